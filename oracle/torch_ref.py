"""FP64 PyTorch (CPU) statement of the relative-velocity scheme, for reference gradients.

TEST INFRASTRUCTURE (see the package docstring). This is the definition of Section 1.2
written with plain torch ops, independent of ``lbmrv_oracle.c``: per node the shifted
moment matrix M(u~)_kj = P_k(v_j - u~) of relation (MatMu) with the polynomials of
relation (mom), m = M(u~) f, m_eq = M(u~) f_eq, the diagonal relaxation (relaxationu),
f* = M(u~)^{-1} m* by ``torch.linalg.solve``, then the exact transport (transport) as a
periodic roll. Reverse-mode differentiation of this program is the reference adjoint:
gradients of a final-time loss with respect to the initial velocity field, the shear
relaxation rate s_nu (shared by p_xx and p_xy) and the amplitude of a prescribed u~.

Conventions match the C oracle: lattice units dx = 1, polynomial second-order
equilibrium, collision at time index t uses u~(x, t) = A u~0(x) cos(2 pi t / P).
"""
from __future__ import annotations

import torch
from torch.utils.checkpoint import checkpoint

CX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
W = (4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36)
F64 = torch.float64


def _c(lam):
    cx = torch.tensor(CX, dtype=F64) * lam
    cy = torch.tensor(CY, dtype=F64) * lam
    return cx, cy


def polynomials(X, Y, lam):
    """The nine polynomials of relation (mom), stacked on a new axis -2 (index k)."""
    r2 = X * X + Y * Y
    l2 = lam * lam
    P = [torch.ones_like(X), X, Y, (3 * r2 - 4 * l2) / l2, (X * X - Y * Y) / l2, X * Y / l2,
         X * (3 * r2 - 5 * l2) / (l2 * lam), Y * (3 * r2 - 5 * l2) / (l2 * lam),
         (4.5 * r2 * r2 - 10.5 * l2 * r2 + 4 * l2 * l2) / (l2 * l2)]
    return torch.stack(P, dim=-2)


def moment_matrix(utx, uty, lam):
    """M(u~) for every node: utx, uty [...] -> [..., 9 (k), 9 (j)]."""
    cx, cy = _c(lam)
    X = cx - utx[..., None]
    Y = cy - uty[..., None]
    return polynomials(X, Y, lam)


def feq(rho, ux, uy, lam):
    """Second-order polynomial equilibrium, [...] -> [..., 9]."""
    cx, cy = _c(lam)
    w = torch.tensor(W, dtype=F64)
    vu = cx * ux[..., None] + cy * uy[..., None]
    uu = (ux * ux + uy * uy)[..., None]
    l2 = lam * lam
    return w * rho[..., None] * (1 + 3 * vu / l2 + 4.5 * vu * vu / (l2 * l2) - 1.5 * uu / l2)


def moments(f, lam):
    """f [9, ny, nx] -> rho, q_x, q_y (relation (rhoq))."""
    cx, cy = _c(lam)
    rho = f.sum(0)
    qx = torch.einsum("j,jyx->yx", cx, f)
    qy = torch.einsum("j,jyx->yx", cy, f)
    return rho, qx, qy


def relative_velocity(mode, f, lam, t, ut0, amp, period):
    ny, nx = f.shape[1:]
    if mode == 0:
        z = torch.zeros((ny, nx), dtype=F64)
        return z, z
    if mode == 1:
        rho, qx, qy = moments(f, lam)
        return qx / rho, qy / rho
    tf = torch.cos(torch.tensor(2 * torch.pi * t / period, dtype=F64)) if period > 0 else 1.0
    return amp * ut0[0] * tf, amp * ut0[1] * tf


def collide(f, lam, s, mode, t, ut0=None, amp=0.0, period=0.0):
    """Relaxation of Section 1.2 at every node; f [9, ny, nx]; s: 9 rates (tensor)."""
    utx, uty = relative_velocity(mode, f, lam, t, ut0, amp, period)
    rho, qx, qy = moments(f, lam)
    fe = feq(rho, qx / rho, qy / rho, lam)              # [ny, nx, 9]
    M = moment_matrix(utx, uty, lam)                    # [ny, nx, 9, 9]
    fn = f.permute(1, 2, 0)                             # [ny, nx, 9]
    m = (M @ fn[..., None])[..., 0]
    meq = (M @ fe[..., None])[..., 0]
    ms = m + s * (meq - m)
    fs = torch.linalg.solve(M, ms[..., None])[..., 0]
    return fs.permute(2, 0, 1)


def stream(f):
    """f_j(x, t+dt) = f*_j(x - c_j), periodic (relation (transport))."""
    return torch.stack([torch.roll(f[j], shifts=(CY[j], CX[j]), dims=(0, 1))
                        for j in range(9)])


def analytic_base_field(nx, ny):
    y = torch.arange(ny, dtype=F64)[:, None].expand(ny, nx)
    x = torch.arange(nx, dtype=F64)[None, :].expand(ny, nx)
    return torch.stack([torch.cos(2 * torch.pi * y / ny), torch.sin(2 * torch.pi * x / nx)])


def rates(s_base, s_nu):
    """9 rates with the two second-order shear rates (p_xx, p_xy) set to s_nu."""
    s = torch.as_tensor(s_base, dtype=F64).clone()
    s_nu = torch.as_tensor(s_nu).to(F64).reshape(1)
    return torch.cat([s[:4], s_nu, s_nu, s[6:]])


def final_state(rho0, u0, lam, s, mode, steps, ut0=None, amp=0.0, period=0.0, chunk=8):
    """f(steps) from f(0) = f_eq(rho0, u0); u0 [2, ny, nx]. Gradient checkpointing every
    `chunk` steps keeps the memory of the reverse pass small."""
    f = feq(rho0, u0[0], u0[1], lam).permute(2, 0, 1)

    def advance(f_in, t_start, n):
        for k in range(n):
            f_in = stream(collide(f_in, lam, s, mode, t_start + k, ut0, amp, period))
        return f_in

    t = 0
    while t < steps:
        n = min(chunk, steps - t)
        f = checkpoint(advance, f, t, n, use_reentrant=False)
        t += n
    return f


def kinetic_energy(f, lam):
    """L = 1/2 sum_x |q|^2 / rho (lattice units)."""
    rho, qx, qy = moments(f, lam)
    return 0.5 * ((qx * qx + qy * qy) / rho).sum()


def loss_and_grads(rho0, u0, lam, s_base, s_nu, mode, steps, ut0=None, amp=0.0, period=0.0):
    """Kinetic energy after `steps` steps and its gradients with respect to u0, s_nu and
    the amplitude of the prescribed u~ (FP64 reverse mode)."""
    u0 = torch.as_tensor(u0, dtype=F64).clone().requires_grad_(True)
    s_nu_t = torch.tensor(float(s_nu), dtype=F64, requires_grad=True)
    amp_t = torch.tensor(float(amp), dtype=F64, requires_grad=True)
    rho0 = torch.as_tensor(rho0, dtype=F64)
    if ut0 is not None:
        ut0 = torch.as_tensor(ut0, dtype=F64)
    s = rates(s_base, s_nu_t)
    f = final_state(rho0, u0, lam, s, mode, steps, ut0, amp_t, period)
    L = kinetic_energy(f, lam)
    gu, gs, ga = torch.autograd.grad(L, (u0, s_nu_t, amp_t), allow_unused=True)
    ga = torch.zeros((), dtype=F64) if ga is None else ga
    return float(L.detach()), gu.detach().numpy(), float(gs), float(ga)


def loss_only(rho0, u0, lam, s_base, s_nu, mode, steps, ut0=None, amp=0.0, period=0.0):
    with torch.no_grad():
        u0 = torch.as_tensor(u0, dtype=F64)
        s = rates(s_base, torch.tensor(float(s_nu), dtype=F64))
        ut = None if ut0 is None else torch.as_tensor(ut0, dtype=F64)
        f = feq(torch.as_tensor(rho0, dtype=F64), u0[0], u0[1], lam).permute(2, 0, 1)
        for k in range(steps):
            f = stream(collide(f, lam, s, mode, k, ut, amp, period))
        return float(kinetic_energy(f, lam))
