"""Helpers that run the CUDA path and the oracle on the same seeded inputs and measure
their difference. Test infrastructure: imports both sides, which never import each other."""
from __future__ import annotations

import numpy as np

import lbm_inputs as inp

S_PAPER = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
MODES = {"zero": 0, "fluid": 1, "prescribed": 2}


def f32_fields(d):
    return tuple(inp.to_f32_exact(d[k]) for k in ("rho", "ux", "uy"))


def reference_populations(rho_ref, u_ref, lam=1.0):
    """Textbook D2Q9 equilibrium of the reference state (the stored offset)."""
    cx = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
    cy = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)
    ux, uy = u_ref[0] / lam, u_ref[1] / lam
    cu = cx * ux + cy * uy
    return W * rho_ref * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy))


def product_populations(rho_ref, u_ref, lam=1.0):
    """Product-form (Maxwellian-moment) equilibrium of the reference state, from its
    definition phi(0, a) = 2/3 - a^2, phi(+-1, a) = (1/3 + a^2 +- a)/2."""
    cx = [0, 1, 0, -1, 0, 1, -1, -1, 1]
    cy = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    phi = lambda c, a: 2 / 3 - a * a if c == 0 else 0.5 * (1 / 3 + a * a + c * a)  # noqa
    ux, uy = u_ref[0] / lam, u_ref[1] / lam
    return np.array([rho_ref * phi(cx[j], ux) * phi(cy[j], uy) for j in range(9)])


def gpu_run(nx, ny, s, mode, steps, fields, storage="fp32", lam=1.0, rho_ref=None,
            ut0=None, amp=0.0, period=0.0, width=0, u_ref=None, cascaded=False):
    """u_ref=None: the library's automatic reference (the mean flow of the fields); a
    tuple fixes it. Populations are rebuilt from the reference the handle reports."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, D2Q9Cascaded

    rho, ux, uy = fields
    cls = D2Q9Cascaded if cascaded else D2Q9
    sim = cls(nx, ny, s, mode=mode, storage=storage, lam=lam, rho_ref=rho_ref, u_ref=u_ref)
    if width:
        sim.set_kernel_width(width)
    if MODES[mode] == 2:
        sim.set_utilde(None if ut0 is None else torch.as_tensor(ut0, dtype=torch.float32),
                       amp, period)
    sim.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    sim.step(steps)
    g = sim.state().double().cpu().numpy()
    ref_pop = product_populations if cascaded else reference_populations
    f = g + ref_pop(sim.rho_ref, sim.u_ref, lam)[:, None, None]
    r, a, b = (t.double().cpu().numpy() for t in sim.moments())
    sim.close()
    return f, (r, a, b)


def oracle_run(nx, ny, s, mode, steps, fields, lam=1.0, ut0=None, amp=0.0, period=0.0,
               method=0, nthreads=8):
    import oracle

    rho, ux, uy = fields
    if method in (oracle.METHOD_GEIER, oracle.METHOD_CASCADED):
        f0 = oracle.init_equilibrium_product(rho, ux, uy, lam)
    else:
        f0 = oracle.init_equilibrium(rho, ux, uy, lam)
    ut = None if ut0 is None else inp.to_f32_exact(ut0)
    S = oracle.post_collision_state(f0, lam, np.asarray(s, float), MODES[mode], steps,
                                    ut0=ut, amp=amp, period=period, method=method,
                                    nthreads=nthreads)
    return S, oracle.moments(S, lam)


def rel_errors(f_g, m_g, f_o, m_o):
    """rho: max|drho| / max|rho|; u: max_x |du(x)|_2 / max_x |u(x)|_2;
    f: max|df| / max|f|."""
    r_g, ux_g, uy_g = m_g
    r_o, ux_o, uy_o = m_o
    e_rho = np.abs(r_g - r_o).max() / np.abs(r_o).max()
    du = np.hypot(ux_g - ux_o, uy_g - uy_o).max()
    e_u = du / max(np.hypot(ux_o, uy_o).max(), 1e-300)
    e_f = np.abs(f_g - f_o).max() / np.abs(f_o).max()
    return e_rho, e_u, e_f


def oracle_kinetic_energy(rho0, u0, s, mode, steps, amp=0.0, period=0.0, ut0=None,
                          method=1, nthreads=8):
    """FP64 oracle: L = 1/2 sum |q|^2 / rho after `steps` steps from f_eq(rho0, u0)."""
    import oracle

    f0 = oracle.init_equilibrium(rho0, u0[0], u0[1], 1.0)
    f = oracle.run(f0, 1.0, np.asarray(s, float), MODES[mode], steps, method=method,
                   ut0=ut0, amp=amp, period=period, nthreads=nthreads)
    r, ux, uy = oracle.moments(f, 1.0)
    return 0.5 * float((r * (ux * ux + uy * uy)).sum())


def gpu_gradients(nx, ny, s, mode, steps, seg, fields, amp=0.0, period=0.0, ut0=None,
                  field_grad=False, u_ref=None, storage="fp32", width=0):
    """Kinetic energy after `steps` steps and its gradients from the CUDA adjoint:
    (L, dL/du0 [2, ny, nx], dL/ds [9], dL/dA, dL/du~0 or None)."""
    import torch

    from paper_1312_3297_gb300 import D2Q9

    rho, ux, uy = fields
    sim = D2Q9(nx, ny, s, mode=mode, u_ref=u_ref, storage=storage)
    if width:
        sim.set_kernel_width(width)
    if MODES[mode] == 2:
        sim.set_utilde(None if ut0 is None else torch.as_tensor(ut0, dtype=torch.float32),
                       amp, period)
    rho_t = torch.as_tensor(rho, dtype=torch.float32, device="cuda")
    u_t = torch.as_tensor(np.stack([ux, uy]), dtype=torch.float32, device="cuda")
    sim.init_equilibrium(rho_t, u_t[0], u_t[1])
    ws = sim.adjoint_workspace(steps, seg)
    sim.forward_checkpointed(steps, seg, ws)
    ke, dLdS = sim.kinetic_energy(grad=True)
    d0, ds, da, dut = sim.adjoint(steps, seg, ws, dLdS, field_grad=field_grad)
    _, du0 = sim.equilibrium_vjp(rho_t, u_t, d0)
    out = (ke, du0.double().cpu().numpy(), ds, da,
           None if dut is None else dut.double().cpu().numpy())
    sim.close()
    return out


# ------------------------------------------------------------------ D3Q19
S3 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3
W3 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
C3 = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
               [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
               [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]], float)


def reference_populations3(rho_ref, u_ref):
    cu = C3.T @ np.asarray(u_ref, float)
    return W3 * rho_ref * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * float(np.dot(u_ref, u_ref)))


def gpu_run3(shape, s, mode, steps, rho, u, storage="fp32", ut0=None, amp=0.0, period=0.0,
             width=0, u_ref=None):
    """shape = (nx, ny, nz); rho (nz, ny, nx), u (3, nz, ny, nx). Returns (f, rho, u)."""
    import torch

    from paper_1312_3297_gb300 import D3Q19

    nx, ny, nz = shape
    sim = D3Q19(nx, ny, nz, s, mode=mode, storage=storage, u_ref=u_ref)
    if width:
        sim.set_kernel_width(width)
    if MODES[mode] == 2:
        sim.set_utilde(torch.as_tensor(ut0, dtype=torch.float32), amp, period)
    sim.init_equilibrium(torch.as_tensor(rho), *(torch.as_tensor(c) for c in u))
    sim.step(steps)
    g = sim.state().double().cpu().numpy()
    f = g + reference_populations3(sim.rho_ref, sim.u_ref)[:, None, None, None]
    m = [t.double().cpu().numpy() for t in sim.moments()]
    sim.close()
    return f, m[0], np.stack(m[1:])


def oracle_run3(s, mode, steps, rho, u, ut0=None, amp=0.0, period=0.0, nthreads=8):
    from oracle import d3q19 as o3

    f0 = o3.init_equilibrium(rho, u, 1.0)
    ut = None if ut0 is None else inp.to_f32_exact(ut0)
    S = o3.post_collision_state(f0, 1.0, np.asarray(s, float), MODES[mode], steps, ut0=ut,
                                amp=amp, period=period, nthreads=nthreads)
    r, uu = o3.moments(S, 1.0)
    return S, r, uu


def rel_errors3(f_g, r_g, u_g, f_o, r_o, u_o):
    e_rho = np.abs(r_g - r_o).max() / np.abs(r_o).max()
    du = np.sqrt(((u_g - u_o) ** 2).sum(0)).max()
    e_u = du / max(np.sqrt((u_o ** 2).sum(0)).max(), 1e-300)
    e_f = np.abs(f_g - f_o).max() / np.abs(f_o).max()
    return e_rho, e_u, e_f
