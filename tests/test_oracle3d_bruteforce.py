"""Brute force on tiny periodic D3Q19 lattices: the C D3Q19 oracle against a second, plain
numpy statement of the scheme of Sections 1.1-1.2 written here.

Per node: rho and q (relation (rhoq)); u~ = 0, q / rho or A u~0(x) cos(2 pi t / P); the
moment matrix M(u~)_kj = P_k(lambda c_j - u~) of the 19 translation-invariant polynomials;
the second-order equilibrium; m* = m + S (m_eq - m); f* = M(u~)^{-1} m* by
numpy.linalg.solve; transport f_j(x) <- f*_j(x - c_j) by numpy.roll. The relaxed
populations do not depend on how each polynomial is normalised (a row scale of M cancels),
so the basis is written here without the oracle's powers of lambda.
"""
import numpy as np
import pytest

from oracle import d3q19 as o3

C3 = np.array([(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
               (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1),
               (1, 0, -1), (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)])
W3 = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
S3 = np.array([0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3)

BASIS = [
    lambda X, Y, Z: 1.0, lambda X, Y, Z: X, lambda X, Y, Z: Y, lambda X, Y, Z: Z,
    lambda X, Y, Z: X * X + Y * Y + Z * Z, lambda X, Y, Z: X * X - Y * Y,
    lambda X, Y, Z: Y * Y - Z * Z, lambda X, Y, Z: X * Y, lambda X, Y, Z: X * Z,
    lambda X, Y, Z: Y * Z, lambda X, Y, Z: X * Y * Y, lambda X, Y, Z: X * Z * Z,
    lambda X, Y, Z: Y * X * X, lambda X, Y, Z: Y * Z * Z, lambda X, Y, Z: Z * X * X,
    lambda X, Y, Z: Z * Y * Y, lambda X, Y, Z: X * X * Y * Y, lambda X, Y, Z: X * X * Z * Z,
    lambda X, Y, Z: Y * Y * Z * Z,
]


def _moment_matrix(ut, lam):
    M = np.empty((19, 19))
    for j in range(19):
        X, Y, Z = lam * C3[j] - ut
        for k in range(19):
            M[k, j] = BASIS[k](X, Y, Z)
    return M


def _feq(rho, u, lam):
    cu = (C3 @ u) / lam
    return W3 * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (u @ u) / lam ** 2)


def _brute_run(f, lam, s, mode, steps, ut0=None, amp=0.0, period=1.0):
    f = f.copy()
    _, nz, ny, nx = f.shape
    for t in range(steps):
        post = np.empty_like(f)
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    g = f[:, z, y, x]
                    rho = g.sum()
                    q = lam * (C3.T @ g)
                    if mode == 0:
                        ut = np.zeros(3)
                    elif mode == 1:
                        ut = q / rho
                    else:
                        ut = amp * ut0[:, z, y, x] * np.cos(2 * np.pi * t / period)
                    M = _moment_matrix(ut, lam)
                    m = M @ g
                    meq = M @ _feq(rho, q / rho, lam)
                    post[:, z, y, x] = np.linalg.solve(M, m + s * (meq - m))
        for j in range(19):
            f[j] = np.roll(post[j], shift=(C3[j, 2], C3[j, 1], C3[j, 0]), axis=(0, 1, 2))
    return f


def test_velocity_order():
    np.testing.assert_array_equal(o3.velocities().T, C3)


@pytest.mark.parametrize("shape", [(3, 3, 3), (4, 3, 2)])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("lam", [1.0, 1.5])
def test_d3q19_oracle_equals_brute_force(shape, mode, lam):
    nx, ny, nz = shape
    rng = np.random.default_rng(200 + 10 * nx + ny + nz + mode)
    rho = 1 + 0.05 * rng.standard_normal((nz, ny, nx))
    u = lam * 0.06 * rng.standard_normal((3, nz, ny, nx))
    f0 = np.empty((19, nz, ny, nx))
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                f0[:, z, y, x] = _feq(rho[z, y, x], u[:, z, y, x], lam)
    f0 *= 1 + 0.05 * rng.standard_normal(f0.shape)  # off-equilibrium in every moment
    kw = {}
    if mode == 2:
        kw = dict(ut0=rng.standard_normal((3, nz, ny, nx)), amp=0.04 * lam, period=7.0)
    steps = 3
    ref = _brute_run(f0, lam, S3, mode, steps, **kw)
    got = o3.run(f0, lam, S3, mode, steps, **kw)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
