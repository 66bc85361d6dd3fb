"""Brute force on tiny periodic lattices: the C definition oracle against a second, plain
numpy statement of the scheme written here from Sections 1.1-1.2.

Per node: rho and q from relation (rhoq); u~ = 0, q / rho or the prescribed field; the
moment matrix M(u~)_kj = P_k(v_j - u~) of the golden polynomials (relation (mom)); the
second-order equilibrium f_eq(rho, q / rho); m* = m + S (m_eq - m) (relation (relaxationu));
f* = M(u~)^{-1} m* by numpy.linalg.solve; then transport f_j(x) <- f*_j(x - v_j), periodic
(relation (transport)). Shares no code with the C oracle (the polynomials are read from the
golden file and evaluated by sympy).
"""
import numpy as np
import pytest
import sympy as sp

from conftest import read_golden_rows

CXY = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
S_PAPER = np.array([0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4])


def _polys():
    X, Y, lam = sp.symbols("X Y lam", real=True)
    ns = {"X": X, "Y": Y, "lam": lam, "Rational": sp.Rational}
    exprs = [sp.sympify(r, locals=ns) for r in read_golden_rows("moment_polynomials.txt")]
    return [sp.lambdify((X, Y, lam), e, "numpy") for e in exprs]


POLYS = _polys()


def _moment_matrix(ut, lam):
    M = np.empty((9, 9))
    for j in range(9):
        X, Y = lam * CXY[j, 0] - ut[0], lam * CXY[j, 1] - ut[1]
        for k in range(9):
            M[k, j] = POLYS[k](X, Y, lam)
    return M


def _feq(rho, u, lam):
    cu = (CXY @ u) / lam
    uu = (u @ u) / lam ** 2
    return W * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * uu)


def _brute_run(f, lam, s, mode, steps, amp=0.0, period=1.0, ut0=None):
    f = f.copy()
    _, ny, nx = f.shape
    for t in range(steps):
        post = np.empty_like(f)
        for y in range(ny):
            for x in range(nx):
                g = f[:, y, x]
                rho = g.sum()
                q = lam * (CXY.T @ g)
                if mode == 0:
                    ut = np.zeros(2)
                elif mode == 1:
                    ut = q / rho
                else:
                    base = (np.array([np.cos(2 * np.pi * y / ny), np.sin(2 * np.pi * x / nx)])
                            if ut0 is None else ut0[:, y, x])
                    ut = amp * base * np.cos(2 * np.pi * t / period)
                M = _moment_matrix(ut, lam)
                m = M @ g
                meq = M @ _feq(rho, q / rho, lam)
                post[:, y, x] = np.linalg.solve(M, m + s * (meq - m))
        for j in range(9):
            f[j] = np.roll(post[j], shift=(CXY[j, 1], CXY[j, 0]), axis=(0, 1))
    return f


def _state(rng, nx, ny, lam):
    rho = 1 + 0.05 * rng.standard_normal((ny, nx))
    u = lam * 0.08 * rng.standard_normal((2, ny, nx))
    f = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f[:, y, x] = _feq(rho[y, x], u[:, y, x], lam)
    # off-equilibrium part so that every moment relaxes
    return f * (1 + 0.05 * rng.standard_normal(f.shape))


@pytest.mark.parametrize("nx,ny", [(3, 3), (4, 5)])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("lam", [1.0, 2.0])
def test_definition_oracle_equals_brute_force(orc, nx, ny, mode, lam):
    rng = np.random.default_rng(100 + 10 * nx + ny + mode)
    f0 = _state(rng, nx, ny, lam)
    kw = dict(amp=0.05 * lam, period=7.0) if mode == 2 else {}
    steps = 4
    ref = _brute_run(f0, lam, S_PAPER, mode, steps, **kw)
    got = orc.run(f0, lam, S_PAPER, mode, steps, method=orc.METHOD_DEFINITION, **kw)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
    got_shift = orc.run(f0, lam, S_PAPER, mode, steps, method=orc.METHOD_SHIFTED, **kw)
    np.testing.assert_allclose(got_shift, ref, rtol=0, atol=1e-12)


def test_prescribed_caller_field_equals_brute_force(orc):
    rng = np.random.default_rng(7)
    nx, ny, lam = 4, 5, 1.0
    f0 = _state(rng, nx, ny, lam)
    ut0 = rng.standard_normal((2, ny, nx))
    kw = dict(amp=0.04, period=5.0)
    ref = _brute_run(f0, lam, S_PAPER, 2, 3, ut0=ut0, **kw)
    got = orc.run(f0, lam, S_PAPER, 2, 3, ut0=ut0, **kw)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- Geier's basis
GEIER = [lambda X, Y: 1.0, lambda X, Y: X, lambda X, Y: Y, lambda X, Y: X * X + Y * Y,
         lambda X, Y: X * X - Y * Y, lambda X, Y: X * Y, lambda X, Y: X * Y * Y,
         lambda X, Y: X * X * Y, lambda X, Y: X * X * Y * Y]
S_GEIER = np.array([0, 0, 0, 1.3, 1.8, 1.8, 1.5, 1.5, 1.2])


def _geier_matrix(ut, lam):
    return np.array([[GEIER[k](lam * CXY[j, 0] - ut[0], lam * CXY[j, 1] - ut[1])
                      for j in range(9)] for k in range(9)])


def _maxwellian_populations(rho, u, lam):
    """The populations whose Geier moments about u are those of the Maxwellian with
    c^2 = lambda^2 / 3: (rho, 0, 0, 2 rho c^2, 0, 0, 0, 0, rho c^4) (the reading of
    Section 1.3 on Geier's equilibria), solved for directly."""
    c2 = lam * lam / 3
    return np.linalg.solve(_geier_matrix(u, lam),
                           np.array([rho, 0, 0, 2 * rho * c2, 0, 0, 0, 0, rho * c2 * c2]))


def _brute_run_geier(f, lam, s, mode, steps, amp=0.0, period=1.0):
    f = f.copy()
    _, ny, nx = f.shape
    for t in range(steps):
        post = np.empty_like(f)
        for y in range(ny):
            for x in range(nx):
                g = f[:, y, x]
                rho = g.sum()
                q = lam * (CXY.T @ g)
                if mode == 0:
                    ut = np.zeros(2)
                elif mode == 1:
                    ut = q / rho
                else:
                    ut = amp * np.array([np.cos(2 * np.pi * y / ny), np.sin(2 * np.pi * x / nx)]
                                        ) * np.cos(2 * np.pi * t / period)
                M = _geier_matrix(ut, lam)
                m = M @ g
                meq = M @ _maxwellian_populations(rho, q / rho, lam)
                post[:, y, x] = np.linalg.solve(M, m + s * (meq - m))
        for j in range(9):
            f[j] = np.roll(post[j], shift=(CXY[j, 1], CXY[j, 0]), axis=(0, 1))
    return f


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("lam", [1.0, 2.0])
def test_geier_definition_oracle_equals_brute_force(orc, mode, lam):
    """The oracle's definition in Geier's basis (product-form equilibrium) against the
    numpy statement above, whose equilibrium is solved from the Maxwellian moments."""
    rng = np.random.default_rng(300 + 10 * mode + int(lam))
    nx, ny = 4, 3
    rho = 1 + 0.05 * rng.standard_normal((ny, nx))
    u = lam * 0.06 * rng.standard_normal((2, ny, nx))
    f0 = np.empty((9, ny, nx))
    for y in range(ny):
        for x in range(nx):
            f0[:, y, x] = _maxwellian_populations(rho[y, x], u[:, y, x], lam)
    f0 *= 1 + 0.05 * rng.standard_normal(f0.shape)
    kw = dict(amp=0.05 * lam, period=7.0) if mode == 2 else {}
    ref = _brute_run_geier(f0, lam, S_GEIER, mode, 3, **kw)
    got = orc.run(f0, lam, S_GEIER, mode, 3, method=orc.METHOD_GEIER, **kw)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)
