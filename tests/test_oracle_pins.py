"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test names the passage it checks. None of them compares the oracle with itself:
the printed matrices of Section 1.3 and Appendix A, the definition T = M(u~) M(0)^{-1},
the morphism proposition, the reduction to d'Humieres MRT, collision invariants, the
equilibrium fixed point, exact transport, and the second-order viscosity of Section 2.3.
"""
import numpy as np
import pytest
import sympy as sp

import lbm_inputs as inp
from conftest import read_golden_rows

S_PAPER = np.array([0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4])


def _sym():
    ux, uy, lam, X, Y = sp.symbols("ux uy lam X Y", real=True)
    return ux, uy, lam, X, Y


def _golden_polys():
    ux, uy, lam, X, Y = _sym()
    ns = {"X": X, "Y": Y, "lam": lam, "Rational": sp.Rational}
    return [sp.sympify(r, locals=ns) for r in read_golden_rows("moment_polynomials.txt")]


CXY = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]


def _sym_T():
    """T = M(u~) M(0)^{-1} from the definition (relation (MatMu) and the definition of T)."""
    ux, uy, lam, X, Y = _sym()
    P = _golden_polys()

    def M(ax, ay):
        return sp.Matrix(9, 9, lambda k, j: sp.simplify(
            P[k].subs({X: lam * CXY[j][0] - ax, Y: lam * CXY[j][1] - ay}, simultaneous=True)))

    return sp.simplify(M(ux, uy) * M(0, 0).inv()), M(0, 0)


@pytest.fixture(scope="module")
def sym_T():
    return _sym_T()


# ----------------------------------------------------------------- Section 1.3 matrices
@pytest.mark.parametrize("lam", [1.0, 2.0, 0.5])
def test_fixed_moment_matrix_matches_printed(orc, lam):
    """Relation (matort): M(0) as printed (rows 1, 2 scaled by lambda)."""
    M_printed = np.array([[float(v) for v in r.split()] for r in read_golden_rows("m0_d2q9.txt")])
    M_printed[1:3] *= lam
    np.testing.assert_array_equal(orc.moment_matrix(0.0, 0.0, lam), M_printed)


def test_printed_m0_rows_orthogonal():
    """Section 1.3 uses the orthogonal set: rows of M(0) are orthogonal, |row|^2 as listed."""
    M = np.array([[float(v) for v in r.split()] for r in read_golden_rows("m0_d2q9.txt")])
    G = M @ M.T
    np.testing.assert_array_equal(G, np.diag([9, 6, 6, 36, 4, 4, 12, 12, 36]).astype(float))


def test_moment_matrix_matches_polynomials_at_shifted_points(orc):
    """Relation (MatMu): M(u~)_kj = P_k(v_j - u~) with the printed polynomials (mom)."""
    ux, uy, lam, X, Y = _sym()
    P = _golden_polys()
    rng = np.random.default_rng(3)
    for _ in range(5):
        a, b = rng.uniform(-0.3, 0.3, 2)
        L = float(rng.uniform(0.5, 2.0))
        M = orc.moment_matrix(a, b, L)
        for k in range(9):
            for j in range(9):
                ref = float(P[k].subs({X: L * CXY[j][0] - a, Y: L * CXY[j][1] - b, lam: L}))
                assert abs(M[k, j] - ref) <= 1e-12 * max(1.0, abs(ref))


# ----------------------------------------------------------------- Appendix A, Prop. 2.1
def test_appendix_a_blocks_vs_definition(sym_T):
    """Appendix A blocks against T = M(u~) M(0)^{-1}; D2 is printed with an extra 1/2."""
    T, _ = sym_T
    ux, uy, lam, X, Y = _sym()
    listed = {}
    for row in read_golden_rows("appendix_a_blocks.txt"):
        name, r, c, expr = row.split(None, 3)
        listed[(int(r), int(c))] = (name, sp.sympify(expr, locals={"ux": ux, "uy": uy, "lam": lam}))
    for r in range(9):
        for c in range(9):
            if (r, c) in listed:
                name, printed = listed[(r, c)]
                diff = sp.simplify(T[r, c] - (2 * printed if name == "D2" else printed))
                assert diff == 0, (name, r, c, T[r, c], printed)
                if name == "D2":
                    assert sp.simplify(T[r, c] - printed) != 0
            else:
                assert T[r, c] == (1 if r == c else 0), (r, c, T[r, c])


def test_oracle_shift_matrix_is_the_definition(orc, sym_T):
    """The oracle's closed-form T(u~) equals M(u~) M(0)^{-1} at random u~, lambda."""
    T, _ = sym_T
    ux, uy, lam, X, Y = _sym()
    f = sp.lambdify((ux, uy, lam), T, "numpy")
    rng = np.random.default_rng(7)
    for _ in range(20):
        a, b = rng.uniform(-0.5, 0.5, 2)
        L = float(rng.uniform(0.5, 3.0))
        np.testing.assert_allclose(orc.shift_matrix(a, b, L), np.array(f(a, b, L), float),
                                   rtol=1e-13, atol=1e-13)


def test_shift_matrix_numeric_definition(orc):
    """Same fact without sympy: T from the oracle's own M(u~) and M(0) by a library solve."""
    rng = np.random.default_rng(11)
    for _ in range(20):
        a, b = rng.uniform(-0.4, 0.4, 2)
        L = float(rng.uniform(0.5, 2.0))
        Mu = orc.moment_matrix(a, b, L)
        M0 = orc.moment_matrix(0.0, 0.0, L)
        T_num = np.linalg.solve(M0.T, Mu.T).T
        np.testing.assert_allclose(orc.shift_matrix(a, b, L), T_num, rtol=1e-11, atol=1e-11)


def test_morphism_of_groups(orc):
    """Proposition 'Morphism of groups': T(u+v) = T(u) T(v) = T(v) T(u), T(u) T(-u) = I."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        u = rng.uniform(-0.3, 0.3, 2)
        v = rng.uniform(-0.3, 0.3, 2)
        L = float(rng.uniform(0.5, 2.0))
        Tu, Tv = orc.shift_matrix(*u, L), orc.shift_matrix(*v, L)
        Tuv = orc.shift_matrix(*(u + v), L)
        np.testing.assert_allclose(Tuv, Tu @ Tv, atol=1e-14)
        np.testing.assert_allclose(Tuv, Tv @ Tu, atol=1e-14)
        np.testing.assert_allclose(Tu @ orc.shift_matrix(*(-u), L), np.eye(9), atol=1e-14)


def test_symbolic_morphism(sym_T):
    T, _ = sym_T
    ux, uy, lam, X, Y = _sym()
    vx, vy = sp.symbols("vx vy", real=True)
    Tv = T.subs({ux: vx, uy: vy}, simultaneous=True)
    Tuv = T.subs({ux: ux + vx, uy: uy + vy}, simultaneous=True)
    assert sp.simplify(Tuv - T * Tv) == sp.zeros(9, 9)


# ----------------------------------------------------------------- equilibrium
def test_equilibrium_textbook_moments(orc):
    """D2Q9 second-order equilibrium: sum f = rho, sum v f = rho u,
    sum v_a v_b f = rho u_a u_b + rho lambda^2/3 delta_ab (c_s^2 = lambda^2/3)."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        rho = float(rng.uniform(0.5, 1.5))
        u = rng.uniform(-0.2, 0.2, 2)
        L = float(rng.uniform(0.5, 2.0))
        f = orc.feq(rho, u[0], u[1], L)
        vx, vy = orc.velocities(L)
        np.testing.assert_allclose(f.sum(), rho, rtol=1e-14)
        np.testing.assert_allclose([vx @ f, vy @ f], rho * u, atol=1e-15)
        Pi = np.array([[vx * vx @ f, vx * vy @ f], [vy * vx @ f, vy * vy @ f]])
        np.testing.assert_allclose(Pi, rho * np.outer(u, u) + rho * L * L / 3 * np.eye(2),
                                   rtol=1e-13, atol=1e-15)


def test_equilibrium_fixed_moments_lallemand_luo(orc):
    """M(0) f_eq equals the Lallemand-Luo equilibrium moments (sympy derivation from the
    textbook equilibrium, not the oracle's code)."""
    rho_s, jx, jy, lam = sp.symbols("rho jx jy lam", positive=True)
    w = [sp.Rational(4, 9)] + [sp.Rational(1, 9)] * 4 + [sp.Rational(1, 36)] * 4
    u = (jx / rho_s, jy / rho_s)
    feq = []
    for j, (a, b) in enumerate(CXY):
        vu = lam * a * u[0] + lam * b * u[1]
        feq.append(w[j] * rho_s * (1 + 3 * vu / lam**2 + sp.Rational(9, 2) * vu**2 / lam**4
                                   - sp.Rational(3, 2) * (u[0]**2 + u[1]**2) / lam**2))
    M0 = np.array([[float(v) for v in r.split()] for r in read_golden_rows("m0_d2q9.txt")])
    M0s = sp.Matrix(M0.astype(int).tolist())
    M0s[1, :] *= lam
    M0s[2, :] *= lam
    meq = sp.simplify(M0s * sp.Matrix(feq))
    expected = [rho_s, jx, jy, -2 * rho_s + 3 * (jx**2 + jy**2) / (lam**2 * rho_s),
                (jx**2 - jy**2) / (lam**2 * rho_s), jx * jy / (lam**2 * rho_s),
                -jx / lam, -jy / lam, rho_s - 3 * (jx**2 + jy**2) / (lam**2 * rho_s)]
    for k in range(9):
        assert sp.simplify(meq[k] - expected[k]) == 0
    rng = np.random.default_rng(4)
    for _ in range(10):
        r = float(rng.uniform(0.5, 1.5)); a, b = rng.uniform(-0.2, 0.2, 2)
        L = float(rng.uniform(0.5, 2.0))
        got = orc.moment_matrix(0, 0, L) @ orc.feq(r, a, b, L)
        ref = [float(e.subs({rho_s: r, jx: r * a, jy: r * b, lam: L})) for e in expected]
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------- per-node relaxation
def _random_state(rng, L=1.0):
    rho = float(rng.uniform(0.8, 1.2))
    u = rng.uniform(-0.1, 0.1, 2)
    import oracle
    f = oracle.feq(rho, u[0], u[1], L)
    return f * (1 + 0.05 * rng.standard_normal(9))


@pytest.mark.parametrize("method", [0, 1, 2])
def test_collision_conserves_rho_and_q(orc, method):
    """Relation (rhoq) and s_k = 0 on conserved moments: rho and q are collision invariants."""
    rng = np.random.default_rng(10 + method)
    for _ in range(50):
        L = float(rng.uniform(0.5, 2.0))
        f = _random_state(rng, L)
        ut = rng.uniform(-0.2, 0.2, 2)
        s = np.concatenate([[0, 0, 0], rng.uniform(0.5, 1.95, 6)])
        fs = orc.collide_node(method, f, ut[0], ut[1], L, s)
        vx, vy = orc.velocities(L)
        np.testing.assert_allclose(fs.sum(), f.sum(), rtol=1e-14)
        np.testing.assert_allclose([vx @ fs, vy @ fs], [vx @ f, vy @ f], atol=1e-14)


@pytest.mark.parametrize("method", [0, 1, 2])
def test_equilibrium_is_fixed_point_of_relaxation(orc, method):
    """Section 1.2: f = f_eq gives m(u~) = m_eq(u~) for every u~, so nothing relaxes."""
    rng = np.random.default_rng(20 + method)
    for _ in range(50):
        L = float(rng.uniform(0.5, 2.0))
        f = orc.feq(float(rng.uniform(0.5, 1.5)), *rng.uniform(-0.2, 0.2, 2), L)
        ut = rng.uniform(-0.3, 0.3, 2)
        s = np.concatenate([[0, 0, 0], rng.uniform(0.5, 1.95, 6)])
        np.testing.assert_allclose(orc.collide_node(method, f, ut[0], ut[1], L, s), f,
                                   rtol=1e-13, atol=1e-15)


def test_shifted_form_equals_definition(orc):
    """Section 1.3: f* = M(0)^{-1} T(-u~) m* equals the definition's M(u~)^{-1} m*."""
    rng = np.random.default_rng(30)
    for _ in range(200):
        L = float(rng.uniform(0.5, 2.0))
        f = _random_state(rng, L)
        ut = rng.uniform(-0.3, 0.3, 2)
        s = np.concatenate([[0, 0, 0], rng.uniform(0.5, 1.95, 6)])
        a = orc.collide_node(0, f, ut[0], ut[1], L, s)
        b = orc.collide_node(1, f, ut[0], ut[1], L, s)
        np.testing.assert_allclose(a, b, rtol=1e-13, atol=1e-14)


def test_relative_velocity_changes_the_relaxation(orc):
    """With unequal rates, u~ != 0 gives a different relaxation from MRT (the scheme is
    not trivially MRT); the difference vanishes linearly as u~ -> 0."""
    rng = np.random.default_rng(31)
    f = _random_state(rng)
    s = S_PAPER
    base = orc.collide_node(2, f, 0, 0, 1.0, s)
    d1 = np.abs(orc.collide_node(0, f, 0.1, 0.05, 1.0, s) - base).max()
    d2 = np.abs(orc.collide_node(0, f, 0.05, 0.025, 1.0, s) - base).max()
    assert d1 > 1e-6
    assert 1.7 < d1 / d2 < 2.3


def test_lu_solve_matches_library(orc):
    import ctypes
    rng = np.random.default_rng(40)
    L = orc.lib()
    for _ in range(20):
        A = rng.standard_normal((9, 9))
        b = rng.standard_normal(9)
        x = np.zeros(9)
        A2, b2 = A.copy(), b.copy()
        P = ctypes.POINTER(ctypes.c_double)
        rc = L.orc_lu_solve(A2.ctypes.data_as(P), b2.ctypes.data_as(P), x.ctypes.data_as(P))
        assert rc == 0
        np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-12)


# ----------------------------------------------------------------- lattice level
def test_transport_moves_each_population_along_its_velocity(orc):
    """Relation (transport): f_j(x, t+dt) = f*_j(x - v_j dt): a population placed at x0
    arrives at x0 + c_j (periodic)."""
    nx, ny = 5, 4
    for j, (cx, cy) in enumerate(CXY):
        f = np.zeros((9, ny, nx))
        f[j, 1, 4] = 1.0
        g = orc.stream(f)
        assert g[j, (1 + cy) % ny, (4 + cx) % nx] == 1.0
        assert g.sum() == 1.0


def _fields(nx, ny, seed=0):
    d = inp.random_sine_flow(nx, ny, seed)
    return d["rho"], d["ux"], d["uy"]


def test_zero_relative_velocity_is_mrt(orc):
    """u~ = 0 gives the d'Humieres scheme (Introduction, Section 1.2): the shifted form is
    bit-for-bit the independently coded MRT; the definition (LU) agrees to rounding."""
    rho, ux, uy = _fields(16, 12)
    f0 = orc.init_equilibrium(rho, ux, uy, 1.0)
    f0 = orc.run(f0, 1.0, S_PAPER, 0, 3, method=2)  # leave equilibrium first
    a = orc.run(f0, 1.0, S_PAPER, 0, 20, method=1)
    b = orc.run(f0, 1.0, S_PAPER, 0, 20, method=2)
    c = orc.run(f0, 1.0, S_PAPER, 0, 20, method=0)
    assert np.array_equal(a, b)
    np.testing.assert_allclose(c, b, rtol=0, atol=1e-14)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_conservation_on_lattice(orc, mode):
    """Mass and momentum are conserved by relaxation and by the periodic transport."""
    rho, ux, uy = _fields(16, 12, seed=1)
    f0 = orc.init_equilibrium(rho, ux, uy, 1.0)
    f = orc.run(f0, 1.0, S_PAPER, mode, 30, amp=0.03, period=50.0)
    r0, a0, b0 = orc.moments(f0, 1.0)
    r1, a1, b1 = orc.moments(f, 1.0)
    np.testing.assert_allclose(r1.sum(), r0.sum(), rtol=1e-13)
    np.testing.assert_allclose((r1 * a1).sum(), (r0 * a0).sum(), atol=1e-13)
    np.testing.assert_allclose((r1 * b1).sum(), (r0 * b0).sum(), atol=1e-13)
    assert np.abs(f - f0).max() > 1e-4  # the state actually evolved


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_uniform_equilibrium_is_steady(orc, mode):
    d = inp.uniform(8, 6, 1.0, (0.07, -0.03))
    f0 = orc.init_equilibrium(d["rho"], d["ux"], d["uy"], 1.0)
    f = orc.run(f0, 1.0, S_PAPER, mode, 25, amp=0.05, period=10.0)
    np.testing.assert_allclose(f, f0, rtol=0, atol=1e-15)


def test_equal_rates_make_scheme_independent_of_relative_velocity(orc):
    """With every non-conserved s_k equal, S = sI commutes with M(u~), so the relaxation
    (relaxationu) does not depend on u~: the three modes give the same trajectory."""
    rho, ux, uy = _fields(12, 10, seed=2)
    f0 = orc.init_equilibrium(rho, ux, uy, 1.0)
    s = np.array([0, 0, 0] + [1.6] * 6)
    runs = [orc.run(f0, 1.0, s, m, 15, amp=0.08, period=40.0) for m in (0, 1, 2)]
    runs.append(orc.run(f0, 1.0, s, 0, 15, method=2))
    for r in runs[1:]:
        np.testing.assert_allclose(r, runs[0], rtol=0, atol=1e-13)


def test_unequal_rates_make_modes_differ(orc):
    rho, ux, uy = _fields(12, 10, seed=2)
    f0 = orc.init_equilibrium(rho, ux, uy, 1.0)
    a = orc.run(f0, 1.0, S_PAPER, 0, 10)
    b = orc.run(f0, 1.0, S_PAPER, 1, 10)
    assert np.abs(a - b).max() > 1e-7


def test_prescribed_field_formula(orc):
    """Prescribed mode at time t uses u~ = A u0(x) cos(2 pi t / P), u0 analytic
    (cos 2 pi y/ny, sin 2 pi x/nx) or a caller field."""
    rng = np.random.default_rng(9)
    nx, ny = 6, 5
    f = np.stack([_random_state(rng) for _ in range(nx * ny)], axis=1).reshape(9, ny, nx)
    A, P, t = 0.04, 30.0, 7
    out = orc.collide(f, 1.0, S_PAPER, 2, t=t, amp=A, period=P)
    base = inp.prescribed_base_field(nx, ny, smooth=False, seed=3)
    out2 = orc.collide(f, 1.0, S_PAPER, 2, t=t, amp=A, period=P, ut0=base)
    tf = np.cos(2 * np.pi * t / P)
    for y in range(ny):
        for x in range(nx):
            ut = (A * np.cos(2 * np.pi * y / ny) * tf, A * np.sin(2 * np.pi * x / nx) * tf)
            np.testing.assert_array_equal(out[:, y, x],
                                          orc.collide_node(0, f[:, y, x], *ut, 1.0, S_PAPER))
            ut2 = (A * base[0, y, x] * tf, A * base[1, y, x] * tf)
            np.testing.assert_array_equal(out2[:, y, x],
                                          orc.collide_node(0, f[:, y, x], *ut2, 1.0, S_PAPER))


# ----------------------------------------------------------------- Section 2.3
def _shear_decay_nu(orc, mode, L=64, s_nu=1.8, steps=300, t_fit=100, method=0):
    s = np.array([0, 0, 0, 1.4, s_nu, s_nu, 1.2, 1.2, 1.4])
    d = inp.shear_wave(L, L, amp=1e-3)
    f = orc.init_equilibrium(d["rho"], d["ux"], d["uy"], 1.0)
    y = np.arange(L)
    sn = np.sin(2 * np.pi * y / L)
    ts, amps = [], []
    chunk = 20
    f = orc.run(f, 1.0, s, mode, t_fit, method=method, amp=0.03, period=0.0, nthreads=8)
    t = t_fit
    while t <= steps:
        _, ux, _ = orc.moments(f, 1.0)
        amps.append((ux.mean(axis=1) @ sn) / (sn @ sn))
        ts.append(t)
        f = orc.run(f, 1.0, s, mode, chunk, t0=t, method=method, amp=0.03, period=0.0,
                    nthreads=8)
        t += chunk
    k = 2 * np.pi / L
    slope = np.polyfit(ts, np.log(amps), 1)[0]
    return -slope / (k * k)


@pytest.mark.slow
def test_shear_wave_viscosity_second_order(orc):
    """Section 2.3 (second-order equivalent equations, corollary): the shear viscosity is
    that of MRT, nu = lambda dx / 3 (1/s_nu - 1/2), independent of u~."""
    nu_th = (1 / 1.8 - 0.5) / 3
    nus = [_shear_decay_nu(orc, m) for m in (0, 1, 2)]
    for nu in nus:
        assert abs(nu / nu_th - 1) < 0.01, (nus, nu_th)
    assert max(nus) / min(nus) - 1 < 1e-3, nus
    nu_other = _shear_decay_nu(orc, 0, s_nu=1.2, method=2)
    assert abs(nu_other / ((1 / 1.2 - 0.5) / 3) - 1) < 0.01


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_taylor_green_decay_rate(orc, mode):
    """Section 2.3: with the MRT viscosity nu = (1/s_nu - 1/2) / 3 (lambda = dx = 1), a
    small Taylor-Green vortex decays as exp(-2 nu k^2 t), k = 2 pi / L, for every u~."""
    L, s_nu, u0 = 32, 1.5, 1e-4
    s = np.array([0, 0, 0, 1.4, s_nu, s_nu, 1.2, 1.2, 1.4])
    d = inp.taylor_green(L, L, u0=u0)
    f = orc.init_equilibrium(d["rho"], d["ux"], d["uy"], 1.0)
    k = 2 * np.pi / L
    x = np.arange(L)[None, :]
    y = np.arange(L)[:, None]
    shape = -np.cos(k * x) * np.sin(k * y)
    ts, amps, t = [], [], 0
    for chunk in (40, 20, 20, 20, 20):
        f = orc.run(f, 1.0, s, mode, chunk, t0=t, amp=0.02, period=0.0, nthreads=4)
        t += chunk
        _, ux, _ = orc.moments(f, 1.0)
        ts.append(t)
        amps.append((ux * shape).sum() / (shape * shape).sum())
    nu = -np.polyfit(ts, np.log(amps), 1)[0] / (2 * k * k)
    assert abs(nu / ((1 / s_nu - 0.5) / 3) - 1) < 1e-3, nu


@pytest.mark.slow
def test_advection_direction(orc):
    """A transverse wave on a uniform flow U moves with the flow (Euler limit of Section
    2.2): uy(x, t) ~ sin(k (x - U t)). Pins the sign of the transport and velocities."""
    L, U, steps = 64, 0.1, 100
    s = np.array([0, 0, 0, 1.4, 1.0, 1.0, 1.2, 1.2, 1.4])
    d = inp.shear_wave(L, 8, amp=1e-4, background=(U, 0.0), axis="x")
    f = orc.init_equilibrium(d["rho"], d["ux"], d["uy"], 1.0)
    f = orc.run(f, 1.0, s, 2, steps, method=2)
    _, _, uy = orc.moments(f, 1.0)
    prof = uy.mean(axis=0)
    x = np.arange(L)
    k = 2 * np.pi / L
    # Fourier phase of the profile: sin(k x - phi) has coefficient ~ -i/2 e^{-i phi}
    c = np.exp(-1j * k * x) @ prof
    phi = np.angle(1j * c) * -1.0
    np.testing.assert_allclose(phi, k * U * steps, rtol=0.05)
    assert np.corrcoef(prof, np.sin(k * (x - U * steps)))[0, 1] > 0.99
