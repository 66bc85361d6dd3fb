"""Pins of the FP64 D3Q19 oracle (the relative-velocity scheme of Section 1.2 on a D3Q19
lattice with a translation-invariant 19-polynomial basis).

The paper gives no 3D basis; what it fixes is the construction (relations (MatMu),
(relaxationu), (transport)) and the property that makes the shifted form work: the
morphism T(u+v) = T(u) T(v) with T lower triangular (Section 1.3). These tests pin the
oracle to that property, to textbook equilibrium moments, collision invariants, the
equilibrium fixed point, exact transport, u~-independence for equal rates, and the
second-order shear viscosity nu = (1/s_nu - 1/2)/3 of Section 2.3.
"""
import numpy as np
import pytest

from oracle import d3q19 as o3

S3 = np.array([0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3)


def test_velocity_set_is_d3q19():
    c = o3.velocities().T
    assert len({tuple(v) for v in c}) == 19
    n2 = (c ** 2).sum(1)
    assert sorted(n2.tolist()) == [0] + [1] * 6 + [2] * 12
    assert (c.sum(0) == 0).all()


@pytest.mark.parametrize("lam", [1.0, 1.7])
def test_basis_is_unisolvent_and_shift_closed(lam):
    M0 = o3.moment_matrix((0, 0, 0), lam)
    assert np.linalg.matrix_rank(M0) == 19
    rng = np.random.default_rng(1)
    T = lambda w: np.linalg.solve(M0.T, o3.moment_matrix(w, lam).T).T  # noqa: E731
    for _ in range(20):
        u, v = rng.uniform(-0.3, 0.3, 3), rng.uniform(-0.3, 0.3, 3)
        np.testing.assert_allclose(T(u + v), T(u) @ T(v), atol=1e-12)
        np.testing.assert_allclose(T(u) @ T(-u), np.eye(19), atol=1e-12)
        assert np.abs(np.triu(T(u), 1)).max() < 1e-12


def test_monomials_at_velocities():
    """A few entries of M(0) by hand: X^2 Y^2 is 1 exactly on the xy-edge velocities."""
    c = o3.velocities().T
    M0 = o3.moment_matrix((0, 0, 0), 1.0)
    for j, (a, b, d) in enumerate(c):
        assert M0[16, j] == (1.0 if (a != 0 and b != 0) else 0.0)
        assert M0[10, j] == a * b * b
        assert M0[4, j] == a * a + b * b + d * d


def test_equilibrium_textbook_moments():
    rng = np.random.default_rng(2)
    c = o3.velocities().astype(float)
    for _ in range(20):
        lam = float(rng.uniform(0.5, 2.0))
        rho = float(rng.uniform(0.5, 1.5))
        u = rng.uniform(-0.15, 0.15, 3)
        f = o3.feq(rho, u, lam)
        v = lam * c
        np.testing.assert_allclose(f.sum(), rho, rtol=1e-14)
        np.testing.assert_allclose(v @ f, rho * u, atol=1e-14)
        Pi = (v[:, None, :] * v[None, :, :] * f).sum(-1)
        np.testing.assert_allclose(Pi, rho * np.outer(u, u) + rho * lam * lam / 3 * np.eye(3),
                                   atol=1e-14)


def _random_state(rng, lam=1.0):
    f = o3.feq(float(rng.uniform(0.8, 1.2)), rng.uniform(-0.1, 0.1, 3), lam)
    return f * (1 + 0.05 * rng.standard_normal(19))


def test_relaxation_invariants_and_fixed_point():
    rng = np.random.default_rng(3)
    c = o3.velocities().astype(float)
    for _ in range(30):
        lam = float(rng.uniform(0.5, 2.0))
        f = _random_state(rng, lam)
        ut = rng.uniform(-0.2, 0.2, 3)
        s = np.concatenate([[0, 0, 0, 0], rng.uniform(0.5, 1.95, 15)])
        fs = o3.collide_node(f, ut, lam, s)
        np.testing.assert_allclose(fs.sum(), f.sum(), rtol=1e-13)
        np.testing.assert_allclose(lam * c @ fs, lam * c @ f, atol=1e-13)
        fe = o3.feq(float(rng.uniform(0.8, 1.2)), rng.uniform(-0.1, 0.1, 3), lam)
        np.testing.assert_allclose(o3.collide_node(fe, ut, lam, s), fe, atol=1e-15)


def test_equal_rates_independent_of_relative_velocity():
    rng = np.random.default_rng(4)
    s = np.array([0, 0, 0, 0] + [1.55] * 15)
    for _ in range(10):
        f = _random_state(rng)
        a = o3.collide_node(f, (0, 0, 0), 1.0, s)
        b = o3.collide_node(f, rng.uniform(-0.2, 0.2, 3), 1.0, s)
        np.testing.assert_allclose(a, b, atol=1e-14)


def test_unequal_rates_depend_on_relative_velocity():
    rng = np.random.default_rng(5)
    f = _random_state(rng)
    a = o3.collide_node(f, (0, 0, 0), 1.0, S3)
    b = o3.collide_node(f, (0.1, -0.05, 0.07), 1.0, S3)
    assert np.abs(a - b).max() > 1e-7


def test_transport_moves_populations_along_velocities():
    c = o3.velocities().T
    nx, ny, nz = 5, 4, 3
    for j, (a, b, d) in enumerate(c):
        f = np.zeros((19, nz, ny, nx))
        f[j, 1, 2, 3] = 1.0
        g = o3.stream(f)
        assert g[j, (1 + d) % nz, (2 + b) % ny, (3 + a) % nx] == 1.0
        assert g.sum() == 1.0


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_lattice_conservation(mode):
    rng = np.random.default_rng(6)
    shape = (3, 5, 4)
    rho = 1 + 0.01 * rng.standard_normal(shape)
    u = 0.03 * rng.standard_normal((3,) + shape)
    ut0 = rng.standard_normal((3,) + shape)
    f0 = o3.init_equilibrium(rho, u, 1.0)
    f = o3.run(f0, 1.0, S3, mode, 12, ut0=ut0, amp=0.05, period=20.0)
    r0, u0 = o3.moments(f0, 1.0)
    r1, u1 = o3.moments(f, 1.0)
    np.testing.assert_allclose(r1.sum(), r0.sum(), rtol=1e-13)
    np.testing.assert_allclose((r1 * u1).sum(axis=(1, 2, 3)), (r0 * u0).sum(axis=(1, 2, 3)),
                               atol=1e-13)


def _shear_nu(mode, axis, s_nu=1.7, L=40, steps=200, t_fit=60):
    s = S3.copy()
    s[5:10] = s_nu
    shape = [4, 4, 4]
    shape[{"y": 1, "z": 0}[axis]] = L  # (nz, ny, nx)
    rho = np.ones(shape)
    u = np.zeros((3,) + tuple(shape))
    coord = np.arange(L)
    prof = 1e-3 * np.sin(2 * np.pi * coord / L)
    if axis == "y":
        u[0] = prof[None, :, None]
    else:
        u[1] = prof[:, None, None]
    ut0 = np.ones((3,) + tuple(shape))
    f = o3.init_equilibrium(rho, u, 1.0)
    f = o3.run(f, 1.0, s, mode, t_fit, ut0=ut0, amp=0.02, nthreads=8)
    ts, amps = [], []
    sn = np.sin(2 * np.pi * coord / L)
    t = t_fit
    while t <= steps:
        _, uu = o3.moments(f, 1.0)
        if axis == "y":
            p = uu[0].mean(axis=(0, 2))
        else:
            p = uu[1].mean(axis=(1, 2))
        amps.append(p @ sn / (sn @ sn))
        ts.append(t)
        f = o3.run(f, 1.0, s, mode, 20, t0=t, ut0=ut0, amp=0.02, nthreads=8)
        t += 20
    k = 2 * np.pi / L
    return -np.polyfit(ts, np.log(amps), 1)[0] / (k * k)


@pytest.mark.slow
def test_shear_viscosity_second_order_3d():
    nu_th = (1 / 1.7 - 0.5) / 3
    nus = [_shear_nu(m, "y") for m in (0, 1, 2)]
    for nu in nus:
        assert abs(nu / nu_th - 1) < 0.015, (nus, nu_th)
    assert max(nus) / min(nus) - 1 < 1e-3
    assert abs(_shear_nu(1, "z") / nu_th - 1) < 0.015
