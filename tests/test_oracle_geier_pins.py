"""Pins of the oracle's Geier (cascaded) scheme, the proposition of Section 1.3 on the
cascaded scheme and its proof in Appendix B.

The oracle holds two independent codes: the relative-velocity definition in the basis of
relation (polgeier) shifted by u~ (method GEIER), and Geier's cascade as Appendix B writes it
(f* = f + M(0)^T g with g from the triangular system C(u) g = Lambda (m_eq - m), with the
2x2 block of relation (casc1) and the cascade of relation (casc2); method CASCADED). The
proposition says they are the same scheme when u~ = q/rho: that is pinned here, together
with the structure the proof relies on and the physics of the equilibrium.
"""
import numpy as np
import pytest

import lbm_inputs as inp

SG = np.array([0, 0, 0, 1.3, 1.8, 1.8, 1.5, 1.5, 1.2])  # rates in the (polgeier) order
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], float)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], float)


def test_geier_basis_is_unisolvent_and_shift_closed(orc):
    M0 = orc.moment_matrix_geier(0, 0, 1.0)
    assert np.linalg.matrix_rank(M0) == 9
    rng = np.random.default_rng(0)
    T = lambda a, b: np.linalg.solve(M0.T, orc.moment_matrix_geier(a, b, 1.0).T).T  # noqa
    for _ in range(20):
        u, v = rng.uniform(-0.3, 0.3, 2), rng.uniform(-0.3, 0.3, 2)
        np.testing.assert_allclose(T(*(u + v)), T(*u) @ T(*v), atol=1e-12)
        assert np.abs(np.triu(T(*u), 1)).max() < 1e-12


def test_product_equilibrium_has_maxwellian_central_moments(orc):
    """In the frame of the fluid velocity, f_eq has the moments of the Maxwellian:
    (rho, 0, 0, 2 rho c^2, 0, 0, 0, 0, rho c^4), c^2 = lambda^2 / 3 (normalised basis)."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        lam = float(rng.uniform(0.5, 2.0))
        rho = float(rng.uniform(0.5, 1.5))
        u = rng.uniform(-0.2, 0.2, 2) * lam
        f = orc.feq_product(rho, u[0], u[1], lam)
        kappa = orc.moment_matrix_geier(u[0], u[1], lam) @ f
        np.testing.assert_allclose(kappa, [rho, 0, 0, 2 * rho / 3, 0, 0, 0, 0, rho / 9],
                                   atol=1e-14)
        v = lam * np.stack([CX, CY])
        np.testing.assert_allclose(v @ f, rho * u, atol=1e-14)
        Pi = (v[:, None, :] * v[None, :, :] * f).sum(-1)
        np.testing.assert_allclose(Pi, rho * np.outer(u, u) + rho * lam * lam / 3 * np.eye(2),
                                   atol=1e-14)


def test_cascade_matrix_is_block_lower_triangular(orc):
    """C(u) = M_g(u) M(0)^T is lower triangular apart from the 2x2 block of the two
    diagonal second-order moments, which is what lets Appendix B solve it as a cascade."""
    M0 = orc.moment_matrix(0, 0, 1.0)
    rng = np.random.default_rng(2)
    for _ in range(10):
        a, b = rng.uniform(-0.2, 0.2, 2)
        X, Y = CX - a, CY - b
        Mg = np.stack([np.ones(9), X, Y, X * X, Y * Y, X * Y, X * Y * Y, X * X * Y, X * X * Y * Y])
        C = Mg @ M0.T
        upper = np.triu(C, 1)
        upper[3, 4] = 0.0
        assert np.abs(upper).max() < 1e-13


def test_cascaded_scheme_is_the_relative_velocity_scheme(orc):
    """Proposition of Section 1.3: Geier's cascade = the scheme with relative velocities in
    the (polgeier) basis shifted by u = q/rho, node by node."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        lam = float(rng.uniform(0.5, 2.0))
        f = orc.feq_product(float(rng.uniform(0.8, 1.2)), *(rng.uniform(-0.1, 0.1, 2) * lam),
                            lam) * (1 + 0.05 * rng.standard_normal(9))
        s = np.concatenate([[0, 0, 0], rng.uniform(0.5, 1.95, 6)])
        rho = f.sum()
        u = lam * np.array([CX @ f, CY @ f]) / rho
        a = orc.collide_node(orc.METHOD_GEIER, f, u[0], u[1], lam, s)
        b = orc.collide_node(orc.METHOD_CASCADED, f, 0.0, 0.0, lam, s)
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-14)


def test_cascaded_lattice_runs_agree(orc):
    d = inp.random_sine_flow(16, 12, seed=4)
    f0 = orc.init_equilibrium_product(d["rho"], d["ux"], d["uy"], 1.0)
    a = orc.run(f0, 1.0, SG, 1, 25, method=orc.METHOD_GEIER)
    b = orc.run(f0, 1.0, SG, 1, 25, method=orc.METHOD_CASCADED)
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-13)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_geier_invariants_and_fixed_point(orc, mode):
    rng = np.random.default_rng(5 + mode)
    for _ in range(30):
        f = orc.feq_product(float(rng.uniform(0.8, 1.2)), *rng.uniform(-0.1, 0.1, 2), 1.0)
        ut = rng.uniform(-0.2, 0.2, 2) if mode else (0.0, 0.0)
        np.testing.assert_allclose(orc.collide_node(orc.METHOD_GEIER, f, *ut, 1.0, SG), f,
                                   atol=1e-15)
        g = f * (1 + 0.05 * rng.standard_normal(9))
        h = orc.collide_node(orc.METHOD_GEIER, g, *ut, 1.0, SG)
        np.testing.assert_allclose(h.sum(), g.sum(), rtol=1e-14)
        np.testing.assert_allclose([CX @ h, CY @ h], [CX @ g, CY @ g], atol=1e-14)


@pytest.mark.slow
def test_geier_shear_viscosity(orc):
    """Second order (Section 2.3): nu = (1/s_nu - 1/2)/3 for the shear rate of X^2-Y^2
    and XY, whatever the basis of the higher moments."""
    L, s_nu = 64, 1.8
    d = inp.shear_wave(L, L, amp=1e-3)
    f = orc.init_equilibrium_product(d["rho"], d["ux"], d["uy"], 1.0)
    y = np.arange(L)
    sn = np.sin(2 * np.pi * y / L)
    f = orc.run(f, 1.0, SG, 1, 100, method=orc.METHOD_CASCADED, nthreads=8)
    ts, amps = [], []
    for t in range(100, 301, 20):
        ux = orc.moments(f, 1.0)[1]
        amps.append((ux.mean(1) @ sn) / (sn @ sn))
        ts.append(t)
        f = orc.run(f, 1.0, SG, 1, 20, t0=t, method=orc.METHOD_CASCADED, nthreads=8)
    k = 2 * np.pi / L
    nu = -np.polyfit(ts, np.log(amps), 1)[0] / (k * k)
    assert abs(nu / ((1 / s_nu - 0.5) / 3) - 1) < 0.01
