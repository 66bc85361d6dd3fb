"""Third-order dependence on the relative velocity (Section 2.4, third-order equivalent
equations): up to second order the scheme does not depend on u~ (same viscosity as MRT),
and the first u~-dependent term is of order Delta^2 in the momentum equation.

Numerical study with the FP64 oracle: a small transverse wave u_y = A sin(k x) advected by
a uniform flow U_x, followed by its complex rate lambda = d/dt log(amplitude). The
difference between the u~ = q/rho (or u~ = U) scheme and MRT (u~ = 0) must vanish faster
than the viscous rate as k -> 0: its dispersive (imaginary) part scales like k^3 and its
dissipative (real) part like k^4, so each doubling of the wavelength divides them by about
8 and 16. There is no closed form to compare the constants with (informative only)."""
import numpy as np
import pytest

import lbm_inputs as inp

S = np.array([0, 0, 0, 1.4, 1.6, 1.6, 1.2, 1.2, 1.4])


def wave_rate(orc, L, mode, U=0.05, A=1e-4, s=S):
    d = inp.shear_wave(L, 4, amp=A, background=(U, 0.0), axis="x")
    f = orc.init_equilibrium(d["rho"], d["ux"], d["uy"], 1.0)
    e = np.exp(-2j * np.pi * np.arange(L) / L)
    ut0 = np.stack([np.ones((4, L)), np.zeros((4, L))])
    kw = dict(method=1, amp=U, period=0.0, ut0=ut0, nthreads=8)
    t1, t2 = L, 3 * L
    f = orc.run(f, 1.0, s, mode, t1, **kw)
    a1 = e @ orc.moments(f, 1.0)[2].mean(0)
    f = orc.run(f, 1.0, s, mode, t2 - t1, t0=t1, **kw)
    a2 = e @ orc.moments(f, 1.0)[2].mean(0)
    return np.log(a2 / a1) / (t2 - t1)


@pytest.mark.slow
def test_relative_velocity_enters_at_third_order(orc):
    Ls = (16, 32, 64)
    diffs = []
    for L in Ls:
        r0 = wave_rate(orc, L, 0)
        k = 2 * np.pi / L
        nu = (1 / 1.6 - 0.5) / 3
        assert abs(-r0.real / (nu * k * k) - 1) < 0.01  # second order: MRT viscosity
        d_fluid = wave_rate(orc, L, 1) - r0
        d_presc = wave_rate(orc, L, 2) - r0
        np.testing.assert_allclose(d_fluid, d_presc, rtol=1e-3)  # q/rho ~ U for a small wave
        assert abs(d_fluid) < 1e-2 * nu * k * k
        diffs.append(d_fluid)
    for a, b in zip(diffs, diffs[1:]):
        assert 7.0 < abs(a.imag / b.imag) < 9.0   # ~ k^3
        assert 13.0 < abs(a.real / b.real) < 19.0  # ~ k^4


def test_no_dependence_at_rest_or_with_equal_rates(orc):
    base = wave_rate(orc, 32, 1) - wave_rate(orc, 32, 0)
    rest = wave_rate(orc, 32, 1, U=0.0) - wave_rate(orc, 32, 0, U=0.0)
    assert abs(rest) < 1e-3 * abs(base)
    s_eq = np.array([0, 0, 0] + [1.6] * 6)
    eq = wave_rate(orc, 32, 1, s=s_eq) - wave_rate(orc, 32, 0, s=s_eq)
    assert abs(eq) < 1e-12
