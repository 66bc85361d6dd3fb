"""The third-order u~-dependence study (Section 2.4) on the CUDA path: the complex rate of an
advected transverse wave, u~ = q/rho minus u~ = 0, against the FP64 oracle, and its k^3 / k^4
scaling. FP32 populations are stored relative to the background flow (lbmrv_set_reference)
so that the small wave is resolved."""
import numpy as np
import pytest

import lbm_inputs as inp

pytestmark = pytest.mark.gpu

S = [0, 0, 0, 1.4, 1.6, 1.6, 1.2, 1.2, 1.4]
U, A = 0.05, 1e-3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _gpu_rate(L, mode):
    import torch

    from paper_1312_3297_gb300 import D2Q9

    d = inp.shear_wave(L, 4, amp=A, background=(U, 0.0), axis="x")
    sim = D2Q9(L, 4, S, mode=mode, u_ref=(U, 0.0))
    sim.set_utilde(torch.stack([torch.ones(4, L), torch.zeros(4, L)]), U, 0.0)
    sim.init_equilibrium(*(torch.as_tensor(inp.to_f32_exact(d[k])) for k in ("rho", "ux", "uy")))
    e = np.exp(-2j * np.pi * np.arange(L) / L)
    sim.step(L)
    a1 = e @ sim.moments()[2].double().cpu().numpy().mean(0)
    sim.step(2 * L)
    a2 = e @ sim.moments()[2].double().cpu().numpy().mean(0)
    sim.close()
    return np.log(a2 / a1) / (2 * L)


def _oracle_rate(L, mode):
    import oracle

    d = inp.shear_wave(L, 4, amp=A, background=(U, 0.0), axis="x")
    f = oracle.init_equilibrium(*(inp.to_f32_exact(d[k]) for k in ("rho", "ux", "uy")), 1.0)
    e = np.exp(-2j * np.pi * np.arange(L) / L)
    ut0 = np.stack([np.ones((4, L)), np.zeros((4, L))])
    kw = dict(method=0, amp=U, period=0.0, ut0=ut0)
    f = oracle.run(f, 1.0, np.array(S, float), mode, L, **kw)
    a1 = e @ oracle.moments(f, 1.0)[2].mean(0)
    f = oracle.run(f, 1.0, np.array(S, float), mode, 2 * L, t0=L, **kw)
    a2 = e @ oracle.moments(f, 1.0)[2].mean(0)
    return np.log(a2 / a1) / (2 * L)


def test_third_order_difference_matches_oracle_and_scales():
    diffs = []
    for L in (16, 32, 64):
        g = _gpu_rate(L, "fluid") - _gpu_rate(L, "zero")
        o = _oracle_rate(L, 1) - _oracle_rate(L, 0)
        assert abs(g.imag - o.imag) <= 0.02 * abs(o.imag), (L, g, o)
        diffs.append(g)
    for a, b in zip(diffs, diffs[1:]):
        assert 7.0 < abs(a.imag / b.imag) < 9.0
