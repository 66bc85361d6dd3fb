"""Pins of the FP64 PyTorch statement of the scheme (the reference for gradients).

Its forward pass is an independent implementation of the definition of Section 1.2
(torch.linalg.solve per node, torch.roll transport) and must agree with the C oracle's
definition stepper to rounding. Its gradients are pinned by central finite differences in
FP64 (not by re-running the same reverse pass)."""
import numpy as np
import pytest
import torch

import lbm_inputs as inp
from oracle import torch_ref as tr

S_BASE = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_forward_matches_c_definition_oracle(orc, mode):
    nx, ny, steps = 12, 10, 15
    d = inp.noisy_shear_wave(nx, ny, seed=1)
    u0 = np.stack([d["ux"], d["uy"]])
    ut0 = tr.analytic_base_field(nx, ny)
    f0 = orc.init_equilibrium(d["rho"], d["ux"], d["uy"], 1.0)
    fC = orc.run(f0, 1.0, np.array(S_BASE, float), mode, steps, amp=0.03, period=40.0)
    with torch.no_grad():
        fT = tr.final_state(torch.tensor(d["rho"]), torch.tensor(u0), 1.0,
                            tr.rates(S_BASE, torch.tensor(1.9, dtype=torch.float64)), mode,
                            steps, ut0, 0.03, 40.0)
    np.testing.assert_allclose(fT.numpy(), fC, rtol=0, atol=1e-14)


def _fd(fun, x, eps):
    return (fun(x + eps) - fun(x - eps)) / (2 * eps)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_gradients_match_central_differences(mode):
    nx, ny, steps = 10, 8, 12
    d = inp.noisy_shear_wave(nx, ny, seed=2, amp=0.05, sigma=0.01)
    u0 = np.stack([d["ux"], d["uy"]])
    ut0 = tr.analytic_base_field(nx, ny)
    args = dict(ut0=ut0, period=30.0)
    L, gu, gs, ga = tr.loss_and_grads(d["rho"], u0, 1.0, S_BASE, 1.9, mode, steps,
                                      amp=0.04, **args)
    fs = _fd(lambda v: tr.loss_only(d["rho"], u0, 1.0, S_BASE, v, mode, steps, amp=0.04,
                                    **args), 1.9, 1e-5)
    assert abs(gs - fs) <= 1e-7 * abs(fs) + 1e-12
    if mode == 2:
        fa = _fd(lambda v: tr.loss_only(d["rho"], u0, 1.0, S_BASE, 1.9, mode, steps, amp=v,
                                        **args), 0.04, 1e-5)
        assert abs(ga - fa) <= 1e-6 * abs(fa) + 1e-12
    else:
        assert ga == 0.0
    rng = np.random.default_rng(3)
    for _ in range(2):
        v = rng.standard_normal(u0.shape)
        fd = _fd(lambda e: tr.loss_only(d["rho"], u0 + e * v, 1.0, S_BASE, 1.9, mode, steps,
                                        amp=0.04, **args), 0.0, 1e-6)
        np.testing.assert_allclose((gu * v).sum(), fd, rtol=1e-6)
