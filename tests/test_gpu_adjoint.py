"""GPU discrete adjoint against the FP64 references.

The CUDA reverse sweep (lbmrv_forward_checkpointed + lbmrv_adjoint, through the C ABI)
gives the gradient of the final kinetic energy L = 1/2 sum |q|^2/rho with respect to the
initial velocity field, the shear rate s_nu and the amplitude A of a prescribed u~. It is
compared with reverse-mode differentiation of the FP64 PyTorch statement of the scheme and
with central differences (eps = 1e-4) of the FP64 C oracle; the bar is 1e-4 relative error.
"""
import json
import os

import numpy as np
import pytest

import lbm_inputs as inp
from pairs import f32_fields, gpu_gradients, oracle_kinetic_energy

pytestmark = pytest.mark.gpu

S = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_adjoint_matches_fp64_reverse_mode(mode):
    from oracle import torch_ref as tr

    nx, ny, steps, seg = 48, 40, 40, 7
    fields = f32_fields(inp.noisy_shear_wave(nx, ny, seed=0))
    rho, ux, uy = fields
    u0 = np.stack([ux, uy])
    amp, period = 0.03, 50.0
    L, du0, ds, da, _ = gpu_gradients(nx, ny, S, mode, steps, seg, fields, amp, period)
    mid = {"zero": 0, "fluid": 1, "prescribed": 2}[mode]
    Lr, gur, gsr, gar = tr.loss_and_grads(rho, u0, 1.0, S, 1.9, mid, steps,
                                          tr.analytic_base_field(nx, ny), amp, period)
    assert abs(L - Lr) <= 1e-6 * abs(Lr)
    assert _rel(du0, gur) <= TOL
    assert abs(ds[4] + ds[5] - gsr) <= TOL * abs(gsr)
    if mode == "prescribed":
        assert abs(da - gar) <= TOL * abs(gar)
    else:
        assert da == 0.0


def test_adjoint_64x64_shear_wave_against_reverse_mode():
    """The 64^2 check of the adjoint workload: noisy shear wave u_x = 0.05 sin 2pi y/L +
    N(0, 0.01), prescribed u~ with A = 0.03, P = 1000."""
    from oracle import torch_ref as tr

    n, steps, seg = 64, 64, 8
    fields = f32_fields(inp.noisy_shear_wave(n, n, seed=0))
    rho, ux, uy = fields
    L, du0, ds, da, _ = gpu_gradients(n, n, S, "prescribed", steps, seg, fields, 0.03, 1000.0)
    Lr, gur, gsr, gar = tr.loss_and_grads(rho, np.stack([ux, uy]), 1.0, S, 1.9, 2, steps,
                                          tr.analytic_base_field(n, n), 0.03, 1000.0)
    assert _rel(du0, gur) <= TOL
    assert abs(ds[4] + ds[5] - gsr) <= TOL * abs(gsr)
    assert abs(da - gar) <= TOL * abs(gar)


def test_adjoint_matches_central_differences_of_the_oracle():
    """Central differences (eps = 1e-4) of the FP64 oracle's kinetic energy, 128^2 x 200
    steps, prescribed u~: s_nu, A, and two random directions of the initial velocity."""
    n, steps, seg = 128, 200, 15
    fields = f32_fields(inp.noisy_shear_wave(n, n, seed=1))
    rho, ux, uy = fields
    u0 = np.stack([ux, uy])
    amp, period = 0.03, 150.0
    base = inp.to_f32_exact(np.stack([
        np.cos(2 * np.pi * np.arange(n)[:, None] / n) * np.ones((1, n)),
        np.sin(2 * np.pi * np.arange(n)[None, :] / n) * np.ones((n, 1))]))
    L, du0, ds, da, _ = gpu_gradients(n, n, S, "prescribed", steps, seg, fields, amp, period)
    eps = 1e-4

    def ke(s_nu=1.9, a=amp, u=u0):
        s = list(S)
        s[4] = s[5] = s_nu
        return oracle_kinetic_energy(rho, u, s, "prescribed", steps, a, period, base)

    fd_s = (ke(s_nu=1.9 + eps) - ke(s_nu=1.9 - eps)) / (2 * eps)
    fd_a = (ke(a=amp + eps) - ke(a=amp - eps)) / (2 * eps)
    assert abs(ds[4] + ds[5] - fd_s) <= TOL * abs(fd_s), (ds[4] + ds[5], fd_s)
    assert abs(da - fd_a) <= TOL * abs(fd_a), (da, fd_a)
    rng = np.random.default_rng(5)
    for _ in range(2):
        v = rng.standard_normal(u0.shape)
        v /= np.abs(v).max()
        fd_v = (ke(u=u0 + eps * v) - ke(u=u0 - eps * v)) / (2 * eps)
        g_v = float((du0 * v).sum())
        assert abs(g_v - fd_v) <= TOL * abs(fd_v), (g_v, fd_v)


def test_field_gradient_is_consistent_with_amplitude_gradient():
    """L depends on A and u~0 only through A u~0(x), so A dL/dA = sum_x u~0 . dL/du~0."""
    nx, ny, steps = 64, 48, 60
    fields = f32_fields(inp.noisy_shear_wave(nx, ny, seed=3))
    ut0 = inp.to_f32_exact(inp.prescribed_base_field(nx, ny, seed=2, smooth=False))
    amp = 0.02
    for field in (None, ut0):
        L, du0, ds, da, dut = gpu_gradients(nx, ny, S, "prescribed", steps, 10, fields, amp,
                                            40.0, ut0=field, field_grad=True)
        base = field if field is not None else np.stack([
            np.cos(2 * np.pi * np.arange(ny)[:, None] / ny) * np.ones((1, nx)),
            np.sin(2 * np.pi * np.arange(nx)[None, :] / nx) * np.ones((ny, 1))])
        np.testing.assert_allclose(amp * da, (base * dut).sum(), rtol=1e-4)


def test_checkpoint_interval_does_not_change_the_gradient():
    nx, ny, steps = 96, 64, 90
    fields = f32_fields(inp.noisy_shear_wave(nx, ny, seed=4))
    outs = [gpu_gradients(nx, ny, S, "fluid", steps, seg, fields) for seg in (1, 9, 13, 90)]
    for o in outs[1:]:
        np.testing.assert_array_equal(o[1], outs[0][1])
        assert o[2] == outs[0][2]


def test_rollout_autograd_function_matches_direct_calls():
    import torch

    from paper_1312_3297_gb300 import D2Q9
    from paper_1312_3297_gb300.autograd import Rollout

    nx, ny, steps = 64, 64, 50
    fields = f32_fields(inp.noisy_shear_wave(nx, ny, seed=6))
    rho, ux, uy = fields
    L, du0, ds, da, _ = gpu_gradients(nx, ny, S, "prescribed", steps, 7, fields, 0.03, 1000.0)
    sim = D2Q9(nx, ny, S, mode="prescribed")
    sim.set_utilde(None, 0.03, 1000.0)
    u0 = torch.tensor(np.stack([ux, uy]), dtype=torch.float32, device="cuda", requires_grad=True)
    s_nu = torch.tensor(1.9, dtype=torch.float64, requires_grad=True)
    amp = torch.tensor(0.03, dtype=torch.float64, requires_grad=True)
    r, u = Rollout.apply(u0, s_nu, amp, sim, steps, 7,
                         torch.as_tensor(rho, dtype=torch.float32, device="cuda"))
    loss = 0.5 * (r.double() * (u.double() ** 2).sum(0)).sum()
    loss.backward()
    np.testing.assert_allclose(loss.item(), L, rtol=1e-6)
    np.testing.assert_allclose(u0.grad.double().cpu().numpy(), du0, rtol=2e-5,
                               atol=2e-5 * np.abs(du0).max())
    np.testing.assert_allclose(s_nu.grad.item(), ds[4] + ds[5], rtol=2e-5)
    np.testing.assert_allclose(amp.grad.item(), da, rtol=2e-5)
    sim.close()


def test_adjoint_full_size_1024_2000_steps():
    """The adjoint workload at full size: 1024^2, 2000 steps, sqrt(N) = 45 checkpoints.
    The gradient does not depend on the checkpoint interval (bitwise), is finite, and the
    identity A dL/dA = sum u~0 . dL/du~0 holds."""
    n, steps = 1024, 2000
    fields = f32_fields(inp.noisy_shear_wave(n, n, seed=0))
    a = gpu_gradients(n, n, S, "prescribed", steps, 45, fields, 0.03, 1000.0, field_grad=True)
    b = gpu_gradients(n, n, S, "prescribed", steps, 400, fields, 0.03, 1000.0)
    np.testing.assert_array_equal(a[1], b[1])
    assert a[2] == b[2] and a[3] == b[3]
    assert np.isfinite(a[1]).all() and np.isfinite(a[2]).all()
    base = np.stack([np.cos(2 * np.pi * np.arange(n)[:, None] / n) * np.ones((1, n)),
                     np.sin(2 * np.pi * np.arange(n)[None, :] / n) * np.ones((n, 1))])
    np.testing.assert_allclose(0.03 * a[3], (base * a[4]).sum(), rtol=1e-4)


def test_adjoint_with_reference_velocity_storage():
    """A reference velocity in the stored state changes no gradient."""
    nx, ny, steps = 48, 40, 30
    fields = f32_fields(inp.noisy_shear_wave(nx, ny, seed=8))
    a = gpu_gradients(nx, ny, S, "fluid", steps, 6, fields)
    b = gpu_gradients(nx, ny, S, "fluid", steps, 6, fields, u_ref=(0.04, -0.01))
    assert abs(a[0] - b[0]) <= 1e-6 * abs(a[0])
    assert _rel(b[1], a[1]) <= 1e-4
    assert abs(b[2][4] + b[2][5] - a[2][4] - a[2][5]) <= 1e-4 * abs(a[2][4] + a[2][5])


@pytest.mark.parametrize("mode", ["fluid", "prescribed"])
def test_velocity_probe_misfit_through_autograd(mode):
    """A velocity-probe misfit L = 1/2 sum_p |u(x_p) - u_p|^2 of the final state, through
    the torch.autograd.Function: gradients with respect to u0, s_nu and the amplitude A of
    the prescribed u~ against FP64 reverse mode of the torch statement of the scheme."""
    import torch

    import oracle.torch_ref as tr
    from paper_1312_3297_gb300 import D2Q9
    from paper_1312_3297_gb300.autograd import Rollout

    nx, ny, steps = 48, 40, 40
    rho, ux, uy = f32_fields(inp.noisy_shear_wave(nx, ny, seed=8))
    rng = np.random.default_rng(9)
    px, py = rng.integers(0, nx, 12), rng.integers(0, ny, 12)
    target = 0.02 * rng.standard_normal((2, 12))
    mid = {"fluid": 1, "prescribed": 2}[mode]

    # FP64 reference
    u0r = torch.tensor(np.stack([ux, uy]), dtype=torch.float64, requires_grad=True)
    snr = torch.tensor(1.9, dtype=torch.float64, requires_grad=True)
    ampr = torch.tensor(0.03, dtype=torch.float64, requires_grad=True)
    f = tr.final_state(torch.as_tensor(rho, dtype=torch.float64), u0r, 1.0, tr.rates(S, snr),
                       mid, steps, tr.analytic_base_field(nx, ny), ampr, 1000.0)
    r_, qx, qy = tr.moments(f, 1.0)
    u_probe = torch.stack([qx / r_, qy / r_])[:, py, px]
    Lr = 0.5 * ((u_probe - torch.as_tensor(target)) ** 2).sum()
    gu, gs, ga = torch.autograd.grad(Lr, (u0r, snr, ampr), allow_unused=True)

    # GPU through the autograd.Function
    sim = D2Q9(nx, ny, S, mode=mode)
    sim.set_utilde(None, 0.03, 1000.0)
    u0 = torch.tensor(np.stack([ux, uy]), dtype=torch.float32, device="cuda", requires_grad=True)
    s_nu = torch.tensor(1.9, dtype=torch.float64, requires_grad=True)
    amp = torch.tensor(0.03, dtype=torch.float64, requires_grad=True)
    r, u = Rollout.apply(u0, s_nu, amp, sim, steps, 7,
                         torch.as_tensor(rho, dtype=torch.float32, device="cuda"))
    tgt = torch.as_tensor(target, dtype=torch.float64, device="cuda")
    L = 0.5 * ((u.double()[:, py, px] - tgt) ** 2).sum()
    L.backward()
    sim.close()
    np.testing.assert_allclose(L.item(), Lr.item(), rtol=1e-5)
    assert _rel(u0.grad.double().cpu().numpy(), gu.numpy()) <= TOL
    assert abs(s_nu.grad.item() - gs.item()) <= TOL * abs(gs.item())
    if mode == "prescribed":
        assert abs(amp.grad.item() - ga.item()) <= TOL * abs(ga.item())


def test_unaligned_gradient_buffers():
    """The C entry point rejects dL/dS buffers that are not 16-byte aligned before queuing
    any work; the Python wrapper copies a misaligned dL/dS view into aligned storage and
    gives the gradient of the aligned call."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B

    nx, ny, steps = 64, 32, 12
    d = inp.noisy_shear_wave(nx, ny, seed=6)
    sim = D2Q9(nx, ny, S, mode="fluid")
    sim.init_equilibrium(*(torch.as_tensor(d[k], dtype=torch.float32) for k in ("rho", "ux", "uy")))
    ws = sim.adjoint_workspace(steps, 4)
    sim.forward_checkpointed(steps, 4, ws)
    _, dlds = sim.kinetic_energy(grad=True)
    n9 = 9 * nx * ny
    big = torch.zeros(n9 + 4, dtype=torch.float32, device="cuda")
    big[1:1 + n9] = dlds.reshape(-1)
    view = big[1:1 + n9].view(9, ny, nx)  # contiguous, 4 bytes past a 16-byte boundary
    out = torch.empty_like(dlds)
    with pytest.raises(B.LbmrvError) as ei:
        B.lbmrv_adjoint(sim.h, steps, 4, ws, ws.numel(), view.data_ptr(), out)
    assert ei.value.status == B.LBMRV_E_INVAL and "aligned" in str(ei.value)
    with pytest.raises(B.LbmrvError):
        B.lbmrv_adjoint(sim.h, steps, 4, ws, ws.numel(), dlds, big[1:1 + n9].data_ptr())
    d_ok = sim.adjoint(steps, 4, ws, dlds)
    d_view = sim.adjoint(steps, 4, ws, view)
    np.testing.assert_array_equal(d_view[0].cpu().numpy(), d_ok[0].cpu().numpy())
    assert d_view[1] == d_ok[1]
    sim.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_adjoint_widths_agree(storage, mode):
    """The reverse step on 4- and 2-node packs (node pairs by packed FP32 instructions) and on
    one node per thread (the scalar form of the same arithmetic). With u~ = 0 or q/rho the
    two packed widths give the same bits of dL/du0 (the forward kernels of those widths
    store the same bits too); with the prescribed field the forward kernels of different
    widths may round the field's product differently. Everything else agrees to rounding
    (1e-6), including the parameter gradients, which are sums taken in a width-dependent
    order. A row of 72 nodes leaves part of a warp idle at 4-node packs."""
    nx, ny, steps = 72, 20, 24
    fields = f32_fields(inp.noisy_shear_wave(nx, ny, seed=8))
    outs = {w: gpu_gradients(nx, ny, S, mode, steps, 5, fields, 0.03, 40.0, storage=storage,
                             width=w) for w in (4, 2, 1)}
    if mode != "prescribed":
        np.testing.assert_array_equal(outs[2][1], outs[4][1])
    for w in (2, 1):
        assert _rel(outs[w][1], outs[4][1]) <= 1e-6
        np.testing.assert_allclose(outs[w][2], outs[4][2], rtol=1e-6, atol=1e-9)
        assert abs(outs[w][3] - outs[4][3]) <= 1e-6 * max(abs(outs[4][3]), 1e-12)


def _report(name, vals):
    out = os.environ.get("LBMRV_PRECISION_REPORT")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps(dict(case=name, **vals)) + "\n")


# Relative gradient errors against FP64 reverse mode measured with 16-bit storage (64^2
# noisy shear wave, prescribed u~, kinetic-energy loss, 64 steps); each bound is the
# measured error with a margin, so that a change that makes it worse is caught.
GRAD16_BOUNDS = {"fp16": dict(du0=3e-3, s_nu=3e-3, amp=3e-3),
                 "bf16": dict(du0=3e-2, s_nu=3e-2, amp=3e-2)}


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_16bit_storage_gradients_against_fp64_reverse_mode(storage):
    """The adjoint workload's shape at 64^2 with the states stored in FP16 / BF16 (the
    checkpoints and the recomputed states are 16-bit; the adjoint vectors FP32): the
    gradients with respect to u0, s_nu and A against FP64 reverse mode of the FP64
    statement of the scheme. The errors are those of the 16-bit forward trajectory."""
    from oracle import torch_ref as tr

    n, steps, seg = 64, 64, 8
    fields = f32_fields(inp.noisy_shear_wave(n, n, seed=0))
    rho, ux, uy = fields
    L, du0, ds, da, _ = gpu_gradients(n, n, S, "prescribed", steps, seg, fields, 0.03, 1000.0,
                                      storage=storage)
    Lr, gur, gsr, gar = tr.loss_and_grads(rho, np.stack([ux, uy]), 1.0, S, 1.9, 2, steps,
                                          tr.analytic_base_field(n, n), 0.03, 1000.0)
    errs = dict(loss=abs(L - Lr) / abs(Lr), du0=_rel(du0, gur),
                s_nu=abs(ds[4] + ds[5] - gsr) / abs(gsr), amp=abs(da - gar) / abs(gar))
    _report(f"adjoint-{storage}-64x64-64", errs)
    for k, bound in GRAD16_BOUNDS[storage].items():
        assert errs[k] <= bound, (k, errs)
