"""GPU parity of the fused D2Q9 relative-velocity step against the FP64 oracle.

All tests call the CUDA library through its C ABI (ctypes binding) and compare with the
oracle on identical seeded inputs (FP32-rounded once, shared by both sides). Tolerances
are those of the specification: FP32 populations give at most 1e-5 relative error in rho
and u (max|drho|/max|rho|, max_x|du|_2/max_x|u|_2); reduced-precision storage at most
2e-3 of max|u|.
"""
import numpy as np
import pytest

import lbm_inputs as inp
from pairs import (S_PAPER, W, f32_fields, gpu_run, oracle_run, reference_populations,
                   rel_errors)

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1312_3297_gb300 import binding

    binding.load()


def _check(nx, ny, mode, steps, fields, tol=TOL, **kw):
    okw = {k: v for k, v in kw.items() if k in ("lam", "ut0", "amp", "period")}
    f_g, m_g = gpu_run(nx, ny, S_PAPER if "s" not in kw else kw["s"], mode, steps, fields,
                       **{k: v for k, v in kw.items() if k != "s"})
    f_o, m_o = oracle_run(nx, ny, S_PAPER if "s" not in kw else kw["s"], mode, steps, fields,
                          **okw)
    e = rel_errors(f_g, m_g, f_o, m_o)
    assert max(e) <= tol, (nx, ny, mode, steps, e)
    return e, f_g


# --------------------------------------------------------------------- small lattice
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
@pytest.mark.parametrize("rho_ref", [0.0, 1.0])
def test_parity_64x64_100_steps(mode, rho_ref):
    """Small-lattice workload: 64^2, rho = 1 + 0.01 N, u = 0.05 (sin, sin) + 0.005 N,
    s = (0,0,0,1.4,1.9,1.9,1.2,1.2,1.4), 100 steps."""
    fields = f32_fields(inp.random_sine_flow(64, 64, seed=0))
    _check(64, 64, mode, 100, fields, rho_ref=rho_ref, amp=0.03, period=1000.0)


@pytest.mark.parametrize("nx,ny", [(37, 23), (96, 33), (130, 7), (64, 48), (260, 5)])
def test_parity_ragged_and_every_kernel_width(nx, ny):
    fields = f32_fields(inp.random_sine_flow(nx, ny, seed=1))
    widths = [w for w in (1, 2, 4) if nx % w == 0]
    states = []
    for w in widths:
        _, f = _check(nx, ny, "fluid", 30, fields, width=w)
        states.append(f)
    for f in states[1:]:
        np.testing.assert_array_equal(f, states[0])  # same arithmetic in every variant


@pytest.mark.parametrize("nx,ny", [(1, 1), (1, 9), (9, 1), (2, 2), (3, 3), (4, 5), (8, 1)])
def test_parity_degenerate_lattices(nx, ny):
    fields = f32_fields(inp.random_sine_flow(nx, ny, seed=2))
    for mode in ("zero", "fluid", "prescribed"):
        _check(nx, ny, mode, 7, fields, amp=0.05, period=9.0)


def test_parity_prescribed_caller_field():
    nx, ny = 48, 40
    fields = f32_fields(inp.random_sine_flow(nx, ny, seed=3))
    ut0 = inp.to_f32_exact(inp.prescribed_base_field(nx, ny, seed=4, smooth=False))
    for w in (1, 4):
        _check(nx, ny, "prescribed", 50, fields, ut0=ut0, amp=0.03, period=25.0, width=w)


@pytest.mark.parametrize("lam", [2.0, 0.5])
def test_parity_other_lambda(lam):
    d = inp.random_sine_flow(32, 24, seed=5)
    fields = f32_fields({"rho": d["rho"], "ux": lam * d["ux"], "uy": lam * d["uy"]})
    for mode in ("zero", "fluid", "prescribed"):
        _check(32, 24, mode, 40, fields, lam=lam, amp=0.03 * lam, period=30.0)


def test_init_equilibrium_matches_oracle():
    fields = f32_fields(inp.random_sine_flow(40, 30, seed=6))
    _check(40, 30, "fluid", 0, fields)


def test_equal_rates_modes_agree_on_gpu():
    s = [0, 0, 0] + [1.6] * 6
    fields = f32_fields(inp.random_sine_flow(64, 64, seed=7))
    outs = [gpu_run(64, 64, s, m, 50, fields, amp=0.08, period=40.0)[0]
            for m in ("zero", "fluid", "prescribed")]
    for f in outs[1:]:
        assert np.abs(f - outs[0]).max() <= 2e-6


def test_uniform_flow_is_steady_on_gpu():
    fields = f32_fields(inp.uniform(64, 32, 1.0, (0.07, -0.03)))
    for mode in ("zero", "fluid", "prescribed"):
        f, (r, ux, uy) = gpu_run(64, 32, S_PAPER, mode, 200, fields, amp=0.05, period=10.0)
        assert np.abs(ux - 0.07).max() < 1e-6 and np.abs(uy + 0.03).max() < 1e-6
        assert np.abs(r - 1.0).max() < 1e-6


# --------------------------------------------------------------------- diagnostics
def test_conserved_sums_and_nonfinite_detection():
    import torch

    from paper_1312_3297_gb300 import D2Q9, LbmrvError

    nx, ny = 96, 64
    rho, ux, uy = f32_fields(inp.random_sine_flow(nx, ny, seed=8))
    sim = D2Q9(nx, ny, S_PAPER, mode="fluid")
    sim.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    c0 = sim.conserved()
    assert c0[3] == 0
    np.testing.assert_allclose(c0[0], rho.sum(), rtol=1e-6)
    np.testing.assert_allclose(c0[1], (rho * ux).sum(), atol=1e-5)
    np.testing.assert_allclose(c0[2], (rho * uy).sum(), atol=1e-5)
    sim.step(200)
    c1 = sim.conserved()
    np.testing.assert_allclose(c1[0], c0[0], rtol=1e-7)
    np.testing.assert_allclose(c1[1:3], c0[1:3], atol=1e-4)
    g = sim.state()
    g[4, 10, 20] = float("nan")
    g[0, 3, 3] = float("inf")
    sim.set_state(g, sim.time)
    with pytest.raises(LbmrvError) as ei:
        sim.conserved()
    assert ei.value.status == -4
    assert sim.conserved(allow_nonfinite=True)[3] == 2
    sim.close()


def test_host_entry_points_match_device_ones():
    import torch

    from paper_1312_3297_gb300 import D2Q9

    nx, ny = 64, 40
    rho, ux, uy = f32_fields(inp.random_sine_flow(nx, ny, seed=9))
    a = D2Q9(nx, ny, S_PAPER, mode="fluid")
    a.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    b = D2Q9(nx, ny, S_PAPER, mode="fluid")
    rh = torch.as_tensor(rho, dtype=torch.float32).reshape(-1).pin_memory()
    uh = torch.as_tensor(np.stack([ux, uy]), dtype=torch.float32).reshape(2, -1).pin_memory()
    b.init_equilibrium_host(rh, uh)
    a.step(25)
    b.step(25)
    torch.testing.assert_close(a.state(), b.state(), rtol=0, atol=0)
    r1, u1x, u1y = a.moments()
    r2, u2 = b.moments_host()
    torch.testing.assert_close(r1.cpu(), r2, rtol=0, atol=0)
    torch.testing.assert_close(torch.stack([u1x, u1y]).cpu(), u2, rtol=0, atol=0)
    a.close()
    b.close()


def test_time_index_and_state_roundtrip():
    import torch

    from paper_1312_3297_gb300 import D2Q9

    nx, ny = 32, 32
    rho, ux, uy = f32_fields(inp.random_sine_flow(nx, ny, seed=10))
    a = D2Q9(nx, ny, S_PAPER, mode="prescribed")
    a.set_utilde(None, 0.04, 12.0)
    a.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    a.step(7)
    assert a.time == 7
    snap = a.state()
    a.step(9)
    ref = a.state()
    a.set_state(snap, 7)
    a.step(9)
    torch.testing.assert_close(a.state(), ref, rtol=0, atol=0)  # resume is exact
    a.close()


def test_zero_steps_is_a_no_op_and_negative_counts_fail():
    import torch

    from paper_1312_3297_gb300 import D2Q9
    from paper_1312_3297_gb300.binding import LbmrvError

    rho, ux, uy = f32_fields(inp.random_sine_flow(16, 8, seed=9))
    sim = D2Q9(16, 8, S_PAPER, mode="fluid")
    sim.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    snap = sim.state()
    sim.step(0)
    assert sim.time == 0
    torch.testing.assert_close(sim.state(), snap, rtol=0, atol=0)
    with pytest.raises(LbmrvError):
        sim.step(-1)
    assert sim.time == 0
    sim.close()


# --------------------------------------------------------------------- full size
def _window_oracle(fields_full, center, R, steps, s, mode, amp, period, nxg, nyg):
    """Oracle of the node `center` of a periodic nxg x nyg lattice after `steps` steps,
    on the (2R+1)^2 window around it (exact while R >= steps: information moves at most
    one node per step)."""
    import oracle

    cx, cy = center
    xs = (cx + np.arange(-R, R + 1)) % nxg
    ys = (cy + np.arange(-R, R + 1)) % nyg
    sub = [a[np.ix_(ys, xs)] for a in fields_full]
    ut0 = np.stack([np.cos(2 * np.pi * ys[:, None] / nyg) * np.ones((1, len(xs))),
                    np.sin(2 * np.pi * xs[None, :] / nxg) * np.ones((len(ys), 1))])
    f0 = oracle.init_equilibrium(*sub, 1.0)
    S = oracle.post_collision_state(f0, 1.0, np.asarray(s, float), mode, steps, ut0=ut0,
                                    amp=amp, period=period)
    return S[:, R, R]


@pytest.mark.parametrize("mode", ["prescribed", "zero", "fluid", "prescribed_stored"])
def test_full_size_4096_sampled_parity(mode):
    """Taylor-Green vortex u0 = 0.04 on 4096^2 in the benchmark's launch configurations:
    sampled nodes (corners, wrap edges, vector-pack and warp boundaries, interior) against
    the oracle on their dependency cone. prescribed_stored: the same u~(x, t), its base
    field (cos 2 pi y/L, sin 2 pi x/L) read from a device array instead of computed."""
    import torch

    from paper_1312_3297_gb300 import D2Q9

    L, steps = 4096, 6
    s = [0, 0, 0, 1.4, 1.8, 1.8, 1.2, 1.2, 1.4]
    d = inp.taylor_green(L, L, u0=0.04)
    fields = f32_fields(d)
    sim = D2Q9(L, L, s, mode="prescribed" if mode == "prescribed_stored" else mode)
    if mode == "prescribed":
        sim.set_utilde(None, 0.03, 1000.0)
    elif mode == "prescribed_stored":
        k = 2 * np.pi * np.arange(L) / L
        base = np.stack([np.repeat(np.cos(k)[:, None], L, axis=1),
                         np.repeat(np.sin(k)[None, :], L, axis=0)]).astype(np.float32)
        sim.set_utilde(torch.as_tensor(base), 0.03, 1000.0)
    sim.init_equilibrium(*(torch.as_tensor(a) for a in fields))
    sim.step(steps)
    g = sim.state()
    rng = np.random.default_rng(0)
    centers = [(0, 0), (L - 1, L - 1), (0, L - 1), (L - 1, 0), (3, 5), (4, 5), (127, 9),
               (128, 9), (511, 2000), (512, 2001), (L - 4, 17), (L - 5, 17)]
    centers += [tuple(int(v) for v in rng.integers(0, L, 2)) for _ in range(6)]
    mid = {"zero": 0, "fluid": 1, "prescribed": 2, "prescribed_stored": 2}[mode]
    fmax = 0.0
    errs = []
    for c in centers:
        ref = _window_oracle(fields, c, steps + 1, steps, s, mid, 0.03, 1000.0, L, L)
        got = g[:, c[1], c[0]].double().cpu().numpy() + reference_populations(
            sim.rho_ref, sim.u_ref)
        errs.append(np.abs(got - ref).max())
        fmax = max(fmax, np.abs(ref).max())
    assert max(errs) / fmax <= TOL, errs
    sim.close()


def test_full_size_4096_conservation_1000_steps():
    """Mass and momentum over 1000 steps of the 4096^2 Taylor-Green workload (prescribed
    u~, analytic field), accumulated in FP64 on the GPU."""
    import torch

    from paper_1312_3297_gb300 import D2Q9

    L = 4096
    s = [0, 0, 0, 1.4, 1.8, 1.8, 1.2, 1.2, 1.4]
    fields = f32_fields(inp.taylor_green(L, L, u0=0.04))
    sim = D2Q9(L, L, s, mode="prescribed")
    sim.set_utilde(None, 0.03, 1000.0)
    sim.init_equilibrium(*(torch.as_tensor(a) for a in fields))
    c0 = sim.conserved()
    sim.step(1000)
    c1 = sim.conserved()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-9
    assert abs(c1[1] - c0[1]) < 1e-6 * c0[0] * 0.04
    assert abs(c1[2] - c0[2]) < 1e-6 * c0[0] * 0.04
    # the vortex decays at the second-order viscosity (Section 2.3): e^{-2 nu k^2 t}
    r, ux, uy = sim.moments()
    nu = (1 / 1.8 - 0.5) / 3
    k = 2 * np.pi / L
    amp = float(torch.sqrt((ux.double() ** 2 + uy.double() ** 2).mean() * 2).item())
    np.testing.assert_allclose(amp / 0.04, np.exp(-2 * nu * k * k * 1000), rtol=1e-3)
    sim.close()


@pytest.mark.parametrize("storage", ["fp32"])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_parity_with_reference_velocity(storage, mode):
    """Storage relative to f_eq(rho_ref, U_ref) is only a change of variables: FP32 results
    match the oracle to the same tolerance, at every kernel width."""
    fields = f32_fields(inp.perturbed_uniform(64, 48, seed=3, U=(0.06, -0.03), drho=1e-2,
                                              du=1e-2))
    for w in (1, 4):
        _check(64, 48, mode, 60, fields, storage=storage, u_ref=(0.06, -0.03), width=w,
               amp=0.03, period=100.0)


def test_conserved_sums_with_reference_velocity():
    import torch

    from paper_1312_3297_gb300 import D2Q9

    nx, ny = 64, 32
    rho, ux, uy = f32_fields(inp.perturbed_uniform(nx, ny, seed=4))
    sim = D2Q9(nx, ny, S_PAPER, mode="fluid", u_ref=(0.05, 0.02))
    sim.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    c0 = sim.conserved()
    np.testing.assert_allclose(c0[0], rho.sum(), rtol=1e-6)
    np.testing.assert_allclose(c0[1], (rho * ux).sum(), rtol=1e-5)
    np.testing.assert_allclose(c0[2], (rho * uy).sum(), rtol=1e-5)
    sim.close()


@pytest.mark.parametrize("lattice", ["d2q9", "cascaded", "d3q19"])
def test_automatic_reference_is_the_mean_flow(lattice):
    """By default each init_equilibrium stores deviations from f_eq(rho_ref, U) with U the
    mean flow sum(rho u) / sum(rho) of its fields (FP64 on the device, against numpy here);
    a fixed reference turns that off and the automatic choice can be turned back on. The
    mean flow is conserved, so the stored state's momentum over its mass stays U."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, D2Q9Cascaded, D3Q19

    if lattice == "d3q19":
        d = inp.random_flow_3d(24, 10, 6, seed=5)
        rho = inp.to_f32_exact(d["rho"])
        u = inp.to_f32_exact(d["u"] + np.array([0.03, -0.02, 0.01])[:, None, None, None])
        sim = D3Q19(24, 10, 6, [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3,
                    mode="fluid", storage="bf16")
        comps = list(u)
    else:
        rho, ux, uy = f32_fields(inp.perturbed_uniform(40, 24, seed=6, U=(0.05, 0.02)))
        cls = D2Q9Cascaded if lattice == "cascaded" else D2Q9
        s = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]
        sim = cls(40, 24, s, mode="fluid", storage="fp16")
        comps = [ux, uy]
    want = np.array([(rho * c).sum() for c in comps]) / rho.sum()
    assert B_ref_auto(sim)
    sim.init_equilibrium(torch.as_tensor(rho), *(torch.as_tensor(c) for c in comps))
    np.testing.assert_allclose(sim.u_ref, want, rtol=1e-12, atol=1e-15)
    sim.step(7)
    c = sim.conserved3()
    np.testing.assert_allclose(np.array(c[1:1 + len(comps)]) / c[0], want, rtol=2e-3,
                               atol=1e-6)
    sim.set_reference(sim.rho_ref, [0.0] * len(comps))
    assert not B_ref_auto(sim)
    sim.init_equilibrium(torch.as_tensor(rho), *(torch.as_tensor(c) for c in comps))
    assert tuple(sim.u_ref) == (0.0,) * len(comps)
    sim.set_reference_auto()
    assert B_ref_auto(sim)
    sim.init_equilibrium(torch.as_tensor(rho), *(torch.as_tensor(c) for c in comps))
    np.testing.assert_allclose(sim.u_ref, want, rtol=1e-12, atol=1e-15)
    sim.close()


def B_ref_auto(sim):
    from paper_1312_3297_gb300 import binding as B

    return B.lbmrv_get_reference(sim.h)[2]


def test_automatic_reference_rejects_nonfinite_fields():
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B

    rho, ux, uy = f32_fields(inp.random_sine_flow(16, 8, seed=1))
    ux = ux.copy()
    ux[3, 4] = np.nan
    sim = D2Q9(16, 8, S_PAPER, mode="fluid")
    with pytest.raises(B.LbmrvError) as ei:
        sim.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    assert ei.value.status == B.LBMRV_E_NONFINITE
    sim.close()


def test_two_handles_on_two_streams_match_single_stream_runs():
    """Handles are independent: a D2Q9 lattice (FP32, prescribed u~) and a D3Q19 lattice
    (FP16, u~ = q/rho) stepped interleaved on two non-default streams end bit for bit where
    each ends alone on the default stream."""
    import torch

    from paper_1312_3297_gb300 import D3Q19, D2Q9

    rho, ux, uy = f32_fields(inp.random_sine_flow(96, 40, seed=21))
    d3 = inp.random_flow_3d(48, 12, 10, seed=22)
    r3, u3 = inp.to_f32_exact(d3["rho"]), inp.to_f32_exact(d3["u"])
    s3 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3

    def make(stream=None):
        a = D2Q9(96, 40, S_PAPER, mode="prescribed", stream=stream)
        a.set_utilde(None, 0.03, 100.0)
        a.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
        return a

    def make3(stream=None):
        b = D3Q19(48, 12, 10, s3, mode="fluid", storage="fp16", stream=stream)
        b.init_equilibrium(torch.as_tensor(r3), *(torch.as_tensor(c) for c in u3))
        return b

    ref_a, ref_b = make(), make3()
    ref_a.step(60)
    ref_b.step(60)
    want_a, want_b = ref_a.state(), ref_b.state()
    ref_a.close()
    ref_b.close()
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    a, b = make(s1), make3(s2)
    for _ in range(6):
        a.step(10)
        b.step(10)
    got_a, got_b = a.state(), b.state()
    torch.testing.assert_close(got_a, want_a, rtol=0, atol=0)
    torch.testing.assert_close(got_b, want_b, rtol=0, atol=0)
    a.close()
    b.close()
