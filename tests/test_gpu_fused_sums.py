"""lbmrv_step_conserved: the FP64 conserved sums (relation (rhoq) summed over the lattice)
taken inside the last step's kernel, against the same steps followed by the separate
reduction pass over the stored state."""
import numpy as np
import pytest

import lbm_inputs as inp

pytestmark = pytest.mark.gpu

S = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pair(cls, shape, mode, storage, width, seed=0, **kw):
    import torch

    nx, ny = shape
    d = inp.random_sine_flow(nx, ny, seed=seed)
    sims = []
    for _ in range(2):
        sim = cls(nx, ny, S, mode=mode, storage=storage, **kw)
        if mode == "prescribed":
            sim.set_utilde(None, 0.03, 40.0)
        if width:
            sim.set_kernel_width(width)
        sim.init_equilibrium(*(torch.as_tensor(d[k], dtype=torch.float32)
                               for k in ("rho", "ux", "uy")))
        sims.append(sim)
    return sims


def _compare(fused_sim, plain_sim, steps, n):
    got = fused_sim.step_conserved(steps)
    plain_sim.step(steps)
    ref = plain_sim.conserved3()
    import torch

    fa, pa = fused_sim.state(), plain_sim.state()  # bitwise (any storage type)
    assert torch.equal(fa.view(torch.uint8), pa.view(torch.uint8))
    assert fused_sim.time == plain_sim.time == steps
    np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=1e-9 * n)
    assert got[4] == ref[4] == 0.0
    return got


@pytest.mark.parametrize("storage,widths", [("fp32", (4, 2)), ("fp16", (8, 4, 2)),
                                            ("bf16", (8, 4, 2))])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_fused_sums_equal_separate_pass(storage, widths, mode):
    """264 x 37: a ragged last block of packs, rows spread over blocks; 7 steps."""
    from paper_1312_3297_gb300 import D2Q9

    shape = (264, 37)
    for w in widths:
        a, b = _pair(D2Q9, shape, mode, storage, w)
        _compare(a, b, 7, shape[0] * shape[1])
        a.close()
        b.close()


def test_fused_sums_cascaded_basis_and_reference_velocity():
    from paper_1312_3297_gb300 import D2Q9, D2Q9Cascaded

    shape = (128, 40)
    a, b = _pair(D2Q9Cascaded, shape, "fluid", "fp16", 8)
    _compare(a, b, 5, shape[0] * shape[1])
    a, b = _pair(D2Q9, shape, "fluid", "bf16", 8, u_ref=(0.05, 0.02))
    _compare(a, b, 5, shape[0] * shape[1])


def test_fused_sums_full_size_4096_fp32():
    """The 4096^2 Taylor-Green workload the benchmark times: 32,768 block partials."""
    import torch

    from paper_1312_3297_gb300 import D2Q9

    L = 4096
    d = inp.taylor_green(L, L, u0=0.04)
    fields = [torch.as_tensor(d[k], dtype=torch.float32) for k in ("rho", "ux", "uy")]
    sims = []
    for _ in range(2):
        sim = D2Q9(L, L, S, mode="prescribed")
        sim.set_utilde(None, 0.03, 1000.0)
        sim.init_equilibrium(*fields)
        sims.append(sim)
    got = _compare(sims[0], sims[1], 3, L * L)
    np.testing.assert_allclose(got[0], float(d["rho"].astype(np.float32).astype(np.float64).sum()),
                               rtol=1e-9)
    for sim in sims:
        sim.close()


def test_fallback_scalar_kernel_matches():
    """The scalar kernel (width 1) has no fused form: the step, then the separate pass."""
    from paper_1312_3297_gb300 import D2Q9

    a, b = _pair(D2Q9, (37, 11), "fluid", "fp32", 1)
    got = a.step_conserved(4)
    b.step(4)
    assert got == b.conserved3()


S19 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3


def _pair3(shape, mode, storage, width, seed=2):
    import torch

    from paper_1312_3297_gb300 import D3Q19

    nx, ny, nz = shape
    d = inp.random_flow_3d(nx, ny, nz, seed=seed)
    ut0 = torch.as_tensor(np.random.default_rng(seed + 7).standard_normal((3, nz, ny, nx)),
                          dtype=torch.float32)
    sims = []
    for _ in range(2):
        sim = D3Q19(nx, ny, nz, S19, mode=mode, storage=storage)
        if mode == "prescribed":
            sim.set_utilde(ut0, 0.03, 40.0)
        sim.set_kernel_width(width)
        sim.init_equilibrium(torch.as_tensor(d["rho"], dtype=torch.float32),
                             *(torch.as_tensor(c, dtype=torch.float32) for c in d["u"]))
        sims.append(sim)
    return sims


@pytest.mark.parametrize("storage,width,shape", [
    ("fp32", 4, (16, 12, 8)), ("fp32", 4, (36, 5, 3)),
    ("fp16", 8, (16, 12, 8)), ("bf16", 8, (16, 12, 8)),
    ("fp16", 8, (264, 3, 2)), ("bf16", 8, (552, 2, 3))])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_fused_sums_d3q19(storage, width, shape, mode):
    """D3Q19 kernels with the sums fused in (FP32 4-node packs, the staged 16-bit kernel,
    including rows of several segments): the same state bit for bit and the same sums to
    FP64 rounding as the step followed by the separate pass."""
    import torch

    a, b = _pair3(shape, mode, storage, width)
    n = shape[0] * shape[1] * shape[2]
    got = a.step_conserved(5)
    b.step(5)
    ref = b.conserved3()
    assert torch.equal(a.state().view(torch.uint8), b.state().view(torch.uint8))
    np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=1e-9 * n)
    assert got[4] == ref[4] == 0.0


@pytest.mark.parametrize("storage,width", [("fp16", 4), ("fp32", 2), ("bf16", 1)])
def test_fallback_d3q19_matches(storage, width):
    """D3Q19 widths without a fused form: the step, then the separate pass (exact)."""
    a, b = _pair3((16, 12, 8), "fluid", storage, width)
    got = a.step_conserved(4)
    b.step(4)
    assert got == b.conserved3()


def test_fused_sums_d3q19_full_size_fp16():
    """The 256^3 FP16 workload the benchmark times (persistent pipeline, one slot per
    block): fused sums against the separate pass."""
    import torch

    from paper_1312_3297_gb300 import D3Q19

    L = 256
    d = inp.taylor_green_3d(L, L, L, u0=0.04)
    fields = [torch.as_tensor(d["rho"], dtype=torch.float32)] + [
        torch.as_tensor(c, dtype=torch.float32) for c in d["u"]]
    del d
    sims = []
    for _ in range(2):
        sim = D3Q19(L, L, L, S19, mode="fluid", storage="fp16")
        sim.init_equilibrium(*fields)
        sims.append(sim)
    got = sims[0].step_conserved(2)
    sims[1].step(2)
    ref = sims[1].conserved3()
    np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=1e-9 * L ** 3)
    assert got[4] == ref[4] == 0.0
    for sim in sims:
        sim.close()


def test_nonfinite_count_matches_and_is_reported():
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding

    a, b = _pair(D2Q9, (64, 16), "fluid", "fp32", 4)
    for sim in (a, b):
        g = sim.state()
        g[3, 5, 7] = float("nan")
        sim.set_state(g, 0)
    got = a.step_conserved(2, allow_nonfinite=True)
    b.step(2)
    ref = b.conserved3(allow_nonfinite=True)
    assert got[4] == ref[4] > 0
    with pytest.raises(binding.LbmrvError):
        a.step_conserved(1)
    with pytest.raises(binding.LbmrvError):
        b.step_conserved(0)


def test_scratch_grows_when_the_width_changes():
    """A call at 4-node packs, then at 2-node packs (twice the step blocks): the scratch is
    reallocated and the sums stay equal to the separate pass."""
    from paper_1312_3297_gb300 import D2Q9

    shape = (512, 64)
    a, b = _pair(D2Q9, shape, "fluid", "fp32", 4)
    _compare(a, b, 3, shape[0] * shape[1])
    for sim in (a, b):
        sim.set_kernel_width(2)
    got = a.step_conserved(2)
    b.step(2)
    ref = b.conserved3()
    np.testing.assert_allclose(got[:4], ref[:4], rtol=1e-12, atol=1e-9 * shape[0] * shape[1])
