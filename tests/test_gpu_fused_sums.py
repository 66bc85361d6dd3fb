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


@pytest.mark.parametrize("width", [1, 0])
def test_fallback_paths_match(width):
    """Scalar kernel (width 1) and D3Q19: the step, then the separate pass."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, D3Q19

    if width == 1:
        a, b = _pair(D2Q9, (37, 11), "fluid", "fp32", 1)
        _compare(a, b, 4, 37 * 11)
        return
    d = inp.random_flow_3d(16, 12, 8, seed=2)
    s19 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3
    sims = []
    for _ in range(2):
        sim = D3Q19(16, 12, 8, s19, mode="fluid", storage="fp16")
        sim.init_equilibrium(torch.as_tensor(d["rho"], dtype=torch.float32),
                             *(torch.as_tensor(c, dtype=torch.float32) for c in d["u"]))
        sims.append(sim)
    got = sims[0].step_conserved(4)
    sims[1].step(4)
    assert got == sims[1].conserved3()


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
