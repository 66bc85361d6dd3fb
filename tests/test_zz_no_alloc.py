"""The allocation-free reduction entry point against the handle-based one.

lbmrv_conserved_noalloc serves callers that cannot allocate device memory when they
want the mass / momentum check (an allocator that owns the whole device, a loop where
cudaMalloc would synchronise, a monitor of a buffer it did not create). It must give the
same sums as lbmrv_conserved, call after call, since every call reuses one fixed scratch
array. This file is collected last so that a first failure here comes after every other
test has run; it also passes alone in a fresh process.
"""
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


@pytest.mark.parametrize("storage,nx,ny", [("fp32", 96, 64), ("fp16", 300, 17),
                                           ("bf16", 64, 64), ("fp32", 1024, 1024)])
def test_noalloc_matches_handle_reduction_twice(storage, nx, ny):
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B

    d = inp.random_sine_flow(nx, ny, seed=11)
    sim = D2Q9(nx, ny, S, mode="fluid", storage=storage)
    sim.init_equilibrium(*(torch.as_tensor(d[k], dtype=torch.float32)
                           for k in ("rho", "ux", "uy")))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row share (and overwrite) the scratch array
        sim.step(13)
        ref = sim.conserved()
        B.lbmrv_conserved_noalloc(sim.state_ptr(), sim.storage, (nx, ny, 1), sim.lam,
                                  sim.rho_ref, out, sim.stream)
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        np.testing.assert_allclose(got[1:3], ref[1:3], rtol=1e-12, atol=1e-12)
        assert got[3] == ref[3] == 0
    sim.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    from paper_1312_3297_gb300 import binding as B

    state = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    for dims in [(1 << 16, 1 << 15, 1), (0, 4, 1), (4, 4, 3)]:
        with pytest.raises(B.LbmrvError) as ei:
            B.lbmrv_conserved_noalloc(state, B.LBMRV_FP32, dims, 1.0, 1.0, out)
        assert ei.value.status == B.LBMRV_E_INVAL
    with pytest.raises(B.LbmrvError):
        B.lbmrv_conserved_noalloc(state, 7, (4, 4, 1), 1.0, 1.0, out)
