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


@pytest.mark.parametrize("storage,nx,ny,u_ref", [("fp32", 96, 64, (0.0, 0.0)),
                                                 ("fp16", 300, 17, None),
                                                 ("bf16", 64, 64, (0.05, 0.02)),
                                                 ("fp32", 1024, 1024, None)])
def test_noalloc_matches_handle_reduction_twice(storage, nx, ny, u_ref):
    """u_ref: the plain form (0, 0), a fixed reference velocity, or the automatic one (the
    mean flow of the initial fields). The entry point reads the state with a zero reference
    velocity, so for a state stored relative to f_eq(rho_ref, U) the header's rule adds
    nx*ny*rho_ref*U to the momentum sums."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B

    d = inp.random_sine_flow(nx, ny, seed=11)
    sim = D2Q9(nx, ny, S, mode="fluid", storage=storage, u_ref=u_ref)
    sim.init_equilibrium(*(torch.as_tensor(d[k], dtype=torch.float32)
                           for k in ("rho", "ux", "uy")))
    U = np.asarray(sim.u_ref, float)
    if u_ref is not None:
        assert tuple(U) == tuple(u_ref)
    else:
        assert np.any(U != 0.0)  # the sine flow's noise leaves a small mean flow
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row share (and overwrite) the scratch array
        sim.step(13)
        ref = sim.conserved()
        B.lbmrv_conserved_noalloc(sim.state_ptr(), sim.storage, (nx, ny, 1), sim.lam,
                                  sim.rho_ref, out, sim.stream)
        got = out.cpu().numpy()
        got[1:3] += nx * ny * sim.rho_ref * U
        np.testing.assert_allclose(got[0], ref[0], rtol=1e-12)
        np.testing.assert_allclose(got[1:3], ref[1:3], rtol=1e-12, atol=1e-10)
        assert got[3] == ref[3] == 0
    sim.close()


def test_noalloc_call_leaves_free_device_memory_unchanged():
    """After a first call (which looks up the scratch address), further calls take no
    device memory: the free memory the driver reports does not move."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B

    nx, ny = 256, 128
    d = inp.random_sine_flow(nx, ny, seed=3)
    sim = D2Q9(nx, ny, S, mode="fluid")
    sim.init_equilibrium(*(torch.as_tensor(d[k], dtype=torch.float32)
                           for k in ("rho", "ux", "uy")))
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    B.lbmrv_conserved_noalloc(sim.state_ptr(), sim.storage, (nx, ny, 1), sim.lam,
                              sim.rho_ref, out, sim.stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        B.lbmrv_conserved_noalloc(sim.state_ptr(), sim.storage, (nx, ny, 1), sim.lam,
                                  sim.rho_ref, out, sim.stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    sim.close()


def test_noalloc_rejects_sizes_beyond_the_maximum():
    import torch

    from paper_1312_3297_gb300 import binding as B

    state = torch.zeros(64, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # raw addresses: the C entry point itself rejects the sizes
    for dims in [(1 << 16, 1 << 15, 1), (0, 4, 1), (4, 4, 3), (4, 4, 0)]:
        with pytest.raises(B.LbmrvError) as ei:
            B.lbmrv_conserved_noalloc(state.data_ptr(), B.LBMRV_FP32, dims, 1.0, 1.0,
                                      out.data_ptr())
        assert ei.value.status == B.LBMRV_E_INVAL
    with pytest.raises(B.LbmrvError):
        B.lbmrv_conserved_noalloc(state.data_ptr(), 7, (4, 4, 1), 1.0, 1.0, out.data_ptr())


def test_noalloc_binding_checks_tensors():
    """Tensors are checked before the call: a state too small for its dims, an output of
    the wrong type or size, a tensor off the device."""
    import torch

    from paper_1312_3297_gb300 import binding as B

    state = torch.zeros(9 * 16, dtype=torch.float32, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    B.lbmrv_conserved_noalloc(state, B.LBMRV_FP32, (4, 4, 1), 1.0, 1.0, out)
    for bad in [dict(dims=(8, 4, 1)),
                dict(out=torch.zeros(4, dtype=torch.float32, device="cuda")),
                dict(out=torch.zeros(3, dtype=torch.float64, device="cuda")),
                dict(out=torch.zeros(4, dtype=torch.float64)),
                dict(state=torch.zeros(9 * 16, dtype=torch.float32))]:
        a = dict(state=state, dims=(4, 4, 1), out=out)
        a.update(bad)
        with pytest.raises(ValueError):
            B.lbmrv_conserved_noalloc(a["state"], B.LBMRV_FP32, a["dims"], 1.0, 1.0, a["out"])
