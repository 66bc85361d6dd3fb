"""The FP64 conserved sums (relation (rhoq) summed over the lattice) of a stored state, at
every vector-pack width the reduction pass chooses.

The pass reads packs of 1 to 8 consecutive nodes per plane, as wide as the lattice's node
count and the planes' alignment allow. Lattices whose node counts are multiples of 8, of 4
but not 8, of 2 but not 4, and odd take each width. The sums must equal those of the state
read back and summed here in FP64: n rho_ref + sum_j g_j and sum_j c_j g_j (a zero
reference velocity, lambda = 1). The GPU adds node moments in FP32 runs of 32 nodes,
hence the tolerance. One planted non-finite population must be counted at every width.
"""
import numpy as np
import pytest

import lbm_inputs as inp

pytestmark = pytest.mark.gpu

C2 = np.array([[0, 1, 0, -1, 0, 1, -1, -1, 1],
               [0, 0, 1, 0, -1, 1, 1, -1, -1]], dtype=np.float64)
C3 = np.array([[0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0],
               [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1],
               [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]],
              dtype=np.float64)
S2 = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]
S3 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _expected(g, c, rho_ref):
    """FP64 sums of the stored deviations g (q, ...) read back from the device."""
    q = g.shape[0]
    flat = g.reshape(q, -1).astype(np.float64)
    n = flat.shape[1]
    per_pop = flat.sum(axis=1)
    return np.concatenate([[n * rho_ref + per_pop.sum()], c @ per_pop])


def _sim(lattice, shape, storage):
    import torch

    from paper_1312_3297_gb300 import D2Q9, D3Q19

    if lattice == "d2q9":
        nx, ny = shape
        d = inp.random_sine_flow(nx, ny, seed=21)
        sim = D2Q9(nx, ny, S2, mode="fluid", storage=storage, u_ref=(0.0, 0.0))
        sim.init_equilibrium(*(torch.as_tensor(d[k], dtype=torch.float32)
                               for k in ("rho", "ux", "uy")))
        return sim, C2
    nx, ny, nz = shape
    d = inp.random_flow_3d(nx, ny, nz, seed=22)
    sim = D3Q19(nx, ny, nz, S3, mode="fluid", storage=storage, u_ref=(0.0, 0.0, 0.0))
    sim.init_equilibrium(torch.as_tensor(d["rho"], dtype=torch.float32),
                         *(torch.as_tensor(c, dtype=torch.float32) for c in d["u"]))
    return sim, C3


SHAPES = {
    # node counts: multiple of 8, 4 (not 8), 2 (not 4), odd; and one spanning many blocks
    "d2q9": [(16, 5), (6, 2), (10, 1), (7, 3), (1030, 77)],
    "d3q19": [(8, 2, 2), (6, 2, 1), (2, 3, 1), (3, 3, 3), (66, 34, 21)],
}


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("lattice", ["d2q9", "d3q19"])
def test_conserved_sums_at_every_pack_width(lattice, storage):
    import torch

    for shape in SHAPES[lattice]:
        sim, c = _sim(lattice, shape, storage)
        sim.step(3)
        g = sim.state()
        want = _expected(g.float().cpu().numpy(), c, sim.rho_ref)
        got = np.asarray(sim.conserved3()[:1 + c.shape[0]])
        scale = float(g.abs().max()) * g[0].numel() + 1e-30
        np.testing.assert_allclose(got[0], want[0], rtol=1e-9, atol=1e-6 * scale,
                                   err_msg=f"{lattice} {shape} {storage}")
        np.testing.assert_allclose(got[1:], want[1:], rtol=1e-6, atol=1e-6 * scale,
                                   err_msg=f"{lattice} {shape} {storage}")
        # one non-finite population, in the last node: counted once, at every width
        bad = g.clone()
        bad.view(g.shape[0], -1)[5, -1] = float("nan")
        sim.set_state(bad, sim.time)
        assert sim.conserved3(allow_nonfinite=True)[-1] == 1.0
        sim.close()
        torch.cuda.empty_cache()
