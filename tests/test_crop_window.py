"""The crop protocol's shrinking window, on the CPU: under exact transport (Section 1.1)
information moves at most one node per step, so running the FP64 oracle on the window of
the central crop's dependency cone as a periodic lattice, and cutting off every m steps the
m-node rim its wrapped edges have reached, leaves the central crop equal bit for bit to the
same region of a run over the whole periodic lattice (the argument of
tests/test_gpu_crop_protocol.py, at a size that runs in seconds)."""
import numpy as np

import lbm_inputs as inp
from pairs import f32_fields

S = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]


def test_shrinking_window_equals_the_whole_lattice(orc):
    n, crop, steps, every = 96, 16, 20, 6
    rho, ux, uy = f32_fields(inp.perturbed_uniform(n, n, seed=0))
    whole = orc.run(orc.init_equilibrium(rho, ux, uy, 1.0), 1.0, np.asarray(S, float),
                    orc.MODE_FLUID, steps, method=orc.METHOD_SHIFTED, nthreads=4)
    c0 = (n - crop) // 2
    idx = np.arange(c0 - steps, c0 + crop + steps) % n
    f = orc.init_equilibrium(rho[np.ix_(idx, idx)], ux[np.ix_(idx, idx)],
                             uy[np.ix_(idx, idx)], 1.0)
    k = 0
    while k < steps:
        m = min(every, steps - k)
        f = orc.run(f, 1.0, np.asarray(S, float), orc.MODE_FLUID, m, t0=k,
                    method=orc.METHOD_SHIFTED, nthreads=4)
        k += m
        f = np.ascontiguousarray(f[:, m:-m, m:-m])
    assert f.shape == (9, crop, crop)
    assert np.array_equal(f, whole[:, c0:c0 + crop, c0:c0 + crop])
    # one step too few cut off would leave contaminated nodes at the edge
    g = orc.init_equilibrium(rho[np.ix_(idx, idx)], ux[np.ix_(idx, idx)],
                             uy[np.ix_(idx, idx)], 1.0)
    g = orc.run(g, 1.0, np.asarray(S, float), orc.MODE_FLUID, steps + 1,
                method=orc.METHOD_SHIFTED, nthreads=4)
    whole1 = orc.run(whole, 1.0, np.asarray(S, float), orc.MODE_FLUID, 1, t0=steps,
                     method=orc.METHOD_SHIFTED, nthreads=4)
    inner = g[:, steps:-steps, steps:-steps]
    assert not np.array_equal(inner, whole1[:, c0:c0 + crop, c0:c0 + crop])
