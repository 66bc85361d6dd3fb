"""GPU parity of the cascaded D2Q9 lattice (Geier's basis and product equilibrium, the
proposition of Section 1.3 and Appendix B) against the FP64 oracle: the relative-velocity
definition in Geier's basis for every u~ mode, and Geier's cascade as Appendix B writes it
for u~ = q/rho."""
import numpy as np
import pytest

import lbm_inputs as inp
from pairs import f32_fields, gpu_run, oracle_run, rel_errors

pytestmark = pytest.mark.gpu

SG = [0, 0, 0, 1.3, 1.8, 1.8, 1.5, 1.5, 1.2]
TOL = 1e-5
GEIER, CASCADED = 3, 4


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _check(nx, ny, mode, steps, fields, method=GEIER, tol=TOL, **kw):
    okw = {k: v for k, v in kw.items() if k in ("ut0", "amp", "period")}
    f_g, m_g = gpu_run(nx, ny, SG, mode, steps, fields, cascaded=True, **kw)
    f_o, m_o = oracle_run(nx, ny, SG, mode, steps, fields, method=method, **okw)
    e = rel_errors(f_g, m_g, f_o, m_o)
    assert max(e) <= tol, (nx, ny, mode, kw, e)
    return f_g


@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_cascaded_lattice_parity_64(mode):
    fields = f32_fields(inp.random_sine_flow(64, 64, seed=0))
    _check(64, 64, mode, 100, fields, amp=0.03, period=1000.0)


def test_geier_scheme_against_appendix_b_cascade():
    fields = f32_fields(inp.random_sine_flow(48, 40, seed=1))
    _check(48, 40, "fluid", 80, fields, method=CASCADED)


@pytest.mark.parametrize("nx,ny", [(37, 23), (96, 33), (1, 1), (3, 5)])
def test_cascaded_ragged_every_width(nx, ny):
    fields = f32_fields(inp.random_sine_flow(nx, ny, seed=2))
    outs = [_check(nx, ny, "fluid", 20, fields, width=w) for w in (1, 2, 4) if nx % w == 0]
    for f in outs[1:]:
        np.testing.assert_array_equal(f, outs[0])


def test_cascaded_reference_velocity_and_fp16():
    fields = f32_fields(inp.perturbed_uniform(64, 48, seed=3, drho=1e-2, du=1e-2))
    _check(64, 48, "fluid", 60, fields, u_ref=(0.05, 0.02))
    _check(64, 48, "fluid", 60, fields, storage="fp16", u_ref=(0.05, 0.02), tol=2e-3)


def test_cascaded_full_size_conservation():
    import torch

    from paper_1312_3297_gb300 import D2Q9Cascaded

    L = 4096
    fields = f32_fields(inp.taylor_green(L, L, u0=0.04))
    sim = D2Q9Cascaded(L, L, SG, mode="fluid")
    sim.init_equilibrium(*(torch.as_tensor(a) for a in fields))
    c0 = sim.conserved()
    sim.step(200)
    c1 = sim.conserved()
    assert abs(c1[0] - c0[0]) / c0[0] < 1e-9
    assert abs(c1[1] - c0[1]) < 1e-6 * c0[0] * 0.04
    sim.close()
