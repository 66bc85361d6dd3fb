"""GPU parity of the cascaded D2Q9 lattice (Geier's basis and product equilibrium, the
proposition of Section 1.3 and Appendix B) against the FP64 oracle: the relative-velocity
definition in Geier's basis for every u~ mode, and Geier's cascade as Appendix B writes it
for u~ = q/rho."""
import numpy as np
import pytest

import lbm_inputs as inp
from pairs import f32_fields, gpu_run, oracle_run, product_populations, rel_errors

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


def test_cascaded_full_size_sampled_parity():
    """The cascaded workload the benchmark times (4096^2 Taylor-Green, u~ = q/rho, 4-node
    packs): sampled nodes against Appendix B's cascade on their dependency windows."""
    import torch

    import oracle
    from paper_1312_3297_gb300 import D2Q9Cascaded

    L, steps = 4096, 4
    rho, ux, uy = f32_fields(inp.taylor_green(L, L, u0=0.04))
    sim = D2Q9Cascaded(L, L, SG, mode="fluid")
    sim.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    sim.step(steps)
    g = sim.state()
    fref = product_populations(sim.rho_ref, sim.u_ref, 1.0)
    R = steps + 1
    rng = np.random.default_rng(4)
    centers = [(0, 0), (L - 1, L - 1), (3, L - 1), (4, 0), (511, 2048), (512, 2049)]
    centers += [tuple(int(v) for v in rng.integers(0, L, 2)) for _ in range(6)]
    errs, fmax = [], 0.0
    for cx, cy in centers:
        xs = (cx + np.arange(-R, R + 1)) % L
        ys = (cy + np.arange(-R, R + 1)) % L
        f0 = oracle.init_equilibrium_product(rho[np.ix_(ys, xs)], ux[np.ix_(ys, xs)],
                                             uy[np.ix_(ys, xs)], 1.0)
        ref = oracle.post_collision_state(f0, 1.0, np.asarray(SG, float), 1, steps,
                                          method=CASCADED)[:, R, R]
        got = g[:, cy, cx].double().cpu().numpy() + fref
        errs.append(float(np.abs(got - ref).max()))
        fmax = max(fmax, float(np.abs(ref).max()))
    sim.close()
    assert max(errs) <= TOL * fmax, errs


@pytest.mark.parametrize("storage,tol", [("fp16", 2e-4), ("bf16", 1.5e-3)])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed", "field"])
def test_cascaded_16bit_every_width(storage, tol, mode):
    """Every 16-bit variant of the cascaded step (one node per thread, 2-, 4- and 8-node
    packs; 8-node packs relax node pairs by packed FP32 instructions) against the oracle's
    Geier scheme, with the automatic reference (the mean flow of the fields), 72 x 21 (a
    partly idle warp, odd ny), 40 steps."""
    nx, ny, steps = 72, 21, 40
    u_mean = (0.05, 0.02)
    fields = f32_fields(inp.perturbed_uniform(nx, ny, seed=13, U=u_mean))
    kw = dict(amp=0.03, period=50.0)
    if mode == "field":
        kw["ut0"] = inp.to_f32_exact(inp.prescribed_base_field(nx, ny, seed=14, smooth=False))
    m = "prescribed" if mode == "field" else mode
    for w in (1, 2, 4, 8):
        _check(nx, ny, m, steps, fields, tol=tol, storage=storage, width=w, **kw)
