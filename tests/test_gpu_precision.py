"""Reduced-precision storage (FP16 / BF16 deviations, FP32 arithmetic) against the FP64
oracle. The bar for the velocity is 2e-3 of max|u| (max_x |du(x)|_2 / max_x |u(x)|_2).

The stored value is g = f - f_eq(rho_ref, U_ref). By default the library takes U_ref to be
the mean flow sum(rho u) / sum(rho) of the initial fields, an invariant of the periodic
scheme, so only the perturbations around the mean flow are rounded. The plain form
(U_ref = 0, g = f - w rho_ref) is kept as a measured case: for a flow with a mean velocity
its deviations are dominated by the mean-flow term w rho (3 c.U + ...), whose 16-bit
rounding is coarse and nearly the same at every node, so the error grows with the number
of steps; on the perturbed uniform flow over 2000 steps it misses the bar (FP16 5.2e-3,
BF16 2.0e-2 of max|u|).

BF16 keeps 8 significant bits (relative rounding up to 2^-8 = 3.9e-3 per stored value).
On flows whose velocity varies by O(|u|) across the lattice (the 64^2 random sine flow)
the deviations from any uniform reference are O(w |u|), and their rounding alone moves
the velocity by about 1e-3 of max|u| per step: BF16 misses the bar there (measured
7.7e-3 to 9.9e-3 of max|u| after 100 steps) and the test states that number.
"""
import json
import os

import numpy as np
import pytest

import lbm_inputs as inp
from pairs import f32_fields, gpu_run, oracle_run, reference_populations, rel_errors

pytestmark = pytest.mark.gpu

S = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]
U_TOL = 2e-3
U_MEAN = (0.05, 0.02)


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _report(name, errs):
    out = os.environ.get("LBMRV_PRECISION_REPORT")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps({"case": name, "e_rho": errs[0], "e_u": errs[1],
                                 "e_f": errs[2]}) + "\n")


@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_fp16_small_lattice(mode):
    """64^2 random sine flow, 100 steps, FP16 with the automatic reference: meets the bar
    (measured 1.03e-3 to 1.10e-3 of max|u|)."""
    fields = f32_fields(inp.random_sine_flow(64, 64, seed=0))
    f_g, m_g = gpu_run(64, 64, S, mode, 100, fields, storage="fp16", amp=0.03, period=1000.0)
    f_o, m_o = oracle_run(64, 64, S, mode, 100, fields, amp=0.03, period=1000.0)
    e = rel_errors(f_g, m_g, f_o, m_o)
    _report(f"fp16-auto-{mode}-64x64-100", e)
    assert e[1] <= U_TOL, e


@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_bf16_small_sine_flow_misses_the_bar_by_a_stated_margin(mode):
    """The same case in BF16: its velocity error is measured at 7.7e-3 to 9.9e-3 of max|u|,
    above the 2e-3 bar (see the module docstring); the test holds it to 1.2e-2 so that a
    change that makes it worse is caught."""
    fields = f32_fields(inp.random_sine_flow(64, 64, seed=0))
    f_g, m_g = gpu_run(64, 64, S, mode, 100, fields, storage="bf16", amp=0.03, period=1000.0)
    f_o, m_o = oracle_run(64, 64, S, mode, 100, fields, amp=0.03, period=1000.0)
    e = rel_errors(f_g, m_g, f_o, m_o)
    _report(f"bf16-auto-{mode}-64x64-100", e)
    assert e[1] <= 1.2e-2, e


@pytest.fixture(scope="module")
def crop_oracle():
    """Perturbed uniform flow U = (0.05, 0.02), drho = du = 1e-3 N(0,1), u~ = q/rho, 2000
    steps on the 512^2 periodic lattice drawn with the same generator and seed as the
    8192^2 throughput workload."""
    fields = f32_fields(inp.perturbed_uniform(512, 512, seed=0, U=U_MEAN))
    return fields, oracle_run(512, 512, S, "fluid", 2000, fields, method=1,
                              nthreads=os.cpu_count())


@pytest.mark.parametrize("storage,u_ref,tol", [
    ("fp16", None, U_TOL),
    ("bf16", None, U_TOL),
    ("fp32", None, 1e-5),
    ("fp32", (0.0, 0.0), 1e-5),
])
def test_perturbed_uniform_flow_512_crop_2000_steps(crop_oracle, storage, u_ref, tol):
    """The precision workload's shape with the library's default (automatic) reference:
    FP16 and BF16 meet 2e-3 of max|u| (measured 2.0e-5 and 4.5e-5), FP32 1e-5 in either
    form."""
    fields, (f_o, m_o) = crop_oracle
    f_g, m_g = gpu_run(512, 512, S, "fluid", 2000, fields, storage=storage, u_ref=u_ref)
    e = rel_errors(f_g, m_g, f_o, m_o)
    _report(f"{storage}-{'plain' if u_ref else 'auto'}-fluid-512x512-2000", e)
    assert e[1] <= tol, e
    assert e[0] <= tol, e


@pytest.mark.parametrize("storage,measured,bound", [("fp16", 5.2e-3, 1e-2),
                                                    ("bf16", 2.0e-2, 3e-2)])
def test_plain_form_misses_the_bar_on_the_crop(crop_oracle, storage, measured, bound):
    """The plain stored form g = f - w rho_ref (U_ref = 0) on the same case: measured at
    `measured` of max|u|, above the 2e-3 bar; held to `bound` so that a change that makes
    it worse is caught. This is why the library's default reference is the mean flow."""
    fields, (f_o, m_o) = crop_oracle
    f_g, m_g = gpu_run(512, 512, S, "fluid", 2000, fields, storage=storage, u_ref=(0.0, 0.0))
    e = rel_errors(f_g, m_g, f_o, m_o)
    _report(f"{storage}-plain-fluid-512x512-2000", e)
    assert U_TOL < e[1] <= bound, e


@pytest.mark.parametrize("storage,tol", [("fp16", 2e-4), ("bf16", 1.5e-3)])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed", "field"])
def test_16bit_every_kernel_width(storage, tol, mode):
    """Every variant of the 16-bit step — one node per thread, 2-, 4- and 8-node packs (the
    8-node packs relax two nodes per packed FP32 instruction) — against the oracle, in the
    automatic reference form, where storage rounding stays far below what a wrong lane,
    term or sign would cost. 72 x 21: nine 8-node packs per row (a partly idle warp), odd ny;
    40 steps of the perturbed uniform flow."""
    nx, ny, steps = 72, 21, 40
    fields = f32_fields(inp.perturbed_uniform(nx, ny, seed=11, U=U_MEAN))
    kw = dict(amp=0.03, period=50.0)
    if mode == "field":
        kw["ut0"] = inp.to_f32_exact(inp.prescribed_base_field(nx, ny, seed=12, smooth=False))
    m = "prescribed" if mode == "field" else mode
    f_o, m_o = oracle_run(nx, ny, S, m, steps, fields, **kw)
    for w in (1, 2, 4, 8):
        f_g, m_g = gpu_run(nx, ny, S, m, steps, fields, storage=storage, width=w, **kw)
        e = rel_errors(f_g, m_g, f_o, m_o)
        assert e[1] <= tol, (w, e)
        assert e[0] <= tol, (w, e)


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_full_size_8192_sampled_parity(storage):
    """The 8192^2 precision workload in the benchmark's launch configuration (8-node packs
    relaxed in pairs, automatic reference): nodes at the corners, wrap edges, pack and warp
    boundaries and random places against the oracle on their dependency windows, in the
    populations and in the velocity (2e-3 of max|u|)."""
    import torch

    import oracle
    from paper_1312_3297_gb300 import D2Q9

    L, steps = 8192, 4
    rho, ux, uy = f32_fields(inp.perturbed_uniform(L, L, seed=0, U=U_MEAN))
    sim = D2Q9(L, L, S, mode="fluid", storage=storage)
    sim.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    sim.step(steps)
    g = sim.state()
    r_g, ux_g, uy_g = sim.moments()
    fref = reference_populations(sim.rho_ref, sim.u_ref, 1.0)
    R = steps + 1
    rng = np.random.default_rng(2)
    centers = [(0, 0), (L - 1, L - 1), (0, L - 1), (L - 1, 0), (7, 3), (8, 3), (1023, 77),
               (1024, 78), (L - 8, 5), (L - 9, L - 2)]
    centers += [tuple(int(v) for v in rng.integers(0, L, 2)) for _ in range(6)]
    errs, du, fmax, umax = [], [], 0.0, 0.0
    for cx, cy in centers:
        xs = (cx + np.arange(-R, R + 1)) % L
        ys = (cy + np.arange(-R, R + 1)) % L
        f0 = oracle.init_equilibrium(rho[np.ix_(ys, xs)], ux[np.ix_(ys, xs)],
                                     uy[np.ix_(ys, xs)], 1.0)
        S_o = oracle.post_collision_state(f0, 1.0, np.asarray(S, float), 1, steps)
        ref = S_o[:, R, R]
        _, uxo, uyo = oracle.moments(S_o, 1.0)
        got = g[:, cy, cx].double().cpu().numpy() + fref
        errs.append(float(np.abs(got - ref).max()))
        du.append(float(np.hypot(float(ux_g[cy, cx]) - uxo[R, R], float(uy_g[cy, cx]) - uyo[R, R])))
        fmax = max(fmax, float(np.abs(ref).max()))
        umax = max(umax, float(np.hypot(uxo[R, R], uyo[R, R])))
    sim.close()
    assert max(errs) <= (1e-4 if storage == "fp16" else 1e-3) * fmax, errs
    assert max(du) <= U_TOL * umax, (max(du) / umax, du)
