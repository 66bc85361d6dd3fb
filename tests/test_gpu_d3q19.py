"""GPU parity of the fused D3Q19 relative-velocity step against the FP64 D3Q19 oracle."""
import json
import os

import numpy as np
import pytest

import lbm_inputs as inp
from pairs import S3, W3, gpu_run3, oracle_run3, reference_populations3, rel_errors3

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fields(shape, seed):
    nx, ny, nz = shape
    d = inp.random_flow_3d(nx, ny, nz, seed=seed)
    return inp.to_f32_exact(d["rho"]), inp.to_f32_exact(d["u"])


def _report(name, errs):
    out = os.environ.get("LBMRV_PRECISION_REPORT")
    if out:
        with open(out, "a") as fh:
            fh.write(json.dumps({"case": name, "e_rho": errs[0], "e_u": errs[1],
                                 "e_f": errs[2]}) + "\n")


# BF16 keeps 8 significant bits. On the random sine flow (u = 0.04 (sin, sin, sin) + noise,
# mean flow near 0) the stored deviations from any uniform reference are O(w |u|), and
# their rounding moves the velocity by about 1e-3 of max|u| per step: after 9 to 20 steps
# the velocity error is measured at 1.7e-3 to 4.7e-3 of max|u|, above the 2e-3 bar, while
# rho and f stay within 2e-4. The BF16 sine-flow tests therefore hold the velocity to the
# stated 6e-3 (so that a change that makes it worse is caught) and rho and f to 2e-3;
# FP16 (measured <= 4.5e-4) and BF16 on the perturbed uniform flow (<= 2.6e-5) meet 2e-3.
BF16_SINE_U_TOL = 6e-3


def _check(shape, mode, steps, tol=TOL, seed=0, flow="sine", u_tol=None, **kw):
    if flow == "sine":
        rho, u = _fields(shape, seed)
    else:
        d = inp.perturbed_uniform_3d(*shape, seed=seed)
        rho, u = inp.to_f32_exact(d["rho"]), inp.to_f32_exact(d["u"])
    nx, ny, nz = shape
    ut0 = None
    if mode == "prescribed":
        ut0 = inp.to_f32_exact(np.random.default_rng(seed + 7).standard_normal((3, nz, ny, nx)))
    f_g, r_g, u_g = gpu_run3(shape, S3, mode, steps, rho, u, ut0=ut0, amp=0.03, period=40.0,
                             **kw)
    f_o, r_o, u_o = oracle_run3(S3, mode, steps, rho, u, ut0=ut0, amp=0.03, period=40.0)
    e = rel_errors3(f_g, r_g, u_g, f_o, r_o, u_o)
    if kw.get("storage", "fp32") != "fp32":
        _report(f"d3q19-{kw['storage']}-{flow}-{mode}-{'x'.join(map(str, shape))}-"
                f"w{kw.get('width', 0)}-{steps}", e)
    assert e[0] <= tol and e[2] <= tol, (shape, mode, kw, e)
    assert e[1] <= (tol if u_tol is None else u_tol), (shape, mode, kw, e)
    return f_g


@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_parity_small_3d_every_width(mode):
    shape = (24, 10, 8)
    outs = [_check(shape, mode, 20, width=w) for w in (1, 2, 4)]
    for f in outs[1:]:
        np.testing.assert_array_equal(f, outs[0])


@pytest.mark.parametrize("storage,u_tol", [("fp16", None), ("bf16", BF16_SINE_U_TOL)])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_16bit_3d_every_width(storage, u_tol, mode):
    """Every 16-bit D3Q19 kernel against the oracle: one node per thread, 2-node packs
    converted to FP32 on load, 4- and 8-node packs kept in storage form (two values per
    register). 40 x 7 x 5: five 8-node packs per row (a partly idle warp; several rows per
    block), odd ny and nz. Kernels of one family agree bit for bit."""
    shape = (40, 7, 5)
    outs = {w: _check(shape, mode, 20, tol=2e-3, u_tol=u_tol, seed=3, storage=storage,
                      width=w)
            for w in (1, 2, 4, 8)}
    np.testing.assert_array_equal(outs[2], outs[1])
    np.testing.assert_array_equal(outs[8], outs[4])


@pytest.mark.parametrize("storage,u_tol", [("fp16", None), ("bf16", BF16_SINE_U_TOL)])
@pytest.mark.parametrize("shape", [(264, 3, 2), (552, 2, 3), (392, 2, 3), (200, 3, 2)])
def test_16bit_3d_rows_of_several_segments(storage, u_tol, shape):
    """Rows longer than one 256-node segment of the staged 8-node-pack kernel, the last
    segment short, with every x-moving population crossing the segment boundaries: the
    kernel against the oracle and bit for bit against 4-node packs. Short last segments of
    one and five packs are packed several rows to an item (the rows of an item in different
    y and z); those of 17 packs (392) and a single segment of 25 (200) keep one row per
    item."""
    outs = {w: _check(shape, "fluid", 12, tol=2e-3, u_tol=u_tol, seed=5, storage=storage,
                      width=w)
            for w in (4, 8)}
    np.testing.assert_array_equal(outs[8], outs[4])


@pytest.mark.parametrize("storage,u_tol", [("fp16", None), ("bf16", BF16_SINE_U_TOL)])
@pytest.mark.parametrize("shape", [(8, 1, 1), (8, 3, 1), (16, 1, 3), (256, 1, 2)])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_16bit_3d_degenerate_8_node_packs(storage, u_tol, shape, mode):
    """The staged 8-node-pack kernel where a row is one pack (the pack its own periodic
    neighbour in x) or where y or z has one row (the row its own neighbour), in every
    relaxation frame (each issues its copies in a different number of plane groups):
    against the oracle and bit for bit against 4-node packs."""
    outs = {w: _check(shape, mode, 9, tol=2e-3, u_tol=u_tol, seed=11, storage=storage,
                      width=w)
            for w in (4, 8)}
    np.testing.assert_array_equal(outs[8], outs[4])


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
@pytest.mark.parametrize("mode", ["zero", "fluid", "prescribed"])
def test_16bit_3d_perturbed_uniform_flow_every_width(storage, mode):
    """The precision workload's shape in 3D (uniform flow U = (0.05, 0.02, 0.01) with
    1e-3 N(0,1) perturbations) with the automatic reference: every 16-bit kernel within
    2e-3 of max|u| in rho, u and f, and kernels of one family bit for bit."""
    shape = (40, 7, 5)
    outs = {w: _check(shape, mode, 20, tol=2e-3, seed=8, flow="uniform", storage=storage,
                      width=w) for w in (1, 2, 4, 8)}
    np.testing.assert_array_equal(outs[2], outs[1])
    np.testing.assert_array_equal(outs[8], outs[4])


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 2, 5), (7, 3, 2), (2, 9, 1), (5, 1, 4)])
def test_parity_degenerate_3d(shape):
    for mode in ("zero", "fluid", "prescribed"):
        _check(shape, mode, 6)


def test_parity_3d_reference_velocity():
    _check((16, 12, 6), "fluid", 25, u_ref=(0.03, -0.02, 0.01))


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_reduced_precision_3d(storage):
    shape = (32, 16, 12)
    rho, u = _fields(shape, 3)
    f_g, r_g, u_g = gpu_run3(shape, S3, "fluid", 40, rho, u, storage=storage)
    f_o, r_o, u_o = oracle_run3(S3, "fluid", 40, rho, u)
    e = rel_errors3(f_g, r_g, u_g, f_o, r_o, u_o)
    _report(f"d3q19-{storage}-sine-fluid-32x16x12-w0-40", e)
    assert e[0] <= 2e-3 and e[2] <= 2e-3, e
    assert e[1] <= (2e-3 if storage == "fp16" else BF16_SINE_U_TOL), e


@pytest.mark.parametrize("storage,tol,u_tol,mass_tol,mom_tol", [
    ("fp32", TOL, TOL, 1e-9, 1e-6),
    ("fp16", 2e-4, 2e-3, 1e-5, 1e-3),
    ("bf16", 3e-3, 2e-3, 1e-4, 1e-2),
])
def test_full_size_256_sampled_parity_and_conservation(storage, tol, u_tol, mass_tol,
                                                       mom_tol):
    """3D Taylor-Green vortex u0 = 0.04 on 256^3 (u~ = q/rho, s_nu = 1.7) in the benchmark's
    launch configuration (FP32: 4-node packs; 16-bit: 8-node packs in storage form): sampled
    nodes against the oracle on their dependency cone, and mass / momentum over 100 steps
    (16-bit storage rounding bounds their drift)."""
    import torch

    from oracle import d3q19 as o3
    from paper_1312_3297_gb300 import D3Q19

    L, steps = 256, 4
    d = inp.taylor_green_3d(L, L, L, u0=0.04)
    rho, u = inp.to_f32_exact(d["rho"]), inp.to_f32_exact(d["u"])
    sim = D3Q19(L, L, L, S3, mode="fluid", storage=storage)
    sim.init_equilibrium(torch.as_tensor(rho), *(torch.as_tensor(c) for c in u))
    c0 = sim.conserved3()
    sim.step(steps)
    g = sim.state()
    m_g = [t for t in sim.moments()]
    fref = reference_populations3(sim.rho_ref, sim.u_ref)
    rng = np.random.default_rng(1)
    centers = [(0, 0, 0), (L - 1, L - 1, L - 1), (1, 0, L - 1), (127, 128, 5), (7, 3, 250),
               (8, 4, 251), (L - 8, 200, 0), (L - 9, 0, 17)]
    centers += [tuple(int(v) for v in rng.integers(0, L, 3)) for _ in range(4)]
    R = steps + 1
    errs, du, fmax, umax = [], [], 0.0, 0.0
    for cx, cy, cz in centers:
        xs = (cx + np.arange(-R, R + 1)) % L
        ys = (cy + np.arange(-R, R + 1)) % L
        zs = (cz + np.arange(-R, R + 1)) % L
        sub_rho = rho[np.ix_(zs, ys, xs)]
        sub_u = u[:, zs][:, :, ys][:, :, :, xs]
        f0 = o3.init_equilibrium(sub_rho, sub_u, 1.0)
        S = o3.post_collision_state(f0, 1.0, np.array(S3, float), 1, steps, nthreads=8)
        ref = S[:, R, R, R]
        got = g[:, cz, cy, cx].double().cpu().numpy() + fref
        errs.append(np.abs(got - ref).max())
        fmax = max(fmax, np.abs(ref).max())
        _, uo = o3.moments(S[:, R - 1:R + 2, R - 1:R + 2, R - 1:R + 2], 1.0)
        ug = np.array([float(m_g[1 + a][cz, cy, cx]) for a in range(3)])
        du.append(float(np.sqrt(((ug - uo[:, 1, 1, 1]) ** 2).sum())))
        umax = max(umax, float(np.sqrt((uo[:, 1, 1, 1] ** 2).sum())))
    _report(f"d3q19-{storage}-tg256-sampled-{steps}", (0.0, max(du) / umax, max(errs) / fmax))
    assert max(errs) / fmax <= tol, errs
    assert max(du) <= u_tol * umax, (max(du) / umax, du)
    sim.step(96)
    c1 = sim.conserved3()
    assert abs(c1[0] - c0[0]) / c0[0] < mass_tol
    for a in (1, 2, 3):
        assert abs(c1[a] - c0[a]) < mom_tol * c0[0] * 0.04
    sim.close()


@pytest.mark.parametrize("storage,tol", [("fp32", TOL), ("fp16", 2e-4)])
def test_512_cubed_plane_offsets_past_31_bits(storage, tol):
    """512^3 (134 M nodes): the offsets j * n of the upper planes pass 2^31 elements, so any
    32-bit plane arithmetic would read the wrong place. Sampled nodes (plane-crossing
    corners, pack and segment edges, random places) against the oracle on their dependency
    cone, in the default kernels (FP32 4-node packs; FP16 the staged 8-node packs)."""
    import torch

    from oracle import d3q19 as o3
    from paper_1312_3297_gb300 import D3Q19

    L, steps = 512, 3
    d = inp.taylor_green_3d(L, L, L, u0=0.04)
    rho, u = inp.to_f32_exact(d["rho"]), inp.to_f32_exact(d["u"])
    del d
    sim = D3Q19(L, L, L, S3, mode="fluid", storage=storage)
    sim.init_equilibrium(torch.as_tensor(rho), *(torch.as_tensor(c) for c in u))
    sim.step(steps)
    g = sim.state()
    fref = reference_populations3(sim.rho_ref, sim.u_ref)
    rng = np.random.default_rng(5)
    centers = [(0, 0, 0), (L - 1, L - 1, L - 1), (255, 256, 511), (256, 511, 0),
               (7, 1, 300), (8, 2, 301), (L - 8, 400, 1)]
    centers += [tuple(int(v) for v in rng.integers(0, L, 3)) for _ in range(3)]
    R = steps + 1
    errs, fmax = [], 0.0
    for cx, cy, cz in centers:
        xs = (cx + np.arange(-R, R + 1)) % L
        ys = (cy + np.arange(-R, R + 1)) % L
        zs = (cz + np.arange(-R, R + 1)) % L
        sub_rho = rho[np.ix_(zs, ys, xs)]
        sub_u = u[:, zs][:, :, ys][:, :, :, xs]
        f0 = o3.init_equilibrium(sub_rho, sub_u, 1.0)
        S = o3.post_collision_state(f0, 1.0, np.array(S3, float), 1, steps, nthreads=8)
        ref = S[:, R, R, R]
        got = g[:, cz, cy, cx].double().cpu().numpy() + fref
        errs.append(np.abs(got - ref).max())
        fmax = max(fmax, np.abs(ref).max())
    assert max(errs) / fmax <= tol, errs
    sim.close()
