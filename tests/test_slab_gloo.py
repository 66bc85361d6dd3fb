"""The slab decomposition's host logic on CPU ranks (gloo), against the single-domain oracle.

Each rank takes its layers from the library's partition plan (lbmrv_slab_plan), builds its
slab with one halo layer on each side, and advances it with the FP64 oracle, one step
S_k = C_k(P S_{k-1}) at a time (the exact transport of Section 1.1, then the relaxation).
Before each step it packs the values the library's index maps (lbmrv_halo_map) name,
exchanges them with its neighbours through the same exchange function the GPU driver uses
(paper_1312_3297_gb300.slab.exchange_faces), and unpacks them where the maps say. The
stitched own layers must equal the single-domain oracle bit for bit, and the all-reduced
FP64 sums of mass and momentum must equal the single-domain sums to rounding.
No GPU is used: the library's host-side plan and maps load without one.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
S2 = [0, 0, 0, 1.4, 1.9, 1.9, 1.2, 1.2, 1.4]
S3 = [0, 0, 0, 0, 1.2] + [1.7] * 5 + [1.9] * 6 + [1.4] * 3
MODES = {"zero": 0, "fluid": 1, "prescribed": 2}
AMP, PERIOD = 0.03, 40.0


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _initial(lattice, dims):
    """Seeded initial state S_0 = f_eq(rho, u) of the whole lattice, and a prescribed base
    field u~0, from the shared input generators; the slab axis is axis 1 of both."""
    import lbm_inputs as inp

    if lattice == "d2q9":
        import oracle

        nx, ny = dims
        d = inp.random_sine_flow(nx, ny, seed=3)
        f0 = oracle.init_equilibrium(*(inp.to_f32_exact(d[k]) for k in ("rho", "ux", "uy")),
                                     1.0)
        ut0 = inp.to_f32_exact(inp.prescribed_base_field(nx, ny, seed=4, smooth=False))
    else:
        from oracle import d3q19 as o3

        nx, ny, nz = dims
        d = inp.random_flow_3d(nx, ny, nz, seed=3)
        f0 = o3.init_equilibrium(inp.to_f32_exact(d["rho"]), inp.to_f32_exact(d["u"]), 1.0)
        ut0 = inp.to_f32_exact(np.random.default_rng(4).standard_normal((3, nz, ny, nx)))
    return f0, ut0


def _step(lattice, S, mode, t, ut0):
    """One step of the oracle from the post-relaxation state: transport, then relaxation
    at time t."""
    if lattice == "d2q9":
        import oracle

        return oracle.collide(oracle.stream(S), 1.0, S2, MODES[mode], t=t, ut0=ut0, amp=AMP,
                              period=PERIOD)
    from oracle import d3q19 as o3

    return o3.collide(o3.stream(S), 1.0, S3, MODES[mode], t=t, ut0=ut0, amp=AMP,
                      period=PERIOD)


def _sums(lattice, S):
    """FP64 mass and momentum of a post-relaxation state (equal to those of f)."""
    if lattice == "d2q9":
        import oracle

        r, ux, uy = oracle.moments(S, 1.0)
        return [r.sum(), (r * ux).sum(), (r * uy).sum()]
    from oracle import d3q19 as o3

    r, u = o3.moments(S, 1.0)
    return [r.sum()] + [(r * u[a]).sum() for a in range(3)]


def _rank(rank, world, port, case, out):
    sys.path[:0] = [ROOT, os.path.join(ROOT, "tests")]
    from paper_1312_3297_gb300 import binding as B
    from paper_1312_3297_gb300.slab import allreduce_sums, exchange_faces

    lattice, dims, mode, steps = case
    if world > 1:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        dist.init_process_group("gloo", rank=rank, world_size=world)
    f0, ut0 = _initial(lattice, dims)
    extent = dims[-1]
    first, count = B.lbmrv_slab_plan(extent, world, rank)
    layers = [(first - 1 + k) % extent for k in range(count + 2)]
    S = np.ascontiguousarray(f0[:, layers])
    ut = np.ascontiguousarray(ut0[:, layers])
    local = tuple(dims[:-1]) + (count + 2,)
    lat = B.LBMRV_D2Q9 if lattice == "d2q9" else B.LBMRV_D3Q19
    send0, recv0 = B.lbmrv_halo_map(lat, local + (1,) * (3 - len(local)), 0)
    send1, recv1 = B.lbmrv_halo_map(lat, local + (1,) * (3 - len(local)), 1)
    for t in range(1, steps + 1):
        flat = S.reshape(-1)
        s_lo, s_hi = torch.from_numpy(flat[send0]), torch.from_numpy(flat[send1])
        r_lo, r_hi = torch.empty_like(s_lo), torch.empty_like(s_hi)
        exchange_faces(s_lo, s_hi, r_lo, r_hi, rank, world)
        flat[recv0] = r_lo.numpy()
        flat[recv1] = r_hi.numpy()
        S = _step(lattice, S, mode, t, ut)
    own = np.ascontiguousarray(S[:, 1:-1])
    sums = allreduce_sums(_sums(lattice, own), world, torch.device("cpu"))
    out[rank] = (first, count, own, sums)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


CASES = [
    # (lattice, global dims, u~ mode, steps, ranks)
    ("d2q9", (24, 30), "fluid", 14, 2),
    ("d2q9", (20, 31), "prescribed", 12, 3),  # ragged: 11, 10, 10 rows
    ("d2q9", (16, 3), "zero", 7, 3),          # one row per rank
    ("d2q9", (12, 9), "fluid", 10, 1),        # one rank: its own neighbour
    ("d3q19", (6, 5, 8), "fluid", 9, 2),
    ("d3q19", (5, 4, 7), "prescribed", 8, 3),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}-{c[1]}-{c[2]}-w{c[4]}" for c in CASES])
def test_slabs_on_gloo_ranks_equal_the_single_domain_oracle(case):
    lattice, dims, mode, steps, world = case
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, case[:4], out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(300)
            assert p.exitcode == 0
        res = dict(out)
    f0, ut0 = _initial(lattice, dims)
    S = f0
    for t in range(1, steps + 1):
        S = _step(lattice, S, mode, t, ut0)
    want = _sums(lattice, S)
    stitched = np.concatenate([res[r][2] for r in range(world)], axis=1)
    assert [res[r][0] for r in range(world)] == sorted(res[r][0] for r in range(world))
    assert sum(res[r][1] for r in range(world)) == dims[-1]
    assert np.array_equal(stitched, S)  # bit for bit
    for r in range(world):
        np.testing.assert_allclose(res[r][3], want, rtol=1e-13, atol=1e-13)


def test_plan_covers_every_layer_once():
    sys.path.insert(0, ROOT)
    from paper_1312_3297_gb300 import binding as B

    for extent in (1, 2, 7, 64, 1001):
        for ranks in range(1, min(extent, 9) + 1):
            seen = []
            for r in range(ranks):
                first, count = B.lbmrv_slab_plan(extent, ranks, r)
                assert count in (extent // ranks, extent // ranks + 1)
                seen += list(range(first, first + count))
            assert seen == list(range(extent))
    for bad in [(4, 5, 0), (4, 0, 0), (4, 2, 2), (4, 2, -1)]:
        with pytest.raises(B.LbmrvError):
            B.lbmrv_slab_plan(*bad)


def test_halo_maps_pair_faces_and_name_crossing_populations():
    """The upper face sends the populations with c = +1 (along the slab axis) of the top own
    layer, which the upper neighbour receives into the same populations of its lower halo
    layer; the lower face likewise with c = -1. Every map entry is inside the state."""
    sys.path.insert(0, ROOT)
    from paper_1312_3297_gb300 import binding as B

    vy2 = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    vz3 = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]
    for lat, dims, axis_v, L in [(B.LBMRV_D2Q9, (7, 5, 1), vy2, 7),
                                 (B.LBMRV_D3Q19, (3, 4, 6), vz3, 12)]:
        m = dims[1] if lat == B.LBMRV_D2Q9 else dims[2]
        n = L * m
        q = len(axis_v)
        assert B.lbmrv_halo_count(lat, dims) == sum(v == 1 for v in axis_v) * L
        for side, (send_layer, send_c, recv_layer, recv_c) in enumerate(
                [(1, -1, 0, 1), (m - 2, 1, m - 1, -1)]):
            send, recv = B.lbmrv_halo_map(lat, dims, side)
            for idx, layer, c in ((send, send_layer, send_c), (recv, recv_layer, recv_c)):
                assert idx.min() >= 0 and idx.max() < q * n
                j, rest = idx // n, idx % n
                assert all(axis_v[k] == c for k in j)
                assert np.all(rest // L == layer)
                assert sorted(set(j)) == [k for k in range(q) if axis_v[k] == c]
        assert B.lbmrv_halo_count(lat, dims[:1] + (2,) + dims[2:]
                                  if lat == B.LBMRV_D2Q9 else dims[:2] + (2,)) == -1


def test_adjoint_halo_maps_run_the_other_way():
    """The adjoint exchange feeds the reverse step's gathers, mu(x + c_j): through the lower
    face a slab sends layer 1's c = +1 populations and receives c = -1 populations into
    layer 0; through the upper face it sends layer m-2's c = -1 populations and receives
    c = +1 populations into layer m-1. So what the lower face sends is what the lower
    neighbour's upper face receives (the same populations), as in the forward exchange."""
    sys.path.insert(0, ROOT)
    from paper_1312_3297_gb300 import binding as B

    vy2 = [0, 0, 1, 0, -1, 1, 1, -1, -1]
    vz3 = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]
    for lat, dims, axis_v, L in [(B.LBMRV_D2Q9, (7, 5, 1), vy2, 7),
                                 (B.LBMRV_D3Q19, (3, 4, 6), vz3, 12)]:
        m = dims[1] if lat == B.LBMRV_D2Q9 else dims[2]
        n = L * m
        maps = [B.lbmrv_halo_map_adjoint(lat, dims, side) for side in (0, 1)]
        expect = [(1, +1, 0, -1), (m - 2, -1, m - 1, +1)]
        for (send, recv), (sl, sc, rl, rc) in zip(maps, expect):
            for idx, layer, c in ((send, sl, sc), (recv, rl, rc)):
                j, rest = idx // n, idx % n
                assert all(axis_v[k] == c for k in j)
                assert np.all(rest // L == layer)
                assert np.all(rest % L == np.tile(np.arange(L), len(set(j))))
        # the buffer sent through one face is received through the other face of the
        # neighbour: the same populations in the same order
        assert np.array_equal(maps[0][0] // n, maps[1][1] // n)
        assert np.array_equal(maps[1][0] // n, maps[0][1] // n)
