"""Slab-decomposed stepping on one GPU, through the C ABI: two slab handles of one periodic
lattice exchange their face buffers with one device copy per buffer before every step
(lbmrv_halo_pack, cudaMemcpyAsync, lbmrv_halo_unpack, lbmrv_step). The stitched own
layers must equal the single-handle run bit for bit (same reference, same kernels, same
per-node arithmetic), stay within the FP32 tolerance of the FP64 oracle, and the slabs'
conserved sums must add up to the single handle's."""
import numpy as np
import pytest

import lbm_inputs as inp
from pairs import S3, S_PAPER, f32_fields, oracle_run, oracle_run3

pytestmark = pytest.mark.gpu
AMP, PERIOD = 0.03, 40.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _two_slabs(cls, dims, s, mode, storage, fields, ut0=None):
    """Two slab handles (ranks 0 and 1 of the library's plan) initialised from the global
    fields, sharing the reference of the summed flow sums. fields: rho (layers first) and
    the d velocity components, as float32 numpy arrays of the global lattice."""
    import torch

    from paper_1312_3297_gb300 import binding as B

    extent = dims[-1]
    slabs = []
    for rank in range(2):
        first, count = B.lbmrv_slab_plan(extent, 2, rank)
        layers = [(first - 1 + k) % extent for k in range(count + 2)]
        local = tuple(dims[:-1]) + (count + 2,)
        sim = cls(*local, s, mode=mode, storage=storage)
        B.lbmrv_set_slab(sim.h, first, extent)
        if mode == "prescribed":
            sim.set_utilde(None if ut0 is None else
                           torch.as_tensor(np.ascontiguousarray(ut0[:, layers])), AMP, PERIOD)
        rho = torch.as_tensor(np.ascontiguousarray(fields[0][layers]), device="cuda")
        u = torch.stack([torch.as_tensor(np.ascontiguousarray(c[layers]), device="cuda")
                         for c in fields[1:]]).contiguous()
        n_face = B.lbmrv_halo_count(cls.LATTICE, local + (1,) * (3 - len(local)))
        bufs = [torch.empty(n_face, dtype=sim.dtype, device="cuda") for _ in range(4)]
        slabs.append(dict(sim=sim, rho=rho, u=u, bufs=bufs, first=first, count=count))
    sums = [sum(v) for v in zip(*(B.lbmrv_flow_sums(sl["sim"].h, sl["rho"], sl["u"])
                                  for sl in slabs))]
    for sl in slabs:
        B.lbmrv_set_reference_sums(sl["sim"].h, sl["sim"].rho_ref, sums)
        sl["sim"].init_equilibrium(sl["rho"], *sl["u"])
    return slabs, sums


def _run_slabs(slabs, steps):
    from paper_1312_3297_gb300 import binding as B

    a, b = slabs
    for _ in range(steps):
        for sl in slabs:  # send_lo, send_hi
            B.lbmrv_halo_pack(sl["sim"].h, sl["bufs"][0], sl["bufs"][1])
        # one device copy per buffer: a's upper face to b's lower halo and so on (periodic)
        a["bufs"][2].copy_(b["bufs"][1])  # a.recv_lo <- b.send_hi
        a["bufs"][3].copy_(b["bufs"][0])  # a.recv_hi <- b.send_lo
        b["bufs"][2].copy_(a["bufs"][1])
        b["bufs"][3].copy_(a["bufs"][0])
        for sl in slabs:
            B.lbmrv_halo_unpack(sl["sim"].h, sl["bufs"][2], sl["bufs"][3])
            sl["sim"].step(1)


def _single(cls, dims, s, mode, storage, fields, sums, ut0=None):
    import torch

    from paper_1312_3297_gb300 import binding as B

    sim = cls(*dims, s, mode=mode, storage=storage)
    B.lbmrv_set_reference_sums(sim.h, sim.rho_ref, sums)
    if mode == "prescribed":
        sim.set_utilde(None if ut0 is None else torch.as_tensor(ut0), AMP, PERIOD)
    sim.init_equilibrium(*(torch.as_tensor(f, device="cuda") for f in fields))
    return sim


@pytest.mark.parametrize("mode,storage,field", [("fluid", "fp32", False),
                                                ("prescribed", "fp32", False),
                                                ("prescribed", "fp32", True),
                                                ("zero", "fp32", False),
                                                ("fluid", "fp16", False),
                                                ("prescribed", "bf16", False)])
def test_two_d2q9_slabs_equal_the_single_handle(mode, storage, field):
    """64^2, 100 steps. The analytic prescribed field is evaluated at each slab's global
    rows (lbmrv_set_slab); a caller field is given per slab, halo rows included."""
    import torch

    from paper_1312_3297_gb300 import D2Q9

    nx = ny = 64
    rho, ux, uy = (a.astype(np.float32) for a in f32_fields(inp.random_sine_flow(nx, ny, seed=7)))
    ut0 = (inp.to_f32_exact(inp.prescribed_base_field(nx, ny, seed=8, smooth=False))
           .astype(np.float32) if field else None)
    slabs, sums = _two_slabs(D2Q9, (nx, ny), S_PAPER, mode, storage, (rho, ux, uy), ut0)
    _run_slabs(slabs, 100)
    one = _single(D2Q9, (nx, ny), S_PAPER, mode, storage, (rho, ux, uy), sums, ut0)
    one.step(100)
    want = one.state()
    got = torch.cat([sl["sim"].state()[:, 1:-1] for sl in slabs], dim=1)
    assert torch.equal(got.view(torch.uint8), want.view(torch.uint8))
    c_one = one.conserved3()
    c_slabs = [sum(v) for v in zip(*(sl["sim"].conserved3() for sl in slabs))]
    np.testing.assert_allclose(c_slabs[:3], c_one[:3], rtol=1e-12, atol=1e-9)
    if storage == "fp32":
        m_g = tuple(torch.cat([m[1:-1] for m in ms], dim=0).double().cpu().numpy()
                    for ms in zip(*(sl["sim"].moments() for sl in slabs)))
        _, m_o = oracle_run(nx, ny, S_PAPER, mode, 100, (rho.astype(float), ux.astype(float),
                                                         uy.astype(float)),
                            ut0=ut0, amp=AMP, period=PERIOD)
        e_rho = np.abs(m_g[0] - m_o[0]).max() / np.abs(m_o[0]).max()
        e_u = (np.hypot(m_g[1] - m_o[1], m_g[2] - m_o[2]).max()
               / np.hypot(m_o[1], m_o[2]).max())
        assert e_rho <= 1e-5 and e_u <= 1e-5, (e_rho, e_u)
    for sl in slabs:
        sl["sim"].close()
    one.close()


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_two_d3q19_slabs_equal_the_single_handle(storage):
    """D3Q19 split along z: 24 x 10 x 12, u~ = q/rho, 40 steps."""
    import torch

    from paper_1312_3297_gb300 import D3Q19

    nx, ny, nz = 24, 10, 12
    d = inp.random_flow_3d(nx, ny, nz, seed=9)
    rho = inp.to_f32_exact(d["rho"]).astype(np.float32)
    u = inp.to_f32_exact(d["u"]).astype(np.float32)
    slabs, sums = _two_slabs(D3Q19, (nx, ny, nz), S3, "fluid", storage, (rho, *u))
    _run_slabs(slabs, 40)
    one = _single(D3Q19, (nx, ny, nz), S3, "fluid", storage, (rho, *u), sums)
    one.step(40)
    want = one.state()
    got = torch.cat([sl["sim"].state()[:, 1:-1] for sl in slabs], dim=1)
    assert torch.equal(got.view(torch.uint8), want.view(torch.uint8))
    if storage == "fp32":
        r_g = torch.cat([sl["sim"].moments()[0][1:-1] for sl in slabs]).double().cpu().numpy()
        _, r_o, _ = oracle_run3(S3, "fluid", 40, rho.astype(float), u.astype(float))
        assert np.abs(r_g - r_o).max() / np.abs(r_o).max() <= 1e-5
    for sl in slabs:
        sl["sim"].close()
    one.close()


def test_slab_driver_one_rank_is_its_own_neighbour():
    """The Slab driver with one rank (no process group): the lattice wraps onto itself
    through the exchange and equals the single handle bit for bit."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B
    from paper_1312_3297_gb300.slab import Slab

    nx, ny = 96, 40
    rho, ux, uy = (a.astype(np.float32) for a in f32_fields(inp.random_sine_flow(nx, ny, seed=5)))
    sl = Slab(D2Q9, (nx, ny), S_PAPER, mode="fluid", storage="fp16")
    sl.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    sl.step(60)
    rho_ref, U, automatic = B.lbmrv_get_reference(sl.sim.h)
    assert not automatic
    one = D2Q9(nx, ny, S_PAPER, mode="fluid", storage="fp16", u_ref=U[:2])
    one.init_equilibrium(*(torch.as_tensor(a, device="cuda") for a in (rho, ux, uy)))
    one.step(60)
    assert torch.equal(sl.own_state().view(torch.uint8), one.state().view(torch.uint8))
    np.testing.assert_allclose(sl.conserved3()[:3], one.conserved3()[:3], rtol=1e-12)
    sl.close()
    one.close()


def test_slab_calls_reject_misuse():
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B

    sim = D2Q9(16, 2, S_PAPER, mode="fluid")
    with pytest.raises(B.LbmrvError):  # fewer than 3 layers
        B.lbmrv_set_slab(sim.h, 0, 8)
    sim.close()
    sim = D2Q9(16, 6, S_PAPER, mode="fluid")
    buf = torch.empty(48, device="cuda")
    with pytest.raises(B.LbmrvError):  # not a slab yet
        B.lbmrv_halo_pack(sim.h, buf, buf)
    for first, extent in [(-1, 8), (8, 8), (0, 3)]:
        with pytest.raises(B.LbmrvError):
            B.lbmrv_set_slab(sim.h, first, extent)
    B.lbmrv_set_slab(sim.h, 2, 8)
    d = inp.random_sine_flow(16, 6, seed=1)
    sim.set_reference_auto()
    with pytest.raises(B.LbmrvError):  # a slab needs the shared reference
        sim.init_equilibrium(*(torch.as_tensor(d[k], dtype=torch.float32)
                               for k in ("rho", "ux", "uy")))
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    with pytest.raises(B.LbmrvError) as ei:  # it would step without the exchanges
        B.lbmrv_forward_checkpointed(sim.h, 4, 2, ws, ws.numel())
    assert ei.value.status == B.LBMRV_E_UNSUPPORTED
    sim.close()


def _single_gradient(nx, ny, mode, steps, seg, fields, u_ref, ut0=None):
    """Kinetic-energy gradient of the single handle (lbmrv_forward_checkpointed +
    lbmrv_adjoint) with a fixed reference: (L, dL/du0 [2, ny, nx], dL/ds, dL/dA)."""
    import torch

    from paper_1312_3297_gb300 import D2Q9

    sim = D2Q9(nx, ny, S_PAPER, mode=mode, u_ref=u_ref)
    if mode == "prescribed":
        sim.set_utilde(None if ut0 is None else torch.as_tensor(ut0), AMP, PERIOD)
    rho = torch.as_tensor(fields[0], device="cuda")
    u = torch.stack([torch.as_tensor(c, device="cuda") for c in fields[1:]]).contiguous()
    sim.init_equilibrium(rho, u[0], u[1])
    ws = sim.adjoint_workspace(steps, seg)
    sim.forward_checkpointed(steps, seg, ws)
    ke, dlds = sim.kinetic_energy(grad=True)
    d0, ds, da, _ = sim.adjoint(steps, seg, ws, dlds)
    _, du0 = sim.equilibrium_vjp(rho, u, d0)
    out = (ke, du0.cpu().numpy(), ds, da)
    sim.close()
    return out


@pytest.mark.parametrize("mode", ["fluid", "prescribed", "zero"])
def test_slab_driver_gradient_equals_the_single_handle(mode):
    """The Slab driver's reverse sweep (one rank, its own neighbour; checkpoints every 6
    steps with recomputation; adjoint exchanges before every gather) against the single
    handle's lbmrv_adjoint: dL/du0 bit for bit (the same per-node arithmetic), the loss and
    the parameter gradients (sums in another order) to 1e-9 and 1e-6."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B
    from paper_1312_3297_gb300.slab import Slab

    nx, ny, steps, seg = 64, 40, 40, 6
    rho, ux, uy = (a.astype(np.float32) for a in f32_fields(inp.noisy_shear_wave(nx, ny, seed=2)))
    sl = Slab(D2Q9, (nx, ny), S_PAPER, mode=mode)
    if mode == "prescribed":
        sl.sim.set_utilde(None, AMP, PERIOD)
    sl.init_equilibrium(torch.as_tensor(rho), torch.as_tensor(ux), torch.as_tensor(uy))
    ke, du0, ds, da = sl.kinetic_energy_gradient(steps, seg)
    U = B.lbmrv_get_reference(sl.sim.h)[1][:2]
    assert sl.time == steps
    sl.close()
    ke1, du1, ds1, da1 = _single_gradient(nx, ny, mode, steps, seg, (rho, ux, uy), U)
    np.testing.assert_array_equal(du0.cpu().numpy(), du1)
    assert abs(ke - ke1) <= 1e-9 * abs(ke1)
    np.testing.assert_allclose(ds, ds1, rtol=1e-6, atol=1e-12)
    assert abs(da - da1) <= 1e-6 * max(abs(da1), 1e-30)


def test_two_slab_handles_reverse_sweep_equals_the_single_handle():
    """Two slab handles on one GPU (64^2, rows 32 + 32) run the forward steps with the
    forward exchange and the reverse sweep with the adjoint exchange, one device copy per
    face buffer each way, every state checkpointed: dL/du0 of the stitched own rows equals
    the single handle's bit for bit; dL/ds and dL/dA, summed over the slabs, to 1e-6."""
    import torch

    from paper_1312_3297_gb300 import D2Q9, binding as B

    nx = ny = 64
    steps = 30
    rho, ux, uy = (a.astype(np.float32) for a in f32_fields(inp.noisy_shear_wave(nx, ny, seed=3)))
    slabs, sums = _two_slabs(D2Q9, (nx, ny), S_PAPER, "prescribed", "fp32", (rho, ux, uy))
    a, b = slabs
    states = {0: [], 1: []}
    for _ in range(steps):  # forward, keeping every state as its step reads it
        for sl in slabs:
            B.lbmrv_halo_pack(sl["sim"].h, sl["bufs"][0], sl["bufs"][1])
        a["bufs"][2].copy_(b["bufs"][1])
        a["bufs"][3].copy_(b["bufs"][0])
        b["bufs"][2].copy_(a["bufs"][1])
        b["bufs"][3].copy_(a["bufs"][0])
        for r, sl in enumerate(slabs):
            B.lbmrv_halo_unpack(sl["sim"].h, sl["bufs"][2], sl["bufs"][3])
            states[r].append(sl["sim"].state())
            sl["sim"].step(1)
    grads = []
    for sl in slabs:
        ke, dlds = sl["sim"].kinetic_energy(grad=True)
        acc = torch.zeros(B.lbmrv_adjoint_acc_doubles(sl["sim"].h), dtype=torch.float64,
                          device="cuda")
        mu = [torch.empty_like(dlds) for _ in range(2)]
        abuf = [torch.empty(3 * nx, device="cuda") for _ in range(4)]
        grads.append(dict(ke=ke, a=dlds, acc=acc, mu=mu, abuf=abuf, pp=0))

    def adjoint_exchange():
        for sl, gr in zip(slabs, grads):
            B.lbmrv_halo_pack_adjoint(sl["sim"].h, gr["a"], gr["abuf"][0], gr["abuf"][1])
        ga, gb = grads
        ga["abuf"][2].copy_(gb["abuf"][1])  # a.recv_lo <- b.send_hi
        ga["abuf"][3].copy_(gb["abuf"][0])  # a.recv_hi <- b.send_lo
        gb["abuf"][2].copy_(ga["abuf"][1])
        gb["abuf"][3].copy_(ga["abuf"][0])
        for sl, gr in zip(slabs, grads):
            B.lbmrv_halo_unpack_adjoint(sl["sim"].h, gr["a"], gr["abuf"][2], gr["abuf"][3])

    for k in range(steps, 0, -1):
        if k < steps:
            adjoint_exchange()
        for r, (sl, gr) in enumerate(zip(slabs, grads)):
            out = gr["mu"][gr["pp"]]
            B.lbmrv_adjoint_step(sl["sim"].h, states[r][k - 1], k, gr["a"], k < steps, out,
                                 gr["acc"])
            gr["a"], gr["pp"] = out, gr["pp"] ^ 1
    adjoint_exchange()
    du, ds, da, ke = [], np.zeros(9), 0.0, 0.0
    for sl, gr in zip(slabs, grads):
        d0 = torch.empty_like(gr["a"])
        B.lbmrv_adjoint_gather(sl["sim"].h, gr["a"], d0)
        _, g = sl["sim"].equilibrium_vjp(sl["rho"], sl["u"], d0)
        du.append(g[:, 1:-1])
        s_, a_ = B.lbmrv_adjoint_acc_sum(sl["sim"].h, gr["acc"])
        ds += np.asarray(s_)
        da += a_
        ke += gr["ke"]
    du = torch.cat(du, dim=1).cpu().numpy()
    U = B.lbmrv_get_reference(a["sim"].h)[1][:2]
    for sl in slabs:
        sl["sim"].close()
    ke1, du1, ds1, da1 = _single_gradient(nx, ny, "prescribed", steps, 1, (rho, ux, uy), U)
    np.testing.assert_array_equal(du, du1)
    assert abs(ke - ke1) <= 1e-9 * abs(ke1)
    np.testing.assert_allclose(ds, ds1, rtol=1e-6, atol=1e-12)
    assert abs(da - da1) <= 1e-6 * abs(da1)
