"""A periodic lattice split into slabs along its last axis, one slab per torch.distributed
rank (or several slab handles driven by one process).

Each rank owns a handle whose lattice holds its own layers plus one halo layer on each
side (include/lbmrv.h, slab decomposition). A step is: pack the edge layers' crossing
populations (a library kernel), exchange the face buffers with the two neighbouring ranks
(point-to-point send/recv: NCCL for CUDA tensors, gloo for CPU tensors), unpack them into
the halo layers (a library kernel), and the ordinary fused step. The conserved sums and
the mean-flow reference are FP64 sums over each rank's own layers, all-reduced. Which
layers a rank owns and which values cross each face come from the library's host-side
plan and index maps. This module only moves buffers between ranks and calls the library.
"""
from __future__ import annotations

import math

import torch

from . import binding as B

# message tags: the buffer sent through the upper face arrives through the neighbour's
# lower face, and vice versa
_TAG_UP, _TAG_DOWN = 0, 1


def exchange_faces(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None):
    """Swap face buffers with the neighbouring ranks of a periodic chain: recv_lo gets the
    lower neighbour's send_hi, recv_hi the upper neighbour's send_lo. With one rank the
    lattice is its own neighbour on both sides."""
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return
    import torch.distributed as dist

    up, down = (rank + 1) % world, (rank - 1) % world
    ops = [dist.P2POp(dist.isend, send_hi, up, group, _TAG_UP),
           dist.P2POp(dist.isend, send_lo, down, group, _TAG_DOWN),
           dist.P2POp(dist.irecv, recv_lo, down, group, _TAG_UP),
           dist.P2POp(dist.irecv, recv_hi, up, group, _TAG_DOWN)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()


def allreduce_sums(values, world: int, device, group=None):
    """FP64 sum of a short list of values over the ranks."""
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist

        dist.all_reduce(t, group=group)
    return [float(v) for v in t.cpu()]


class Slab:
    """Rank `rank` of `world` slabs of a periodic lattice of global dims (nx, ny) (D2Q9 and
    D2Q9Cascaded, split along y) or (nx, ny, nz) (D3Q19, split along z).

    ``cls`` is D2Q9, D2Q9Cascaded or D3Q19 from ``simulation``; ``kw`` goes to it (mode,
    storage, lam, rho_ref, device, stream)."""

    def __init__(self, cls, dims, s, rank: int = 0, world: int = 1, group=None, **kw):
        dims = tuple(int(v) for v in dims)
        self.cls, self.global_dims = cls, dims
        self.rank, self.world, self.group = int(rank), int(world), group
        self.extent = dims[-1]
        self.first, self.count = B.lbmrv_slab_plan(self.extent, self.world, self.rank)
        local = dims[:-1] + (self.count + 2,)
        kw.pop("u_ref", None)  # the reference is the global mean flow, set at init
        self.sim = cls(*local, s, **kw)
        B.lbmrv_set_slab(self.sim.h, self.first, self.extent)
        n_face = B.lbmrv_halo_count(cls.LATTICE, local + (1,) * (3 - len(local)))
        dev, dt = self.sim.device, self.sim.dtype
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = (
            torch.empty(n_face, dtype=dt, device=dev) for _ in range(4))
        # the adjoint exchange's buffers (FP32 adjoint vectors)
        self.a_send_lo, self.a_send_hi, self.a_recv_lo, self.a_recv_hi = (
            torch.empty(n_face, dtype=torch.float32, device=dev) for _ in range(4))
        self._fields = None

    # -- lifecycle
    def close(self):
        self.sim.close()

    @property
    def time(self) -> int:
        return self.sim.time

    # -- fields: the rank's own layers, shaped (..., count, ...) like the lattice
    def _with_halo(self, t):
        """Own layers plus a halo layer on each side (copies of the edge layers: finite
        placeholders, replaced by the first exchange)."""
        return torch.cat([t[-1:], t, t[:1]], dim=0).contiguous()  # layers lead

    def init_equilibrium(self, rho_own, *u_own):
        """rho_own: the own layers' density (layers first .. first+count-1), u_own: the d
        velocity components likewise. The stored reference is the global mean flow: FP64
        sums over each rank's own layers, all-reduced."""
        dev = self.sim.device
        rho = self._with_halo(torch.as_tensor(rho_own, dtype=torch.float32, device=dev))
        u = torch.stack([self._with_halo(torch.as_tensor(c, dtype=torch.float32, device=dev))
                         for c in u_own]).contiguous()
        sums = allreduce_sums(B.lbmrv_flow_sums(self.sim.h, rho, u), self.world,
                              self._comm_device(), self.group)
        B.lbmrv_set_reference_sums(self.sim.h, self.sim.rho_ref, sums)
        self.sim.init_equilibrium(rho, *u)
        self._fields = (rho, u)  # for the adjoint of the initialisation

    def _comm_device(self):
        import torch.distributed as dist

        if self.world > 1 and dist.get_backend(self.group) == "nccl":
            return self.sim.device
        return torch.device("cpu")

    # -- stepping
    def exchange(self):
        if self.world == 1:  # its own neighbour: pack straight into the other face's halo
            B.lbmrv_halo_pack(self.sim.h, self.recv_hi, self.recv_lo)
        else:
            B.lbmrv_halo_pack(self.sim.h, self.send_lo, self.send_hi)
            exchange_faces(self.send_lo, self.send_hi, self.recv_lo, self.recv_hi, self.rank,
                           self.world, self.group)
        B.lbmrv_halo_unpack(self.sim.h, self.recv_lo, self.recv_hi)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange()
            self.sim.step(1)

    def exchange_adjoint(self, mu):
        """Fill the halo layers of the adjoint vector mu (FP32, the state's shape) with the
        neighbours' values that the reverse step's gathers read."""
        h = self.sim.h
        if self.world == 1:  # its own neighbour: pack straight into the other face's halo
            B.lbmrv_halo_pack_adjoint(h, mu, self.a_recv_hi, self.a_recv_lo)
        else:
            B.lbmrv_halo_pack_adjoint(h, mu, self.a_send_lo, self.a_send_hi)
            exchange_faces(self.a_send_lo, self.a_send_hi, self.a_recv_lo, self.a_recv_hi,
                           self.rank, self.world, self.group)
        B.lbmrv_halo_unpack_adjoint(h, mu, self.a_recv_lo, self.a_recv_hi)

    def kinetic_energy_gradient(self, n: int, seg: int = 0):
        """Advance n steps from the state set by init_equilibrium (time 0) with a checkpoint
        every seg steps (sqrt(n) when 0), and return the kinetic energy L of the final state
        and its gradients: (L, dL/du0 of the own layers [d, count, ...], dL/ds [q], dL/dA).
        L, dL/ds and dL/dA are FP64 sums over the slabs (all-reduced). The reverse sweep
        recomputes each segment from its checkpoint, with the forward exchanges, and
        exchanges the adjoint vector before each gather. The handle ends at the final
        state (time n)."""
        sim, h = self.sim, self.sim.h
        if self._fields is None or sim.time != 0:
            raise ValueError("kinetic_energy_gradient starts from init_equilibrium (time 0)")
        n = int(n)
        seg = int(seg) if seg else max(1, int(math.ceil(math.sqrt(n))))
        # forward: checkpoints are the states as the steps read them (halos exchanged)
        ck = []
        for k in range(1, n + 1):
            self.exchange()
            if (k - 1) % seg == 0:
                ck.append(sim.state())
            sim.step(1)
        final = sim.state()
        ke, dlds = sim.kinetic_energy(grad=True)
        dev = sim.device
        acc = torch.zeros(B.lbmrv_adjoint_acc_doubles(h), dtype=torch.float64, device=dev)
        mu = [torch.empty_like(dlds) for _ in range(2)]
        a, gather, pp = dlds, False, 0
        for c in range(len(ck) - 1, -1, -1):
            base = c * seg
            khi = min(base + seg, n)
            states = [ck[c]]
            if khi - base > 1:  # recompute the segment's states, with their exchanges
                sim.set_state(ck[c], base)
                for _ in range(base + 1, khi):
                    sim.step(1)
                    self.exchange()
                    states.append(sim.state())
            for k in range(khi, base, -1):
                if gather:
                    self.exchange_adjoint(a)
                B.lbmrv_adjoint_step(h, states[k - 1 - base], k, a, gather, mu[pp], acc)
                a, gather, pp = mu[pp], True, pp ^ 1
        self.exchange_adjoint(a)
        d0 = torch.empty_like(dlds)
        B.lbmrv_adjoint_gather(h, a, d0)
        ds, da = B.lbmrv_adjoint_acc_sum(h, acc)
        rho, u = self._fields
        _, du = sim.equilibrium_vjp(rho, u, d0)
        sim.set_state(final, n)
        tot = allreduce_sums([ke] + list(ds) + [da], self.world, self._comm_device(),
                             self.group)
        return tot[0], du[:, 1:-1].contiguous(), tot[1:1 + len(ds)], tot[-1]

    # -- results
    def conserved3(self):
        """Global [sum rho, sum q_x, sum q_y, sum q_z, non-finite nodes]: FP64 sums over
        each rank's own layers, all-reduced."""
        own = self.sim.conserved3(allow_nonfinite=True)
        return allreduce_sums(own, self.world, self._comm_device(), self.group)

    def own_state(self) -> torch.Tensor:
        """The stored state of the own layers, shape (q, count, ...) along the slab axis."""
        g = self.sim.state()
        return g[:, 1:-1].contiguous()

    def own_moments(self):
        """rho and the velocity components of the own layers."""
        return tuple(t[1:-1] for t in self.sim.moments())
