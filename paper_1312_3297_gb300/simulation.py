"""Convenience wrapper around one lbmrv handle, with PyTorch owning the device memory.

``D2Q9`` allocates the two population buffers as torch tensors on the current CUDA
device, enqueues on torch's current stream, and forwards every operation to the C
entry points of ``binding``. It does no arithmetic of its own.
"""
from __future__ import annotations

import torch

from . import binding as B

_MODES = {"zero": B.LBMRV_UT_ZERO, "fluid": B.LBMRV_UT_FLUID,
          "prescribed": B.LBMRV_UT_PRESCRIBED}
_STORAGES = {"fp32": B.LBMRV_FP32, "fp16": B.LBMRV_FP16, "bf16": B.LBMRV_BF16}
STORAGE_DTYPES = {B.LBMRV_FP32: torch.float32, B.LBMRV_FP16: torch.float16,
                  B.LBMRV_BF16: torch.bfloat16}


def mode_id(mode) -> int:
    return _MODES[mode] if isinstance(mode, str) else int(mode)


def storage_id(storage) -> int:
    return _STORAGES[storage] if isinstance(storage, str) else int(storage)


class D2Q9:
    """A periodic nx x ny D2Q9 lattice advanced by the relative-velocity scheme.

    The stored state is g = f - f_eq(rho_ref, u_ref). With ``u_ref=None`` (the default)
    the library sets u_ref at each init_equilibrium to the mean flow of the fields it is
    given; a tuple fixes it ((0, 0) is the plain form g = f - w rho_ref)."""

    LATTICE = B.LBMRV_D2Q9
    Q = 9
    DIM = 2

    def __init__(self, nx: int, ny: int, s, mode="fluid", storage="fp32", lam: float = 1.0,
                 rho_ref: float | None = None, device=None, stream=None, u_ref=None, nz: int = 1):
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz
        self.shape = (self.ny, self.nx) if self.DIM == 2 else (self.nz, self.ny, self.nx)
        self.mode = mode_id(mode)
        self.storage = storage_id(storage)
        self.lam = float(lam)
        if rho_ref is None:
            rho_ref = 1.0  # store deviations from the rest state: smaller rounding error
        self.rho_ref = float(rho_ref)
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        dims = (self.nx, self.ny, self.nz)
        nbytes = B.lbmrv_state_bytes(self.LATTICE, dims, self.storage)
        if nbytes <= 0:
            raise ValueError(f"invalid lattice {dims}")
        self._bufs = [torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                      for _ in range(2)]
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.h = B.lbmrv_create(self.LATTICE, dims, self.lam, list(s), self.mode,
                                    self.storage, self.rho_ref, self.stream,
                                    self._bufs[0], self._bufs[1])
        if u_ref is not None:
            B.lbmrv_set_reference(self.h, self.rho_ref, tuple(float(v) for v in u_ref))
        self._ut0 = None
        self.s = [float(v) for v in s]
        self.amp, self.period = 0.0, 0.0
        self.dtype = STORAGE_DTYPES[self.storage]

    # -- stream order between torch's current stream and the handle's stream
    def _sync_in(self):
        """The handle's stream waits for work already queued on torch's current stream
        (inputs that torch produced)."""
        cur = torch.cuda.current_stream(self.device)
        if isinstance(self.stream, torch.cuda.Stream) and cur != self.stream:
            self.stream.wait_stream(cur)

    def _sync_out(self):
        """Torch's current stream waits for the handle's queued work (outputs torch will
        read)."""
        cur = torch.cuda.current_stream(self.device)
        if isinstance(self.stream, torch.cuda.Stream) and cur != self.stream:
            cur.wait_stream(self.stream)

    # -- lifecycle
    def close(self):
        if getattr(self, "h", None):
            B.lbmrv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- configuration
    @property
    def u_ref(self) -> tuple:
        """Reference velocity of the stored deviations (d components, physical units)."""
        return B.lbmrv_get_reference(self.h)[1][:self.DIM]

    def set_reference(self, rho_ref: float, u_ref):
        """Fix the reference state (turns the automatic choice off)."""
        B.lbmrv_set_reference(self.h, rho_ref, tuple(float(v) for v in u_ref))
        self.rho_ref = float(rho_ref)

    def set_reference_auto(self, rho_ref: float | None = None):
        """Let each init_equilibrium take u_ref from the mean flow of its fields."""
        if rho_ref is not None:
            self.rho_ref = float(rho_ref)
        B.lbmrv_set_reference_auto(self.h, self.rho_ref)

    def set_kernel_width(self, nodes_per_thread: int):
        B.lbmrv_set_kernel_width(self.h, nodes_per_thread)

    def set_rates(self, s):
        B.lbmrv_set_rates(self.h, list(s))
        self.s = [float(v) for v in s]

    def set_utilde(self, ut0=None, amplitude: float = 0.0, period: float = 0.0):
        self.amp, self.period = float(amplitude), float(period)
        if ut0 is not None:
            ut0 = torch.as_tensor(ut0, dtype=torch.float32, device=self.device).contiguous()
            if ut0.numel() != self.DIM * self.n:
                raise ValueError(f"u~0 must hold {self.DIM} * n values")
        self._ut0 = ut0  # keep the field alive while the handle refers to it
        self._sync_in()
        B.lbmrv_set_utilde(self.h, ut0, amplitude, period)

    # -- state
    def init_equilibrium(self, rho, *u_components):
        """rho and the d velocity components, each shaped like the lattice."""
        if len(u_components) != self.DIM:
            raise ValueError(f"expected {self.DIM} velocity components")
        rho = torch.as_tensor(rho, dtype=torch.float32, device=self.device).contiguous()
        u = torch.stack([torch.as_tensor(c, dtype=torch.float32, device=self.device)
                         for c in u_components]).contiguous()
        self._sync_in()
        B.lbmrv_init_equilibrium(self.h, rho, u)
        self._keep = (rho, u)  # the copy is asynchronous on the stream

    def init_equilibrium_host(self, rho_host, u_host):
        """rho_host: CPU float32 [n] (pinned for speed); u_host: CPU float32 [2, n]."""
        B.lbmrv_init_equilibrium_host(self.h, rho_host, u_host)

    def step(self, n: int = 1):
        B.lbmrv_step(self.h, n)

    @property
    def time(self) -> int:
        return B.lbmrv_time(self.h)

    def moments(self):
        """rho and the d velocity components (device tensors shaped like the lattice)."""
        rho = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        u = torch.empty((self.DIM,) + self.shape, dtype=torch.float32, device=self.device)
        B.lbmrv_moments(self.h, rho, u)
        self._sync_out()
        return (rho,) + tuple(u[a] for a in range(self.DIM))

    def moments_host(self, rho_host=None, u_host=None):
        if rho_host is None:
            rho_host = torch.empty(self.shape, dtype=torch.float32, pin_memory=True)
        if u_host is None:
            u_host = torch.empty((self.DIM,) + self.shape, dtype=torch.float32,
                                 pin_memory=True)
        B.lbmrv_moments_host(self.h, rho_host, u_host)
        return rho_host, u_host

    def conserved(self, allow_nonfinite: bool = False):
        """[sum rho, sum q_x, sum q_y, non-finite nodes] (D2Q9 layout)."""
        return B.lbmrv_conserved(self.h, allow_nonfinite=allow_nonfinite)

    def conserved3(self, allow_nonfinite: bool = False):
        """[sum rho, sum q_x, sum q_y, sum q_z, non-finite nodes]."""
        return B.lbmrv_conserved3(self.h, allow_nonfinite=allow_nonfinite)

    def step_conserved(self, n: int = 1, allow_nonfinite: bool = False):
        """n steps, the last with the sums of conserved3() of its result taken in the same
        kernel (D2Q9 vector widths, D3Q19 default widths; otherwise a separate pass)."""
        return B.lbmrv_step_conserved(self.h, n, allow_nonfinite=allow_nonfinite)

    def state(self) -> torch.Tensor:
        """Copy of the stored state g = f - f_eq(rho_ref, u_ref), shape (9, ny, nx), in the
        storage dtype."""
        out = torch.empty((self.Q,) + self.shape, dtype=self.dtype, device=self.device)
        B.lbmrv_get_state(self.h, out)
        self._sync_out()
        return out

    def set_state(self, g: torch.Tensor, t: int = 0):
        g = g.to(device=self.device, dtype=self.dtype).contiguous()
        if g.numel() != self.Q * self.n:
            raise ValueError(f"state must hold {self.Q} * n values")
        self._sync_in()
        B.lbmrv_set_state(self.h, g, t)
        self._keep = g

    def state_ptr(self) -> int:
        return B.lbmrv_state_ptr(self.h)

    # -- adjoint (FP32 storage)
    def adjoint_workspace(self, n: int, seg: int) -> torch.Tensor:
        nbytes = B.lbmrv_adjoint_workspace_bytes(self.h, n, seg)
        if nbytes <= 0:
            raise ValueError(f"invalid adjoint window n={n}, seg={seg}")
        return torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def forward_checkpointed(self, n: int, seg: int, ws: torch.Tensor):
        B.lbmrv_forward_checkpointed(self.h, n, seg, ws, ws.numel())

    def adjoint(self, n: int, seg: int, ws: torch.Tensor, dL_dS: torch.Tensor,
                field_grad: bool = False):
        """Reverse sweep of the last forward_checkpointed(n, seg, ws). Returns
        (dL/dS_0 [9, ny, nx], dL/ds [9], dL/dA, dL/du~0 [2, ny, nx] or None)."""
        d0 = torch.empty((9, self.ny, self.nx), dtype=torch.float32, device=self.device)
        dut = (torch.empty((2, self.ny, self.nx), dtype=torch.float32, device=self.device)
               if field_grad else None)
        dL_dS = dL_dS.contiguous()
        if dL_dS.data_ptr() % 16:  # the library reads it in 16-byte packs
            dL_dS = dL_dS.clone()
        self._sync_in()
        ds, da = B.lbmrv_adjoint(self.h, n, seg, ws, ws.numel(), dL_dS, d0, dut)
        self._sync_out()
        return d0, ds, da, dut

    def kinetic_energy(self, grad: bool = False):
        g = (torch.empty((9, self.ny, self.nx), dtype=torch.float32, device=self.device)
             if grad else None)
        ke = B.lbmrv_kinetic_energy(self.h, g)
        self._sync_out()
        return ke, g

    def moments_vjp(self, dL_drho=None, dL_du=None) -> torch.Tensor:
        out = torch.empty((9, self.ny, self.nx), dtype=torch.float32, device=self.device)
        if dL_drho is not None:
            dL_drho = dL_drho.to(torch.float32).contiguous()
        if dL_du is not None:
            dL_du = dL_du.to(torch.float32).contiguous()
        self._sync_in()
        B.lbmrv_moments_vjp(self.h, dL_drho, dL_du, out)
        self._sync_out()
        self._keep = (dL_drho, dL_du)
        return out

    def equilibrium_vjp(self, rho, u, dL_dS0):
        """rho [ny, nx] or None, u [2, ny, nx] (device float32)."""
        drho = torch.empty((self.ny, self.nx), dtype=torch.float32, device=self.device)
        du = torch.empty((2, self.ny, self.nx), dtype=torch.float32, device=self.device)
        rho = None if rho is None else rho.contiguous()
        u, dL_dS0 = u.contiguous(), dL_dS0.contiguous()
        self._sync_in()
        B.lbmrv_equilibrium_vjp(self.h, rho, u, dL_dS0, drho, du)
        self._sync_out()
        self._keep = (rho, u, dL_dS0)
        return drho, du


class D3Q19(D2Q9):
    """A periodic nx x ny x nz D3Q19 lattice advanced by the relative-velocity scheme
    (19 rates in the order of the 3D basis of include/lbmrv.h). No adjoint."""

    LATTICE = B.LBMRV_D3Q19
    Q = 19
    DIM = 3

    def __init__(self, nx: int, ny: int, nz: int, s, **kw):
        super().__init__(nx, ny, s, nz=nz, **kw)


class D2Q9Cascaded(D2Q9):
    """D2Q9 with Geier's cascaded basis and product-form equilibrium (rates in the order
    1, X, Y, X^2+Y^2, X^2-Y^2, XY, XY^2, X^2Y, X^2Y^2). mode="fluid" is Geier's scheme."""

    LATTICE = B.LBMRV_D2Q9_CASCADED
