"""Thin ctypes binding of the lbmrv C ABI (include/lbmrv.h).

Each ``lbmrv_*`` function here has the name, arguments and meaning of the C entry
point; this module only marshals arguments (torch tensors become device or host
pointers, CUDA streams become handles) and turns negative status codes into
``LbmrvError``. All computation runs in the CUDA library; there is no Python or CPU
fallback, and importing fails loudly when the library cannot be built or loaded.
"""
from __future__ import annotations

import ctypes
import threading

from . import build as _build

LBMRV_OK = 0
LBMRV_E_INVAL = -1
LBMRV_E_CUDA = -2
LBMRV_E_NOMEM = -3
LBMRV_E_NONFINITE = -4
LBMRV_E_TIMEOUT = -5
LBMRV_E_UNSUPPORTED = -6

LBMRV_D2Q9 = 0
LBMRV_D3Q19 = 1
LBMRV_D2Q9_CASCADED = 2
LBMRV_UT_ZERO = 0
LBMRV_UT_FLUID = 1
LBMRV_UT_PRESCRIBED = 2
LBMRV_FP32 = 0
LBMRV_FP16 = 1
LBMRV_BF16 = 2

_STATUS_NAMES = {
    LBMRV_E_INVAL: "LBMRV_E_INVAL", LBMRV_E_CUDA: "LBMRV_E_CUDA",
    LBMRV_E_NOMEM: "LBMRV_E_NOMEM", LBMRV_E_NONFINITE: "LBMRV_E_NONFINITE",
    LBMRV_E_TIMEOUT: "LBMRV_E_TIMEOUT", LBMRV_E_UNSUPPORTED: "LBMRV_E_UNSUPPORTED",
}

# (name, restype, argtypes) of every exported entry point.
_VP = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_I64P = ctypes.POINTER(ctypes.c_int64)
SIGNATURES = [
    ("lbmrv_version", _I, []),
    ("lbmrv_state_bytes", _I64, [_I, _I64P, _I]),
    ("lbmrv_create", _I, [ctypes.POINTER(_VP), _I, _I64P, _D, _DP, _I, _I, _D, _VP, _VP, _VP]),
    ("lbmrv_destroy", _I, [_VP]),
    ("lbmrv_last_error", ctypes.c_char_p, [_VP]),
    ("lbmrv_set_stream", _I, [_VP, _VP]),
    ("lbmrv_set_kernel_width", _I, [_VP, _I]),
    ("lbmrv_set_utilde", _I, [_VP, _VP, _D, _D]),
    ("lbmrv_init_equilibrium", _I, [_VP, _VP, _VP]),
    ("lbmrv_init_equilibrium_host", _I, [_VP, _VP, _VP]),
    ("lbmrv_step", _I, [_VP, _I64]),
    ("lbmrv_moments", _I, [_VP, _VP, _VP]),
    ("lbmrv_moments_host", _I, [_VP, _VP, _VP]),
    ("lbmrv_conserved", _I, [_VP, _DP]),
    ("lbmrv_get_state", _I, [_VP, _VP]),
    ("lbmrv_set_state", _I, [_VP, _VP, _I64]),
    ("lbmrv_state_ptr", _I, [_VP, ctypes.POINTER(_VP)]),
    ("lbmrv_time", _I64, [_VP]),
    ("lbmrv_conserved_noalloc", _I, [_VP, _I, _I64P, _D, _D, _VP, _VP]),
    ("lbmrv_set_rates", _I, [_VP, _DP]),
    ("lbmrv_set_reference", _I, [_VP, _D, _DP]),
    ("lbmrv_set_reference_auto", _I, [_VP, _D]),
    ("lbmrv_get_reference", _I, [_VP, _DP, _DP]),
    ("lbmrv_slab_plan", _I, [_I64, _I, _I, _I64P, _I64P]),
    ("lbmrv_halo_count", _I64, [_I, _I64P]),
    ("lbmrv_halo_map", _I, [_I, _I64P, _I, _VP, _VP]),
    ("lbmrv_set_slab", _I, [_VP, _I64, _I64]),
    ("lbmrv_halo_pack", _I, [_VP, _VP, _VP]),
    ("lbmrv_halo_unpack", _I, [_VP, _VP, _VP]),
    ("lbmrv_flow_sums", _I, [_VP, _VP, _VP, _DP]),
    ("lbmrv_set_reference_sums", _I, [_VP, _D, _DP]),
    ("lbmrv_halo_map_adjoint", _I, [_I, _I64P, _I, _VP, _VP]),
    ("lbmrv_halo_pack_adjoint", _I, [_VP, _VP, _VP, _VP]),
    ("lbmrv_halo_unpack_adjoint", _I, [_VP, _VP, _VP, _VP]),
    ("lbmrv_adjoint_acc_doubles", _I64, [_VP]),
    ("lbmrv_adjoint_step", _I, [_VP, _VP, _I64, _VP, _I, _VP, _VP, _VP]),
    ("lbmrv_adjoint_acc_sum", _I, [_VP, _VP, _DP, _DP]),
    ("lbmrv_adjoint_gather", _I, [_VP, _VP, _VP]),
    ("lbmrv_conserved3", _I, [_VP, _DP]),
    ("lbmrv_step_conserved", _I, [_VP, _I64, _DP]),
    ("lbmrv_adjoint_workspace_bytes", _I64, [_VP, _I64, _I64]),
    ("lbmrv_forward_checkpointed", _I, [_VP, _I64, _I64, _VP, ctypes.c_size_t]),
    ("lbmrv_adjoint", _I, [_VP, _I64, _I64, _VP, ctypes.c_size_t, _VP, _VP, _DP, _DP, _VP]),
    ("lbmrv_kinetic_energy", _I, [_VP, _DP, _VP]),
    ("lbmrv_moments_vjp", _I, [_VP, _VP, _VP, _VP]),
    ("lbmrv_equilibrium_vjp", _I, [_VP, _VP, _VP, _VP, _VP, _VP]),
]

_lock = threading.Lock()
_lib = None


class LbmrvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_needed: bool = True) -> ctypes.CDLL:
    """Load liblbmrv.so (building it first when stale). Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_needed else _build.LIB_PATH
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _err(h) -> str:
    msg = load().lbmrv_last_error(h)
    return msg.decode() if msg else ""


def _check(rc: int, h=None) -> int:
    if rc < 0:
        raise LbmrvError(rc, _err(h))
    return rc


def _addr(x) -> int | None:
    """Pointer of a torch tensor (or an int address / None)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_contiguous():
        raise ValueError("lbmrv needs contiguous tensors")
    return x.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s or None
    return s.cuda_stream or None


def _dims(dims) -> ctypes.Array:
    d = list(dims) + [1] * (3 - len(dims))
    return (ctypes.c_int64 * 3)(*d)


# ------------------------------------------------------------------ entry points
def lbmrv_version() -> int:
    return load().lbmrv_version()


def lbmrv_state_bytes(lattice: int, dims, storage: int) -> int:
    return load().lbmrv_state_bytes(lattice, _dims(dims), storage)


def lbmrv_create(lattice: int, dims, lam: float, s, umode: int, storage: int,
                 rho_ref: float, stream=None, f_a=None, f_b=None) -> int:
    h = _VP()
    sv = (ctypes.c_double * len(s))(*[float(v) for v in s])
    rc = load().lbmrv_create(ctypes.byref(h), lattice, _dims(dims), float(lam), sv, umode,
                             storage, float(rho_ref), _stream(stream), _addr(f_a), _addr(f_b))
    _check(rc, None)
    return h.value


def lbmrv_destroy(h) -> None:
    _check(load().lbmrv_destroy(h), None)


def lbmrv_last_error(h) -> str:
    return _err(h)


def lbmrv_set_stream(h, stream) -> None:
    _check(load().lbmrv_set_stream(h, _stream(stream)), h)


def lbmrv_set_kernel_width(h, nodes_per_thread: int) -> None:
    _check(load().lbmrv_set_kernel_width(h, int(nodes_per_thread)), h)


def lbmrv_set_utilde(h, ut0, amplitude: float, period: float) -> None:
    _check(load().lbmrv_set_utilde(h, _addr(ut0), float(amplitude), float(period)), h)


def lbmrv_init_equilibrium(h, rho, u) -> None:
    _check(load().lbmrv_init_equilibrium(h, _addr(rho), _addr(u)), h)


def lbmrv_init_equilibrium_host(h, rho, u) -> None:
    _check(load().lbmrv_init_equilibrium_host(h, _addr(rho), _addr(u)), h)


def lbmrv_step(h, n: int) -> None:
    _check(load().lbmrv_step(h, int(n)), h)


def lbmrv_moments(h, rho, u) -> None:
    _check(load().lbmrv_moments(h, _addr(rho), _addr(u)), h)


def lbmrv_moments_host(h, rho, u) -> None:
    _check(load().lbmrv_moments_host(h, _addr(rho), _addr(u)), h)


def lbmrv_conserved(h, allow_nonfinite: bool = False):
    out = (ctypes.c_double * 4)()
    rc = load().lbmrv_conserved(h, out)
    if rc == LBMRV_E_NONFINITE and allow_nonfinite:
        return list(out)
    _check(rc, h)
    return list(out)


def lbmrv_get_state(h, dst) -> None:
    _check(load().lbmrv_get_state(h, _addr(dst)), h)


def lbmrv_set_state(h, src, t: int) -> None:
    _check(load().lbmrv_set_state(h, _addr(src), int(t)), h)


def lbmrv_state_ptr(h) -> int:
    p = _VP()
    _check(load().lbmrv_state_ptr(h, ctypes.byref(p)), h)
    return p.value


def lbmrv_time(h) -> int:
    return load().lbmrv_time(h)


_STORAGE_BYTES = {LBMRV_FP32: 4, LBMRV_FP16: 2, LBMRV_BF16: 2}


def _check_noalloc_tensors(state, storage, dims, out):
    """No handle stands between the caller and the kernel here, so the tensors are checked
    before the call: the state must hold 9 planes of nx*ny values of the storage type and
    ``out`` 4 doubles, both on the current CUDA device."""
    import torch

    d = list(dims) + [1] * (3 - len(dims))
    need = 9 * int(d[0]) * int(d[1]) * _STORAGE_BYTES.get(int(storage), 0)
    if torch.is_tensor(state):
        if not state.is_cuda or state.device.index != torch.cuda.current_device():
            raise ValueError("state must be on the current CUDA device")
        if state.numel() * state.element_size() < need:
            raise ValueError(f"state holds fewer than the {need} bytes of 9 x {d[0]} x {d[1]} "
                             "values of the storage type")
    if torch.is_tensor(out):
        if not out.is_cuda or out.device.index != torch.cuda.current_device():
            raise ValueError("out must be on the current CUDA device")
        if out.dtype != torch.float64 or out.numel() < 4:
            raise ValueError("out must hold at least 4 float64 values")


def lbmrv_conserved_noalloc(state, storage: int, dims, lam: float, rho_ref: float, out,
                            stream=None) -> None:
    """Sums of a caller-owned state into ``out`` (4 device doubles) without allocating."""
    _check_noalloc_tensors(state, storage, dims, out)
    rc = load().lbmrv_conserved_noalloc(_addr(state), int(storage), _dims(dims), float(lam),
                                        float(rho_ref), _addr(out), _stream(stream))
    if rc < 0:
        raise LbmrvError(rc, "lbmrv_conserved_noalloc failed")


def lbmrv_set_rates(h, s) -> None:
    sv = (ctypes.c_double * len(s))(*[float(v) for v in s])
    _check(load().lbmrv_set_rates(h, sv), h)


def lbmrv_set_reference(h, rho_ref: float, u_ref) -> None:
    u = (ctypes.c_double * 3)(*([float(v) for v in u_ref] + [0.0] * (3 - len(u_ref))))
    _check(load().lbmrv_set_reference(h, float(rho_ref), u), h)


def lbmrv_set_reference_auto(h, rho_ref: float) -> None:
    _check(load().lbmrv_set_reference_auto(h, float(rho_ref)), h)


def lbmrv_get_reference(h):
    """Returns (rho_ref, (u_x, u_y, u_z), automatic)."""
    r = ctypes.c_double()
    u = (ctypes.c_double * 3)()
    rc = _check(load().lbmrv_get_reference(h, ctypes.byref(r), u), h)
    return r.value, tuple(u), bool(rc)


def lbmrv_slab_plan(extent: int, ranks: int, rank: int):
    """Returns (first, count): the layers slab `rank` of `ranks` owns."""
    first, count = ctypes.c_int64(), ctypes.c_int64()
    rc = load().lbmrv_slab_plan(int(extent), int(ranks), int(rank), ctypes.byref(first),
                                ctypes.byref(count))
    if rc < 0:
        raise LbmrvError(rc, f"lbmrv_slab_plan({extent}, {ranks}, {rank})")
    return first.value, count.value


def lbmrv_halo_count(lattice: int, dims) -> int:
    return load().lbmrv_halo_count(int(lattice), _dims(dims))


def lbmrv_halo_map(lattice: int, dims, side: int):
    """Returns (send_idx, recv_idx) as numpy int64 arrays."""
    import numpy as np

    count = lbmrv_halo_count(lattice, dims)
    if count < 0:
        raise LbmrvError(LBMRV_E_INVAL, f"lbmrv_halo_count: bad slab dims {tuple(dims)}")
    send = np.empty(count, dtype=np.int64)
    recv = np.empty(count, dtype=np.int64)
    rc = load().lbmrv_halo_map(int(lattice), _dims(dims), int(side), send.ctypes.data,
                               recv.ctypes.data)
    if rc < 0:
        raise LbmrvError(rc, f"lbmrv_halo_map(side={side})")
    return send, recv


def lbmrv_halo_map_adjoint(lattice: int, dims, side: int):
    """Returns (send_idx, recv_idx) of the adjoint exchange as numpy int64 arrays."""
    import numpy as np

    count = lbmrv_halo_count(lattice, dims)
    if count < 0:
        raise LbmrvError(LBMRV_E_INVAL, f"lbmrv_halo_count: bad slab dims {tuple(dims)}")
    send = np.empty(count, dtype=np.int64)
    recv = np.empty(count, dtype=np.int64)
    rc = load().lbmrv_halo_map_adjoint(int(lattice), _dims(dims), int(side), send.ctypes.data,
                                       recv.ctypes.data)
    if rc < 0:
        raise LbmrvError(rc, f"lbmrv_halo_map_adjoint(side={side})")
    return send, recv


def lbmrv_halo_pack_adjoint(h, mu, send_lo, send_hi) -> None:
    _check(load().lbmrv_halo_pack_adjoint(h, _addr(mu), _addr(send_lo), _addr(send_hi)), h)


def lbmrv_halo_unpack_adjoint(h, mu, recv_lo, recv_hi) -> None:
    _check(load().lbmrv_halo_unpack_adjoint(h, _addr(mu), _addr(recv_lo), _addr(recv_hi)), h)


def lbmrv_adjoint_acc_doubles(h) -> int:
    return load().lbmrv_adjoint_acc_doubles(h)


def lbmrv_adjoint_step(h, s_prev, t: int, a, gather: bool, mu, acc, dL_dut0=None) -> None:
    _check(load().lbmrv_adjoint_step(h, _addr(s_prev), int(t), _addr(a), int(bool(gather)),
                                     _addr(mu), _addr(acc), _addr(dL_dut0)), h)


def lbmrv_adjoint_acc_sum(h, acc):
    """Returns (dL/ds as 9 floats, dL/dA)."""
    ds = (ctypes.c_double * 9)()
    da = ctypes.c_double()
    _check(load().lbmrv_adjoint_acc_sum(h, _addr(acc), ds, ctypes.byref(da)), h)
    return list(ds), da.value


def lbmrv_adjoint_gather(h, mu, out) -> None:
    _check(load().lbmrv_adjoint_gather(h, _addr(mu), _addr(out)), h)


def lbmrv_set_slab(h, first: int, extent: int) -> None:
    _check(load().lbmrv_set_slab(h, int(first), int(extent)), h)


def lbmrv_halo_pack(h, send_lo, send_hi) -> None:
    _check(load().lbmrv_halo_pack(h, _addr(send_lo), _addr(send_hi)), h)


def lbmrv_halo_unpack(h, recv_lo, recv_hi) -> None:
    _check(load().lbmrv_halo_unpack(h, _addr(recv_lo), _addr(recv_hi)), h)


def lbmrv_flow_sums(h, rho, u):
    out = (ctypes.c_double * 4)()
    _check(load().lbmrv_flow_sums(h, _addr(rho), _addr(u), out), h)
    return list(out)


def lbmrv_set_reference_sums(h, rho_ref: float, sums) -> None:
    sv = (ctypes.c_double * 4)(*[float(v) for v in sums])
    _check(load().lbmrv_set_reference_sums(h, float(rho_ref), sv), h)


def lbmrv_conserved3(h, allow_nonfinite: bool = False):
    out = (ctypes.c_double * 5)()
    rc = load().lbmrv_conserved3(h, out)
    if rc == LBMRV_E_NONFINITE and allow_nonfinite:
        return list(out)
    _check(rc, h)
    return list(out)


def lbmrv_step_conserved(h, n: int, allow_nonfinite: bool = False):
    out = (ctypes.c_double * 5)()
    rc = load().lbmrv_step_conserved(h, int(n), out)
    if rc == LBMRV_E_NONFINITE and allow_nonfinite:
        return list(out)
    _check(rc, h)
    return list(out)


def lbmrv_adjoint_workspace_bytes(h, n: int, seg: int) -> int:
    return load().lbmrv_adjoint_workspace_bytes(h, int(n), int(seg))


def lbmrv_forward_checkpointed(h, n: int, seg: int, ws, ws_bytes: int) -> None:
    _check(load().lbmrv_forward_checkpointed(h, int(n), int(seg), _addr(ws), int(ws_bytes)), h)


def lbmrv_adjoint(h, n: int, seg: int, ws, ws_bytes: int, dL_dS, dL_dS0, dL_dut0=None):
    """Returns (dL/ds as 9 floats, dL/dA)."""
    ds = (ctypes.c_double * 9)()
    da = ctypes.c_double()
    _check(load().lbmrv_adjoint(h, int(n), int(seg), _addr(ws), int(ws_bytes), _addr(dL_dS),
                                _addr(dL_dS0), ds, ctypes.byref(da), _addr(dL_dut0)), h)
    return list(ds), da.value


def lbmrv_kinetic_energy(h, dL_dS=None) -> float:
    ke = ctypes.c_double()
    _check(load().lbmrv_kinetic_energy(h, ctypes.byref(ke), _addr(dL_dS)), h)
    return ke.value


def lbmrv_moments_vjp(h, dL_drho, dL_du, dL_dS) -> None:
    _check(load().lbmrv_moments_vjp(h, _addr(dL_drho), _addr(dL_du), _addr(dL_dS)), h)


def lbmrv_equilibrium_vjp(h, rho, u, dL_dS0, dL_drho, dL_du) -> None:
    _check(load().lbmrv_equilibrium_vjp(h, _addr(rho), _addr(u), _addr(dL_dS0), _addr(dL_drho),
                                        _addr(dL_du)), h)
