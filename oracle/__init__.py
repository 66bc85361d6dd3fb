"""FP64 CPU oracle for the lattice Boltzmann scheme with relative velocities.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` import this package. It shares no code with the CUDA library in
``paper_1312_3297_gb300`` and never imports it; the two meet only through the seeded
input generators of ``lbm_inputs``.

Two independent implementations live here:

* ``lbmrv_oracle.c`` (plain C, FP64, ``-ffp-contract=off``): the scheme of Section 1.2
  taken literally (per-node shifted moment matrix and LU solve), the shifted form of
  Section 1.3 with the T(u~) blocks of Appendix A, and the fixed-moment d'Humieres MRT
  of Section 1.1. This module wraps it with ctypes.
* ``lbmrv_oracle3d.c`` (wrapped by ``d3q19.py``): the same definition on a D3Q19 lattice
  with a translation-invariant 19-polynomial basis.
* ``torch_ref.py`` (plain PyTorch CPU ops in FP64): the same definition written with
  ``torch.linalg.solve`` so that reverse-mode differentiation of the definition gives
  the reference adjoint.

Parity unpinned: nothing here. Every function is pinned by a ``-m "not gpu"`` test
against what the paper fixes (printed matrices, the morphism, the reduction to MRT,
invariants, the second-order viscosity).
"""
from __future__ import annotations

import ctypes
import os
import shutil
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbmrv_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "lbmrv_oracle3d.c")]
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liblbmrv_oracle.so")

METHOD_DEFINITION = 0
METHOD_SHIFTED = 1
METHOD_MRT = 2
METHOD_GEIER = 3       # definition in Geier's basis, product (Maxwellian-moment) equilibrium
METHOD_CASCADED = 4    # Geier's cascade as written in Appendix B (u~ = q/rho)
MODE_ZERO = 0
MODE_FLUID = 1
MODE_PRESCRIBED = 2

_lock = threading.Lock()
_lib = None
_openmp = False


def _compile(out_path: str, extra=(), srcs=None) -> bool:
    """gcc the C oracle into out_path (OpenMP when available); returns whether OpenMP is
    on. `extra` are additional compiler flags; `srcs` replaces the two C sources (the
    mutation tests compile edited copies of them)."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("no C compiler found to build the oracle")
    base = [cc, "-O2", "-fPIC", "-shared", "-std=c99", "-ffp-contract=off",
            "-fno-fast-math", *extra, *(srcs or _SRCS), "-o", out_path + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
        omp = True
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
        omp = False
    os.replace(out_path + ".tmp", out_path)
    return omp


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP when available). Returns the .so path."""
    global _openmp
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(p) for p in _SRCS)):
        _openmp = _probe_openmp_flag()
        return _LIB_PATH
    _openmp = _compile(_LIB_PATH)
    with open(_LIB_PATH + ".omp", "w") as fh:
        fh.write("1" if _openmp else "0")
    return _LIB_PATH


def _probe_openmp_flag() -> bool:
    try:
        with open(_LIB_PATH + ".omp") as fh:
            return fh.read().strip() == "1"
    except OSError:
        return False


def openmp_enabled() -> bool:
    lib()
    return _openmp


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _bind(path: str) -> ctypes.CDLL:
    """Load an oracle library and declare its entry points."""
    L = ctypes.CDLL(path)
    D = ctypes.c_double
    P = ctypes.POINTER(ctypes.c_double)
    I64 = ctypes.c_int64
    I = ctypes.c_int
    L.orc_poly.restype = D
    L.orc_poly.argtypes = [I, D, D, D]
    L.orc_moment_matrix.argtypes = [D, D, D, P]
    L.orc_shift_matrix.argtypes = [D, D, D, P]
    L.orc_feq.argtypes = [D, D, D, D, P]
    L.orc_lu_solve.restype = I
    L.orc_lu_solve.argtypes = [P, P, P]
    L.orc_collide_definition.restype = I
    L.orc_collide_definition.argtypes = [P, D, D, D, P, P]
    L.orc_collide_shifted.argtypes = [P, D, D, D, P, P]
    L.orc_collide_mrt.argtypes = [P, D, P, P]
    L.orc_collide_lattice.restype = I
    L.orc_collide_lattice.argtypes = [I, I64, I64, D, P, I, P, D, D, I64, P, P, I]
    L.orc_stream.argtypes = [I64, I64, P, P, I]
    L.orc_run.restype = I
    L.orc_run.argtypes = [I, I64, I64, D, P, I, P, D, D, I64, I64, P, P, I]
    L.orc_init_equilibrium.argtypes = [I64, I64, D, P, P, P, P]
    L.orc_moments.argtypes = [I64, I64, D, P, P, P, P]
    L.orc_velocities.argtypes = [D, P, P]
    L.orc_poly_geier.restype = D
    L.orc_poly_geier.argtypes = [I, D, D, D]
    L.orc_moment_matrix_geier.argtypes = [D, D, D, P]
    L.orc_feq_product.argtypes = [D, D, D, D, P]
    L.orc_collide_geier.restype = I
    L.orc_collide_geier.argtypes = [P, D, D, D, P, P]
    L.orc_collide_cascaded.restype = I
    L.orc_collide_cascaded.argtypes = [P, D, P, P]
    L.orc_init_equilibrium_product.argtypes = [I64, I64, D, P, P, P, P]
    IP = ctypes.POINTER(ctypes.c_int)  # D3Q19 oracle (lbmrv_oracle3d.c, wrapped by d3q19.py)
    L.orc3_velocities.argtypes = [IP, IP, IP]
    L.orc3_poly.restype = D
    L.orc3_poly.argtypes = [I, D, D, D, D]
    L.orc3_moment_matrix.argtypes = [D, D, D, D, P]
    L.orc3_feq.argtypes = [D, D, D, D, D, P]
    L.orc3_collide_node.restype = I
    L.orc3_collide_node.argtypes = [P, P, D, P, P]
    L.orc3_collide_lattice.restype = I
    L.orc3_collide_lattice.argtypes = [I64, I64, I64, D, P, I, P, D, D, I64, P, P, I]
    L.orc3_stream.argtypes = [I64, I64, I64, P, P, I]
    L.orc3_run.restype = I
    L.orc3_run.argtypes = [I64, I64, I64, D, P, I, P, D, D, I64, I64, P, P, I]
    L.orc3_init_equilibrium.argtypes = [I64, D, P, P, P]
    L.orc3_moments.argtypes = [I64, D, P, P, P]
    return L


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _optr(a):
    return None if a is None else _ptr(a)


# ---------------------------------------------------------------- per-node pieces
def poly(k: int, X: float, Y: float, lam: float) -> float:
    return lib().orc_poly(k, X, Y, lam)


def moment_matrix(utx: float, uty: float, lam: float) -> np.ndarray:
    M = np.zeros((9, 9))
    lib().orc_moment_matrix(utx, uty, lam, _ptr(M))
    return M


def shift_matrix(utx: float, uty: float, lam: float) -> np.ndarray:
    T = np.zeros((9, 9))
    lib().orc_shift_matrix(utx, uty, lam, _ptr(T))
    return T


def feq(rho: float, ux: float, uy: float, lam: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, lam, _ptr(out))
    return out


def velocities(lam: float):
    vx, vy = np.zeros(9), np.zeros(9)
    lib().orc_velocities(lam, _ptr(vx), _ptr(vy))
    return vx, vy


def collide_node(method: int, f, utx: float, uty: float, lam: float, s) -> np.ndarray:
    f = _f64(f)
    s = _f64(s)
    out = np.zeros(9)
    if method == METHOD_DEFINITION:
        rc = lib().orc_collide_definition(_ptr(f), utx, uty, lam, _ptr(s), _ptr(out))
        if rc != 0:
            raise FloatingPointError("singular shifted moment matrix")
    elif method == METHOD_SHIFTED:
        lib().orc_collide_shifted(_ptr(f), utx, uty, lam, _ptr(s), _ptr(out))
    elif method == METHOD_MRT:
        lib().orc_collide_mrt(_ptr(f), lam, _ptr(s), _ptr(out))
    elif method == METHOD_GEIER:
        if lib().orc_collide_geier(_ptr(f), utx, uty, lam, _ptr(s), _ptr(out)) != 0:
            raise FloatingPointError("singular shifted moment matrix")
    else:
        if lib().orc_collide_cascaded(_ptr(f), lam, _ptr(s), _ptr(out)) != 0:
            raise FloatingPointError("singular cascade")
    return out


def moment_matrix_geier(utx: float, uty: float, lam: float) -> np.ndarray:
    M = np.zeros((9, 9))
    lib().orc_moment_matrix_geier(utx, uty, lam, _ptr(M))
    return M


def feq_product(rho: float, ux: float, uy: float, lam: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_feq_product(rho, ux, uy, lam, _ptr(out))
    return out


def init_equilibrium_product(rho, ux, uy, lam: float) -> np.ndarray:
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    ny, nx = rho.shape
    f = np.zeros((9, ny, nx))
    lib().orc_init_equilibrium_product(nx, ny, lam, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(f))
    return f


# ---------------------------------------------------------------- lattice level
def init_equilibrium(rho, ux, uy, lam: float) -> np.ndarray:
    rho, ux, uy = _f64(rho), _f64(ux), _f64(uy)
    ny, nx = rho.shape
    f = np.zeros((9, ny, nx))
    lib().orc_init_equilibrium(nx, ny, lam, _ptr(rho), _ptr(ux), _ptr(uy), _ptr(f))
    return f


def collide(f, lam: float, s, mode: int, t: int = 0, method: int = METHOD_DEFINITION,
            ut0=None, amp: float = 0.0, period: float = 0.0, nthreads: int = 1) -> np.ndarray:
    """Relaxation at every node at collision time t (no transport)."""
    f = _f64(f)
    s = _f64(s)
    ut0 = None if ut0 is None else _f64(ut0)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    rc = lib().orc_collide_lattice(method, nx, ny, lam, _ptr(s), mode, _optr(ut0), amp,
                                   period, t, _ptr(f), _ptr(out), nthreads)
    if rc != 0:
        raise FloatingPointError("singular shifted moment matrix")
    return out


def stream(f, nthreads: int = 1) -> np.ndarray:
    f = _f64(f)
    _, ny, nx = f.shape
    out = np.empty_like(f)
    lib().orc_stream(nx, ny, _ptr(f), _ptr(out), nthreads)
    return out


def run(f, lam: float, s, mode: int, steps: int, t0: int = 0,
        method: int = METHOD_DEFINITION, ut0=None, amp: float = 0.0, period: float = 0.0,
        nthreads: int = 1) -> np.ndarray:
    """``steps`` time steps (relax at t0.., then transport) from the pre-collision f."""
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    s = _f64(s)
    ut0 = None if ut0 is None else _f64(ut0)
    _, ny, nx = f.shape
    work = np.empty_like(f)
    rc = lib().orc_run(method, nx, ny, lam, _ptr(s), mode, _optr(ut0), amp, period, t0,
                       steps, _ptr(f), _ptr(work), nthreads)
    if rc != 0:
        raise FloatingPointError("singular shifted moment matrix")
    return f


def run_inplace(f: np.ndarray, work: np.ndarray, lam: float, s, mode: int, steps: int,
                t0: int = 0, method: int = METHOD_DEFINITION, ut0=None, amp: float = 0.0,
                period: float = 0.0, nthreads: int = 1) -> None:
    """Same as ``run`` but advances ``f`` in place using the caller's ``work`` buffer."""
    s = _f64(s)
    ut0 = None if ut0 is None else _f64(ut0)
    _, ny, nx = f.shape
    assert work.shape == f.shape
    rc = lib().orc_run(method, nx, ny, lam, _ptr(s), mode, _optr(ut0), amp, period, t0,
                       steps, _ptr(f), _ptr(work), nthreads)
    if rc != 0:
        raise FloatingPointError("singular shifted moment matrix")


def moments(f, lam: float):
    f = _f64(f)
    _, ny, nx = f.shape
    rho, ux, uy = (np.zeros((ny, nx)) for _ in range(3))
    lib().orc_moments(nx, ny, lam, _ptr(f), _ptr(rho), _ptr(ux), _ptr(uy))
    return rho, ux, uy


def post_collision_state(f0, lam: float, s, mode: int, steps: int, **kw) -> np.ndarray:
    """State after ``steps`` steps in post-collision form, C_steps(f(steps)).

    A stepper that stores the post-collision state S_k = C_k(f(k)) (pull streaming
    fused before the relaxation) and starts from S_0 = f_eq holds exactly this after
    ``steps`` steps, because f(k+1) is the transport of S_k."""
    method = kw.pop("method", METHOD_DEFINITION)
    nthreads = kw.pop("nthreads", 1)
    f = run(f0, lam, s, mode, steps, method=method, nthreads=nthreads, **kw)
    return collide(f, lam, s, mode, t=steps, method=method, nthreads=nthreads, **kw)
