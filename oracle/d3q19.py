"""ctypes wrappers of the FP64 D3Q19 oracle (``lbmrv_oracle3d.c``).

TEST INFRASTRUCTURE (see the package docstring). Arrays are FP64, populations shaped
(19, nz, ny, nx), velocity fields (3, nz, ny, nx).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _f64, _optr, _ptr, lib

Q = 19


def velocities():
    c = [(ctypes.c_int * Q)() for _ in range(3)]
    lib().orc3_velocities(*c)
    return np.array([list(v) for v in c], dtype=int)  # (3, 19)


def poly(k, X, Y, Z, lam):
    return lib().orc3_poly(k, X, Y, Z, lam)


def moment_matrix(ut, lam):
    M = np.zeros((Q, Q))
    lib().orc3_moment_matrix(float(ut[0]), float(ut[1]), float(ut[2]), lam, _ptr(M))
    return M


def feq(rho, u, lam):
    out = np.zeros(Q)
    lib().orc3_feq(rho, float(u[0]), float(u[1]), float(u[2]), lam, _ptr(out))
    return out


def collide_node(f, ut, lam, s):
    f, s, ut = _f64(f), _f64(s), _f64(ut)
    out = np.zeros(Q)
    if lib().orc3_collide_node(_ptr(f), _ptr(ut), lam, _ptr(s), _ptr(out)) != 0:
        raise FloatingPointError("singular shifted moment matrix")
    return out


def init_equilibrium(rho, u, lam):
    rho, u = _f64(rho), _f64(u)
    f = np.zeros((Q,) + rho.shape)
    lib().orc3_init_equilibrium(rho.size, lam, _ptr(rho), _ptr(u), _ptr(f))
    return f


def moments(f, lam):
    f = _f64(f)
    shape = f.shape[1:]
    rho, u = np.zeros(shape), np.zeros((3,) + shape)
    lib().orc3_moments(rho.size, lam, _ptr(f), _ptr(rho), _ptr(u))
    return rho, u


def collide(f, lam, s, mode, t=0, ut0=None, amp=0.0, period=0.0, nthreads=1):
    f, s = _f64(f), _f64(s)
    ut0 = None if ut0 is None else _f64(ut0)
    nz, ny, nx = f.shape[1:]
    out = np.empty_like(f)
    rc = lib().orc3_collide_lattice(nx, ny, nz, lam, _ptr(s), mode, _optr(ut0), amp, period, t,
                                    _ptr(f), _ptr(out), nthreads)
    if rc != 0:
        raise FloatingPointError(f"D3Q19 oracle relaxation failed ({rc})")
    return out


def stream(f, nthreads=1):
    f = _f64(f)
    nz, ny, nx = f.shape[1:]
    out = np.empty_like(f)
    lib().orc3_stream(nx, ny, nz, _ptr(f), _ptr(out), nthreads)
    return out


def run(f, lam, s, mode, steps, t0=0, ut0=None, amp=0.0, period=0.0, nthreads=1):
    f = np.array(f, dtype=np.float64, order="C", copy=True)
    s = _f64(s)
    ut0 = None if ut0 is None else _f64(ut0)
    nz, ny, nx = f.shape[1:]
    work = np.empty_like(f)
    rc = lib().orc3_run(nx, ny, nz, lam, _ptr(s), mode, _optr(ut0), amp, period, t0, steps,
                        _ptr(f), _ptr(work), nthreads)
    if rc != 0:
        raise FloatingPointError(f"D3Q19 oracle step failed ({rc})")
    return f


def post_collision_state(f0, lam, s, mode, steps, **kw):
    """C_steps(f(steps)): the state a pull-then-relax stepper stores after `steps` steps."""
    nthreads = kw.pop("nthreads", 1)
    f = run(f0, lam, s, mode, steps, nthreads=nthreads, **kw)
    return collide(f, lam, s, mode, t=steps, nthreads=nthreads, **kw)
