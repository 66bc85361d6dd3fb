"""Seeded synthetic initial fields, shared by the oracle side and the GPU side.

This module only draws and shapes the initial macroscopic fields (density and velocity
on a periodic lattice, in lattice units dx = 1). It holds none of the lattice Boltzmann
arithmetic: each side turns these fields into populations with its own equilibrium.

All fields are FP64 arrays of shape (ny, nx), row-major with x fastest. Random draws use
``numpy.random.default_rng(seed)`` in a fixed order: density noise first, then the
x-velocity noise plane, then the y-velocity noise plane.

``to_f32_exact`` rounds a field to FP32 and back so that the FP32 GPU path and the FP64
oracle start from bit-identical inputs.
"""
from __future__ import annotations

import numpy as np

TWO_PI = 2.0 * np.pi


def _grid(nx: int, ny: int):
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    return x, y


def to_f32_exact(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def random_sine_flow(nx: int, ny: int, seed: int = 0, amp: float = 0.05,
                     u_noise: float = 0.005, rho_noise: float = 0.01):
    """Small-lattice parity workload: rho = 1 + 0.01 N(0,1),
    u = 0.05 (sin 2 pi y/ny, sin 2 pi x/nx) + 0.005 N(0,1) per component."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    rho = 1.0 + rho_noise * rng.standard_normal((ny, nx))
    nxn = rng.standard_normal((ny, nx))
    nyn = rng.standard_normal((ny, nx))
    ux = amp * np.sin(TWO_PI * y / ny) + u_noise * nxn
    uy = amp * np.sin(TWO_PI * x / nx) + u_noise * nyn
    return {"rho": rho, "ux": ux, "uy": uy}


def taylor_green(nx: int, ny: int, u0: float = 0.04, rho0: float = 1.0, lam: float = 1.0):
    """2D Taylor-Green vortex, k = 2 pi / L per axis:
    ux = -u0 cos(kx x) sin(ky y), uy = u0 sin(kx x) cos(ky y),
    p = -rho0 u0^2 / 4 (cos 2 kx x + cos 2 ky y), rho = rho0 + 3 p / lambda^2."""
    x, y = _grid(nx, ny)
    kx, ky = TWO_PI / nx, TWO_PI / ny
    ux = -u0 * np.cos(kx * x) * np.sin(ky * y)
    uy = u0 * np.sin(kx * x) * np.cos(ky * y)
    p = -rho0 * u0 * u0 / 4.0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y))
    rho = rho0 + 3.0 * p / (lam * lam)
    return {"rho": rho, "ux": ux, "uy": uy}


def perturbed_uniform(nx: int, ny: int, seed: int = 0, U=(0.05, 0.02), drho: float = 1e-3,
                      du: float = 1e-3, rho0: float = 1.0):
    """Randomly perturbed uniform flow: rho = rho0 + drho N(0,1), u = U + du N(0,1)."""
    rng = np.random.default_rng(seed)
    rho = rho0 + drho * rng.standard_normal((ny, nx))
    ux = U[0] + du * rng.standard_normal((ny, nx))
    uy = U[1] + du * rng.standard_normal((ny, nx))
    return {"rho": rho, "ux": ux, "uy": uy}


def noisy_shear_wave(nx: int, ny: int, seed: int = 0, amp: float = 0.05, sigma: float = 0.01):
    """Shear wave ux = amp sin(2 pi y/ny) plus N(0, sigma) noise (sigma is the standard
    deviation) on both components; rho = 1."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    rho = np.ones((ny, nx))
    ux = amp * np.sin(TWO_PI * y / ny) + sigma * rng.standard_normal((ny, nx))
    uy = sigma * rng.standard_normal((ny, nx))
    return {"rho": rho, "ux": ux, "uy": uy}


def shear_wave(nx: int, ny: int, amp: float = 1e-3, background=(0.0, 0.0), kmode: int = 1,
               axis: str = "y"):
    """Transverse shear wave on an optional uniform background flow.

    axis="y": ux = bx + amp sin(2 pi k y / ny), uy = by.
    axis="x": ux = bx, uy = by + amp sin(2 pi k x / nx)."""
    x, y = _grid(nx, ny)
    rho = np.ones((ny, nx))
    ux = np.full((ny, nx), float(background[0]))
    uy = np.full((ny, nx), float(background[1]))
    if axis == "y":
        ux = ux + amp * np.sin(TWO_PI * kmode * y / ny)
    else:
        uy = uy + amp * np.sin(TWO_PI * kmode * x / nx)
    return {"rho": rho, "ux": ux, "uy": uy}


def uniform(nx: int, ny: int, rho0: float = 1.0, U=(0.0, 0.0)):
    return {"rho": np.full((ny, nx), rho0), "ux": np.full((ny, nx), float(U[0])),
            "uy": np.full((ny, nx), float(U[1]))}


def prescribed_base_field(nx: int, ny: int, seed: int = 0, smooth: bool = True):
    """A caller-supplied base field u~0(x), shape (2, ny, nx), for the prescribed mode:
    smooth=True gives (sin 2 pi (x+y)/n, cos 2 pi x/nx); otherwise N(0,1) draws."""
    if smooth:
        x, y = _grid(nx, ny)
        return np.stack([np.sin(TWO_PI * (x / nx + y / ny)), np.cos(TWO_PI * x / nx)])
    rng = np.random.default_rng(seed)
    return rng.standard_normal((2, ny, nx))


# ------------------------------------------------------------------ 3D fields (nz, ny, nx)
def _grid3(nx: int, ny: int, nz: int):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def taylor_green_3d(nx: int, ny: int, nz: int, u0: float = 0.04, rho0: float = 1.0,
                    lam: float = 1.0):
    """3D Taylor-Green vortex, k = 2 pi / L per axis:
    u = u0 (sin kx cos ky cos kz, -cos kx sin ky cos kz, 0),
    p = rho0 u0^2 / 16 (cos 2kx + cos 2ky)(cos 2kz + 2), rho = rho0 + 3 p / lambda^2.
    Returns rho (nz, ny, nx) and u (3, nz, ny, nx)."""
    x, y, z = _grid3(nx, ny, nz)
    kx, ky, kz = TWO_PI / nx, TWO_PI / ny, TWO_PI / nz
    ux = u0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    uy = -u0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z)
    uz = np.zeros_like(ux)
    p = rho0 * u0 * u0 / 16.0 * (np.cos(2 * kx * x) + np.cos(2 * ky * y)) * (np.cos(2 * kz * z) + 2)
    return {"rho": rho0 + 3.0 * p / (lam * lam), "u": np.stack([ux, uy, uz])}


def random_flow_3d(nx: int, ny: int, nz: int, seed: int = 0, amp: float = 0.04,
                   u_noise: float = 0.005, rho_noise: float = 0.01):
    """Small-lattice 3D parity workload: rho = 1 + 0.01 N(0,1), u = amp (sin 2pi y/ny,
    sin 2pi z/nz, sin 2pi x/nx) + u_noise N(0,1) per component (draws: rho, u_x, u_y, u_z)."""
    rng = np.random.default_rng(seed)
    x, y, z = _grid3(nx, ny, nz)
    rho = 1.0 + rho_noise * rng.standard_normal((nz, ny, nx))
    noise = [rng.standard_normal((nz, ny, nx)) for _ in range(3)]
    u = np.stack([amp * np.sin(TWO_PI * y / ny) + u_noise * noise[0],
                  amp * np.sin(TWO_PI * z / nz) + u_noise * noise[1],
                  amp * np.sin(TWO_PI * x / nx) + u_noise * noise[2]])
    return {"rho": rho, "u": u}


def perturbed_uniform_3d(nx: int, ny: int, nz: int, seed: int = 0, U=(0.05, 0.02, 0.01),
                         drho: float = 1e-3, du: float = 1e-3, rho0: float = 1.0):
    """Randomly perturbed uniform 3D flow: rho = rho0 + drho N(0,1), u = U + du N(0,1) per
    component (draws: rho, u_x, u_y, u_z). Returns rho (nz, ny, nx) and u (3, nz, ny, nx)."""
    rng = np.random.default_rng(seed)
    rho = rho0 + drho * rng.standard_normal((nz, ny, nx))
    u = np.stack([U[a] + du * rng.standard_normal((nz, ny, nx)) for a in range(3)])
    return {"rho": rho, "u": u}
