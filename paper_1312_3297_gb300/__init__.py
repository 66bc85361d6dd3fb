"""lbmrv: lattice Boltzmann schemes with relative velocities (arXiv:1312.3297) as
hand-written sm_103a CUDA kernels behind a C ABI (include/lbmrv.h).

``binding`` holds the one-to-one ctypes binding of the C entry points; ``simulation``
a small torch-owned-memory wrapper. The CUDA library is built in-tree by ``build``.
"""
from . import binding
from .binding import LbmrvError
from .simulation import D2Q9, D2Q9Cascaded, D3Q19

__all__ = ["binding", "LbmrvError", "D2Q9", "D2Q9Cascaded", "D3Q19"]
