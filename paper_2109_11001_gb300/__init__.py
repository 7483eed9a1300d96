"""GB300 (sm_103a) implementation of the hot path of the core-softened
double-bridging hybrid (DBH) equilibration of semiflexible Kremer-Grest melts
(Dietz & Hoy, arXiv:2109.11001): the MD step and the double-bridging Monte
Carlo sweep, behind the C ABI of ``include/kg.h``.

``binding`` exposes the C entry points under their own names; ``build``
compiles ``libkg.so`` in-tree.
"""
from .binding import *  # noqa: F401,F403
from .binding import EXPORTS, KGError, load, make_params, stage, torch_allocator  # noqa: F401
