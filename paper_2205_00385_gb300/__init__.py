"""GB300-native AARMR topology optimisation (arXiv 2205.00385).

The compute path is libtopo.so (CUDA, sm_103a), reached through the C ABI
in include/topo.h; ``binding`` wraps it one-to-one and ``driver`` runs the
design loop of Algorithm 1 on top of it.
"""

from . import binding  # noqa: F401

__all__ = ["binding", "driver"]
