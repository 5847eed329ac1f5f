"""GB300-native Wilson-clover quark solver with the restricted additive
Schwarz preconditioner (Osaki & Ishikawa, "Domain Decomposition method on GPU
cluster", Lattice 2010).

The product is libqdd.so (CUDA kernels for sm_103a behind the C ABI in
include/qdd.h); ``paper_1011_3318_gb300.qdd`` is its Python binding and
``paper_1011_3318_gb300.build`` compiles it.
"""

__all__ = ["build", "qdd"]
