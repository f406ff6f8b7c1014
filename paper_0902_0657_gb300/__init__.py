"""GB300 (sm_103a) adaptive LP decoder.

The decoder (MALP-A/MALP-B cut search, interior-point LP solver with PCG
and the column-wise MTS preconditioner, optimal-vertex recovery) runs in
hand-written CUDA kernels behind the C ABI of include/lpdec.h; ``lpdec``
is its Python binding and ``build`` compiles the library in-tree.
"""
