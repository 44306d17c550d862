"""GB300-native variational (Galerkin) FFT solver for finite-strain
polycrystals (Lucarini & Segurado, arXiv:1806.10599).

The solver is the CUDA library libgff.so (C ABI declared in include/gff.h,
sources in csrc/); `gff` is its thin ctypes binding and `build` compiles it
for sm_103a.  Import `paper_1806_10599_gb300.gff` to use it.
"""
