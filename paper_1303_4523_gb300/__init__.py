"""GB300-native ENUF-DPD: the reciprocal-space Ewald sum for Slater-smeared
charges evaluated with the non-uniform FFT (Wang, Laaksonen & Lu,
arXiv 1303.4523), plus the fused real-space + DPD pair forces, as sm_103a CUDA
kernels behind a C ABI (include/enuf.h).

Importing the package is cheap; the CUDA library is loaded on first use of the
binding (``paper_1303_4523_gb300.enuf``) and raises if it is missing.
"""
