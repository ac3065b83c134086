"""CPU oracle for the FLINTS lensing remap: plain, slow, FP64, written from the paper.

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import or run it; the library's
product path never does.  It shares no code with the CUDA path.

Modules: ``healpix`` (RING geometry), ``xi`` (correlation functions, direct and
tabulated), ``kriging`` (displacement, exact K-nearest stencil, covariance,
Cholesky with nugget, conditional mean and variance), ``sht`` (spherical
harmonic synthesis at arbitrary directions: the exact benchmark of Sec. 3.2).
"""
