"""GB300-native KP-SVD preconditioned Tikhonov deblurring (arXiv 2311.15393).

The compute path is a CUDA C-ABI library (``libkpsvd.so``, built for sm_103a);
this package holds its thin ctypes binding (``kpsvd``) and the seeded input
generator (``synth``).
"""
