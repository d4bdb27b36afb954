"""GB300-native batched forward model, Gaussian log-likelihood and adjoint for
sub-stellar atmospheric retrieval (Exo Skryer, arXiv 2602.19687).

The compute path is the C-ABI library ``libexoskry.so`` (hand-written CUDA for
sm_103a); ``binding`` is a thin ctypes layer over it.
"""
