"""GB300-native low-rank K^-1 A for huge, nearly rank-deficient covariance matrices
(Banerjee, Vogelstein & Dunson, arXiv:1312.1869): structured random sketch, blocked TSQR
and low-rank solve as sm_103a CUDA kernels behind a C ABI (include/ckinv.h).

`paper_1312_1869_gb300.ckinv` is the Python binding; `paper_1312_1869_gb300.build` compiles
the library in-tree.
"""
__all__ = ["ckinv", "build"]
