"""GB300-native RNA / ARNA distributed-resampling particle filter.

Implements the hot path of Demirel et al., "An Adaptive Distributed
Resampling Algorithm with Non-Proportional Allocation" (arXiv:1310.4624): one
SIR time step split into G groups (the paper's processing elements), with
propagation, Gaussian-PSF image likelihood, per-group exact systematic
resampling and RNA / ARNA ring exchange, all in hand-written CUDA for sm_103a
behind the C ABI declared in include/pfarna.h.

Importing the package loads nothing; the CUDA library is opened on first use
of :mod:`paper_1310_4624_gb300.binding`.
"""
__all__ = ["synth", "binding", "filter"]
