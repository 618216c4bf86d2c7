"""GB300-native D-GAMP-CT: the per-iteration hot path of denoising GAMP for
sparse-view CT (Perelli, Lexa, Can, Davies) as hand-written sm_103a CUDA
kernels behind the C ABI in include/dgamp_ct.h.

``Plan`` (see :mod:`paper_1609_04661_gb300.binding`) wraps one geometry;
build the library first with ``python -m paper_1609_04661_gb300.build``.
"""
from .binding import CNN, Batch, DgampError, Plan, default_options, load, schedule_lpt, solve_batched  # noqa: F401

__all__ = ["CNN", "Batch", "Plan", "DgampError", "default_options", "load", "schedule_lpt", "solve_batched"]
