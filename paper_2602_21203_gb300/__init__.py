"""Squint visual-SAC learner for GB300 (sm_103a): CUDA kernels behind a C ABI.

The compiled library is loaded on first use by `paper_2602_21203_gb300.lib`;
importing the package itself loads nothing.
"""
