"""FP64 CPU oracle of the Squint update and actor inference.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline leg may import this package.  It shares no code with the CUDA
path and never calls it.
"""
