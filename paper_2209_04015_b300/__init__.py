"""B300-native phaseless AFQMC walker step (arXiv:2209.04015) behind a C ABI.

The compute path is libafqmc.so (hand-written CUDA for sm_103a, declared in
include/afqmc.h); ``afqmc`` is a ctypes binding with the same entry-point names.
``synthetic`` draws the seeded inputs used by tests and benchmarks.
"""
from .afqmc import AfqBatch, AfqContext, AfqError, load_library  # noqa: F401
