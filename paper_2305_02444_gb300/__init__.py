"""GB300-native fault-tolerant DGEMM (FT-GEMM, HPDC'23) for sm_103a.

The compute path is libftgemm.so (hand-written CUDA, C ABI in
include/ftgemm.h); `ftgemm` is its thin ctypes binding and `inputs` holds the
seeded synthetic input generators.
"""
from . import ftgemm, inputs  # noqa: F401
from .ftgemm import (ftgemm_d, ftgemm_d_host, ftgemm_d_noft, ftgemm_encode_operands,  # noqa: F401
                     ftgemm_finalize, ftgemm_injection_log, ftgemm_launch_count,
                     ftgemm_selftest_wait_timeout, ftgemm_set_injection, ftgemm_strerror)
