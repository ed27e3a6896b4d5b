"""GB300-native randomized HSS compression (arXiv:1503.05464).

The library is libhss.so (C ABI in include/hss.h, CUDA kernels for sm_103a in
csrc/); ``hss`` is its ctypes binding.
"""
from . import hss  # noqa: F401
from .hss import (HSS, HssBatch, HssError, hss_compress, hss_compress_batched,  # noqa: F401
                  hss_compress_matfree, hss_default_opts, hss_factor,
                  hss_factor_batched, hss_solve_batched,
                  hss_id_batched, hss_info, hss_matvec, hss_node_ranks, hss_random_gaussian,
                  hss_sample, hss_sample_noalloc, hss_solve)
