"""B300-native Cholesky-decomposed two-electron integrals (arXiv 2609.00306).

The compute path is the CUDA library ``libcderi.so`` (C ABI in
``include/cderi.h``); this package is its ctypes binding.
"""
from .cderi import (CD_ALG_FULL, CD_ALG_SPAN, CD_ALG_TWOSTEP, CD_ECUDA, CD_EINVAL, CD_ENOMEM, CD_ENOTPSD,
                    CD_ETIMEOUT, CD_FP64, CD_JK_BF16X3, CD_JK_BF16X4, CD_JK_BF16X5, CD_JK_FP64, CD_OK,
                    CD_UPDATE_FP64, CD_UPDATE_SLICE, CD_VEC_FP32, CDError, Factor, System, batch_persistent, batch_run,
                    cd_eri_factor, cd_eri_factor_sys, cd_version, kernel_launches, load, set_wait_limit,
                    slice_matmul)

__all__ = ["CD_ALG_FULL", "CD_ALG_SPAN", "CD_ALG_TWOSTEP", "CD_ECUDA", "CD_EINVAL", "CD_ENOMEM", "CD_ENOTPSD",
           "CD_ETIMEOUT", "CD_FP64", "CD_JK_BF16X3", "CD_JK_BF16X4", "CD_JK_BF16X5", "CD_JK_FP64", "CD_OK",
           "CD_UPDATE_FP64", "CD_UPDATE_SLICE", "CD_VEC_FP32", "CDError", "Factor", "System", "batch_persistent",
           "batch_run",
           "cd_eri_factor", "cd_eri_factor_sys", "cd_version", "kernel_launches", "load", "set_wait_limit",
           "slice_matmul"]
