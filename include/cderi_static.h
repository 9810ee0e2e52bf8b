/*
 * cderi_static.h -- Coulomb build without device allocation (libcderi.so).
 * Conventions as in cderi.h.
 */
#ifndef CDERI_STATIC_H
#define CDERI_STATIC_H

#include "cderi.h"

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Coulomb build without device allocation ------------------------------ */
/* The paper has no counterpart to this entry point.  It exists for callers
 * that cannot allocate device memory (an arena or pool that owns all device
 * memory, or a host application whose own allocator must not be bypassed).
 * J = cd_jk(f, C, n_occ, J, NULL, CD_JK_FP64 | CD_JK_DEVICE | CD_JK_ONLY_J),
 * with C_occ_dev [N][n_occ] and J_dev [N][N] device pointers owned by the
 * caller.  Scratch comes from one static device array of 16.25 MiB per GPU
 * (held until the process exits): at most 1,048,576 rows and 32,768 vectors,
 * larger factors are rejected with CD_EINVAL.  No cudaMalloc/cudaFree or
 * allocating library call is made.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) once; later calls reuse it.
 * All calls share the array: calls that overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 * Asynchronous on `stream`. */
int cd_jk_coulomb_static(const cd_factor_t* f, const double* C_occ_dev, int32_t n_occ, double* J_dev,
                         void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CDERI_STATIC_H */
