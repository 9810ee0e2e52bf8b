// colupd.cu -- kernel (c): the blocked column update of Eq. (subtr),
//   col_j(r) -= sum_{K in [k0,k1)} L^K_r L^K_{c_j},
// as an FP64 GEMM (rows x K) x (K x b), plus a generic strided FP64 GEMM used
// by the exchange build.  On this GPU the FP64 pipe (about 1.1 TFLOP/s for
// both DFMA and the legacy DMMA path, measured) bounds both, so the kernels
// are register-tiled DFMA loops with shared-memory staging; arithmetic
// intensity is 2 flop per 8-byte L element per column of the block.
#include "internal.cuh"
#include "pivot.cuh"

namespace cd {
namespace {

constexpr int kTR = 128, kTC = 32, kTK = 16;

__global__ void __launch_bounds__(256) colupd_kernel(double* __restrict__ cols, int64_t ld,
                                                     const int32_t* __restrict__ slots, int nb,
                                                     const double* __restrict__ L, int64_t k0, int64_t k1,
                                                     const double* __restrict__ Bg, int64_t n) {
  __shared__ double As[kTK][kTR];
  __shared__ double Bs[kTK][kTC];
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int64_t r0 = (int64_t)blockIdx.x * kTR;
  const int j0 = blockIdx.y * kTC;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
  for (int64_t kk = k0; kk < k1; kk += kTK) {
#pragma unroll
    for (int t = 0; t < (kTK * kTR) / 256; ++t) {
      const int idx = tid + 256 * t, k = idx / kTR, r = idx % kTR;
      As[k][r] = (kk + k < k1 && r0 + r < n) ? L[(kk + k) * ld + r0 + r] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < (kTK * kTC) / 256; ++t) {
      const int idx = tid + 256 * t, k = idx / kTC, j = idx % kTC;
      Bs[k][j] = (kk + k < k1 && j0 + j < nb) ? Bg[(kk + k - k0) * nb + j0 + j] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kTK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tx + 32 * i];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[k][ty * 4 + c];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[i][c] = fma(a[i], b[c], acc[i][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = j0 + ty * 4 + c;
    if (j >= nb) continue;
    double* C = cols + (int64_t)slots[j] * ld;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = r0 + tx + 32 * i;
      if (r < n) C[r] -= acc[i][c];
    }
  }
}

constexpr int kGM = 64, kGN = 64, kGK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(int m, int n, int k, int batch, double alpha,
                                                    const double* __restrict__ A, int64_t ars, int64_t acs, int64_t abs_,
                                                    const double* __restrict__ B, int64_t brs, int64_t bcs, int64_t bbs,
                                                    double* __restrict__ C, int64_t ldc, int64_t cbs, int reduce_batch,
                                                    int accumulate) {
  __shared__ double As[kGK][kGM];
  __shared__ double Bs[kGK][kGN + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * kGM, j0 = blockIdx.y * kGN;
  double acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
  const int b_begin = reduce_batch ? 0 : blockIdx.z;
  const int b_end = reduce_batch ? batch : blockIdx.z + 1;
  for (int b = b_begin; b < b_end; ++b) {
    const double* Ab = A + (int64_t)b * abs_;
    const double* Bb = B + (int64_t)b * bbs;
    for (int kk = 0; kk < k; kk += kGK) {
#pragma unroll
      for (int t = 0; t < (kGK * kGM) / 256; ++t) {
        const int idx = tid + 256 * t, kx = idx / kGM, ix = idx % kGM;
        const int gi = i0 + ix, gk = kk + kx;
        As[kx][ix] = (gi < m && gk < k) ? Ab[(int64_t)gi * ars + (int64_t)gk * acs] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < (kGK * kGN) / 256; ++t) {
        const int idx = tid + 256 * t, kx = idx / kGN, jx = idx % kGN;
        const int gj = j0 + jx, gk = kk + kx;
        Bs[kx][jx] = (gj < n && gk < k) ? Bb[(int64_t)gk * brs + (int64_t)gj * bcs] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kx = 0; kx < kGK; ++kx) {
        double a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kx][tx + 16 * i];
#pragma unroll
        for (int c = 0; c < 4; ++c) bb[c] = Bs[kx][ty + 16 * c];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[i][c] = fma(a[i], bb[c], acc[i][c]);
      }
      __syncthreads();
    }
  }
  double* Cb = C + (reduce_batch ? 0 : (int64_t)blockIdx.z * cbs);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + tx + 16 * i;
    if (gi >= m) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int gj = j0 + ty + 16 * c;
      if (gj >= n) continue;
      double* p = Cb + (int64_t)gi * ldc + gj;
      *p = accumulate ? fma(alpha, acc[i][c], *p) : alpha * acc[i][c];
    }
  }
}

}  // namespace

int launch_colupd(double* cols, int64_t ld, const int32_t* slots_dev, int nb, const double* L,
                  int64_t k0, int64_t k1, const double* Bg, int64_t n, cudaStream_t st) {
  if (nb <= 0 || k1 <= k0 || n <= 0) return CD_OK;
  dim3 grid((unsigned)((n + kTR - 1) / kTR), (unsigned)((nb + kTC - 1) / kTC));
  colupd_kernel<<<grid, 256, 0, st>>>(cols, ld, slots_dev, nb, L, k0, k1, Bg, n);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_dgemm(int m, int n, int k, int batch, double alpha,
                 const double* A, int64_t ars, int64_t acs, int64_t abs_,
                 const double* B, int64_t brs, int64_t bcs, int64_t bbs,
                 double* C, int64_t ldc, int64_t cbs, bool reduce_batch, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0 || batch <= 0) return CD_OK;
  dim3 grid((unsigned)((m + kGM - 1) / kGM), (unsigned)((n + kGN - 1) / kGN), reduce_batch ? 1u : (unsigned)batch);
  dgemm_kernel<<<grid, 256, 0, st>>>(m, n, k, batch, alpha, A, ars, acs, abs_, B, brs, bcs, bbs, C, ldc, cbs,
                                      reduce_batch ? 1 : 0, reduce_batch ? 1 : 0);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

}  // namespace cd
