// jk.cu -- kernels (d) and (e): Coulomb and exchange matrices from the vectors
// (Sec. 4.1).  Packed density d_r = D_{mu nu} (2 - delta_{mu nu}), D = 2 C C^T.
//   J: v_P = sum_r L^P_r d_r (pass 1 over L), J_r = sum_P L^P_r v_P (pass 2).
//   K: B^P = unpack(L^P) C (N x O), K = 2 sum_P B^P B^P^T.
#include <algorithm>
#include "internal.cuh"
#include "pivot.cuh"

namespace cd {
namespace {

__global__ void density_packed_kernel(const double* __restrict__ C, int N, int O, const int32_t* __restrict__ mu,
                                      const int32_t* __restrict__ nu, int64_t n, double* __restrict__ d) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int a = mu[r], b = nu[r];
  const double* ca = C + (int64_t)a * O;
  const double* cb = C + (int64_t)b * O;
  double s = 0.0;
  for (int i = 0; i < O; ++i) s = fma(ca[i], cb[i], s);
  d[r] = (a == b ? 2.0 : 4.0) * s;
}

// ---- J, pass 1: v_P = sum_r L^P_r d_r.  A CTA takes VB consecutive vectors
// and streams them against one read of d, 16 bytes per load (double2 for FP64
// vectors, float4 for FP32; rows start on 256-byte boundaries because ld is a
// multiple of 32).  The scalar tail covers n not divisible by the vector width.
template <class T> struct Vec;
template <> struct Vec<double> { using V = double2; static constexpr int W = 2; };
template <> struct Vec<float> { using V = float4; static constexpr int W = 4; };

// acc += l . dd with one FP64 FMA per element (the FP64 pipe, not HBM, bounds J
// on this GPU: 2 FP64 operations/clk/SM), split over two accumulators
__device__ __forceinline__ void dot_w(double2 l, const double* dd, double& a0, double& a1) {
  a0 = fma(l.x, dd[0], a0);
  a1 = fma(l.y, dd[1], a1);
}
__device__ __forceinline__ void dot_w(float4 l, const double* dd, double& a0, double& a1) {
  a0 = fma((double)l.x, dd[0], a0);
  a1 = fma((double)l.y, dd[1], a1);
  a0 = fma((double)l.z, dd[2], a0);
  a1 = fma((double)l.w, dd[3], a1);
}
__device__ __forceinline__ void axpy_w(double2 l, double vp, double* a) { a[0] = fma(l.x, vp, a[0]); a[1] = fma(l.y, vp, a[1]); }
__device__ __forceinline__ void axpy_w(float4 l, double vp, double* a) {
  a[0] = fma((double)l.x, vp, a[0]); a[1] = fma((double)l.y, vp, a[1]);
  a[2] = fma((double)l.z, vp, a[2]); a[3] = fma((double)l.w, vp, a[3]);
}

constexpr int kJThreads = 256;
constexpr int kJVB = 4;   // vectors per CTA in pass 1

// grid (vector groups, row slabs): a CTA covers groups of W rows [w0, w1) of
// its vectors and adds its partial sums into v (cleared by the launcher), so
// that the grid is many waves deep and the last wave is short
template <class T>
__global__ void __launch_bounds__(kJThreads) j_pass1_kernel(const T* __restrict__ L, int64_t ld, int64_t M, int64_t n,
                                                            const double* __restrict__ d, double* __restrict__ v,
                                                            int64_t wchunk) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
  const int64_t P0 = (int64_t)blockIdx.x * kJVB;
  const int nv = (int)min((int64_t)kJVB, M - P0);
  double acc[kJVB], acc2[kJVB];
#pragma unroll
  for (int j = 0; j < kJVB; ++j) acc[j] = acc2[j] = 0.0;
  const int64_t nw = n / W;
  const int64_t w0 = (int64_t)blockIdx.y * wchunk;
  const int64_t w1 = min(nw, w0 + wchunk);
  const V* rowv[kJVB];
#pragma unroll
  for (int j = 0; j < kJVB; ++j) rowv[j] = reinterpret_cast<const V*>(L + (P0 + (j < nv ? j : 0)) * ld);
#pragma unroll 2
  for (int64_t i = w0 + threadIdx.x; i < w1; i += kJThreads) {
    double dd[W];
    if constexpr (W == 2) {
      const double2 x = __ldg(reinterpret_cast<const double2*>(d) + i);
      dd[0] = x.x; dd[1] = x.y;
    } else {
      const double2 x0 = __ldg(reinterpret_cast<const double2*>(d) + 2 * i);
      const double2 x1 = __ldg(reinterpret_cast<const double2*>(d) + 2 * i + 1);
      dd[0] = x0.x; dd[1] = x0.y; dd[2] = x1.x; dd[3] = x1.y;
    }
#pragma unroll
    for (int j = 0; j < kJVB; ++j)
      if (j < nv) dot_w(__ldg(rowv[j] + i), dd, acc[j], acc2[j]);
  }
#pragma unroll
  for (int j = 0; j < kJVB; ++j) acc[j] += acc2[j];
  if (blockIdx.y == gridDim.y - 1)   // the rows past the last whole group of W
    for (int64_t r = nw * W + threadIdx.x; r < n; r += kJThreads)
#pragma unroll
      for (int j = 0; j < kJVB; ++j)
        if (j < nv) acc[j] = fma((double)L[(P0 + j) * ld + r], d[r], acc[j]);
  // CTA reduction of the kJVB sums
  __shared__ double sh[kJThreads / 32][kJVB];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < kJVB; ++j) {
    double x = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) sh[w][j] = x;
  }
  __syncthreads();
  if (threadIdx.x < kJVB && (int)threadIdx.x < nv) {
    double x = 0.0;
#pragma unroll
    for (int k = 0; k < kJThreads / 32; ++k) x += sh[k][threadIdx.x];
    atomicAdd(v + P0 + threadIdx.x, x);
  }
}

// ---- J, pass 2: y_r = sum_P L^P_r v_P.  A thread owns W consecutive rows and
// walks the vectors [P0, P1) of its slab (16-byte loads, coalesced across the
// warp); with one slab it stores y, with several it adds atomically into a
// cleared y.
template <class T>
__global__ void __launch_bounds__(kJThreads) j_pass2_kernel(const T* __restrict__ L, int64_t ld, int64_t M, int64_t n,
                                                            const double* __restrict__ v, double* __restrict__ y,
                                                            int64_t pchunk, int atomic) {
  using V = typename Vec<T>::V;
  constexpr int W = Vec<T>::W;
  const int64_t i = (int64_t)blockIdx.x * kJThreads + threadIdx.x;   // group of W rows
  const int64_t r0 = i * W;
  if (r0 >= n) return;
  const int64_t P0 = (int64_t)blockIdx.y * pchunk;
  const int64_t P1 = min(M, P0 + pchunk);
  double a[W];
#pragma unroll
  for (int k = 0; k < W; ++k) a[k] = 0.0;
  if (r0 + W <= n) {
    const V* base = reinterpret_cast<const V*>(L) + i;
    const int64_t ldv = ld / W;
    int64_t P = P0;
    for (; P + 4 <= P1; P += 4) {
      const V l0 = __ldg(base + (P + 0) * ldv), l1 = __ldg(base + (P + 1) * ldv);
      const V l2 = __ldg(base + (P + 2) * ldv), l3 = __ldg(base + (P + 3) * ldv);
      axpy_w(l0, __ldg(v + P + 0), a); axpy_w(l1, __ldg(v + P + 1), a);
      axpy_w(l2, __ldg(v + P + 2), a); axpy_w(l3, __ldg(v + P + 3), a);
    }
    for (; P < P1; ++P) axpy_w(__ldg(base + P * ldv), __ldg(v + P), a);
  } else {
    for (int64_t P = P0; P < P1; ++P)
      for (int k = 0; k < W && r0 + k < n; ++k) a[k] = fma((double)L[P * ld + r0 + k], v[P], a[k]);
  }
#pragma unroll
  for (int k = 0; k < W; ++k) {
    if (r0 + k >= n) break;
    if (atomic) atomicAdd(y + r0 + k, a[k]);
    else y[r0 + k] = a[k];
  }
}

__global__ void unpack_sym_kernel(const double* __restrict__ packed, const int32_t* __restrict__ mu,
                                  const int32_t* __restrict__ nu, int64_t n, int N, double* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double v = packed[r];
  out[(int64_t)mu[r] * N + nu[r]] = v;
  out[(int64_t)nu[r] * N + mu[r]] = v;
}

template <class T, class TO>
__global__ void unpack_vectors_kernel(const T* __restrict__ L, int64_t ld, int64_t P0, const int32_t* __restrict__ mu,
                                      const int32_t* __restrict__ nu, int64_t n, int N, TO* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (r >= n) return;
  const TO v = (TO)L[(P0 + p) * ld + r];
  TO* o = out + (int64_t)p * N * N;
  o[(int64_t)mu[r] * N + nu[r]] = v;
  o[(int64_t)nu[r] * N + mu[r]] = v;
}

}  // namespace

int launch_density_packed(const double* C, int N, int O, const int32_t* mu, const int32_t* nu, int64_t n,
                          double* d, cudaStream_t st) {
  if (n <= 0) return CD_OK;
  density_packed_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(C, N, O, mu, nu, n, d);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

// resident CTAs of the J kernels (256 threads, < 64 registers: 8 per SM) and the
// grid depth aimed at, in waves
constexpr int64_t kJResident = 148 * 8;
constexpr int64_t kJWaves = 8;

template <class T>
int launch_gemv_rows(const T* L, int64_t ld, int64_t M, int64_t n, const double* x, double* y, cudaStream_t st) {
  if (M <= 0) return CD_OK;
  if (ld % Vec<T>::W) { set_error("J: vector leading dimension not a multiple of the load width"); return CD_EINVAL; }
  const int64_t groups = (M + kJVB - 1) / kJVB;
  const int64_t nw = n / Vec<T>::W;
  int64_t rs = (kJWaves * kJResident + groups - 1) / groups;          // row slabs per vector group
  rs = std::max<int64_t>(1, std::min<int64_t>(rs, (nw + kJThreads - 1) / kJThreads));
  const int64_t wchunk = std::max<int64_t>(1, (nw + rs - 1) / rs);
  rs = std::max<int64_t>(1, (nw + wchunk - 1) / wchunk);
  CD_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * M, st));
  j_pass1_kernel<T><<<dim3((unsigned)groups, (unsigned)rs), kJThreads, 0, st>>>(L, ld, M, n, x, y, wchunk);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template <class T>
int launch_gemv_cols(const T* L, int64_t ld, int64_t M, int64_t n, const double* v, double* y, cudaStream_t st) {
  if (n <= 0) return CD_OK;
  if (ld % Vec<T>::W) { set_error("J: vector leading dimension not a multiple of the load width"); return CD_EINVAL; }
  constexpr int W = Vec<T>::W;
  const int64_t tiles = (n + (int64_t)W * kJThreads - 1) / ((int64_t)W * kJThreads);
  // split the vectors into slabs so that the grid is kJWaves waves deep
  int64_t splits = (kJWaves * kJResident + tiles - 1) / tiles;
  if (splits > M) splits = M;
  if (splits < 1) splits = 1;
  const int64_t pchunk = M > 0 ? (M + splits - 1) / splits : 0;
  if (M > 0) splits = (M + pchunk - 1) / pchunk;
  // y is stored directly by a single slab; several slabs (and M = 0: y = 0) need it cleared
  if (splits > 1 || M <= 0) CD_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n, st));
  if (M <= 0) return CD_OK;
  dim3 grid((unsigned)tiles, (unsigned)splits);
  j_pass2_kernel<T><<<grid, kJThreads, 0, st>>>(L, ld, M, n, v, y, pchunk, splits > 1 ? 1 : 0);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_unpack_sym(const double* packed, const int32_t* mu, const int32_t* nu, int64_t n, int N, double* out,
                      cudaStream_t st) {
  CD_CUDA(cudaMemsetAsync(out, 0, sizeof(double) * N * N, st));
  if (n <= 0) return CD_OK;
  unpack_sym_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(packed, mu, nu, n, N, out);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template <class T, class TO>
int launch_unpack_vectors(const T* L, int64_t ld, int64_t P0, int Pc, const int32_t* mu, const int32_t* nu,
                          int64_t n, int N, TO* out, cudaStream_t st) {
  CD_CUDA(cudaMemsetAsync(out, 0, sizeof(TO) * (size_t)Pc * N * N, st));
  if (n <= 0 || Pc <= 0) return CD_OK;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)Pc);
  unpack_vectors_kernel<T, TO><<<grid, 256, 0, st>>>(L, ld, P0, mu, nu, n, N, out);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template int launch_gemv_rows<double>(const double*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_gemv_rows<float>(const float*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_gemv_cols<double>(const double*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_gemv_cols<float>(const float*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_unpack_vectors<double, double>(const double*, int64_t, int64_t, int, const int32_t*,
                                                   const int32_t*, int64_t, int, double*, cudaStream_t);
template int launch_unpack_vectors<float, double>(const float*, int64_t, int64_t, int, const int32_t*,
                                                  const int32_t*, int64_t, int, double*, cudaStream_t);

}  // namespace cd
