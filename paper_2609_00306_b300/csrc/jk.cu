// jk.cu -- kernels (d) and (e): Coulomb and exchange matrices from the vectors
// (Sec. 4.1).  Packed density d_r = D_{mu nu} (2 - delta_{mu nu}), D = 2 C C^T.
//   J: v_P = sum_r L^P_r d_r (pass 1 over L), J_r = sum_P L^P_r v_P (pass 2).
//   K: B^P = unpack(L^P) C (N x O), K = 2 sum_P B^P B^P^T.
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

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  return v;
}

template <class T>
__global__ void __launch_bounds__(256) gemv_rows_kernel(const T* __restrict__ L, int64_t ld, int64_t n,
                                                        const double* __restrict__ x, double* __restrict__ y) {
  const int64_t P = blockIdx.x;
  const T* row = L + P * ld;
  double s = 0.0;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s = fma((double)row[r], x[r], s);
  s = block_sum(s);
  if (threadIdx.x == 0) y[P] = s;
}

template <class T>
__global__ void __launch_bounds__(256) gemv_cols_kernel(const T* __restrict__ L, int64_t ld, int64_t M, int64_t n,
                                                        const double* __restrict__ v, double* __restrict__ y,
                                                        int64_t pchunk) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t P0 = (int64_t)blockIdx.y * pchunk;
  const int64_t P1 = min(M, P0 + pchunk);
  if (r >= n) return;
  double s = 0.0;
  for (int64_t P = P0; P < P1; ++P) s = fma((double)L[P * ld + r], v[P], s);
  atomicAdd(y + r, s);
}

__global__ void unpack_sym_kernel(const double* __restrict__ packed, const int32_t* __restrict__ mu,
                                  const int32_t* __restrict__ nu, int64_t n, int N, double* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double v = packed[r];
  out[(int64_t)mu[r] * N + nu[r]] = v;
  out[(int64_t)nu[r] * N + mu[r]] = v;
}

template <class T>
__global__ void unpack_vectors_kernel(const T* __restrict__ L, int64_t ld, int64_t P0, const int32_t* __restrict__ mu,
                                      const int32_t* __restrict__ nu, int64_t n, int N, T* __restrict__ out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (r >= n) return;
  const T v = L[(P0 + p) * ld + r];
  T* o = out + (int64_t)p * N * N;
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

template <class T>
int launch_gemv_rows(const T* L, int64_t ld, int64_t M, int64_t n, const double* x, double* y, cudaStream_t st) {
  if (M <= 0) return CD_OK;
  gemv_rows_kernel<T><<<(unsigned)M, 256, 0, st>>>(L, ld, n, x, y);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template <class T>
int launch_gemv_cols(const T* L, int64_t ld, int64_t M, int64_t n, const double* v, double* y, cudaStream_t st) {
  if (n <= 0) return CD_OK;
  // y accumulates with atomics: clear it first, also when there is no vector
  // (M = 0 gives y = 0)
  CD_CUDA(cudaMemsetAsync(y, 0, sizeof(double) * n, st));
  if (M <= 0) return CD_OK;
  const int64_t tiles = (n + 255) / 256;
  int64_t splits = (148 * 8 + tiles - 1) / tiles;
  if (splits < 1) splits = 1;
  if (splits > M) splits = M;
  const int64_t pchunk = (M + splits - 1) / splits;
  splits = (M + pchunk - 1) / pchunk;
  dim3 grid((unsigned)tiles, (unsigned)splits);
  gemv_cols_kernel<T><<<grid, 256, 0, st>>>(L, ld, M, n, v, y, pchunk);
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

template <class T>
int launch_unpack_vectors(const T* L, int64_t ld, int64_t P0, int Pc, const int32_t* mu, const int32_t* nu,
                          int64_t n, int N, T* out, cudaStream_t st) {
  CD_CUDA(cudaMemsetAsync(out, 0, sizeof(T) * (size_t)Pc * N * N, st));
  if (n <= 0 || Pc <= 0) return CD_OK;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)Pc);
  unpack_vectors_kernel<T><<<grid, 256, 0, st>>>(L, ld, P0, mu, nu, n, N, out);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template int launch_gemv_rows<double>(const double*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_gemv_rows<float>(const float*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_gemv_cols<double>(const double*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_gemv_cols<float>(const float*, int64_t, int64_t, int64_t, const double*, double*, cudaStream_t);
template int launch_unpack_vectors<double>(const double*, int64_t, int64_t, int, const int32_t*, const int32_t*,
                                           int64_t, int, double*, cudaStream_t);
template int launch_unpack_vectors<float>(const float*, int64_t, int64_t, int, const int32_t*, const int32_t*,
                                          int64_t, int, float*, cudaStream_t);

}  // namespace cd
