// mixed.cu -- mixed-precision J/K.  The decomposition itself is FP64; the
// vectors are rounded once to FP32 and contracted on the tensor cores:
//   B^P = L^P C      (S BF16 slices of the FP32 rows of L^P and of C^T)
//   K   = 2 sum_P B^P B^P^T   (S BF16 slices of the rows of B, kept in FP64)
// Each product runs through the exact-slice GEMM (ozaki.cu): BF16 integer
// slices, exact FP32 accumulation inside a k-chunk, 64-bit fixed-point sums;
// the only roundings are the FP32 storage of L, the 8S-bit slicing of each
// operand row below its maximum, and the final FP64 scaling.  J accumulates FP32 vector entries against the
// FP64 packed density in FP64.
#include <cuda_bf16.h>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "internal.cuh"
#include "ozaki.cuh"
#include "pivot.cuh"

namespace cd {
namespace {

__global__ void to_fp32_kernel(const double* __restrict__ src, int64_t total, float* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __double2float_rn(src[i]);
}

// one warp per row: e[r] = frexp exponent of max_k |X[r][k]| (0 for a zero row);
// the maximum is taken on the magnitude bit patterns (integer compares only)
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long mag_bits(float x) {
  return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
}
template <class T>
__global__ void row_exp_warp_kernel(const T* __restrict__ X, int64_t ldx, int64_t rows, int64_t k,
                                    int32_t* __restrict__ e) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= rows) return;
  unsigned long long m = 0;
  for (int64_t c = lane; c < k; c += 32) m = max(m, mag_bits(X[r * ldx + c]));
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) {
    int ex = 0;
    if (m != 0) {
      const double mx = sizeof(T) == 8 ? __longlong_as_double((long long)m) : (double)__uint_as_float((unsigned)m);
      frexp(mx, &ex);
    }
    e[r] = ex;
  }
}

// dst[s][r][k] = s-th 8-bit slice of X[r][k] / 2^e[r]  (S = 3 or 4 slices: 24 or 32 bits
// of fixed point below the row maximum); one multiply by a power of two and one
// conversion per element, then integer digit extraction
template <class T, int S>
__global__ void slice_kernel(const T* __restrict__ X, int64_t ldx, int64_t rows, int64_t k,
                             const int32_t* __restrict__ e, __nv_bfloat16* __restrict__ dst, int64_t kpitch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * kpitch) return;
  const int64_t r = t / kpitch, c = t % kpitch;
  long long v = 0;
  if (c < k) v = scaled_double_to_ll(X[r * ldx + c], 8 * S - 1 - e[r]);  // integer ops only
  float a[S];
  fixed_digits<S>(v, a);
#pragma unroll
  for (int s = 0; s < S; ++s) dst[((int64_t)s * rows + r) * kpitch + c] = __float2bfloat16_rn(a[s]);
}

// idx[mu*N + nu] = row of the pair (max(mu, nu), min(mu, nu)); the caller
// fills idx with -1 first, which then marks the screened-out pairs
__global__ void pair_index_kernel(const int32_t* __restrict__ mu, const int32_t* __restrict__ nu, int64_t n, int N,
                                  int32_t* __restrict__ idx) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int a = mu[r], b = nu[r];
  idx[(int64_t)a * N + b] = (int32_t)r;
  idx[(int64_t)b * N + a] = (int32_t)r;
}

// One CTA per dense row (p, mu) of the chunk's vectors L^{P0+p} (symmetric
// N x N unpacking of a packed vector): the row is gathered straight from the
// packed vector through idx, its exponent e = frexp exponent of the row
// maximum is found, and the row is cut into S exact 8-bit slices of
// x / 2^e, written in the k-contiguous layout dst[s][row][kpitch] that the
// tensor-core product loads by TMA.  The two sweeps over the row read the
// packed vector twice; the second read comes from L2.  This replaces a dense
// FP64/FP32 unpacking (a cleared N x N matrix per vector), a separate
// row-exponent pass and a separate slicing pass.
constexpr int kUnpackThreads = 128;
template <class T, int S>
__global__ void __launch_bounds__(kUnpackThreads) unpack_slice_kernel(const T* __restrict__ L, int64_t ld, int64_t P0,
                                                                      const int32_t* __restrict__ idx, int N,
                                                                      int64_t rows, int64_t kpitch,
                                                                      int32_t* __restrict__ e,
                                                                      __nv_bfloat16* __restrict__ dst) {
  const int64_t row = blockIdx.x;                  // p * N + mu
  const int64_t p = row / N, mu = row % N;
  const T* __restrict__ Lp = L + (P0 + p) * ld;
  const int32_t* __restrict__ ir = idx + mu * N;
  unsigned long long m = 0;
  for (int nu = threadIdx.x; nu < N; nu += kUnpackThreads) {
    const int32_t r = __ldg(ir + nu);
    if (r >= 0) m = max(m, mag_bits(__ldg(Lp + r)));
  }
  __shared__ unsigned long long sh[kUnpackThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
#pragma unroll
  for (int w = 0; w < kUnpackThreads / 32; ++w) m = max(m, sh[w]);
  int ex = 0;
  if (m != 0) {
    const double mx = sizeof(T) == 8 ? __longlong_as_double((long long)m) : (double)__uint_as_float((unsigned)m);
    frexp(mx, &ex);
  }
  if (threadIdx.x == 0) e[row] = ex;
  const int k = 8 * S - 1 - ex;
  for (int64_t nu = threadIdx.x; nu < kpitch; nu += kUnpackThreads) {
    long long v = 0;
    if (nu < N) {
      const int32_t r = __ldg(ir + nu);
      if (r >= 0) v = scaled_double_to_ll(__ldg(Lp + r), k);   // integer operations only
    }
    float a[S];
    fixed_digits<S>(v, a);
#pragma unroll
    for (int s = 0; s < S; ++s) dst[((int64_t)s * rows + row) * kpitch + nu] = __float2bfloat16_rn(a[s]);
  }
}

// B chunk from the fixed-point product: D[i][p*N + mu] (i < O) -> Bm[mu][p*Op + i]
__global__ void half_finalize_kernel(const unsigned long long* __restrict__ D, int64_t ldd, int Pc, int N, int O,
                                     int Op, const int32_t* __restrict__ eL, const int32_t* __restrict__ eC, int F,
                                     double* __restrict__ Bm) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = (int64_t)Pc * N * O;
  if (t >= tot) return;
  const int i = (int)(t % O);
  const int64_t row = t / O;  // p*N + mu
  const int p = (int)(row / N), mu = (int)(row % N);
  const double v = ldexp((double)(long long)D[(int64_t)i * ldd + row], eL[row] + eC[i] - F);
  Bm[(int64_t)mu * ((int64_t)Pc * Op) + (int64_t)p * Op + i] = v;
}

// K[mu][nu] += 2 * 2^(e_mu + e_nu - F) * D[max][min]  (only the upper triangle of
// the symmetric product is computed: row index <= column index)
__global__ void k_accumulate_kernel(const unsigned long long* __restrict__ D, int N, const int32_t* __restrict__ eB,
                                    int F, double* __restrict__ K) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * N) return;
  const int mu = (int)(t / N), nu = (int)(t % N);
  const int lo = min(mu, nu), hi = max(mu, nu);
  K[t] += ldexp((double)(long long)D[(int64_t)hi * N + lo], eB[mu] + eB[nu] - F + 1);
}

template <class T>
int launch_row_exp_warp(const T* X, int64_t ldx, int64_t rows, int64_t k, int32_t* e, cudaStream_t st) {
  if (rows <= 0) return CD_OK;
  row_exp_warp_kernel<T><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(X, ldx, rows, k, e);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template <class T>
int launch_slice3(const T* X, int64_t ldx, int64_t rows, int64_t k, const int32_t* e, void* dst, int64_t kpitch,
                  int S, cudaStream_t st) {
  const int64_t tot = rows * kpitch;
  if (tot <= 0) return CD_OK;
  const unsigned grid = (unsigned)((tot + 255) / 256);
  if (S == 3) slice_kernel<T, 3><<<grid, 256, 0, st>>>(X, ldx, rows, k, e, (__nv_bfloat16*)dst, kpitch);
  else if (S == 4) slice_kernel<T, 4><<<grid, 256, 0, st>>>(X, ldx, rows, k, e, (__nv_bfloat16*)dst, kpitch);
  else if (S == 5) slice_kernel<T, 5><<<grid, 256, 0, st>>>(X, ldx, rows, k, e, (__nv_bfloat16*)dst, kpitch);
  else slice_kernel<T, 7><<<grid, 256, 0, st>>>(X, ldx, rows, k, e, (__nv_bfloat16*)dst, kpitch);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

// pair -> row table of the dense unpacking ([N][N] int32, -1 = screened out)
int build_pair_index(const int32_t* mu, const int32_t* nu, int64_t n, int N, int32_t* idx, cudaStream_t st) {
  CD_CUDA(cudaMemsetAsync(idx, 0xFF, sizeof(int32_t) * (size_t)N * N, st));
  if (n <= 0) return CD_OK;
  pair_index_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mu, nu, n, N, idx);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

// rows (p, mu) of vectors P0 .. P0+pc-1: exponents e [pc*N] and slices dst [S][pc*N][kpitch]
template <class T>
int launch_unpack_slice(const T* L, int64_t ld, int64_t P0, int pc, const int32_t* idx, int N, int64_t kpitch,
                        int S, int32_t* e, void* dst, cudaStream_t st) {
  const int64_t rows = (int64_t)pc * N;
  if (rows <= 0) return CD_OK;
  __nv_bfloat16* d = (__nv_bfloat16*)dst;
  const unsigned grid = (unsigned)rows;
  if (S == 3) unpack_slice_kernel<T, 3><<<grid, kUnpackThreads, 0, st>>>(L, ld, P0, idx, N, rows, kpitch, e, d);
  else if (S == 4) unpack_slice_kernel<T, 4><<<grid, kUnpackThreads, 0, st>>>(L, ld, P0, idx, N, rows, kpitch, e, d);
  else if (S == 5) unpack_slice_kernel<T, 5><<<grid, kUnpackThreads, 0, st>>>(L, ld, P0, idx, N, rows, kpitch, e, d);
  else if (S == 7) unpack_slice_kernel<T, 7><<<grid, kUnpackThreads, 0, st>>>(L, ld, P0, idx, N, rows, kpitch, e, d);
  else { set_error("unpack_slice: unsupported slice count"); return CD_EINVAL; }
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int ilog2_ceil(int64_t v) {
  int l = 0;
  while ((1ll << l) < v) ++l;
  return l;
}

}  // namespace

int launch_to_fp32(const double* src, int64_t ld, int64_t M, int64_t n, float* dst, cudaStream_t st) {
  const int64_t total = M * ld;
  if (total <= 0) return CD_OK;
  (void)n;
  to_fp32_kernel<<<148 * 8, 256, 0, st>>>(src, total, dst);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

namespace {
struct MixedBufs {
  cudaStream_t st = nullptr;
  void* Ls = nullptr;
  void* Cs = nullptr;
  double* Ct = nullptr;
  int32_t *eL = nullptr, *eC = nullptr, *eB = nullptr;
  unsigned long long *D1 = nullptr, *D2 = nullptr;
  double* Bm = nullptr;
  void* Bs = nullptr;
  double *d = nullptr, *v = nullptr, *Jp = nullptr;
  int32_t* idx = nullptr;
  int* err = nullptr;
  ~MixedBufs() {
    for (void* p : {Ls, Cs, (void*)Ct, (void*)eL, (void*)eC, (void*)eB, (void*)D1, (void*)D2, (void*)Bm,
                    Bs, (void*)d, (void*)v, (void*)Jp, (void*)idx, (void*)err})
      scratch_free(p, st);
  }
};
__global__ void transpose_kernel(const double* __restrict__ C, int N, int O, double* __restrict__ Ct) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)N * O) return;
  const int nu = (int)(t / O), i = (int)(t % O);
  Ct[(int64_t)i * N + nu] = C[t];
}
}  // namespace

// Optional stage timing (environment variable CDERI_TIMING=1): CUDA events
// around the stages of the exchange build, summed over chunks, on stderr.
struct StageTimer {
  bool on = false;
  cudaStream_t st = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<int> stage;
  void mark(int s) {
    if (!on) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, st);
    ev.push_back(e);
    stage.push_back(s);
  }
  void report(const char* names[], int nst) {
    if (!on || ev.empty()) return;
    cudaEventSynchronize(ev.back());
    std::vector<double> t(nst, 0.0);
    for (size_t i = 1; i < ev.size(); ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
      t[stage[i]] += ms;
    }
    for (int i = 0; i < nst; ++i) fprintf(stderr, "[cderi timing] %-12s %9.2f ms\n", names[i], t[i]);
    for (auto e : ev) cudaEventDestroy(e);
  }
};

template <class TL>
int jk_mixed_t(const TL* L32, int64_t ld, int64_t M, int64_t n, int N, int O, const double* C_dev,
               const int32_t* mu, const int32_t* nu, double* J_dev, double* K_dev, bool wantJ, bool wantK,
               int S, cudaStream_t st) {
  StageTimer tm;
  tm.on = getenv("CDERI_TIMING") != nullptr;
  tm.st = st;
  const char* names[] = {"start", "J", "unused", "unpack_slice_L", "gemm_BLC", "finalize_B", "slice_B", "gemm_K", "accum_K"};
  tm.mark(0);
  MixedBufs b;
  b.st = st;
  if (wantJ) {
    CD_TRY(scratch_alloc(&b.d, (size_t)n, st));
    CD_TRY(scratch_alloc(&b.v, (size_t)M, st));
    CD_TRY(scratch_alloc(&b.Jp, (size_t)n, st));
    CD_TRY(launch_density_packed(C_dev, N, O, mu, nu, n, b.d, st));
    CD_TRY(launch_gemv_rows<TL>(L32, ld, M, n, b.d, b.v, st));
    CD_TRY(launch_gemv_cols<TL>(L32, ld, M, n, b.v, b.Jp, st));
    CD_TRY(launch_unpack_sym(b.Jp, mu, nu, n, N, J_dev, st));
    tm.mark(1);
  }
  if (wantK) {
    const int64_t Np = (N + 7) / 8 * 8;                     // k pitch of the first product (16-byte rows)
    const int Op = (O + 63) / 64 * 64;                      // padded occupied count (k blocks of the second product)
    // chunk of vectors: k-dim of the second product Pc*Op, scratch ~ Pc*N^2*(4 + 6) bytes
    int Pc = (int)std::max<int64_t>(1, std::min<int64_t>(M, (int64_t)(2.0e9 / (2.0 * S * N * (double)N))));
    Pc = std::min(Pc, 64);
    CD_TRY(scratch_alloc(&b.idx, (size_t)N * N, st));
    CD_TRY(build_pair_index(mu, nu, n, N, b.idx, st));
    CD_TRY(scratch_alloc((uint16_t**)&b.Ls, (size_t)S * Pc * N * Np, st));
    CD_TRY(scratch_alloc((uint16_t**)&b.Cs, (size_t)S * O * Np, st));
    CD_TRY(scratch_alloc(&b.Ct, (size_t)O * N, st));
    CD_TRY(scratch_alloc(&b.eL, (size_t)Pc * N, st));
    CD_TRY(scratch_alloc(&b.eC, (size_t)O, st));
    CD_TRY(scratch_alloc(&b.eB, (size_t)N, st));
    CD_TRY(scratch_alloc(&b.D1, (size_t)O * Pc * N, st));
    CD_TRY(scratch_alloc(&b.D2, (size_t)N * N, st));
    CD_TRY(scratch_alloc(&b.Bm, (size_t)N * Pc * Op, st));
    CD_TRY(scratch_alloc((uint16_t**)&b.Bs, (size_t)S * N * Pc * Op, st));
    CD_TRY(scratch_alloc(&b.err, 1, st));
    CD_CUDA(cudaMemsetAsync(b.err, 0, sizeof(int), st));
    CD_CUDA(cudaMemsetAsync(K_dev, 0, sizeof(double) * N * N, st));
    // C^T slices (rows i, k = nu)
    transpose_kernel<<<(unsigned)(((int64_t)N * O + 255) / 256), 256, 0, st>>>(C_dev, N, O, b.Ct);
    count_launch();
    CD_TRY(launch_row_exp_warp<double>(b.Ct, N, O, N, b.eC, st));
    CD_TRY(launch_slice3<double>(b.Ct, N, O, N, b.eC, b.Cs, Np, S, st));
    OzakiPlan p1, p2;
    p1.SA = p1.SB = S; p1.KEEP = S + 1; p1.F = 61 - ilog2_ceil(N);
    p2.SA = p2.SB = S; p2.KEEP = S + 1;
    for (int64_t P0 = 0; P0 < M; P0 += Pc) {
      const int pc = (int)std::min<int64_t>(Pc, M - P0);
      // rows (p, mu) of the dense L^P gathered from the packed vectors, their exponents and slices
      tm.mark(0);
      CD_TRY(launch_unpack_slice<TL>(L32, ld, P0, pc, b.idx, N, Np, S, b.eL, b.Ls, st));
      tm.mark(3);
      // B^P = L^P C for the chunk: D1[i][p*N+mu]
      CD_CUDA(cudaMemsetAsync(b.D1, 0, sizeof(unsigned long long) * O * pc * N, st));
      CD_TRY(ozaki_gemm(p1, b.Ls, (int64_t)pc * N, Np, b.Cs, O, Np, N, b.D1, (int64_t)pc * N, 1, b.err, st));
      tm.mark(4);
      CD_CUDA(cudaMemsetAsync(b.Bm, 0, sizeof(double) * N * pc * Op, st));
      {
        const int64_t tot = (int64_t)pc * N * O;
        half_finalize_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b.D1, (int64_t)pc * N, pc, N, O, Op, b.eL,
                                                                            b.eC, p1.F, b.Bm);
        count_launch();
      }
      tm.mark(5);
      // K += 2 B B^T over the chunk's (p, i)
      const int64_t kd = (int64_t)pc * Op;
      CD_TRY(launch_row_exp_warp<double>(b.Bm, kd, N, kd, b.eB, st));
      CD_TRY(launch_slice3<double>(b.Bm, kd, N, kd, b.eB, b.Bs, kd, S, st));
      p2.F = 61 - ilog2_ceil(kd);
      tm.mark(6);
      CD_CUDA(cudaMemsetAsync(b.D2, 0, sizeof(unsigned long long) * N * N, st));
      CD_TRY(ozaki_gemm(p2, b.Bs, N, kd, b.Bs, N, kd, kd, b.D2, N, 2, b.err, st, true));
      tm.mark(7);
      k_accumulate_kernel<<<(unsigned)(((int64_t)N * N + 255) / 256), 256, 0, st>>>(b.D2, N, b.eB, p2.F, K_dev);
      count_launch();
      tm.mark(8);
    }
    tm.report(names, 9);
    int herr = 0;
    CD_CUDA(cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CD_CUDA(cudaStreamSynchronize(st));
    if (herr) { set_error("mixed K: a bounded tensor-core pipeline wait timed out"); return CD_ETIMEOUT; }
  }
  CD_CUDA(cudaStreamSynchronize(st));
  return CD_OK;
}

namespace {
// Bt[(p*n_mo + i)*Np + mu] = B^P[mu][i] from the fixed-point product D[i][p*N + mu]
__global__ void mo_half_kernel(const unsigned long long* __restrict__ D, int64_t ldd, int Pc, int N, int n_mo,
                               int64_t Np, const int32_t* __restrict__ eL, const int32_t* __restrict__ eC, int F,
                               double* __restrict__ Bt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)Pc * N * n_mo) return;
  const int i = (int)(t % n_mo);
  const int64_t row = t / n_mo;  // p*N + mu
  const int p = (int)(row / N), mu = (int)(row % N);
  Bt[((int64_t)p * n_mo + i) * Np + mu] = ldexp((double)(long long)D[(int64_t)i * ldd + row], eL[row] + eC[i] - F);
}
// out[p][i][j] = 2^(eB[p*n_mo+i] + eC[j] - F) * D[(p*n_mo + i)][j]
__global__ void mo_out_kernel(const unsigned long long* __restrict__ D, int Pc, int n_mo,
                              const int32_t* __restrict__ eB, const int32_t* __restrict__ eC, int F,
                              double* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)Pc * n_mo * n_mo) return;
  const int j = (int)(t % n_mo);
  const int64_t row = t / n_mo;  // p*n_mo + i
  out[t] = ldexp((double)(long long)D[t], eB[row] + eC[j] - F);
}
}  // namespace

// CV -> MO transformation (Sec. 4.1: the vectors transformed to the MO basis
// for CASSCF / CC), out[P - P0][i][j] = sum_{mu nu} C[mu][i] L^P_{mu nu} C[nu][j],
// as two exact-slice products per chunk of vectors: B^P = L^P C, then C^T B^P.
template <class TL>
int mo_vectors_sliced_t(const TL* L, int64_t ld, int64_t P0, int64_t nP, int64_t n, int N, int n_mo,
                        const double* C_dev, const int32_t* mu, const int32_t* nu, int S, double* out_dev,
                        cudaStream_t st) {
  if (nP <= 0) return CD_OK;
  const int64_t Np = (N + 7) / 8 * 8;
  int Pc = (int)std::max<int64_t>(1, std::min<int64_t>(nP, (int64_t)(1.5e9 / (2.0 * S * N * (double)N))));
  Pc = std::min(Pc, 64);
  MixedBufs b;
  b.st = st;
  unsigned long long* D3 = nullptr;
  int32_t* eBt = nullptr;
  struct Extra {
    cudaStream_t st;
    unsigned long long** d3;
    int32_t** e;
    ~Extra() { scratch_free(*d3, st); scratch_free(*e, st); }
  } extra{st, &D3, &eBt};
  CD_TRY(scratch_alloc(&b.idx, (size_t)N * N, st));
  CD_TRY(build_pair_index(mu, nu, n, N, b.idx, st));
  CD_TRY(scratch_alloc((uint16_t**)&b.Ls, (size_t)S * Pc * N * Np, st));
  CD_TRY(scratch_alloc((uint16_t**)&b.Cs, (size_t)S * n_mo * Np, st));
  CD_TRY(scratch_alloc(&b.Ct, (size_t)n_mo * N, st));
  CD_TRY(scratch_alloc(&b.eL, (size_t)Pc * N, st));
  CD_TRY(scratch_alloc(&b.eC, (size_t)n_mo, st));
  CD_TRY(scratch_alloc(&eBt, (size_t)Pc * n_mo, st));
  CD_TRY(scratch_alloc(&b.D1, (size_t)n_mo * Pc * N, st));
  CD_TRY(scratch_alloc(&D3, (size_t)Pc * n_mo * n_mo, st));
  CD_TRY(scratch_alloc(&b.Bm, (size_t)Pc * n_mo * Np, st));
  CD_TRY(scratch_alloc((uint16_t**)&b.Bs, (size_t)S * Pc * n_mo * Np, st));
  CD_TRY(scratch_alloc(&b.err, 1, st));
  CD_CUDA(cudaMemsetAsync(b.err, 0, sizeof(int), st));
  transpose_kernel<<<(unsigned)(((int64_t)N * n_mo + 255) / 256), 256, 0, st>>>(C_dev, N, n_mo, b.Ct);
  count_launch();
  CD_TRY(launch_row_exp_warp<double>(b.Ct, N, n_mo, N, b.eC, st));
  CD_TRY(launch_slice3<double>(b.Ct, N, n_mo, N, b.eC, b.Cs, Np, S, st));
  OzakiPlan pl;
  pl.SA = pl.SB = S;
  pl.KEEP = S + 1;
  pl.F = 61 - ilog2_ceil(N);
  for (int64_t Q0 = P0; Q0 < P0 + nP; Q0 += Pc) {
    const int pc = (int)std::min<int64_t>(Pc, P0 + nP - Q0);
    CD_TRY(launch_unpack_slice<TL>(L, ld, Q0, pc, b.idx, N, Np, S, b.eL, b.Ls, st));
    // B^P[mu][i]: D1[i][p*N + mu]
    CD_CUDA(cudaMemsetAsync(b.D1, 0, sizeof(unsigned long long) * n_mo * pc * N, st));
    CD_TRY(ozaki_gemm(pl, b.Ls, (int64_t)pc * N, Np, b.Cs, n_mo, Np, N, b.D1, (int64_t)pc * N, 1, b.err, st));
    CD_CUDA(cudaMemsetAsync(b.Bm, 0, sizeof(double) * pc * n_mo * Np, st));
    {
      const int64_t tot = (int64_t)pc * N * n_mo;
      mo_half_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(b.D1, (int64_t)pc * N, pc, N, n_mo, Np, b.eL,
                                                                    b.eC, pl.F, b.Bm);
      count_launch();
    }
    // (C^T B^P)[i][j] = sum_mu B^P[mu][i] C[mu][j]: rows (p, i) of Bt against rows j of C^T
    CD_TRY(launch_row_exp_warp<double>(b.Bm, Np, (int64_t)pc * n_mo, N, eBt, st));
    CD_TRY(launch_slice3<double>(b.Bm, Np, (int64_t)pc * n_mo, N, eBt, b.Bs, Np, S, st));
    CD_CUDA(cudaMemsetAsync(D3, 0, sizeof(unsigned long long) * pc * n_mo * n_mo, st));
    CD_TRY(ozaki_gemm(pl, b.Cs, n_mo, Np, b.Bs, (int64_t)pc * n_mo, Np, N, D3, n_mo, 1, b.err, st));
    {
      const int64_t tot = (int64_t)pc * n_mo * n_mo;
      mo_out_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(D3, pc, n_mo, eBt, b.eC, pl.F,
                                                                   out_dev + (Q0 - P0) * (int64_t)n_mo * n_mo);
      count_launch();
    }
  }
  int herr = 0;
  CD_CUDA(cudaMemcpyAsync(&herr, b.err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CD_CUDA(cudaStreamSynchronize(st));
  if (herr) { set_error("MO transform: a bounded tensor-core pipeline wait timed out"); return CD_ETIMEOUT; }
  return CD_OK;
}

int mo_vectors_sliced(const float* L32, const double* L64, int64_t ld, int64_t P0, int64_t nP, int64_t n, int N,
                      int n_mo, const double* C_dev, const int32_t* mu, const int32_t* nu, int S, double* out_dev,
                      cudaStream_t st) {
  if (L32) return mo_vectors_sliced_t<float>(L32, ld, P0, nP, n, N, n_mo, C_dev, mu, nu, S, out_dev, st);
  return mo_vectors_sliced_t<double>(L64, ld, P0, nP, n, N, n_mo, C_dev, mu, nu, S, out_dev, st);
}

int jk_mixed(const float* L32, const double* L64, int64_t ld, int64_t M, int64_t n, int N, int O, const double* C_dev,
             const int32_t* mu, const int32_t* nu, double* J_dev, double* K_dev, bool wantJ, bool wantK,
             int S, cudaStream_t st) {
  if (L32) return jk_mixed_t<float>(L32, ld, M, n, N, O, C_dev, mu, nu, J_dev, K_dev, wantJ, wantK, S, st);
  return jk_mixed_t<double>(L64, ld, M, n, N, O, C_dev, mu, nu, J_dev, K_dev, wantJ, wantK, S, st);
}

}  // namespace cd
