// pivot.cu -- kernel (b): vector finalisation, residual-diagonal update and the
// global argmax of the residual diagonal (ties to the lowest row index).
//
// One step of the recursion of Sec. 2 for pivot row p:
//   L^K_r = (col_r - sum_{J in [Kb,K)} L^J_r L^J_p) / sqrt(D_p)   Eq. (subtr)
//   D'_r  = D_r - (L^K_r)^2                                       Eq. (diag)
// where col already holds (r|p) - sum_{J<Kb} L^J_r L^J_p (column-update GEMM)
// and the vectors of the current block [Kb, K) are applied here.  D is double
// buffered (read D, write D') so that D_p stays readable by every CTA.
// The argmax is reduced warp -> CTA (shuffles) -> grid (last CTA to finish).
#include <float.h>
#include <math.h>
#include <string>
#include "internal.cuh"
#include "pivot.cuh"

namespace cd {
namespace {

__device__ __forceinline__ bool better(double v1, int64_t i1, double v2, int64_t i2) {
  return v1 > v2 || (v1 == v2 && i1 < i2);
}

__device__ __forceinline__ void warp_argmax(double& v, int64_t& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(v2, i2, v, i)) { v = v2; i = i2; }
  }
}

// block-level argmax of (v, i) held by every thread; result valid in thread 0
__device__ void block_argmax(double& v, int64_t& i) {
  __shared__ double sv[32];
  __shared__ int64_t si[32];
  warp_argmax(v, i);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sv[w] = v; si[w] = i; }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    v = lane < nw ? sv[lane] : -DBL_MAX;
    i = lane < nw ? si[lane] : INT64_MAX;
    warp_argmax(v, i);
  }
  __syncthreads();
}

// grid-level finish: every CTA writes its partial; the last one reduces them
__device__ void grid_finish(double v, int64_t i, int bad, StepScratch* sc, StepResult* res) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    sc->part_val[blockIdx.x] = v;
    sc->part_idx[blockIdx.x] = i;
    if (bad) atomicOr(&sc->bad, 1);
    __threadfence();
    unsigned t = atomicAdd(&sc->counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double bv = -DBL_MAX;
  int64_t bi = INT64_MAX;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    double v2 = ((volatile double*)sc->part_val)[b];
    int64_t i2 = ((volatile int64_t*)sc->part_idx)[b];
    if (better(v2, i2, bv, bi)) { bv = v2; bi = i2; }
  }
  block_argmax(bv, bi);
  if (threadIdx.x == 0) {
    res->dmax = bv;
    res->idx = bi;
    res->bad = *(volatile int*)&sc->bad;
    sc->bad = 0;
    sc->counter = 0;
    __threadfence();
  }
}

__global__ void __launch_bounds__(kStepThreads) argmax_kernel(const double* __restrict__ D, int64_t n,
                                                              const uint8_t* __restrict__ cand,
                                                              StepScratch* sc, StepResult* res) {
  double bv = -DBL_MAX;
  int64_t bi = INT64_MAX;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    double d = D[r];
    if ((!cand || cand[r]) && better(d, r, bv, bi)) { bv = d; bi = r; }
  }
  block_argmax(bv, bi);
  grid_finish(bv, bi, 0, sc, res);
}

__global__ void __launch_bounds__(kStepThreads) finalize_kernel(
    const double* __restrict__ col, const double* __restrict__ L, int64_t ld, int64_t Kb, int64_t K,
    int64_t prow, const double* __restrict__ Din, double* __restrict__ Dout, double* __restrict__ Lout,
    int64_t n, double neg_tol, const uint8_t* __restrict__ cand, StepScratch* sc, StepResult* res) {
  __shared__ double g[kMaxBlock];
  const int nk = (int)(K - Kb);
  for (int k = threadIdx.x; k < nk; k += blockDim.x) g[k] = L[(Kb + k) * ld + prow];
  __syncthreads();
  const double dp = Din[prow];
  const double inv = 1.0 / sqrt(dp);
  double bv = -DBL_MAX;
  int64_t bi = INT64_MAX;
  int bad = 0;
  const double* Lb = L + Kb * ld;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    // two independent FMA chains (even / odd in-block vectors) keep the FP64 pipe fed
    double acc = col[r], acc2 = 0.0;
    int k = 0;
    for (; k + 4 <= nk; k += 4) {
      double a0 = Lb[(k + 0) * ld + r], a1 = Lb[(k + 1) * ld + r];
      double a2 = Lb[(k + 2) * ld + r], a3 = Lb[(k + 3) * ld + r];
      acc = fma(-a0, g[k + 0], acc);
      acc2 = fma(-a1, g[k + 1], acc2);
      acc = fma(-a2, g[k + 2], acc);
      acc2 = fma(-a3, g[k + 3], acc2);
    }
    for (; k < nk; ++k) acc = fma(-Lb[k * ld + r], g[k], acc);
    acc += acc2;
    const double v = acc * inv;
    Lout[r] = v;
    const double d = fma(-v, v, Din[r]);
    Dout[r] = d;
    if (d < neg_tol) bad = 1;
    if ((!cand || cand[r]) && better(d, r, bv, bi)) { bv = d; bi = r; }
  }
  block_argmax(bv, bi);
  grid_finish(bv, bi, bad, sc, res);
}

// One device-driven step (see DevStep).  Thread 0 of every CTA reads the
// state; all CTAs reach the same decision because the state only changes at
// the end of a step, after every CTA of that step has read it (the last CTA to
// finish writes it).
__global__ void __launch_bounds__(kStepThreads) finalize_dev_kernel(
    DevStep* __restrict__ ds, int32_t* __restrict__ slot_of_row, const double* __restrict__ pool,
    const double* __restrict__ L, int64_t ld, int64_t n, double neg_tol, const uint8_t* __restrict__ cand,
    int64_t* __restrict__ piv, double* __restrict__ pivd, StepScratch* sc) {
  __shared__ int s_go;
  __shared__ int64_t s_p, s_K, s_Kb;
  __shared__ int s_slot, s_odd;
  __shared__ double s_dp;
  __shared__ double g[kMaxBlock];
  if (threadIdx.x == 0) {
    const volatile DevStep* v = ds;
    int reason = 0;
    const int64_t K = v->K, Kb = v->Kb, idx = v->res.idx;
    const double dmax = v->res.dmax;
    int slot = -1;
    double dp = 0.0;
    const int odd = (int)((K - Kb) & 1);
    if (v->done) reason = -1;
    else if (v->res.bad) reason = kStepNotPsd;
    else if (!(dmax >= v->tau) || idx < 0 || idx >= n) reason = kStepConverged;
    else if (K >= v->Kcap || K - Kb >= kMaxBlock) reason = kStepCapacity;
    else {
      slot = slot_of_row[idx];
      if (slot < 0) reason = kStepOutside;
      else {
        const double* Din = odd ? v->Dnext0 : v->Dcur0;
        dp = Din[idx];
        if (!(dp > 0.0)) reason = kStepNotPsd;
      }
    }
    s_go = reason == 0;
    s_p = idx; s_K = K; s_Kb = Kb; s_slot = slot; s_odd = odd; s_dp = dp;
    if (reason > 0 && blockIdx.x == 0) {
      ds->done = 1;
      ds->reason = reason;
    }
  }
  __syncthreads();
  if (!s_go) return;
  const int64_t prow = s_p, K = s_K, Kb = s_Kb;
  const double* Din = s_odd ? ds->Dnext0 : ds->Dcur0;
  double* Dout = s_odd ? const_cast<double*>(ds->Dcur0) : ds->Dnext0;
  const double* col = pool + (int64_t)s_slot * ld;
  double* Lout = const_cast<double*>(L) + K * ld;
  const int nk = (int)(K - Kb);
  for (int k = threadIdx.x; k < nk; k += blockDim.x) g[k] = L[(Kb + k) * ld + prow];
  __syncthreads();
  const double inv = 1.0 / sqrt(s_dp);
  double bv = -DBL_MAX;
  int64_t bi = INT64_MAX;
  int bad = 0;
  const double* Lb = L + Kb * ld;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    // two independent FMA chains (even / odd in-block vectors) keep the FP64 pipe fed
    double acc = col[r], acc2 = 0.0;
    int k = 0;
    for (; k + 4 <= nk; k += 4) {
      double a0 = Lb[(k + 0) * ld + r], a1 = Lb[(k + 1) * ld + r];
      double a2 = Lb[(k + 2) * ld + r], a3 = Lb[(k + 3) * ld + r];
      acc = fma(-a0, g[k + 0], acc);
      acc2 = fma(-a1, g[k + 1], acc2);
      acc = fma(-a2, g[k + 2], acc);
      acc2 = fma(-a3, g[k + 3], acc2);
    }
    for (; k < nk; ++k) acc = fma(-Lb[k * ld + r], g[k], acc);
    acc += acc2;
    const double vv = acc * inv;
    Lout[r] = vv;
    const double d = fma(-vv, vv, Din[r]);
    Dout[r] = d;
    if (d < neg_tol) bad = 1;
    if ((!cand || cand[r]) && better(d, r, bv, bi)) { bv = d; bi = r; }
  }
  block_argmax(bv, bi);
  // grid finish: the last CTA reduces the partial argmaxes and advances the state
  __shared__ bool last;
  if (threadIdx.x == 0) {
    sc->part_val[blockIdx.x] = bv;
    sc->part_idx[blockIdx.x] = bi;
    if (bad) atomicOr(&sc->bad, 1);
    __threadfence();
    unsigned t = atomicAdd(&sc->counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  bv = -DBL_MAX;
  bi = INT64_MAX;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
    double v2 = ((volatile double*)sc->part_val)[b];
    int64_t i2 = ((volatile int64_t*)sc->part_idx)[b];
    if (better(v2, i2, bv, bi)) { bv = v2; bi = i2; }
  }
  block_argmax(bv, bi);
  if (threadIdx.x == 0) {
    ds->res.dmax = bv;
    ds->res.idx = bi;
    ds->res.bad = *(volatile int*)&sc->bad;
    sc->bad = 0;
    sc->counter = 0;
    piv[K] = prow;
    pivd[K] = s_dp;
    slot_of_row[prow] = -1;
    ds->K = K + 1;
    __threadfence();
  }
}

__global__ void slot_map_kernel(int32_t* __restrict__ slot_of_row, const int64_t* __restrict__ rows,
                                const int32_t* __restrict__ slots, int nb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nb) slot_of_row[rows[j]] = slots[j];
}

// Bg[k][j] = L[k][rows[j]] for k in [k0, k1), j < nb (row-major, leading dim nb)
template <class T>
__global__ void gather_kernel(const T* __restrict__ L, int64_t ld, const int64_t* __restrict__ rows, int nb,
                              int64_t k0, int64_t k1, double* __restrict__ Bg) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nk = k1 - k0;
  if (t >= nk * nb) return;
  const int64_t k = t / nb;
  const int j = (int)(t % nb);
  Bg[t] = L[(k0 + k) * ld + rows[j]];
}

// dst[c * ldd + i] = src[c * lds + idx[i]] for c < ncol, i < m (row compaction of
// column-stored vectors: idx increasing, so reads stay mostly coalesced)
__global__ void compact_f64_kernel(const double* __restrict__ src, int64_t lds, const int32_t* __restrict__ idx,
                                   int64_t m, int64_t ncol, double* __restrict__ dst, int64_t ldd) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * ncol) return;
  const int64_t c = t / m, i = t % m;
  dst[c * ldd + i] = src[c * lds + __ldg(idx + i)];
}

// rows of 16-byte words: dst[(g * m + i) * w + x] = src[(g * n_old + idx[i]) * w + x]
// for g < groups (slices), i < m, x < w
__global__ void compact_rows16_kernel(const uint4* __restrict__ src, int64_t n_old, const int32_t* __restrict__ idx,
                                      int64_t m, int groups, int64_t w, uint4* __restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = m * w;
  if (t >= per * groups) return;
  const int64_t g = t / per, r = t % per;
  const int64_t i = r / w, x = r % w;
  dst[(g * m + i) * w + x] = src[(g * n_old + __ldg(idx + i)) * w + x];
}

__global__ void compact_i32_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ idx, int64_t m,
                                   int32_t* __restrict__ dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) dst[i] = src[__ldg(idx + i)];
}

// out[j] = D[rows[j]] (or -inf for rows[j] < 0), j < nb
__global__ void gather_vals_kernel(const double* __restrict__ D, const int64_t* __restrict__ rows, int nb,
                                   double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nb) out[j] = rows[j] >= 0 ? D[rows[j]] : -INFINITY;
}

}  // namespace

int launch_compact_f64(const double* src, int64_t lds, const int32_t* idx, int64_t m, int64_t ncol, double* dst,
                       int64_t ldd, cudaStream_t st) {
  const int64_t tot = m * ncol;
  if (tot <= 0) return CD_OK;
  compact_f64_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(src, lds, idx, m, ncol, dst, ldd);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_compact_rows16(const void* src, int64_t n_old, const int32_t* idx, int64_t m, int groups, int64_t row_bytes,
                          void* dst, cudaStream_t st) {
  if (row_bytes % 16) { set_error("compact_rows16: row not a multiple of 16 bytes"); return CD_EINVAL; }
  const int64_t w = row_bytes / 16, tot = m * w * groups;
  if (tot <= 0) return CD_OK;
  compact_rows16_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>((const uint4*)src, n_old, idx, m, groups, w,
                                                                       (uint4*)dst);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_compact_i32(const int32_t* src, const int32_t* idx, int64_t m, int32_t* dst, cudaStream_t st) {
  if (m <= 0) return CD_OK;
  compact_i32_kernel<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(src, idx, m, dst);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_gather_vals(const double* D, const int64_t* rows, int nb, double* out, cudaStream_t st) {
  if (nb <= 0) return CD_OK;
  gather_vals_kernel<<<(nb + 255) / 256, 256, 0, st>>>(D, rows, nb, out);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_argmax(const double* D, int64_t n, StepScratch* sc, StepResult* res, cudaStream_t st, const uint8_t* cand) {
  argmax_kernel<<<kStepGrid, kStepThreads, 0, st>>>(D, n, cand, sc, res);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_finalize(const double* col, const double* L, int64_t ld, int64_t Kb, int64_t K, int64_t prow,
                    const double* Din, double* Dout, double* Lout, int64_t n, double neg_tol,
                    StepScratch* sc, StepResult* res, cudaStream_t st, const uint8_t* cand) {
  if (K - Kb > kMaxBlock) { set_error("finalize: block too large"); return CD_EINVAL; }
  finalize_kernel<<<kStepGrid, kStepThreads, 0, st>>>(col, L, ld, Kb, K, prow, Din, Dout, Lout, n, neg_tol, cand, sc,
                                                      res);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_finalize_dev(DevStep* ds, int32_t* slot_of_row, const double* pool, const double* L, int64_t ld,
                        int64_t n, double neg_tol, const uint8_t* cand, int64_t* piv, double* pivd,
                        StepScratch* sc, cudaStream_t st) {
  finalize_dev_kernel<<<kStepGrid, kStepThreads, 0, st>>>(ds, slot_of_row, pool, L, ld, n, neg_tol, cand, piv, pivd,
                                                          sc);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int build_step_graph(cudaGraphExec_t* exec, int nsteps, DevStep* ds, int32_t* slot_of_row, const double* pool,
                     const double* L, int64_t ld, int64_t n, double neg_tol, const uint8_t* cand, int64_t* piv,
                     double* pivd, StepScratch* sc) {
  // built node by node (no stream capture, so work that other threads put on
  // the device meanwhile cannot disturb it)
  *exec = nullptr;
  cudaGraph_t g = nullptr;
  CD_CUDA(cudaGraphCreate(&g, 0));
  void* args[] = {(void*)&ds, (void*)&slot_of_row, (void*)&pool, (void*)&L, (void*)&ld, (void*)&n,
                  (void*)&neg_tol, (void*)&cand, (void*)&piv, (void*)&pivd, (void*)&sc};
  cudaKernelNodeParams p = {};
  p.func = (void*)finalize_dev_kernel;
  p.gridDim = dim3(kStepGrid);
  p.blockDim = dim3(kStepThreads);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  p.extra = nullptr;
  cudaGraphNode_t prev = nullptr;
  for (int i = 0; i < nsteps; ++i) {
    cudaGraphNode_t node = nullptr;
    cudaError_t e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &p);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaGraphDestroy(g);
      set_error(std::string("step graph: ") + cudaGetErrorString(e));
      return CD_ECUDA;
    }
    prev = node;
  }
  cudaError_t e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *exec = nullptr;
    set_error(std::string("step graph: ") + cudaGetErrorString(e));
    return CD_ECUDA;
  }
  return CD_OK;
}

int launch_slot_map(int32_t* slot_of_row, int64_t n, const int64_t* rows, const int32_t* slots, int nb,
                    cudaStream_t st) {
  if (n > 0) CD_CUDA(cudaMemsetAsync(slot_of_row, 0xFF, sizeof(int32_t) * n, st));
  if (nb <= 0) return CD_OK;
  slot_map_kernel<<<(nb + 127) / 128, 128, 0, st>>>(slot_of_row, rows, slots, nb);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template <class T>
static int launch_gather_t(const T* L, int64_t ld, const int64_t* rows_dev, int nb, int64_t k0, int64_t k1,
                           double* Bg, cudaStream_t st) {
  int64_t tot = (k1 - k0) * nb;
  if (tot <= 0) return CD_OK;
  gather_kernel<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(L, ld, rows_dev, nb, k0, k1, Bg);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}
int launch_gather(const double* L, int64_t ld, const int64_t* rows_dev, int nb, int64_t k0, int64_t k1,
                  double* Bg, cudaStream_t st) {
  return launch_gather_t(L, ld, rows_dev, nb, k0, k1, Bg, st);
}
int launch_gather(const float* L, int64_t ld, const int64_t* rows_dev, int nb, int64_t k0, int64_t k1,
                  double* Bg, cudaStream_t st) {
  return launch_gather_t(L, ld, rows_dev, nb, k0, k1, Bg, st);
}

}  // namespace cd

// ---------------------------------------------------------------------------
// Candidate selection: the b largest residual diagonals with D >= tau, by a
// radix select over the IEEE-754 bit patterns (monotone for positive doubles,
// 8 bits per pass, histograms in shared memory, the last CTA of each pass
// picks the byte), then one compaction of every row at or above the b-th key.
namespace cd {
namespace {

__device__ __forceinline__ unsigned long long dkey(double d, double tau) {
  return d >= tau ? (unsigned long long)__double_as_longlong(d) : 0ull;
}

__global__ void __launch_bounds__(256) select_pass_kernel(const double* __restrict__ D, int64_t n, double tau, int pass,
                                                          int b, SelectState* stt, const uint8_t* __restrict__ cand) {
  __shared__ unsigned sh[256];
  __shared__ bool last;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const unsigned long long prefix = stt->prefix, mask = stt->mask;
  const int shift = 56 - 8 * pass;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = (cand && !cand[r]) ? 0ull : dkey(D[r], tau);
    if (k != 0ull && (k & mask) == prefix) atomicAdd(&sh[(k >> shift) & 255ull], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&stt->hist[pass][i], sh[i]);
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(&stt->counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  if (pass > 0 && *(volatile int*)&stt->all) {  // decided in an earlier pass: nothing left to narrow
    stt->counter = 0;
    __threadfence();
    return;
  }
  volatile unsigned* h = stt->hist[pass];
  long long need = pass == 0 ? (long long)b : (long long)stt->need;
  long long cum = 0, total = 0;
  int chosen = -1;
  for (int bin = 255; bin >= 0; --bin) total += h[bin];
  if (pass == 0) stt->total = total;
  if (total <= need) {
    // every remaining key qualifies: threshold = smallest key with this prefix;
    // later passes leave prefix, mask and need unchanged
    stt->all = 1;
    stt->need = need;
  } else {
    for (int bin = 255; bin >= 0; --bin) {
      cum += h[bin];
      if (cum >= need) { chosen = bin; need -= cum - h[bin]; break; }
    }
    stt->prefix = prefix | ((unsigned long long)chosen << shift);
    stt->mask = mask | (255ull << shift);
    stt->need = need;
  }
  stt->counter = 0;
  __threadfence();
}

__global__ void __launch_bounds__(256) select_compact_kernel(const double* __restrict__ D, int64_t n, double tau,
                                                             SelectState* stt, int64_t* __restrict__ rows_out,
                                                             double* __restrict__ vals_out, int cap,
                                                             const uint8_t* __restrict__ cand) {
  const unsigned long long thr = stt->all ? (stt->prefix & stt->mask) : stt->prefix;
  const bool all = stt->all != 0;
  const unsigned long long mask = stt->mask, prefix = stt->prefix;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long k = (cand && !cand[r]) ? 0ull : dkey(D[r], tau);
    if (k == 0ull) continue;
    const bool take = all ? ((k & mask) >= prefix) : (k >= thr);
    if (take) {
      const int slot = (int)atomicAdd(&stt->count, 1u);
      if (slot < cap) { rows_out[slot] = r; vals_out[slot] = D[r]; }
    }
  }
}

}  // namespace

int launch_select(const double* D, int64_t n, double tau, int b, SelectState* stt, int64_t* rows_out,
                  double* vals_out, int cap, cudaStream_t st, const uint8_t* cand) {
  CD_CUDA(cudaMemsetAsync(stt, 0, sizeof(SelectState), st));
  for (int pass = 0; pass < 8; ++pass) {
    select_pass_kernel<<<kStepGrid, 256, 0, st>>>(D, n, tau, pass, b, stt, cand);
    count_launch();
  }
  select_compact_kernel<<<kStepGrid, 256, 0, st>>>(D, n, tau, stt, rows_out, vals_out, cap, cand);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

}  // namespace cd
