// pivot.cuh -- step kernels of the pivoted decomposition (see pivot.cu).
#pragma once
#include "internal.cuh"

namespace cd {

constexpr int kStepThreads = 256;
constexpr int kStepGrid = 148 * 4;     // 4 CTAs per SM on 148 SMs
constexpr int kMaxBlock = 256;          // largest speculative block

struct StepResult {        // written by the last CTA of a step kernel
  double dmax;             // max residual diagonal after the step
  int64_t idx;             // its row (lowest on ties)
  int32_t bad;             // 1 if some D < neg_tol (not PSD)
  int32_t pad;
};

struct StepScratch {       // device scratch of the grid-wide argmax
  double part_val[kStepGrid];
  int64_t part_idx[kStepGrid];
  unsigned counter;        // CTAs finished (reset by the last one)
  int bad;
};

// cand (optional, [n]): rows with cand[r] == 0 are not candidates for the argmax / the selection
int launch_argmax(const double* D, int64_t n, StepScratch* sc, StepResult* res, cudaStream_t st,
                  const uint8_t* cand = nullptr);

// radix select of the b largest D >= tau (see pivot.cu)
struct SelectState {
  unsigned long long prefix, mask;
  unsigned long long need;   // keys still to take below the current prefix (set before pass 0)
  long long total;           // keys >= tau (pass 0)
  int all;                   // fewer than b keys: take everything matching the prefix
  unsigned counter;          // CTAs done in the current pass
  unsigned count;            // compacted rows
  unsigned hist[8][256];
};
int launch_select(const double* D, int64_t n, double tau, int b, SelectState* stt, int64_t* rows_out,
                  double* vals_out, int cap, cudaStream_t st, const uint8_t* cand = nullptr);
int launch_finalize(const double* col, const double* L, int64_t ld, int64_t Kb, int64_t K, int64_t prow,
                    const double* Din, double* Dout, double* Lout, int64_t n, double neg_tol,
                    StepScratch* sc, StepResult* res, cudaStream_t st, const uint8_t* cand = nullptr);
int launch_gather(const double* L, int64_t ld, const int64_t* rows_dev, int nb, int64_t k0, int64_t k1,
                  double* Bg, cudaStream_t st);
int launch_gather(const float* L, int64_t ld, const int64_t* rows_dev, int nb, int64_t k0, int64_t k1,
                  double* Bg, cudaStream_t st);

// ---- device-driven pivot steps of one block (full pivoting) ----------------
// The state the step kernels read at their start and the last CTA of each
// step updates: the host uploads it once per block, enqueues up to b step
// launches (captured once in a CUDA graph) and reads it back once per block,
// instead of a round trip per step.
struct DevStep {
  StepResult res;          // argmax of the current residual diagonal
  int64_t K;               // vectors so far
  int64_t Kb;              // vectors at the start of the block (in-block vectors: [Kb, K))
  int64_t Kcap;            // vector capacity of L
  const double* Dcur0;     // residual diagonal at the block's first step; steps alternate
  double* Dnext0;          //   Dcur0 -> Dnext0 -> Dcur0 ...
  double tau;
  int32_t done;            // set once a step declines to run; later steps do nothing
  int32_t reason;          // kStep* below
};
constexpr int kStepConverged = 1;   // max D < tau (or no candidate)
constexpr int kStepOutside = 2;     // argmax row has no column in the block: start a new block
constexpr int kStepCapacity = 3;    // K reached Kcap
constexpr int kStepNotPsd = 4;      // pivot diagonal <= 0 or a residual below the tolerance

// slot_of_row [n]: pool slot of each row in the block, -1 elsewhere.  Step k
// of the block: p = res.idx; L^K from pool column slot_of_row[p] (vectors
// [Kb, K) applied), D' = D - (L^K)^2, argmax of D'; piv[K] = p, pivd[K] = D_p,
// slot_of_row[p] = -1, K += 1.
int launch_finalize_dev(DevStep* ds, int32_t* slot_of_row, const double* pool, const double* L, int64_t ld,
                        int64_t n, double neg_tol, const uint8_t* cand, int64_t* piv, double* pivd,
                        StepScratch* sc, cudaStream_t st);
// CUDA graph of nsteps launches of the step kernel above, in order
int build_step_graph(cudaGraphExec_t* exec, int nsteps, DevStep* ds, int32_t* slot_of_row, const double* pool,
                     const double* L, int64_t ld, int64_t n, double neg_tol, const uint8_t* cand, int64_t* piv,
                     double* pivd, StepScratch* sc);
// slot_of_row[rows[j]] = slots[j] for j < nb (after clearing all n entries to -1)
int launch_slot_map(int32_t* slot_of_row, int64_t n, const int64_t* rows, const int32_t* slots, int nb,
                    cudaStream_t st);

// row compaction (first step of the two-step scheme): keep rows idx[0..m) (increasing)
int launch_compact_f64(const double* src, int64_t lds, const int32_t* idx, int64_t m, int64_t ncol, double* dst,
                       int64_t ldd, cudaStream_t st);
int launch_compact_rows16(const void* src, int64_t n_old, const int32_t* idx, int64_t m, int groups, int64_t row_bytes,
                          void* dst, cudaStream_t st);
int launch_compact_i32(const int32_t* src, const int32_t* idx, int64_t m, int32_t* dst, cudaStream_t st);
// out[j] = D[rows[j]] (-inf where rows[j] < 0)
int launch_gather_vals(const double* D, const int64_t* rows, int nb, double* out, cudaStream_t st);

// column update (colupd.cu): cols[slot[j]] -= L[k0:k1]^T Bg  (Bg row-major [k1-k0][nb])
int launch_colupd(double* cols, int64_t ld, const int32_t* slots_dev, int nb, const double* L,
                  int64_t k0, int64_t k1, const double* Bg, int64_t n, cudaStream_t st);

// J / K helpers (jk.cu)
int launch_density_packed(const double* C, int N, int O, const int32_t* mu, const int32_t* nu, int64_t n,
                          double* d, cudaStream_t st);
template <class T>
int launch_gemv_rows(const T* L, int64_t ld, int64_t M, int64_t n, const double* x, double* y, cudaStream_t st);
template <class T>
int launch_gemv_cols(const T* L, int64_t ld, int64_t M, int64_t n, const double* v, double* y, cudaStream_t st);
int launch_unpack_sym(const double* packed, const int32_t* mu, const int32_t* nu, int64_t n, int N, double* out,
                      cudaStream_t st);
// dense symmetric N x N unpacking of vectors P0 .. P0+Pc-1 (T: stored type, TO: output type)
template <class T, class TO>
int launch_unpack_vectors(const T* L, int64_t ld, int64_t P0, int Pc, const int32_t* mu, const int32_t* nu,
                          int64_t n, int N, TO* out, cudaStream_t st);
// generic FP64 GEMM: C[b] (+)= alpha * A[b] B[b]; element (i,k) of A at A + i*ars + k*acs + b*abs
int launch_dgemm(int m, int n, int k, int batch, double alpha,
                 const double* A, int64_t ars, int64_t acs, int64_t abs_,
                 const double* B, int64_t brs, int64_t bcs, int64_t bbs,
                 double* C, int64_t ldc, int64_t cbs, bool reduce_batch, cudaStream_t st);

}  // namespace cd
