// batch.cu -- many independent systems decomposed and contracted in one
// persistent kernel launch, recorded in a CUDA graph.
//
// Every system runs the fully pivoted decomposition of Sec. 2 in the blocked
// form of the single-system path (b candidate columns computed and brought up
// to date together, then pivot steps while the global argmax of the residual
// diagonal stays among them) and then the J/K build of Sec. 4.1.  Everything is
// FP64 except, in the default tensor-core build, the column update, which is
// the exact 7-slice BF16 product of the single-system path (FP64-equivalent).
// A system's work is a sequence of jobs, each a set of independent items:
//
//   SELECT  1 item: the b largest residual diagonals >= tau (ties: lowest row)
//           become the block's candidates (radix select over the IEEE-754 bit
//           patterns); pool slots of columns still wanted are kept, the new
//           rows get ket groups
//   COLS    the pivot rows of the existing vectors gathered for the update
//           (256 vectors per item; their slices in the tensor-core build), and
//           the ERI columns of the new candidates (kernel a: 128 bra shell
//           pairs x one ket group per item)
//   UPDATE  col -= L Lp^T over the vectors not yet applied, Eq. (subtr): 128
//           rows x 32 columns per item on the tensor cores (tcgen05, operands
//           copied to shared memory with cp.async), or 128 x <= 64 DFMA tiles
//   STEP    one pivot step, Eq. (subtr) in-block terms and Eq. (diag), over
//           1024 rows per item, each item leaving its partial argmax
//   SLICE   tensor-core build, after a block: its vectors (an FP64 block
//           buffer) written once into the BF16 slice store
//   JK1     d = packed density (1024 rows per item); B^P = L^P C (through a
//           row list per basis function; 32 vectors x 8 basis functions per
//           item from the slice store, or one vector per item)
//   JK2     v = L d; partial K tiles sum_P B^P B^P^T (64 x 64 tile x 128
//           vectors per item)
//   JK3     J_p = L^T v (1024 rows per item); K tiles = 2 x the sum of partials
//   JK4     J unpacked to N x N
//
// Jobs and stage flags.  A system holds one job at a time in a 64-bit word
// (generation | item count | next item).  A CTA claims an item with one
// atomic add on the word.  The CTA that completes a job's last item (counted
// per system) runs the job's finish: it writes the next job's parameters and
// then publishes the next word; the STEP finish reduces the step's argmax and
// decides between another step, a new block and the J/K build.  Items never
// wait for each other, so the launch needs no co-residency; the one wait is a
// CTA's wait for work, which gives up and makes the call return CD_ETIMEOUT
// once no item anywhere has completed for the wait limit (cd_set_wait_limit).
// CTAs scan the systems largest first, so the largest systems take the GPU
// first and the small ones fill the gaps.
//
// Memory is reserved per system before the launch (vectors for max_vectors,
// default 8 N, plus the K intermediates); a system that needs more vectors
// stops with CD_ENOMEM.  Loads of data that change during the launch (residual
// diagonals, columns, gathered rows, slices, job state) bypass L1
// (ld.global.cg, cp.async.cg or volatile): another SM may have rewritten them
// since this SM last cached them.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <thread>
#include <vector>
#include <cuda_bf16.h>
#include "internal.cuh"
#include "eri_dev.cuh"
#include "ozaki.cuh"
#include "tc.cuh"

namespace cd {
unsigned long long device_wait_limit_ns();  // ozaki.cu (cd_set_wait_limit)

namespace {

constexpr int kBT = 128;          // threads per CTA
constexpr int kBMaxB = 64;        // largest block of the batch kernel
constexpr int kStepRows = 1024;   // rows per STEP / DENS / JP / JUNPACK item
constexpr int kRowTile = 128;     // rows per UPDATE item
constexpr int kGatherQ = 256;     // vectors per gather item
constexpr int kJvVec = 4;         // vectors per JV item
constexpr int kKtSplit = 128;     // vectors per partial K tile
constexpr int kKt = 64;           // K tile edge
constexpr int kTieCap = 1024;     // tie-bin entries ranked directly by SELECT
constexpr int kSmemBytes = 32768;     // scratch of the FP64 items
// exact-slice update items (tcgen05): A = 7 BF16 slices of 128 rows x 32 vectors,
// B = 7 slices of 32 columns x 32 vectors, 64-byte swizzled rows
constexpr int kTcSlices = 7, kTcBN = 32, kTcBK = 32;
constexpr int kTcABytes = kTcSlices * 128 * kTcBK * 2;    // 57,344
constexpr int kTcBBytes = kTcSlices * kTcBN * kTcBK * 2;  // 14,336
constexpr int kTcF = 60;          // fixed-point fraction bits of the update sums
constexpr int kTcChunk = 4;       // k-blocks per drain: 7 products x 128 k x 129^2 < 2^24 (exact FP32 sums)
constexpr int kTcTmemCols = 256;  // 7 accumulator groups x 32 columns = 224 used
constexpr int kDynSmem = (kTcABytes + kTcBBytes > kSmemBytes ? kTcABytes + kTcBBytes : kSmemBytes) + 1024;

enum JobType : int { kJobNone = 0, kJobSelect, kJobCols, kJobUpdate, kJobStep, kJobJk1, kJobJk2, kJobJk3, kJobJk4,
                     kJobSlice = 9 /* tensor-core mode: the finished block's vectors into the slice store */,
                     kJobConverged = 100 /* pseudo job: the decomposition has converged */ };

__host__ __device__ constexpr unsigned long long job_word(unsigned gen, unsigned count, unsigned next) {
  return ((unsigned long long)(gen & 0xffffu) << 48) | ((unsigned long long)(count & 0xffffffu) << 24) |
         (unsigned long long)(next & 0xffffffu);
}
__host__ __device__ constexpr unsigned job_gen(unsigned long long w) { return (unsigned)(w >> 48); }
__host__ __device__ constexpr unsigned job_count(unsigned long long w) { return (unsigned)((w >> 24) & 0xffffffu); }
__host__ __device__ constexpr unsigned job_next(unsigned long long w) { return (unsigned)(w & 0xffffffu); }
constexpr unsigned kMaxJobItems = 1u << 23;   // far below the 24-bit fields, so over-claims cannot carry

// Mutable per-system state (device).  Written only by a job's finish (one CTA,
// while no item of the system is outstanding) and by SELECT (the only item of
// its job); read by the items of the next job after they claim it.
struct SysState {
  unsigned long long word;   // current job
  unsigned done;             // items of the current job completed
  int type;                  // JobType of the current job
  int status;                // CD_OK or the system's error code
  int bad;                   // a residual diagonal fell below neg_tol in this step
  int cur;                   // D[cur] is the current residual diagonal
  int pslot;                 // pool slot of the current pivot
  int converged;             // SELECT found max D < tau
  int after_slice;           // job after a SLICE job: kJobSelect or kJobConverged
  int ngroups;               // ERI ket groups of the block
  int64_t K, Kb;             // vectors done; first vector of the current block
  int64_t prow;              // pivot row of the current step
  double dp;                 // its residual diagonal
  double dmax;               // max of D[cur] and its row (ties: lowest row)
  int64_t idx;
  int nitems[2];             // items of the two parts of a job
  int gitems[2];             // gather items of the two update groups
  int nb[2];                 // update groups (new slots, kept slots): columns
  int64_t k0[2];             // and the first vector each still needs
  int32_t uslot[2][kBMaxB];
  int64_t urow[2][kBMaxB];
  int64_t slot_row[kBMaxB];  // pool slot -> row (-1 = free)
  int64_t slot_valid[kBMaxB];// vectors [0, slot_valid) are applied to the slot's column
};

static_assert(sizeof(KetGroup) % 16 == 0, "ket groups are copied in 16-byte words");

// Immutable per-system descriptor (device; copied to shared memory per item).
struct __align__(16) SysDesc {
  int64_t n, ld, Mcap;
  int N, O, Op, b;
  double tau, neg_tol;
  PairSet bra, ket;                 // screened bra shell pairs (by class), all shell pairs
  int64_t cls[4], all_cls[4];
  int ntile[3], nsplit_cap;
  int64_t nnz;                      // entries of the row lists (2 n minus the diagonal pairs)
  int tc;                           // column update: 1 = exact 7-slice BF16 products on the tensor cores, 0 = DFMA
  int pad0;
  const int32_t* erow;              // [n] row exponents: |L^K_r| <= sqrt(D^1_r) < 2^erow[r]
  __nv_bfloat16* Bsl;               // [2][7][64][bpitch] slices of the gathered pivot rows (tc)
  int64_t bpitch;
  const int32_t* row_allsp;         // [n] shell pair (in ket) of each row
  const int8_t* row_kc;             // [n] canonical components of each row
  const int8_t* row_kd;
  const int32_t* row_mu;            // [n] mu >= nu of each row
  const int32_t* row_nu;
  const int32_t* csr_off;           // [N+1] row list per basis function mu:
  const int32_t* csr_nu;            //   partner nu and row r of every screened pair (mu nu)
  const int32_t* csr_row;
  const double* C;                  // [N][Op] occupied coefficients (rows zero-padded to Op)
  double* D0;                       // [ld] residual diagonals (double buffered)
  double* D1;
  double* pool;                     // [b][ld] candidate columns
  double* L;                        // [Mcap][ld] vectors (DFMA mode; NULL with tc)
  __nv_bfloat16* Ls;                // tc: vectors as 7 BF16 slices, [ceil(Mcap/32)][7][n][32] (zeroed)
  double* Lblk;                     // tc: the current block's vectors in FP64, [kBMaxB][ld]
  int64_t* piv;                     // [Mcap] pivot rows
  double* pivd;                     // [Mcap] their residual diagonals
  double* Bg0;                      // [Mcap][b] gathered pivot rows (new slots)
  double* Bg1;                      // [b][b] (kept slots)
  KetGroup* groups;                 // [b]
  double* part_val;                 // [ceil(n / kStepRows)] partial argmax
  int64_t* part_idx;
  double* dpk;                      // [ld] packed density
  double* v;                        // [Mcap] v_P
  double* Jp;                       // [ld] packed J
  double* B;                        // [Mcap][N][Op] half-transformed vectors
  double* Kpart;                    // [nsplit_cap][N][N] partial K tiles
  double* J;                        // [N][N]
  double* Kx;                       // [N][N]
  SysState* st;
};

constexpr int kJobKinds = 16;
struct BatchCtl {
  unsigned done_sys;            // systems finished (converged or failed)
  int abort;                    // stop claiming work
  int timed_out;                // a CTA's wait for work ran out
  int tc_err;                   // a bounded tensor-core (MMA completion) wait gave up
  unsigned long long progress;  // items completed, all systems
  unsigned long long kind_ns[kJobKinds];     // CTA time per item kind (incl. its job finish)
  unsigned long long kind_items[kJobKinds];  // items per kind
  unsigned long long kind_ops[kJobKinds];    // FP64-pipe operations per kind (one per FMA; ERI: executed)
  unsigned long long idle_ns;                // CTA time spent looking for work
  unsigned long long tc_ns[4];               // tensor-core update items: operand copies, MMA issue + wait, drain, result
};

// ------------------------------------------------------------ helpers ----
__device__ __forceinline__ long long globaltimer_ns() {
  long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
template <class T>
__device__ __forceinline__ T vload(const T* p) { return *(const volatile T*)p; }

__device__ __forceinline__ bool better(double v1, int64_t i1, double v2, int64_t i2) {
  return v1 > v2 || (v1 == v2 && i1 < i2);
}
__device__ __forceinline__ void warp_argmax(double& v, int64_t& i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    const int64_t i2 = __shfl_xor_sync(0xffffffffu, i, o);
    if (better(v2, i2, v, i)) { v = v2; i = i2; }
  }
}
// CTA argmax; result valid in every thread
__device__ void cta_argmax(double& v, int64_t& i, double* sv, int64_t* si) {
  warp_argmax(v, i);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) { sv[w] = v; si[w] = i; }
  __syncthreads();
  v = sv[0]; i = si[0];
  for (int k = 1; k < kBT / 32; ++k)
    if (better(sv[k], si[k], v, i)) { v = sv[k]; i = si[k]; }
  __syncthreads();
}
__device__ double cta_sum(double x, double* sv) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sv[w] = x;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < kBT / 32; ++k) s += sv[k];
  __syncthreads();
  return s;
}
__device__ int cta_sum_int(int x, int* sv) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sv[w] = x;
  __syncthreads();
  int s = 0;
  for (int k = 0; k < kBT / 32; ++k) s += sv[k];
  __syncthreads();
  return s;
}
__device__ __forceinline__ const double* dcur(const SysDesc& d, int cur) { return cur ? d.D1 : d.D0; }
__device__ __forceinline__ double* dnext(const SysDesc& d, int cur) { return cur ? d.D0 : d.D1; }
__device__ __forceinline__ unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// reduction scratch shared by the helpers
struct Red {
  double v[kBT / 32];
  int64_t i[kBT / 32];
  int n[kBT / 32];
};

// --------------------------------------------------------------- SELECT ----
// Candidates of a new block: the b rows with the largest residual diagonals
// >= tau, ordered by (D descending, row ascending); the exact top b of that
// order.  Positive doubles compare like their bit patterns, so a radix select
// over 12-bit digits of the bit pattern finds the bin of the b-th value; the
// rows of that bin (at most kTieCap, or all of one value) are ranked directly.
__device__ void select_item(const SysDesc& d, unsigned char* smem, Red* red, int64_t* s_cand, int* s_int) {
  SysState* st = d.st;
  const int tid = threadIdx.x;
  const int64_t n = d.n;
  const int cur = vload(&st->cur);
  const double dmax = vload(&st->dmax);
  const double tau = d.tau;
  if (!(dmax >= tau)) {
    if (tid == 0) st->converged = 1;
    return;
  }
  const double* D = dcur(d, cur);
  unsigned* hist = (unsigned*)smem;                           // [4096]
  unsigned long long* tkey = (unsigned long long*)(smem + 16384);   // [kTieCap]
  int64_t* trow = (int64_t*)(smem + 16384 + 8 * kTieCap);     // [kTieCap]
  const int b = d.b;
  int cnt = 0;
  for (int64_t r = tid; r < n; r += kBT) cnt += (__ldcg(D + r) >= tau) ? 1 : 0;
  cnt = cta_sum_int(cnt, red->n);
  // s_int: 0 n_cand, 1 n_tie, 2 need, 3 sel bin, 4 fixed bits, 5 stop
  unsigned long long prefix = 0;
  int fixed = 0, need = b;
  if (cnt > b) {
    for (;;) {
      const int dig = min(12, 64 - fixed);
      const int shift = 64 - fixed - dig;
      const unsigned nbin = 1u << dig;
      for (unsigned k = tid; k < nbin; k += kBT) hist[k] = 0;
      __syncthreads();
      for (int64_t r = tid; r < n; r += kBT) {
        const double x = __ldcg(D + r);
        if (!(x >= tau)) continue;
        const unsigned long long key = (unsigned long long)__double_as_longlong(x);
        if (fixed > 0 && (key >> (64 - fixed)) != prefix) continue;
        atomicAdd(&hist[(unsigned)((key >> shift) & (nbin - 1))], 1u);
      }
      __syncthreads();
      // bin of the need-th largest: chunk sums (32 bins per thread), then one scan
      const unsigned per = (nbin + kBT - 1) / kBT;
      unsigned csum = 0;
      for (unsigned k = tid * per; k < min(nbin, (tid + 1) * per); ++k) csum += hist[k];
      unsigned* chunk = (unsigned*)(smem + 16384);  // tkey area is free during the passes
      chunk[tid] = csum;
      __syncthreads();
      if (tid == 0) {
        unsigned above = 0;
        int c = kBT - 1;
        for (; c > 0; --c) {
          if (above + chunk[c] >= (unsigned)need) break;
          above += chunk[c];
        }
        unsigned bin = min(nbin, (unsigned)(c + 1) * per);
        unsigned sel = (unsigned)c * per;
        for (unsigned k = bin; k-- > (unsigned)c * per;) {
          if (above + hist[k] >= (unsigned)need) { sel = k; break; }
          above += hist[k];
        }
        s_int[2] = need - (int)above;
        s_int[3] = (int)sel;
        s_int[5] = (hist[sel] <= (unsigned)kTieCap || fixed + dig == 64) ? 1 : 0;
      }
      __syncthreads();
      need = s_int[2];
      prefix = (prefix << dig) | (unsigned long long)s_int[3];
      fixed += dig;
      const int stop = s_int[5];
      __syncthreads();
      if (stop) break;
    }
  }
  // collect: rows above the bin (all taken) and the bin's rows, in row order
  if (tid == 0) { s_int[0] = 0; s_int[1] = 0; }
  __syncthreads();
  for (int64_t r0 = 0; r0 < n; r0 += kBT) {
    const int64_t r = r0 + tid;
    int kind = 0;   // 1 above, 2 in the bin
    unsigned long long key = 0;
    if (r < n) {
      const double x = __ldcg(D + r);
      if (x >= tau) {
        key = (unsigned long long)__double_as_longlong(x);
        if (cnt <= b) kind = 1;
        else {
          const unsigned long long hi = key >> (64 - fixed);
          kind = hi > prefix ? 1 : (hi == prefix ? 2 : 0);
        }
      }
    }
    const unsigned ma = __ballot_sync(0xffffffffu, kind == 1);
    const unsigned mt = __ballot_sync(0xffffffffu, kind == 2);
    const int w = tid >> 5, lane = tid & 31;
    if (lane == 0) { red->n[w] = __popc(ma) | (__popc(mt) << 8); }
    __syncthreads();
    int base_a = s_int[0], base_t = s_int[1];
    for (int k = 0; k < w; ++k) { base_a += red->n[k] & 0xff; base_t += red->n[k] >> 8; }
    const unsigned below = (1u << lane) - 1u;
    if (kind == 1) s_cand[base_a + __popc(ma & below)] = r;
    if (kind == 2) {
      const int t = base_t + __popc(mt & below);
      if (t < kTieCap) { tkey[t] = key; trow[t] = r; }
    }
    __syncthreads();
    if (tid == 0) {
      int ta = 0, tt = 0;
      for (int k = 0; k < kBT / 32; ++k) { ta += red->n[k] & 0xff; tt += red->n[k] >> 8; }
      s_int[0] += ta;
      s_int[1] += tt;
    }
    __syncthreads();
  }
  if (cnt > b) {
    const int nab = s_int[0];
    const int nt = min(s_int[1], kTieCap);
    for (int e = tid; e < nt; e += kBT) {
      int rank = 0;
      for (int f = 0; f < nt; ++f)
        rank += (tkey[f] > tkey[e] || (tkey[f] == tkey[e] && trow[f] < trow[e])) ? 1 : 0;
      if (rank < need) s_cand[nab + rank] = trow[e];
    }
    __syncthreads();
    if (tid == 0) s_int[0] = nab + need;
    __syncthreads();
  }
  const int nc = min(s_int[0], b);
  // slots: free the ones no longer wanted, keep the others, new rows take free slots
  if (tid == 0) {
    volatile SysState* st = d.st;
    // candidates in row order (deterministic slot assignment)
    for (int i = 1; i < nc; ++i) {
      const int64_t x = s_cand[i];
      int j = i - 1;
      while (j >= 0 && s_cand[j] > x) { s_cand[j + 1] = s_cand[j]; --j; }
      s_cand[j + 1] = x;
    }
    const int64_t K = st->K;
    bool kept[kBMaxB];
    for (int s = 0; s < b; ++s) {
      const int64_t r = st->slot_row[s];
      bool want = false;
      if (r >= 0)
        for (int i = 0; i < nc; ++i) want = want || (s_cand[i] == r);
      if (r >= 0 && !want) st->slot_row[s] = -1;
      kept[s] = r >= 0 && want;
    }
    // update groups: new slots need vectors [0, K), kept ones [valid, K)
    int nnew = 0, nkeep = 0;
    int64_t kvalid = K;
    KetDesc kd[kBMaxB];
    int nk = 0;
    for (int i = 0; i < nc; ++i) {
      const int64_t r = s_cand[i];
      int slot = -1;
      for (int s = 0; s < b; ++s)
        if (kept[s] && st->slot_row[s] == r) slot = s;
      if (slot >= 0) continue;
      for (int s = 0; s < b && slot < 0; ++s)
        if (st->slot_row[s] < 0) slot = s;
      if (slot < 0) break;   // cannot happen: at most b candidates, kept ones hold their slots
      st->slot_row[slot] = r;
      kept[slot] = false;
      st->uslot[0][nnew] = slot;
      st->urow[0][nnew] = r;
      ++nnew;
      KetDesc k;
      k.sp = __ldg(d.row_allsp + r);
      k.slot = slot;
      k.kc = __ldg(d.row_kc + r);
      k.kd = __ldg(d.row_kd + r);
      if (k.sp < d.all_cls[1]) { k.lc = 0; k.ld = 0; }
      else if (k.sp < d.all_cls[2]) { k.lc = 1; k.ld = 0; }
      else { k.lc = 1; k.ld = 1; }
      kd[nk++] = k;
    }
    for (int s = 0; s < b; ++s)
      if (kept[s] && st->slot_valid[s] < K) {
        st->uslot[1][nkeep] = s;
        st->urow[1][nkeep] = st->slot_row[s];
        kvalid = min(kvalid, st->slot_valid[s]);
        ++nkeep;
      }
    st->nb[0] = K > 0 ? nnew : 0;
    st->k0[0] = 0;
    st->nb[1] = nkeep;
    st->k0[1] = kvalid;
    for (int s = 0; s < b; ++s)
      if (st->slot_row[s] >= 0) st->slot_valid[s] = K;
    // ket groups: same shell pair together (sorted by shell pair, kc, kd), up to
    // 9 components for a (pp) shell pair and 3 otherwise
    for (int i = 1; i < nk; ++i) {
      const KetDesc x = kd[i];
      int j = i - 1;
      while (j >= 0 && (kd[j].sp > x.sp || (kd[j].sp == x.sp && (kd[j].kc > x.kc || (kd[j].kc == x.kc && kd[j].kd > x.kd))))) {
        kd[j + 1] = kd[j];
        --j;
      }
      kd[j + 1] = x;
    }
    int ng = 0;
    for (int i = 0; i < nk;) {
      const int cap = (kd[i].lc == 1 && kd[i].ld == 1) ? kMaxKetGroup : 3;
      int j = i;
      while (j < nk && kd[j].sp == kd[i].sp && j - i < cap) ++j;
      KetGroup g;
      memset(&g, 0, sizeof(g));
      g.sp = kd[i].sp;
      g.lc = kd[i].lc;
      g.ld = kd[i].ld;
      g.nc = (int8_t)(j - i);
      for (int c = 0; c < j - i; ++c) {
        g.kc[c] = kd[i + c].kc;
        g.kd[c] = kd[i + c].kd;
        g.slot[c] = kd[i + c].slot;
      }
      d.groups[ng++] = g;
      i = j;
    }
    st->ngroups = ng;
    st->Kb = K;
    for (int g = 0; g < 2; ++g) {
      // DFMA: vectors [k0, K); tensor cores: the whole 32-vector blocks that hold them
      const int64_t lo = d.tc ? st->k0[g] / kTcBK * kTcBK : st->k0[g];
      const int64_t hi = d.tc ? (K + kTcBK - 1) / kTcBK * kTcBK : K;
      st->gitems[g] = st->nb[g] > 0 ? (int)ceil_div(hi - lo, kGatherQ) : 0;
    }
    int64_t neri = 0;
    for (int c = 0; c < 3; ++c) neri += (int64_t)d.ntile[c] * ng;
    st->nitems[0] = st->gitems[0] + st->gitems[1];
    st->nitems[1] = (int)neri;
  }
}

// ----------------------------------------------------------------- COLS ----
__device__ void gather_item(const SysDesc& d, unsigned it) {
  SysState* st = d.st;
  const int g0 = vload(&st->gitems[0]);
  const int g = (int)it < g0 ? 0 : 1;
  const unsigned chunk = g == 0 ? it : it - g0;
  const int nb = vload(&st->nb[g]);
  const int64_t k0 = vload(&st->k0[g]), K = vload(&st->K);
  const int64_t q0 = k0 + (int64_t)chunk * kGatherQ;
  const int64_t q1 = min(K, q0 + kGatherQ);
  double* Bg = g ? d.Bg1 : d.Bg0;
  const int64_t tot = (q1 - q0) * nb;
  for (int64_t e = threadIdx.x; e < tot; e += kBT) {
    const int64_t q = q0 + e / nb;
    const int j = (int)(e % nb);
    const int64_t row = vload(&st->urow[g][j]);
    Bg[(q - k0) * nb + j] = __ldcg(d.L + q * d.ld + row);
  }
}

// 16-byte global -> shared copy that bypasses registers (src_bytes = 0: zero fill)
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_u32(sdst)), "l"(gsrc), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// element (q, r) of slice t in the chunked slice store
__device__ __forceinline__ int64_t ls_index(int64_t n, int64_t q, int t, int64_t r) {
  return (((q / kTcBK) * kTcSlices + t) * n + r) * kTcBK + q % kTcBK;
}

// Slices of the gathered pivot rows for the tensor-core update: group g, column
// j, vector q in the 32-vector blocks covering [k0, K): the 7 slices of
// L[q][row_j] from the slice store (zero outside [k0, K)), Bsl[g][s][j][q - kbase].
__device__ void gather_tc_item(const SysDesc& d, unsigned it) {
  SysState* st = d.st;
  const int g0 = vload(&st->gitems[0]);
  const int g = (int)it < g0 ? 0 : 1;
  const unsigned chunk = g == 0 ? it : it - g0;
  const int nb = vload(&st->nb[g]);
  const int64_t k0 = vload(&st->k0[g]), K = vload(&st->K);
  const int64_t kbase = k0 / kTcBK * kTcBK, kpad = (K + kTcBK - 1) / kTcBK * kTcBK;
  const int64_t q0 = kbase + (int64_t)chunk * kGatherQ;
  const int64_t nq = min(kpad, q0 + kGatherQ) - q0;
  __nv_bfloat16* B = d.Bsl + (int64_t)g * kTcSlices * 64 * d.bpitch;
  const int64_t tot = nq * nb;
  for (int64_t e = threadIdx.x; e < tot; e += kBT) {
    const int j = (int)(e / nq);
    const int64_t q = q0 + e % nq;
    const int64_t row = vload(&st->urow[g][j]);
    const bool in = q >= k0 && q < K;
#pragma unroll
    for (int t = 0; t < kTcSlices; ++t)
      B[((int64_t)t * 64 + j) * d.bpitch + (q - kbase)] =
          in ? __ldcg(d.Ls + ls_index(d.n, q, t, row)) : __float2bfloat16_rn(0.0f);
  }
}

// Column update on the tensor cores, exact 7-slice products (the same
// arithmetic as the single-system sliced update): 128 rows x 32 columns of one
// update group over its vectors [k0, K).  Per block of 32 vectors every thread
// copies its row of the 7 slice planes into A (64-byte swizzled rows: the
// 16-byte chunk c of row r sits at chunk c ^ ((r >> 1) & 3)), the CTA copies
// the 32 columns' slices into B, and thread 0 issues one MMA per A slice s
// against the stacked B slices 0..6-s (N = 32 (7 - s)), so that the product
// (s, t) lands in accumulator group s + t.  Every 4 blocks the 7 groups are
// drained from tensor memory into 64-bit fixed-point sums (thread = row); at
// the end col -= 2^(e_r + e_c - 60) * sum.
__device__ bool update_tc_item(const SysDesc& d, unsigned it, unsigned char* smem, uint32_t tmem, uint64_t* mbar,
                               uint32_t& mphase, int* s_fail, BatchCtl* ctl, long long wait_ns) {
  SysState* st = d.st;
  const int n0 = vload(&st->nitems[0]);
  const int g = (int)it < n0 ? 0 : 1;
  const int64_t li = g == 0 ? it : it - n0;
  const int nb = vload(&st->nb[g]);
  const int ctn = (nb + kTcBN - 1) / kTcBN;
  const int64_t rt = li / ctn;
  const int ct = (int)(li % ctn);
  const int64_t k0 = vload(&st->k0[g]), K = vload(&st->K);
  const int64_t n = d.n, ld = d.ld, r0 = rt * 128;
  const int tid = threadIdx.x, w = tid >> 5;
  const int64_t r = r0 + tid;
  const int er = r < n ? __ldg(d.erow + r) : 0;
  const int kb0 = (int)(k0 / kTcBK), kb1 = (int)((K + kTcBK - 1) / kTcBK);
  (void)ld;
  const int64_t kbase = (int64_t)kb0 * kTcBK;
  unsigned char* A = smem;
  unsigned char* Bm = smem + kTcABytes;
  const __nv_bfloat16* Bg = d.Bsl + (int64_t)g * kTcSlices * 64 * d.bpitch;
  const int sw = (tid >> 1) & 3;
  long long run[kTcBN];
#pragma unroll
  for (int c = 0; c < kTcBN; ++c) run[c] = 0;
  if (tid == 0) *s_fail = 0;
  long long tt[4] = {0, 0, 0, 0};
  long long tprev = tid == 0 ? globaltimer_ns() : 0;
  auto mark = [&](int k) {
    if (tid == 0) {
      const long long t = globaltimer_ns();
      tt[k] += t - tprev;
      tprev = t;
    }
  };
  for (int kb = kb0; kb < kb1; kb += kTcChunk) {
    const int kbe = min(kb1, kb + kTcChunk);
    for (int b = kb; b < kbe; ++b) {
      // A: this thread's row of the 7 slice planes of vector block b (64 bytes each),
      // B: 7 slices x 32 columns x 32 vectors of the gathered slices; all copies
      // in flight at once (cp.async), rows past n and columns past nb zero-filled
#pragma unroll
      for (int t = 0; t < kTcSlices; ++t) {
        const __nv_bfloat16* src = d.Ls + (((int64_t)b * kTcSlices + t) * n + (r < n ? r : 0)) * kTcBK;
#pragma unroll
        for (int c = 0; c < 4; ++c)
          cp_async16(A + t * (128 * 64) + tid * 64 + ((c ^ sw) * 16), src + c * 8, r < n ? 16 : 0);
      }
      for (int t = tid; t < kTcSlices * kTcBN * 4; t += kBT) {
        const int sl = t / (kTcBN * 4), jj = (t / 4) % kTcBN, c = t % 4;
        const int j = ct * kTcBN + jj;
        const __nv_bfloat16* src = Bg + ((int64_t)sl * 64 + (j < nb ? j : 0)) * d.bpitch + ((int64_t)b * kTcBK - kbase) + c * 8;
        cp_async16(Bm + sl * (kTcBN * 64) + jj * 64 + ((c ^ ((jj >> 1) & 3)) * 16), src, j < nb ? 16 : 0);
      }
      cp_async_wait_all();
      tc::fence_proxy_async();
      __syncthreads();
      mark(0);
      if (tid == 0) {
        tc::tc_fence_after();
        const uint32_t a0 = tc::smem_u32(A), b0 = tc::smem_u32(Bm);
#pragma unroll
        for (int sa = 0; sa < kTcSlices; ++sa) {
          const int nt = kTcSlices - sa;
          const uint32_t idesc = tc::idesc_bf16_f32_n(128, nt * kTcBN);
#pragma unroll
          for (int kk = 0; kk < kTcBK / 16; ++kk)
            tc::umma_bf16(tmem + (uint32_t)(sa * kTcBN), sdesc_k_sw64(a0 + sa * (128 * 64) + kk * 32),
                          sdesc_k_sw64(b0 + kk * 32), idesc, (b == kb && sa == 0 && kk == 0) ? 0u : 1u);
        }
        tc::umma_commit(mbar);
      }
      if (tid == 0) {
        volatile int ab = 0;
        if (!tc::mbar_wait(mbar, mphase, &ab, &ctl->tc_err, 1, (unsigned long long)wait_ns)) {
          tc::mbar_settle(mbar, mphase);
          *s_fail = 1;
          atomicExch(&ctl->abort, 1);
        }
        mphase ^= 1u;
      }
      __syncthreads();
      mark(1);
      if (*(volatile int*)s_fail) return false;
    }
    // drain the 7 groups into the fixed-point sums (thread = TMEM lane = tile row)
    tc::tc_fence_after();
    const uint32_t acc = tmem + ((uint32_t)(w * 32) << 16);
#pragma unroll
    for (int gq = 0; gq < kTcSlices; ++gq) {
      const int sh = kTcF - 8 * (gq + 2) + 2;
#pragma unroll
      for (int cb = 0; cb < kTcBN / 16; ++cb) {
        uint32_t v[16];
        tc::tmem_ld16(acc + (uint32_t)(gq * kTcBN + cb * 16), v);
        tc::tmem_ld_wait();
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const long long iv = exact_float_to_ll(__uint_as_float(v[c]));
          run[cb * 16 + c] += sh >= 0 ? (iv << sh) : ((iv + (1ll << (-sh - 1))) >> (-sh));
        }
      }
    }
    tc::tc_fence_before();
    __syncthreads();
    mark(2);
  }
  if (r < n) {
#pragma unroll
    for (int c = 0; c < kTcBN; ++c) {
      const int j = ct * kTcBN + c;
      if (j >= nb) continue;
      double* col = d.pool + (int64_t)vload(&st->uslot[g][j]) * ld;
      const int ec = __ldg(d.erow + vload(&st->urow[g][j]));
      col[r] = __ldcg(col + r) - ldexp((double)run[c], er + ec - kTcF);
    }
  }
  __syncthreads();
  mark(3);
  if (tid == 0)
    for (int k = 0; k < 4; ++k) atomicAdd(&ctl->tc_ns[k], (unsigned long long)tt[k]);
  return true;
}

__device__ void eri_item(const SysDesc& d, unsigned it, const double* boys, KetGroup* sg,
                         unsigned long long* ops_out) {
  SysState* st = d.st;
  const int ng = vload(&st->ngroups);
  int64_t j = (int64_t)it - vload(&st->nitems[0]);
  int c = 2;
  for (; c > 0; --c) {
    const int64_t cnt = (int64_t)d.ntile[c] * ng;
    if (j < cnt) break;
    j -= cnt;
  }
  const int64_t tile = j / ng;
  const int g = (int)(j % ng);
  if (threadIdx.x < (int)(sizeof(KetGroup) / 16))
    ((int4*)sg)[threadIdx.x] = __ldcg((const int4*)(d.groups + g) + threadIdx.x);
  __syncthreads();
  unsigned long long ops = 0;
  if (c == 0) column_item<0, 0>(d.bra, nullptr, d.cls[0], d.cls[1], d.ket, sg, tile, 0, d.pool, d.ld, boys, ops);
  else if (c == 1) column_item<1, 0>(d.bra, nullptr, d.cls[1], d.cls[2], d.ket, sg, tile, 0, d.pool, d.ld, boys, ops);
  else column_item<1, 1>(d.bra, nullptr, d.cls[2], d.cls[3], d.ket, sg, tile, 0, d.pool, d.ld, boys, ops);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ops += __shfl_xor_sync(0xffffffffu, ops, o);
  if ((threadIdx.x & 31) == 0 && ops) atomicAdd(ops_out, ops);
}

// --------------------------------------------------------------- UPDATE ----
// pool[slot_j][r] -= sum_{q in [k0, K)} L[q][r] Bg[q - k0][j] for 128 rows and
// the nb <= NC columns of one update group (NC = 64, or 32 for narrow groups).
// Thread (tx, ty) owns rows tx + 16 i (i < 8) and columns CPT ty + c (c < CPT).
template <int NC>
__device__ void update_tile(const SysDesc& d, unsigned it, unsigned char* smem) {
  constexpr int CPT = NC / 8;
  SysState* st = d.st;
  const int n0 = vload(&st->nitems[0]);
  const int g = (int)it < n0 ? 0 : 1;
  const int64_t tile = g == 0 ? it : it - n0;
  const int nb = vload(&st->nb[g]);
  const int64_t k0 = vload(&st->k0[g]), K = vload(&st->K);
  const int64_t n = d.n, ld = d.ld, r0 = tile * kRowTile;
  const double* Bg = g ? d.Bg1 : d.Bg0;
  double (*As)[kRowTile] = (double (*)[kRowTile])smem;                  // [16][128]
  double (*Bs)[NC] = (double (*)[NC])(smem + 16 * kRowTile * 8);  // [16][NC]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[8][CPT];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < CPT; ++c) acc[i][c] = 0.0;
  for (int64_t kk = k0; kk < K; kk += 16) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const int e = tid + kBT * t;
      const int k = e >> 6, rp = (e & 63) * 2;
      const int64_t q = kk + k, r = r0 + rp;
      double2 x = make_double2(0.0, 0.0);
      if (q < K) {
        const double* src = d.L + q * ld + r;
        if (r + 1 < n) x = __ldcg((const double2*)src);
        else if (r < n) x.x = __ldcg(src);
      }
      *(double2*)&As[k][rp] = x;
    }
#pragma unroll
    for (int t = 0; t < NC / 8; ++t) {
      const int e = tid + kBT * t;
      const int k = e / NC, j = e % NC;
      const int64_t q = kk + k;
      Bs[k][j] = (q < K && j < nb) ? __ldcg(Bg + (q - k0) * nb + j) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      double a[8], bb[CPT];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = As[k][tx + 16 * i];
#pragma unroll
      for (int c = 0; c < CPT; ++c) bb[c] = Bs[k][ty * CPT + c];
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int c = 0; c < CPT; ++c) acc[i][c] = fma(a[i], bb[c], acc[i][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < CPT; ++c) {
    const int j = ty * CPT + c;
    if (j >= nb) continue;
    double* col = d.pool + (int64_t)vload(&st->uslot[g][j]) * ld;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t r = r0 + tx + 16 * i;
      if (r < n) col[r] = __ldcg(col + r) - acc[i][c];
    }
  }
}

__device__ void update_item(const SysDesc& d, unsigned it, unsigned char* smem) {
  const SysState* st = d.st;
  const int g = (int)it < vload(&st->nitems[0]) ? 0 : 1;
  if (vload(&st->nb[g]) <= 32) update_tile<32>(d, it, smem);
  else update_tile<64>(d, it, smem);
}

// ----------------------------------------------------------------- STEP ----
// L^K_r = (col_r - sum_{k in [Kb, K)} L^k_r L^k_p) / sqrt(D_p), D'_r = D_r - (L^K_r)^2
// for 1024 rows; the item's argmax of D' goes to part_val / part_idx.
__device__ void step_item(const SysDesc& d, unsigned it, unsigned char* smem, Red* red) {
  SysState* st = d.st;
  const int64_t K = vload(&st->K), Kb = vload(&st->Kb), prow = vload(&st->prow);
  const int pslot = vload(&st->pslot), cur = vload(&st->cur);
  const double dp = vload(&st->dp);
  const int64_t n = d.n, ld = d.ld;
  double* g = (double*)smem;
  const int nk = (int)(K - Kb);
  // the block's earlier vectors: rows Kb.. of L, or the FP64 block buffer (tensor-core mode)
  const double* Lb = d.tc ? d.Lblk : d.L + Kb * ld;
  for (int k = threadIdx.x; k < nk; k += kBT) g[k] = __ldcg(Lb + k * ld + prow);
  __syncthreads();
  const int64_t r0 = (int64_t)it * kStepRows + threadIdx.x;
  constexpr int R = kStepRows / kBT;
  double acc[R];
  const double* col = d.pool + (int64_t)pslot * ld;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int64_t r = r0 + (int64_t)j * kBT;
    acc[j] = r < n ? __ldcg(col + r) : 0.0;
  }
  for (int k = 0; k < nk; ++k) {
    const double gk = g[k];
    const double* Lk = Lb + k * ld;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int64_t r = r0 + (int64_t)j * kBT;
      if (r < n) acc[j] = fma(-__ldcg(Lk + r), gk, acc[j]);
    }
  }
  const double inv = 1.0 / sqrt(dp);
  const double* Din = dcur(d, cur);
  double* Dout = dnext(d, cur);
  double* Lout = d.tc ? d.Lblk + (K - Kb) * ld : d.L + K * ld;
  double bv = -1.0e300;
  int64_t bi = INT64_MAX;
  int bad = 0;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int64_t r = r0 + (int64_t)j * kBT;
    if (r < n) {
      const double vv = acc[j] * inv;
      Lout[r] = vv;
      const double dd = fma(-vv, vv, __ldcg(Din + r));
      Dout[r] = dd;
      bad |= dd < d.neg_tol;
      if (better(dd, r, bv, bi)) { bv = dd; bi = r; }
    }
  }
  cta_argmax(bv, bi, red->v, red->i);
  if (bad) atomicOr(&d.st->bad, 1);
  if (threadIdx.x == 0) {
    d.part_val[it] = bv;
    d.part_idx[it] = bi;
  }
}

// ---------------------------------------------------------------- SLICE ----
// Tensor-core mode, after a block: its vectors [Kb, K) (FP64 block buffer) as
// 7 BF16 slices in the store, round(L 2^(55 - e_r)) in balanced base-256 digits
// (the representation of the single-system sliced update), 1024 rows per item,
// 8 vectors per 16-byte store (partial groups keep the neighbouring blocks' values).
__device__ void slice_item(const SysDesc& d, unsigned it) {
  const SysState* st = d.st;
  const int64_t K = vload(&st->K), Kb = vload(&st->Kb), n = d.n;
  const int64_t r0 = (int64_t)it * kStepRows;
  for (int64_t r = r0 + threadIdx.x; r < min(n, r0 + kStepRows); r += kBT) {
    const int er = __ldg(d.erow + r);
    for (int64_t q8 = Kb / 8 * 8; q8 < K; q8 += 8) {
      unsigned short h[kTcSlices][8];
      const bool full = q8 >= Kb && q8 + 8 <= K;
      if (!full) {
#pragma unroll
        for (int t = 0; t < kTcSlices; ++t) {
          const uint4 v = __ldcg((const uint4*)(d.Ls + ls_index(n, q8, t, r)));
          const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int m = 0; m < 4; ++m) {
            h[t][2 * m] = (unsigned short)(w[m] & 0xffffu);
            h[t][2 * m + 1] = (unsigned short)(w[m] >> 16);
          }
        }
      }
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int64_t q = q8 + e;
        if (q < Kb || q >= K) continue;
        float a[kTcSlices];
        fixed_digits<kTcSlices>(scaled_double_to_ll(__ldcg(d.Lblk + (q - Kb) * d.ld + r), 8 * kTcSlices - 1 - er), a);
#pragma unroll
        for (int t = 0; t < kTcSlices; ++t) {
          const __nv_bfloat16 bv = __float2bfloat16_rn(a[t]);
          h[t][e] = *(const unsigned short*)&bv;
        }
      }
#pragma unroll
      for (int t = 0; t < kTcSlices; ++t) {
        uint4 v;
        v.x = (uint32_t)h[t][0] | ((uint32_t)h[t][1] << 16);
        v.y = (uint32_t)h[t][2] | ((uint32_t)h[t][3] << 16);
        v.z = (uint32_t)h[t][4] | ((uint32_t)h[t][5] << 16);
        v.w = (uint32_t)h[t][6] | ((uint32_t)h[t][7] << 16);
        *(uint4*)(d.Ls + ls_index(n, q8, t, r)) = v;
      }
    }
  }
}

// ------------------------------------------------------------------- JK ----
// d_r = D_{mu nu} (2 - delta_{mu nu}), D = 2 C C^T
__device__ void dens_item(const SysDesc& d, unsigned it) {
  const int64_t r0 = (int64_t)it * kStepRows;
  for (int64_t r = r0 + threadIdx.x; r < min(d.n, r0 + kStepRows); r += kBT) {
    const int mu = __ldg(d.row_mu + r), nu = __ldg(d.row_nu + r);
    const double* cm = d.C + (int64_t)mu * d.Op;
    const double* cn = d.C + (int64_t)nu * d.Op;
    double s = 0.0;
    for (int i = 0; i < d.O; ++i) s = fma(__ldg(cm + i), __ldg(cn + i), s);
    d.dpk[r] = 2.0 * s * (mu == nu ? 1.0 : 2.0);
  }
}

// B^P[mu][i] = sum_nu L^P_{mu nu} C[nu][i] for one vector P (warp per mu, lanes over i)
__device__ void kb_item(const SysDesc& d, unsigned P) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const double* Lp = d.L + (int64_t)P * d.ld;   // DFMA mode (the slice store has kb_tc_item)
  double* Bp = d.B + (int64_t)P * d.N * d.Op;
  for (int mu = w; mu < d.N; mu += kBT / 32) {
    const int e0 = __ldg(d.csr_off + mu), e1 = __ldg(d.csr_off + mu + 1);
    for (int i0 = 0; i0 < d.Op; i0 += 32) {
      const int i = i0 + lane;
      double s = 0.0;
      if (i < d.O)
        for (int e = e0; e < e1; ++e) {
          const double l = __ldcg(Lp + __ldg(d.csr_row + e));
          s = fma(l, __ldg(d.C + (int64_t)__ldg(d.csr_nu + e) * d.Op + i), s);
        }
      if (i < d.Op) Bp[(int64_t)mu * d.Op + i] = s;
    }
  }
}

// tensor-core mode: B^P[mu][i] = sum_nu L^P_{mu nu} C[nu][i] for the 32 vectors
// of slice chunk c (lane = vector: each row's 7 slice rows are read as 64-byte
// rows across the warp) and 8 basis functions mu (2 per warp); all columns i in
// one pass when the padded occupied count is at most 72, else passes of 24
template <int NI>
__device__ __forceinline__ void kb_tc_mu(const SysDesc& d, int64_t c, int mu, int i0, int lane, int64_t P, int64_t M) {
  const int e0 = __ldg(d.csr_off + mu), e1 = __ldg(d.csr_off + mu + 1);
  double acc[NI];
#pragma unroll
  for (int q = 0; q < NI; ++q) acc[q] = 0.0;
  for (int e = e0; e < e1; ++e) {
    const int32_t row = __ldg(d.csr_row + e), nu = __ldg(d.csr_nu + e);
    long long v = 0;
#pragma unroll
    for (int t = 0; t < kTcSlices; ++t)
      v = v * 256 + (long long)(int)__bfloat162float(__ldcg(d.Ls + ((c * kTcSlices + t) * d.n + row) * kTcBK + lane));
    const double x = ldexp((double)v, __ldg(d.erow + row) - (8 * kTcSlices - 1));
    // C rows are zero-padded to Op (a multiple of 8), so NI columns from i0 are in the array
    const double2* cr = (const double2*)(d.C + (int64_t)nu * d.Op + i0);
#pragma unroll
    for (int q = 0; q < NI / 2; ++q) {
      const double2 c2 = __ldg(cr + q);
      acc[2 * q] = fma(x, c2.x, acc[2 * q]);
      acc[2 * q + 1] = fma(x, c2.y, acc[2 * q + 1]);
    }
  }
  if (P < M) {
    double* Bp = d.B + ((int64_t)P * d.N + mu) * d.Op + i0;
#pragma unroll
    for (int q = 0; q < NI; ++q)
      if (i0 + q < d.Op) Bp[q] = acc[q];
  }
}

__device__ void kb_tc_item(const SysDesc& d, unsigned it, int64_t M) {
  const int nmu = (d.N + 7) / 8;
  const int64_t c = it / nmu;
  const int mb = (int)(it % nmu);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t P = c * 32 + lane;
  for (int mu = mb * 8 + w; mu < min(d.N, mb * 8 + 8); mu += kBT / 32) {
    if (d.Op <= 72) {
      // every column in one pass: each entry's 7 slice reads and its rebuild are done once
      kb_tc_mu<72>(d, c, mu, 0, lane, P, M);
    } else {
      for (int i0 = 0; i0 < d.Op; i0 += 24) kb_tc_mu<24>(d, c, mu, i0, lane, P, M);
    }
  }
}

// v_P = sum_r L^P_r d_r for kJvVec vectors
__device__ void jv_item(const SysDesc& d, unsigned it, int64_t M, Red* red) {
  for (int t = 0; t < kJvVec; ++t) {
    const int64_t P = (int64_t)it * kJvVec + t;
    if (P >= M) break;
    const double* Lp = d.L + P * d.ld;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < d.n; r += kBT) s = fma(__ldcg(Lp + r), __ldcg(d.dpk + r), s);
    s = cta_sum(s, red->v);
    if (threadIdx.x == 0) d.v[P] = s;
  }
}

// the 8 integers round(L^P_r 2^(55 - e_r)) of vectors 32 c + 8 g8 .. + 7 of row r
__device__ __forceinline__ void ls_ints8(const __nv_bfloat16* __restrict__ Ls, int64_t n, int64_t c, int g8, int64_t r,
                                         long long (&v)[8]) {
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = 0;
#pragma unroll
  for (int t = 0; t < kTcSlices; ++t) {
    const uint4 w4 = __ldcg((const uint4*)(Ls + ((c * kTcSlices + t) * n + r) * kTcBK + g8 * 8));
    const uint32_t w[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const unsigned short lo = (unsigned short)(w[m] & 0xffffu), hi = (unsigned short)(w[m] >> 16);
      v[2 * m] = v[2 * m] * 256 + (long long)(int)__bfloat162float(*(const __nv_bfloat16*)&lo);
      v[2 * m + 1] = v[2 * m + 1] * 256 + (long long)(int)__bfloat162float(*(const __nv_bfloat16*)&hi);
    }
  }
}

// tensor-core mode: v_P = sum_r L^P_r d_r for the 32 vectors of slice chunk `it`
// (every row's 7 x 64-byte slice rows read once), reduced over the CTA in shared memory
__device__ void jv_tc_item(const SysDesc& d, unsigned it, int64_t M, unsigned char* smem) {
  double acc[32];
#pragma unroll
  for (int e = 0; e < 32; ++e) acc[e] = 0.0;
  for (int64_t r = threadIdx.x; r < d.n; r += kBT) {
    const double sc = ldexp(__ldcg(d.dpk + r), __ldg(d.erow + r) - (8 * kTcSlices - 1));
#pragma unroll
    for (int g8 = 0; g8 < 4; ++g8) {
      long long v[8];
      ls_ints8(d.Ls, d.n, it, g8, r, v);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc[g8 * 8 + e] = fma((double)v[e], sc, acc[g8 * 8 + e]);
    }
  }
  double* red = (double*)smem;   // [32][kBT]
#pragma unroll
  for (int e = 0; e < 32; ++e) red[e * kBT + threadIdx.x] = acc[e];
  __syncthreads();
  if (threadIdx.x < 32) {
    const int64_t P = (int64_t)it * 32 + threadIdx.x;
    double sum = 0.0;
    for (int k = 0; k < kBT; ++k) sum += red[threadIdx.x * kBT + k];
    if (P < M) d.v[P] = sum;
  }
}

// tensor-core mode: J_r = sum_P L^P_r v_P for 1024 rows from the slice store
__device__ void jp_tc_item(const SysDesc& d, unsigned it, int64_t M, unsigned char* smem) {
  double* vs = (double*)smem;   // [1024]
  const int64_t r0 = (int64_t)it * kStepRows + threadIdx.x;
  constexpr int R = kStepRows / kBT;
  double acc[R];
#pragma unroll
  for (int j = 0; j < R; ++j) acc[j] = 0.0;
  for (int64_t P0 = 0; P0 < M; P0 += 1024) {
    const int np = (int)min((int64_t)1024, M - P0);
    __syncthreads();
    for (int k = threadIdx.x; k < 1024; k += kBT) vs[k] = k < np ? __ldcg(d.v + P0 + k) : 0.0;
    __syncthreads();
    for (int c = 0; c < (np + 31) / 32; ++c) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int64_t r = r0 + (int64_t)j * kBT;
        if (r >= d.n) continue;
#pragma unroll
        for (int g8 = 0; g8 < 4; ++g8) {
          long long v[8];
          ls_ints8(d.Ls, d.n, P0 / 32 + c, g8, r, v);
#pragma unroll
          for (int e = 0; e < 8; ++e) acc[j] = fma((double)v[e], vs[c * 32 + g8 * 8 + e], acc[j]);
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int64_t r = r0 + (int64_t)j * kBT;
    if (r < d.n) d.Jp[r] = ldexp(acc[j], __ldg(d.erow + r) - (8 * kTcSlices - 1));
  }
}

__device__ __forceinline__ void tile_of(unsigned t, int& bi, int& bj) {
  int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((i + 1) * (i + 2) / 2 <= (int)t) ++i;
  while (i * (i + 1) / 2 > (int)t) --i;
  bi = i;
  bj = (int)t - i * (i + 1) / 2;
}

// Kpart[s][mu][nu] = sum_{P in split s} sum_i B^P[mu][i] B^P[nu][i] over one
// 64 x 64 tile (block row bi >= block column bj).  Thread (tx, ty) owns
// mu = tx + 16 a (a < 4) and nu = ty + 8 c (c < 8).
__device__ void kt_item(const SysDesc& d, unsigned it, int64_t M, int ntiles, unsigned char* smem) {
  const int s = (int)(it / ntiles);
  int bi, bj;
  tile_of(it % ntiles, bi, bj);
  const int mu0 = bi * kKt, nu0 = bj * kKt, N = d.N, Op = d.Op;
  double (*As)[kKt] = (double (*)[kKt])smem;               // [8][64]
  double (*Bs)[kKt] = (double (*)[kKt])(smem + 8 * kKt * 8);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double acc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[a][c] = 0.0;
  const int64_t P0 = (int64_t)s * kKtSplit, P1 = min(M, P0 + kKtSplit);
  for (int64_t P = P0; P < P1; ++P) {
    const double* Bp = d.B + P * N * Op;
    for (int i0 = 0; i0 < Op; i0 += 8) {
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int e = tid + kBT * t;
        const int ii = e & 7, m = e >> 3;
        const int mu = mu0 + m, nu = nu0 + m;
        As[ii][m] = mu < N ? __ldcg(Bp + (int64_t)mu * Op + i0 + ii) : 0.0;
        Bs[ii][m] = nu < N ? __ldcg(Bp + (int64_t)nu * Op + i0 + ii) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        double a[4], bb[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] = As[k][tx + 16 * q];
#pragma unroll
        for (int c = 0; c < 8; ++c) bb[c] = Bs[k][ty + 8 * c];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[q][c] = fma(a[q], bb[c], acc[q][c]);
      }
      __syncthreads();
    }
  }
  double* Kp = d.Kpart + (int64_t)s * N * N;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int mu = mu0 + tx + 16 * q;
    if (mu >= N) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int nu = nu0 + ty + 8 * c;
      if (nu < N) Kp[(int64_t)mu * N + nu] = acc[q][c];
    }
  }
}

// J_r = sum_P L^P_r v_P for 1024 rows (v staged through shared memory)
__device__ void jp_item(const SysDesc& d, unsigned it, int64_t M, unsigned char* smem) {
  double* vs = (double*)smem;   // [1024]
  const int64_t r0 = (int64_t)it * kStepRows + threadIdx.x;
  constexpr int R = kStepRows / kBT;
  double acc[R];
#pragma unroll
  for (int j = 0; j < R; ++j) acc[j] = 0.0;
  for (int64_t P0 = 0; P0 < M; P0 += 1024) {
    const int np = (int)min((int64_t)1024, M - P0);
    __syncthreads();
    for (int k = threadIdx.x; k < np; k += kBT) vs[k] = __ldcg(d.v + P0 + k);
    __syncthreads();
    for (int k = 0; k < np; ++k) {
      const double vk = vs[k];
      const double* Lk = d.L + (P0 + k) * d.ld;
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int64_t r = r0 + (int64_t)j * kBT;
        if (r < d.n) acc[j] = fma(__ldcg(Lk + r), vk, acc[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int64_t r = r0 + (int64_t)j * kBT;
    if (r < d.n) d.Jp[r] = acc[j];
  }
}

// K[mu][nu] = K[nu][mu] = 2 sum_s Kpart[s][mu][nu] over one tile
__device__ void ksum_item(const SysDesc& d, unsigned t, int nsplit) {
  int bi, bj;
  tile_of(t, bi, bj);
  const int N = d.N;
  for (int e = threadIdx.x; e < kKt * kKt; e += kBT) {
    const int mu = bi * kKt + e / kKt, nu = bj * kKt + e % kKt;
    if (mu >= N || nu >= N) continue;
    double s = 0.0;
    for (int q = 0; q < nsplit; ++q) s += __ldcg(d.Kpart + ((int64_t)q * N + mu) * N + nu);
    d.Kx[(int64_t)mu * N + nu] = 2.0 * s;
    d.Kx[(int64_t)nu * N + mu] = 2.0 * s;
  }
}

__device__ void junpack_item(const SysDesc& d, unsigned it) {
  const int64_t r0 = (int64_t)it * kStepRows;
  for (int64_t r = r0 + threadIdx.x; r < min(d.n, r0 + kStepRows); r += kBT) {
    const int mu = __ldg(d.row_mu + r), nu = __ldg(d.row_nu + r);
    const double x = __ldcg(d.Jp + r);
    d.J[(int64_t)mu * d.N + nu] = x;
    d.J[(int64_t)nu * d.N + mu] = x;
  }
}

// -------------------------------------------------------------- finishes ----
// Thread 0 only: publish the next job (parameters first, then the word).
__device__ void publish(volatile SysState* st, int type, unsigned count) {
  st->type = type;
  st->done = 0;
  __threadfence();
  const unsigned long long w = st->word;
  atomicExch((unsigned long long*)&st->word, job_word(job_gen(w) + 1, count, 0));
}
__device__ void end_system(volatile SysState* st, BatchCtl* ctl, int status) {
  if (status != CD_OK) st->status = status;
  publish(st, kJobNone, 0);
  __threadfence();
  atomicAdd(&ctl->done_sys, 1u);
}

__device__ __forceinline__ int ntiles_k(int N) { const int nb = (N + kKt - 1) / kKt; return nb * (nb + 1) / 2; }

// Runs in thread 0: moves a system from the end of job `type` to its next
// non-empty job (or ends it).
__device__ void advance(const SysDesc& d, int type, BatchCtl* ctl) {
  volatile SysState* st = d.st;
  const unsigned nrow = ceil_div(d.n, kStepRows);
  for (;;) {
    const int64_t K = st->K;
    switch (type) {
      case kJobSelect: {
        if (st->converged) { type = kJobConverged; break; }
        const unsigned c = (unsigned)(st->nitems[0] + st->nitems[1]);
        if (c > 0) { publish(st, kJobCols, c); return; }
        type = kJobCols;
        break;
      }
      case kJobCols: {
        const unsigned t = ceil_div(d.n, kRowTile);
        for (int g = 0; g < 2; ++g) {
          const int ctn = d.tc ? (st->nb[g] + kTcBN - 1) / kTcBN : 1;   // tensor cores: 32-column tiles
          st->nitems[g] = (st->nb[g] > 0 && K > st->k0[g]) ? (int)t * ctn : 0;
        }
        const unsigned c = (unsigned)(st->nitems[0] + st->nitems[1]);
        if (c > 0) { publish(st, kJobUpdate, c); return; }
        type = kJobUpdate;
        break;
      }
      case kJobUpdate: {
        // first step of the block: the pivot is the argmax (one of the candidates)
        const int64_t p = st->idx;
        int slot = -1;
        for (int s = 0; s < d.b; ++s)
          if (st->slot_row[s] == p) slot = s;
        const double dp = __ldcg(dcur(d, st->cur) + p);
        if (slot < 0 || !(dp > 0.0)) { end_system(st, ctl, slot < 0 ? CD_EINVAL : CD_ENOTPSD); return; }
        st->prow = p;
        st->pslot = slot;
        st->dp = dp;
        publish(st, kJobStep, nrow);
        return;
      }
      case kJobConverged: {   // J/K build
        const int64_t M = K;
        st->nitems[0] = (int)nrow;
        st->nitems[1] = d.tc ? (int)(ceil_div(M, 32) * ((d.N + 7) / 8)) : (int)M;
        const unsigned c = (unsigned)(st->nitems[0] + st->nitems[1]);
        if (c > 0) { publish(st, kJobJk1, c); return; }
        type = kJobJk1;
        break;
      }
      case kJobJk1: {
        const int64_t M = K;
        const int nsplit = (int)ceil_div(M, kKtSplit);
        st->nitems[0] = (int)ceil_div(M, d.tc ? 32 : kJvVec);
        st->nitems[1] = nsplit * ntiles_k(d.N);
        const unsigned c = (unsigned)(st->nitems[0] + st->nitems[1]);
        if (c > 0) { publish(st, kJobJk2, c); return; }
        type = kJobJk2;
        break;
      }
      case kJobJk2: {
        st->nitems[0] = (int)nrow;
        st->nitems[1] = ntiles_k(d.N);
        publish(st, kJobJk3, (unsigned)(st->nitems[0] + st->nitems[1]));
        return;
      }
      case kJobJk3: {
        if (nrow > 0) { publish(st, kJobJk4, nrow); return; }
        type = kJobJk4;
        break;
      }
      case kJobJk4:
        end_system(st, ctl, CD_OK);
        return;
      case kJobSlice:
        if (st->after_slice == kJobSelect) { publish(st, kJobSelect, 1); return; }
        type = kJobConverged;
        break;
      default:
        end_system(st, ctl, CD_EINVAL);
        return;
    }
  }
}

// End of a pivot step (whole CTA): the step's argmax from the item partials,
// the pivot recorded, then the next job.
__device__ void finish_step(const SysDesc& d, BatchCtl* ctl, Red* red) {
  volatile SysState* st = d.st;
  const unsigned nit = ceil_div(d.n, kStepRows);
  double bv = -1.0e300;
  int64_t bi = INT64_MAX;
  for (unsigned k = threadIdx.x; k < nit; k += kBT) {
    const double v2 = __ldcg(d.part_val + k);
    const int64_t i2 = __ldcg(d.part_idx + k);
    if (better(v2, i2, bv, bi)) { bv = v2; bi = i2; }
  }
  cta_argmax(bv, bi, red->v, red->i);
  if (threadIdx.x != 0) return;
  const int64_t K = st->K;
  d.piv[K] = st->prow;
  d.pivd[K] = st->dp;
  st->slot_row[st->pslot] = -1;
  st->K = K + 1;
  st->cur ^= 1;
  st->dmax = bv;
  st->idx = bi;
  const int bad = st->bad;
  st->bad = 0;
  if (bad) { end_system(st, ctl, CD_ENOTPSD); return; }
  if (!(bv >= d.tau)) {
    if (d.tc) { st->after_slice = kJobConverged; publish(st, kJobSlice, nit); }
    else advance(d, kJobConverged, ctl);
    return;
  }
  if (K + 1 >= d.Mcap) { end_system(st, ctl, CD_ENOMEM); return; }
  int slot = -1;
  for (int s = 0; s < d.b; ++s)
    if (st->slot_row[s] == bi) slot = s;
  if (slot < 0) {
    if (d.tc) { st->after_slice = kJobSelect; publish(st, kJobSlice, nit); }
    else publish(st, kJobSelect, 1);
    return;
  }
  const double dp = __ldcg(dcur(d, st->cur) + bi);
  if (!(dp > 0.0)) { end_system(st, ctl, CD_ENOTPSD); return; }
  st->prow = bi;
  st->pslot = slot;
  st->dp = dp;
  publish(st, kJobStep, nit);
}

// FMAs of one item as the algorithm counts them (no tile padding), read before
// the item runs (the job's parameters do not change while it is outstanding)
__device__ unsigned long long item_work(const SysDesc& d, int type, int kind, unsigned it) {
  const SysState* st = d.st;
  const int64_t K = vload(&st->K);
  if (type == kJobUpdate) {
    const int n0 = vload(&st->nitems[0]);
    const int g = (int)it < n0 ? 0 : 1;
    const int64_t li = g == 0 ? it : it - n0;
    const int nb = vload(&st->nb[g]);
    int64_t tile = li, cols = nb;
    if (d.tc) {
      const int ctn = (nb + kTcBN - 1) / kTcBN;
      tile = li / ctn;
      cols = min((int64_t)kTcBN, (int64_t)nb - (li % ctn) * kTcBN);
    }
    const int64_t rows = min((int64_t)kRowTile, d.n - tile * kRowTile);
    return (unsigned long long)(rows * cols * (K - vload(&st->k0[g])));
  }
  if (type == kJobStep) {
    const int64_t rows = min((int64_t)kStepRows, d.n - (int64_t)it * kStepRows);
    return (unsigned long long)(rows * (K - vload(&st->Kb) + 1));
  }
  if (kind == kJobJk1 + 8) {   // B^P = L^P C: every screened pair twice (mu nu and nu mu), O each
    if (d.tc) {
      const unsigned j = it - (unsigned)vload(&st->nitems[0]);
      const int nmu = (d.N + 7) / 8;
      const int64_t c = j / nmu;
      const int mb = (int)(j % nmu);
      const int64_t nv = min((int64_t)32, K - c * 32);
      const int64_t deg = __ldg(d.csr_off + min(d.N, mb * 8 + 8)) - __ldg(d.csr_off + mb * 8);
      return (unsigned long long)(nv * deg * d.O);
    }
    return (unsigned long long)d.nnz * (unsigned long long)d.O;
  }
  if (kind == kJobJk2 + 8) {   // partial K tile: tile elements x vectors x O
    const int ntl = ntiles_k(d.N);
    const int s = (int)(it - (unsigned)vload(&st->nitems[0])) / ntl;
    int bi, bj;
    tile_of((it - (unsigned)vload(&st->nitems[0])) % ntl, bi, bj);
    const int64_t nm = min(kKt, d.N - bi * kKt), nn = min(kKt, d.N - bj * kKt);
    const int64_t np = min((int64_t)kKtSplit, K - (int64_t)s * kKtSplit);
    return (unsigned long long)(nm * nn * np * d.O);
  }
  if (kind == kJobJk2) {       // v = L d
    const int64_t per = d.tc ? 32 : kJvVec;
    const int64_t nv = min(per, K - (int64_t)it * per);
    return (unsigned long long)(nv * d.n);
  }
  if (kind == kJobJk3) {       // J_p = L^T v
    const int64_t rows = min((int64_t)kStepRows, d.n - (int64_t)it * kStepRows);
    return (unsigned long long)(rows * K);
  }
  return 0;
}

// ---------------------------------------------------------------- kernel ----
// TC = true: the build with the tensor-core update items.  A kernel that contains
// tcgen05 instructions is resident at one CTA per SM, so the FP64-only build
// (TC = false, two CTAs per SM) serves batches whose systems all use the DFMA update.
template <bool TC>
__global__ void __launch_bounds__(kBT, 2) batch_kernel(const SysDesc* __restrict__ sys, int n_sys, BatchCtl* ctl,
                                                       const double* __restrict__ boys, long long wait_ns) {
  constexpr int use_tc = TC ? 1 : 0;
  // item scratch (dynamic, 1024-byte aligned for the swizzled tensor-core operands)
  extern __shared__ __align__(1024) unsigned char dsmem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)dsmem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ SysDesc sd;
  __shared__ __align__(8) uint64_t s_mbar;   // MMA completion of the tensor-core update items
  __shared__ uint32_t s_tmem;
  __shared__ int s_tcfail;
  __shared__ Red red;
  __shared__ __align__(16) KetGroup sg;   // filled with 16-byte copies
  __shared__ int64_t s_cand[kBMaxB + kBT];
  __shared__ int s_int[8];
  __shared__ int s_sys, s_last, s_type;
  __shared__ unsigned s_item, s_count;
  long long idle_since = -1, last_idle = 0;
  unsigned long long seen = 0;
  uint32_t mphase = 0;   // thread 0: parity of the next MMA-completion phase
  // tensor memory for the update accumulators: 256 columns per CTA (two CTAs per SM),
  // held for the whole launch
  if (threadIdx.x == 0) {
    tc::mbar_init(&s_mbar, 1);
    tc::fence_mbar_init();
    s_tcfail = 0;
  }
  if constexpr (TC) {
    if (threadIdx.x < 32) tc::tmem_alloc<kTcTmemCols>(&s_tmem);
    tc::tc_fence_before();
  }
  __syncthreads();
  if constexpr (TC) tc::tc_fence_after();
  const uint32_t tmem = use_tc ? s_tmem : 0u;
  for (;;) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int found = -1;
      unsigned item = 0, count = 0;
      int stop = 0;
      if (lane == 0) stop = vload(&ctl->abort) || vload(&ctl->done_sys) >= (unsigned)n_sys;
      stop = __shfl_sync(0xffffffffu, stop, 0);
      if (!stop) {
        for (int base = 0; base < n_sys && found < 0; base += 32) {
          const int s = base + lane;
          unsigned long long w = 0;
          if (s < n_sys) w = vload(&sys[s].st->word);
          const bool avail = s < n_sys && job_next(w) < job_count(w);
          unsigned mask = __ballot_sync(0xffffffffu, avail);
          while (mask && found < 0) {
            const int l = __ffs(mask) - 1;
            mask &= mask - 1;
            unsigned long long old = 0;
            if (lane == l) old = atomicAdd(&sys[base + l].st->word, 1ull);
            old = __shfl_sync(0xffffffffu, old, l);
            if (job_next(old) < job_count(old)) {
              found = base + l;
              item = job_next(old);
              count = job_count(old);
            }
          }
        }
      }
      if (lane == 0) {
        s_sys = stop ? -2 : found;
        s_item = item;
        s_count = count;
      }
    }
    __syncthreads();
    const int s = s_sys;
    if (s == -2) break;
    if (s < 0) {
      // no work: a bounded wait (no item completed anywhere for wait_ns -> give up)
      if (threadIdx.x == 0) {
        const unsigned long long p = vload(&ctl->progress);
        const long long now = globaltimer_ns();
        if (idle_since >= 0) atomicAdd(&ctl->idle_ns, (unsigned long long)(now - last_idle));
        last_idle = now;
        if (idle_since < 0 || p != seen) {
          idle_since = now;
          seen = p;
        } else if (now - idle_since > wait_ns) {
          atomicExch(&ctl->timed_out, 1);
          atomicExch(&ctl->abort, 1);
        }
        __nanosleep(500);
      }
      __syncthreads();
      continue;
    }
    if (threadIdx.x == 0) idle_since = -1;
    for (int k = threadIdx.x; k < (int)(sizeof(SysDesc) / 16); k += kBT)
      ((int4*)&sd)[k] = __ldg((const int4*)(sys + s) + k);
    __threadfence();
    if (threadIdx.x == 0) s_type = vload(&sys[s].st->type);
    __syncthreads();
    const unsigned it = s_item;
    const int type = s_type;
    const SysState* st = sd.st;
    const long long t_item = threadIdx.x == 0 ? globaltimer_ns() : 0;
    int kind = type;   // item kind for the timing: the second part of a combined job counts as type + 8
    unsigned long long item_fma = 0;   // FMAs of the item (thread 0; algorithmic, no padding)
    if (threadIdx.x == 0) {
      if ((type == kJobCols || type == kJobJk1 || type == kJobJk2 || type == kJobJk3) && (int)it >= vload(&st->nitems[0]))
        kind = type + 8;
      item_fma = item_work(sd, type, kind, it);
    }
    switch (type) {
      case kJobSelect: select_item(sd, smem, &red, s_cand, s_int); break;
      case kJobCols:
        if ((int)it < vload(&st->nitems[0])) {
          if (sd.tc) gather_tc_item(sd, it);
          else gather_item(sd, it);
        }
        else eri_item(sd, it, boys, &sg, &ctl->kind_ops[kJobCols + 8]);
        break;
      case kJobUpdate:
        if constexpr (TC) {
          if (sd.tc) update_tc_item(sd, it, smem, tmem, &s_mbar, mphase, &s_tcfail, ctl, wait_ns);
          else update_item(sd, it, smem);
        } else {
          update_item(sd, it, smem);
        }
        break;
      case kJobStep: step_item(sd, it, smem, &red); break;
      case kJobJk1:
        if ((int)it < vload(&st->nitems[0])) dens_item(sd, it);
        else if (sd.tc) kb_tc_item(sd, it - (unsigned)vload(&st->nitems[0]), vload(&st->K));
        else kb_item(sd, it - (unsigned)vload(&st->nitems[0]));
        break;
      case kJobJk2: {
        const int n0 = vload(&st->nitems[0]);
        if ((int)it < n0) {
          if (sd.tc) jv_tc_item(sd, it, vload(&st->K), smem);
          else jv_item(sd, it, vload(&st->K), &red);
        }
        else kt_item(sd, it - (unsigned)n0, vload(&st->K), ntiles_k(sd.N), smem);
        break;
      }
      case kJobJk3: {
        const int n0 = vload(&st->nitems[0]);
        if ((int)it < n0) {
          if (sd.tc) jp_tc_item(sd, it, vload(&st->K), smem);
          else jp_item(sd, it, vload(&st->K), smem);
        }
        else ksum_item(sd, it - (unsigned)n0, (int)ceil_div(vload(&st->K), kKtSplit));
        break;
      }
      case kJobJk4: junpack_item(sd, it); break;
      case kJobSlice: slice_item(sd, it); break;
      default: break;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned t = atomicAdd(&sd.st->done, 1u);
      s_last = (t + 1 == s_count) ? 1 : 0;
      atomicAdd(&ctl->progress, 1ull);
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      if (type == kJobStep) {
        finish_step(sd, ctl, &red);
      } else if (threadIdx.x == 0) {
        advance(sd, type, ctl);
      }
    }
    if (threadIdx.x == 0 && kind >= 0 && kind < kJobKinds) {
      atomicAdd(&ctl->kind_ns[kind], (unsigned long long)(globaltimer_ns() - t_item));
      atomicAdd(&ctl->kind_items[kind], 1ull);
      if (item_fma) atomicAdd(&ctl->kind_ops[kind], item_fma);
    }
    __syncthreads();
  }
  if constexpr (TC) tc::tc_fence_before();
  __syncthreads();
  if constexpr (TC) {
    if (threadIdx.x < 32) {
      tc::tc_fence_after();
      tc::tmem_dealloc<kTcTmemCols>(tmem);
    }
  }
}

}  // namespace

// ------------------------------------------------------------------ host ----
namespace {
size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

}  // namespace cd

extern "C" int cd_batch_persistent(int32_t n_sys, const cd_basis_t* bases, const cd_opts_t* opts,
                                   const double* const* C_occ, const int32_t* n_occ, double* const* J,
                                   double* const* K, int64_t* M_out, double* stats, void* stream) {
  using namespace cd;
  if (n_sys < 0 || (n_sys > 0 && (!bases || !opts || !C_occ || !n_occ || !J || !K))) {
    set_error("cd_batch_persistent: bad argument");
    return CD_EINVAL;
  }
  if (n_sys == 0) return CD_OK;
  for (int i = 0; i < n_sys; ++i) {
    const cd_opts_t& o = opts[i];
    std::string why;
    if (!(o.tau > 0.0) || !std::isfinite(o.tau)) why = "tau must be finite and > 0";
    else if (o.block < 0 || o.block > kBMaxB) why = "block must be in [0, 64] (0 = 64)";
    else if (o.vec_precision != CD_FP64) why = "vectors are FP64";
    else if (o.algorithm != CD_ALG_FULL || o.forced_pivots || o.candidates || o.diag_shift != 0.0)
      why = "only the fully pivoted decomposition (CD_ALG_FULL, no forced pivots, mask or shift)";
    else if (o.max_vectors < 0) why = "max_vectors < 0";
    else if (o.update != CD_UPDATE_SLICE && o.update != CD_UPDATE_FP64) why = "bad update mode";
    else if (n_occ[i] <= 0 || !C_occ[i] || !J[i] || !K[i]) why = "n_occ, C_occ, J, K";
    if (!why.empty()) {
      set_error("cd_batch_persistent: system " + std::to_string(i) + ": " + why);
      return CD_EINVAL;
    }
  }
  const double t0 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
  auto now_ms = []() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
  };
  int dev = 0;
  CD_CUDA(cudaGetDevice(&dev));
  cudaStream_t ust = (cudaStream_t)stream;
  // ---- set-up of every system (screening, diagonal, pair records) on host workers
  std::vector<cd_system_t*> systems(n_sys, nullptr);
  std::vector<int> rcs(n_sys, CD_OK);
  std::vector<std::string> msgs(n_sys);
  {
    const int nw = std::max(1, std::min<int>(n_sys, (int)std::thread::hardware_concurrency()));
    std::atomic<int> next{0};
    auto work = [&]() {
      cudaSetDevice(dev);
      cudaStream_t st = nullptr;
      if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { cudaGetLastError(); st = nullptr; }
      for (;;) {
        const int i = next.fetch_add(1);
        if (i >= n_sys) break;
        const int rc = cd_system_create(&bases[i], opts[i].schwarz, st, &systems[i]);
        rcs[i] = rc;
        if (rc != CD_OK) msgs[i] = cd_last_error();
      }
      if (st) { cudaStreamSynchronize(st); cudaStreamDestroy(st); }
    };
    std::vector<std::thread> th;
    for (int w = 1; w < std::min(nw, 16); ++w) th.emplace_back(work);
    work();
    for (auto& t : th) t.join();
  }
  auto release_systems = [&]() {
    for (auto* s : systems)
      if (s) cd_system_free(s);
  };
  for (int i = 0; i < n_sys; ++i)
    if (rcs[i] != CD_OK) {
      release_systems();
      set_error("cd_batch_persistent: system " + std::to_string(i) + ": " + msgs[i]);
      return rcs[i];
    }
  const double t_setup = now_ms();
  // ---- sizes of every system's buffers (offsets relative to the system's base)
  struct Plan {
    int64_t n, ld, Mcap;
    int N, O, Op, b, nsplit;
    size_t off[28];
    int64_t bpitch;
    size_t bytes;
    std::vector<int32_t> csr_off, csr_nu, csr_row, allsp;
    std::vector<int8_t> kc, kd;
    double dmax;
    int64_t idx;
  };
  std::vector<Plan> plan(n_sys);
  size_t max_items = 0;
  for (int i = 0; i < n_sys; ++i) {
    cd_system* s = systems[i];
    Plan& p = plan[i];
    p.n = s->n_rows;
    p.ld = s->n_rows_pad;
    p.N = s->hb.nbf;
    p.O = n_occ[i];
    p.Op = (p.O + 7) / 8 * 8;
    p.b = opts[i].block ? opts[i].block : kBMaxB;
    int64_t mcap = opts[i].max_vectors > 0 ? opts[i].max_vectors : (int64_t)8 * p.N;
    p.Mcap = std::max<int64_t>(1, std::min<int64_t>(mcap, std::max<int64_t>(p.n, 1)));
    p.nsplit = (int)((p.Mcap + kKtSplit - 1) / kKtSplit);
    const int64_t nst = std::max<int64_t>(1, (p.n + kStepRows - 1) / kStepRows);
    const size_t N2 = (size_t)p.N * p.N;
    size_t sz[] = {
        sizeof(double) * (size_t)p.ld,               // 0 D0
        sizeof(double) * (size_t)p.ld,               // 1 D1
        sizeof(double) * (size_t)p.b * p.ld,         // 2 pool
        opts[i].update == CD_UPDATE_SLICE ? (size_t)16 : sizeof(double) * (size_t)p.Mcap * p.ld,   // 3 L (DFMA)
        sizeof(int64_t) * (size_t)p.Mcap,            // 4 piv
        sizeof(double) * (size_t)p.Mcap,             // 5 pivd
        sizeof(double) * (size_t)p.Mcap * p.b,       // 6 Bg0
        sizeof(double) * (size_t)p.b * p.b,          // 7 Bg1
        sizeof(KetGroup) * (size_t)p.b,              // 8 groups
        sizeof(double) * (size_t)nst,                // 9 part_val
        sizeof(int64_t) * (size_t)nst,               // 10 part_idx
        sizeof(double) * (size_t)p.ld,               // 11 dpk
        sizeof(double) * (size_t)p.Mcap,             // 12 v
        sizeof(double) * (size_t)p.ld,               // 13 Jp
        sizeof(double) * (size_t)p.Mcap * p.N * p.Op,// 14 B
        sizeof(double) * (size_t)p.nsplit * N2,      // 15 Kpart
        sizeof(double) * N2,                         // 16 J
        sizeof(double) * N2,                         // 17 K
        sizeof(SysState),                            // 18 state
        sizeof(double) * ((size_t)p.N * p.Op + 80),   // 19 C (rows padded to Op, + room for the last 72-column read)
        sizeof(int32_t) * (size_t)(p.N + 1),         // 20 csr_off
        sizeof(int32_t) * (size_t)std::max<int64_t>(1, 2 * p.n),   // 21 csr_nu
        sizeof(int32_t) * (size_t)std::max<int64_t>(1, 2 * p.n),   // 22 csr_row
        sizeof(int32_t) * (size_t)std::max<int64_t>(1, p.n) + 2 * align256((size_t)std::max<int64_t>(1, p.n)),  // 23 allsp, kc, kd
        sizeof(int32_t) * (size_t)std::max<int64_t>(1, p.n),                     // 24 erow
        opts[i].update == CD_UPDATE_SLICE ? (size_t)2 * kTcSlices * 64 * (size_t)((p.Mcap + 2 * kTcBK) / kTcBK * kTcBK) * 2
                                          : (size_t)16,                          // 25 pivot-row slices
        opts[i].update == CD_UPDATE_SLICE
            ? (size_t)((p.Mcap + kTcBK - 1) / kTcBK) * kTcSlices * (size_t)std::max<int64_t>(1, p.n) * kTcBK * 2
            : (size_t)16,                                                        // 26 slice store
        opts[i].update == CD_UPDATE_SLICE ? sizeof(double) * (size_t)kBMaxB * p.ld : (size_t)16,   // 27 block buffer
    };
    p.bpitch = (p.Mcap + 2 * kTcBK) / kTcBK * kTcBK;
    size_t o = 0;
    for (int k = 0; k < 28; ++k) {
      p.off[k] = o;
      o += align256(sz[k]);
    }
    p.bytes = o;
    // row list per basis function: (mu nu) under mu and, if mu != nu, under nu
    p.csr_off.assign(p.N + 1, 0);
    std::vector<int32_t> mu(p.n), nu(p.n);
    for (int64_t r = 0; r < p.n; ++r) {
      const int64_t pk = s->row_packed[r];
      int64_t m = (int64_t)((std::sqrt(8.0 * (double)pk + 1.0) - 1.0) / 2.0);
      while (m * (m + 1) / 2 > pk) --m;
      while ((m + 1) * (m + 2) / 2 <= pk) ++m;
      mu[r] = (int32_t)m;
      nu[r] = (int32_t)(pk - m * (m + 1) / 2);
      p.csr_off[mu[r] + 1]++;
      if (mu[r] != nu[r]) p.csr_off[nu[r] + 1]++;
    }
    for (int k = 0; k < p.N; ++k) p.csr_off[k + 1] += p.csr_off[k];
    p.csr_nu.assign(std::max<int32_t>(1, p.csr_off[p.N]), 0);
    p.csr_row.assign(std::max<int32_t>(1, p.csr_off[p.N]), 0);
    std::vector<int32_t> fill(p.csr_off.begin(), p.csr_off.end() - 1);
    for (int64_t r = 0; r < p.n; ++r) {
      int32_t e = fill[mu[r]]++;
      p.csr_nu[e] = nu[r];
      p.csr_row[e] = (int32_t)r;
      if (mu[r] != nu[r]) {
        e = fill[nu[r]]++;
        p.csr_nu[e] = mu[r];
        p.csr_row[e] = (int32_t)r;
      }
    }
    p.dmax = -1.0;
    p.idx = -1;
    for (int64_t r = 0; r < p.n; ++r)
      if (s->row_diag[r] > p.dmax) { p.dmax = s->row_diag[r]; p.idx = r; }
    // largest job of the system (queue words hold 24-bit counts)
    int64_t neri = 0;
    for (int c = 0; c < 3; ++c) neri += (s->bra_class_off[c + 1] - s->bra_class_off[c] + 127) / 128 * p.b;
    const int64_t nb_k = (p.N + kKt - 1) / kKt;
    const int64_t jobs[] = {neri + 2 * ((p.Mcap + kGatherQ - 1) / kGatherQ), 2 * ((p.n + kRowTile - 1) / kRowTile),
                            nst + p.Mcap, (p.Mcap + kJvVec - 1) / kJvVec + p.nsplit * nb_k * (nb_k + 1) / 2};
    for (int64_t j : jobs) max_items = std::max<size_t>(max_items, (size_t)j);
  }
  if (max_items >= kMaxJobItems) {
    release_systems();
    set_error("cd_batch_persistent: a system needs more than 2^23 work items in one job");
    return CD_EINVAL;
  }
  for (int i = 1; i < n_sys; ++i)
    if (systems[i]->boys != systems[0]->boys) {
      release_systems();
      set_error("cd_batch_persistent: systems on different Boys tables");
      return CD_EINVAL;
    }
  // ---- waves: systems largest first (CTAs scan them in this order), each put
  // into the first wave whose buffers still fit the budget; one launch per wave
  size_t freeb = 0, totb = 0;
  CD_CUDA(cudaMemGetInfo(&freeb, &totb));
  const double budget = opts[0].mem_budget_gb > 0 ? opts[0].mem_budget_gb * 1e9 : 0.9 * (double)freeb;
  std::vector<int> order(n_sys);
  for (int i = 0; i < n_sys; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)plan[a].n * plan[a].N > (double)plan[b].n * plan[b].N;
  });
  std::vector<std::vector<int>> waves;
  std::vector<size_t> wave_bytes;
  for (int i : order) {
    if ((double)plan[i].bytes > budget) {
      release_systems();
      set_error("cd_batch_persistent: system " + std::to_string(i) + ": its device memory (" +
                std::to_string(plan[i].bytes / 1e9) + " GB) exceeds the budget (" + std::to_string(budget / 1e9) +
                " GB)");
      return CD_ENOMEM;
    }
    size_t w = 0;
    while (w < waves.size() && (double)(wave_bytes[w] + plan[i].bytes) > budget) ++w;
    if (w == waves.size()) {
      waves.emplace_back();
      wave_bytes.push_back(0);
    }
    waves[w].push_back(i);
    wave_bytes[w] += plan[i].bytes;
  }
  size_t max_wave = 0, max_sys = 0;
  for (size_t w = 0; w < waves.size(); ++w) {
    max_wave = std::max(max_wave, wave_bytes[w]);
    max_sys = std::max(max_sys, waves[w].size());
  }
  unsigned char* arena = nullptr;
  SysDesc* desc_dev = nullptr;
  BatchCtl* ctl_dev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  auto free_wave = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  };
  auto cleanup = [&]() {
    free_wave();
    if (cs) cudaStreamDestroy(cs);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(desc_dev);
    cudaFree(ctl_dev);
    cudaFree(arena);
    release_systems();
  };
  auto fail = [&](int code) {
    cleanup();
    return code;
  };
#define BP_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t _e = (call);                                                            \
    if (_e != cudaSuccess) {                                                            \
      cudaGetLastError();                                                               \
      set_error(std::string("cd_batch_persistent: ") + cudaGetErrorString(_e) + " at " + \
                std::to_string(__LINE__));                                              \
      return fail(CD_ECUDA);                                                            \
    }                                                                                   \
  } while (0)
  // one arena the size of the largest wave, reused by every wave
  if (cudaMalloc(&arena, max_wave) != cudaSuccess) {
    cudaGetLastError();
    arena = nullptr;
    set_error("cd_batch_persistent: cudaMalloc of " + std::to_string(max_wave) + " bytes failed");
    return fail(CD_ENOMEM);
  }
  BP_CUDA(cudaMalloc(&desc_dev, sizeof(SysDesc) * max_sys));
  BP_CUDA(cudaMalloc(&ctl_dev, sizeof(BatchCtl)));
  BP_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  BP_CUDA(cudaEventCreate(&e0));
  BP_CUDA(cudaEventCreate(&e1));
  BP_CUDA(cudaStreamSynchronize(ust));
  // the kernel build and its grid: the tensor-core build if any system wants it
  int use_tc = 0;
  for (int i = 0; i < n_sys; ++i) use_tc |= opts[i].update == CD_UPDATE_SLICE ? 1 : 0;
  auto kfn = use_tc ? batch_kernel<true> : batch_kernel<false>;
  int per_sm = 0, sms = 0;
  BP_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem));
  BP_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  BP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBT, kDynSmem));
  BP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (use_tc && per_sm >= 1) {
    // the occupancy calculator reports one CTA per SM for any kernel with tcgen05
    // instructions; registers (2 x 128 x 256) and shared memory (2 x 77 KB) allow
    // two, each holding half of the SM's tensor memory.  A CTA that is not
    // resident at once only starts after another exits and then finds no work.
    cudaFuncAttributes fa;
    BP_CUDA(cudaFuncGetAttributes(&fa, kfn));
    int smem_sm = 0;
    BP_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    const int by_regs = 65536 / (kBT * ((fa.numRegs + 7) / 8 * 8));
    const int by_smem = smem_sm / (int)(kDynSmem + fa.sharedSizeBytes + 1024);
    per_sm = std::max(per_sm, std::min(by_regs, by_smem));
  }
  // at most two CTAs per SM (each would hold half of the SM's tensor memory)
  const int grid = std::max(1, std::min(per_sm, 2)) * sms;
  if (getenv("CDERI_DEBUG"))
    fprintf(stderr, "[cderi] batch_kernel<%s>: %d CTAs per SM, grid %d, %zu wave(s)\n",
            use_tc ? "tensor-core update" : "FP64", per_sm, grid, waves.size());
  const long long wait_ns = (long long)device_wait_limit_ns();
  double upload_ms = 0.0, launch_host_ms = 0.0, device_ms = 0.0;
  BatchCtl sum;
  memset(&sum, 0, sizeof(sum));
  for (size_t w = 0; w < waves.size(); ++w) {
    const std::vector<int>& members = waves[w];
    const int nw = (int)members.size();
    const double tw0 = now_ms();
    std::vector<SysDesc> hd(nw);
    size_t base = 0;
    for (int k = 0; k < nw; ++k) {
      const int i = members[k];
      cd_system* s = systems[i];
      Plan& p = plan[i];
      unsigned char* sys_base = arena + base;
      base += p.bytes;
      auto at = [&](int slot) { return (void*)(sys_base + p.off[slot]); };
      SysDesc& d = hd[k];
      memset(&d, 0, sizeof(d));
      d.n = p.n;
      d.ld = p.ld;
      d.Mcap = p.Mcap;
      d.N = p.N;
      d.O = p.O;
      d.Op = p.Op;
      d.b = p.b;
      d.tau = opts[i].tau;
      double d1max = 0.0;
      for (double v : s->row_diag) d1max = std::max(d1max, v);
      d.neg_tol = -1e-10 * d1max;
      d.bra = s->bra;
      d.ket = s->all;
      for (int c = 0; c < 4; ++c) {
        d.cls[c] = s->bra_class_off[c];
        d.all_cls[c] = s->all_class_off[c];
      }
      for (int c = 0; c < 3; ++c) d.ntile[c] = (int)((d.cls[c + 1] - d.cls[c] + 127) / 128);
      d.nsplit_cap = p.nsplit;
      d.nnz = p.csr_off[p.N];
      d.D0 = (double*)at(0);
      d.D1 = (double*)at(1);
      d.pool = (double*)at(2);
      d.L = (double*)at(3);
      d.piv = (int64_t*)at(4);
      d.pivd = (double*)at(5);
      d.Bg0 = (double*)at(6);
      d.Bg1 = (double*)at(7);
      d.groups = (KetGroup*)at(8);
      d.part_val = (double*)at(9);
      d.part_idx = (int64_t*)at(10);
      d.dpk = (double*)at(11);
      d.v = (double*)at(12);
      d.Jp = (double*)at(13);
      d.B = (double*)at(14);
      d.Kpart = (double*)at(15);
      d.J = (double*)at(16);
      d.Kx = (double*)at(17);
      d.st = (SysState*)at(18);
      d.C = (const double*)at(19);
      d.csr_off = (const int32_t*)at(20);
      d.csr_nu = (const int32_t*)at(21);
      d.csr_row = (const int32_t*)at(22);
      unsigned char* rt = (unsigned char*)at(23);
      d.row_allsp = (const int32_t*)rt;
      d.row_kc = (const int8_t*)(rt + align256(sizeof(int32_t) * (size_t)std::max<int64_t>(1, p.n)));
      d.row_kd = d.row_kc + align256((size_t)std::max<int64_t>(1, p.n));
      d.row_mu = s->row_mu_dev;
      d.row_nu = s->row_nu_dev;
      d.tc = opts[i].update == CD_UPDATE_SLICE ? 1 : 0;
      d.erow = (const int32_t*)at(24);
      d.Bsl = (__nv_bfloat16*)at(25);
      d.bpitch = p.bpitch;
      d.Ls = (__nv_bfloat16*)at(26);
      d.Lblk = (double*)at(27);
      if (d.tc) d.L = nullptr;
      {
        // row exponents: sqrt(D^1_r) < 2^e_r (frexp), so every |L^K_r| / 2^e_r <= 1
        std::vector<int32_t> er(std::max<int64_t>(1, p.n), 0);
        for (int64_t r = 0; r < p.n; ++r) {
          int ex = 0;
          if (s->row_diag[r] > 0.0) std::frexp(std::sqrt(s->row_diag[r]), &ex);
          er[r] = ex;
        }
        BP_CUDA(cudaMemcpyAsync((void*)d.erow, er.data(), sizeof(int32_t) * er.size(), cudaMemcpyHostToDevice, cs));
        BP_CUDA(cudaStreamSynchronize(cs));   // er is a temporary
      }
      // uploads
      SysState h;
      memset(&h, 0, sizeof(h));
      h.word = job_word(1, 1, 0);
      h.type = kJobSelect;
      h.dmax = p.dmax;
      h.idx = p.idx;
      for (int x = 0; x < kBMaxB; ++x) h.slot_row[x] = -1;
      BP_CUDA(cudaMemcpyAsync(d.st, &h, sizeof(h), cudaMemcpyHostToDevice, cs));
      BP_CUDA(cudaMemcpyAsync(d.D0, s->diag_dev, sizeof(double) * p.ld, cudaMemcpyDeviceToDevice, cs));
      {
        std::vector<double> cp((size_t)p.N * p.Op + 80, 0.0);
        for (int mu = 0; mu < p.N; ++mu)
          for (int k2 = 0; k2 < p.O; ++k2) cp[(size_t)mu * p.Op + k2] = C_occ[i][(size_t)mu * p.O + k2];
        BP_CUDA(cudaMemcpyAsync((void*)d.C, cp.data(), sizeof(double) * cp.size(), cudaMemcpyHostToDevice, cs));
        BP_CUDA(cudaStreamSynchronize(cs));   // cp and h are temporaries
      }
      BP_CUDA(cudaMemcpyAsync((void*)d.csr_off, p.csr_off.data(), sizeof(int32_t) * p.csr_off.size(), cudaMemcpyHostToDevice, cs));
      BP_CUDA(cudaMemcpyAsync((void*)d.csr_nu, p.csr_nu.data(), sizeof(int32_t) * p.csr_nu.size(), cudaMemcpyHostToDevice, cs));
      BP_CUDA(cudaMemcpyAsync((void*)d.csr_row, p.csr_row.data(), sizeof(int32_t) * p.csr_row.size(), cudaMemcpyHostToDevice, cs));
      if (p.n > 0) {
        BP_CUDA(cudaMemcpyAsync((void*)d.row_allsp, s->row_allsp.data(), sizeof(int32_t) * p.n, cudaMemcpyHostToDevice, cs));
        BP_CUDA(cudaMemcpyAsync((void*)d.row_kc, s->row_kc.data(), (size_t)p.n, cudaMemcpyHostToDevice, cs));
        BP_CUDA(cudaMemcpyAsync((void*)d.row_kd, s->row_kd.data(), (size_t)p.n, cudaMemcpyHostToDevice, cs));
      }
    }
    BP_CUDA(cudaMemcpyAsync(desc_dev, hd.data(), sizeof(SysDesc) * nw, cudaMemcpyHostToDevice, cs));
    BP_CUDA(cudaStreamSynchronize(cs));
    const double tw1 = now_ms();
    upload_ms += tw1 - tw0;
    // ---- the launch, recorded in a CUDA graph: clear J, the slice store and the
    // control block, one persistent kernel
    BP_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (int k = 0; k < nw; ++k) {
      cudaMemsetAsync(hd[k].J, 0, sizeof(double) * (size_t)hd[k].N * hd[k].N, cs);
      // the slice store starts at zero: the last 32-vector block of a system is read whole by the update
      if (hd[k].tc)
        cudaMemsetAsync(hd[k].Ls, 0,
                        (size_t)((hd[k].Mcap + kTcBK - 1) / kTcBK) * kTcSlices * (size_t)std::max<int64_t>(1, hd[k].n) *
                            kTcBK * 2, cs);
    }
    cudaMemsetAsync(ctl_dev, 0, sizeof(BatchCtl), cs);
    kfn<<<grid, kBT, kDynSmem, cs>>>(desc_dev, nw, ctl_dev, systems[0]->boys, wait_ns);
    BP_CUDA(cudaStreamEndCapture(cs, &graph));
    BP_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    BP_CUDA(cudaEventRecord(e0, cs));
    BP_CUDA(cudaGraphLaunch(exec, cs));
    count_launch();
    BP_CUDA(cudaEventRecord(e1, cs));
    BP_CUDA(cudaStreamSynchronize(cs));
    float kms = 0.0f;
    cudaEventElapsedTime(&kms, e0, e1);
    device_ms += kms;
    BatchCtl hctl;
    std::vector<SysState> hst(nw);
    BP_CUDA(cudaMemcpy(&hctl, ctl_dev, sizeof(BatchCtl), cudaMemcpyDeviceToHost));
    for (int k = 0; k < nw; ++k) BP_CUDA(cudaMemcpy(&hst[k], hd[k].st, sizeof(SysState), cudaMemcpyDeviceToHost));
    if (hctl.tc_err) {
      set_error("cd_batch_persistent: a bounded tensor-core wait gave up (MMA completion)");
      return fail(CD_ETIMEOUT);
    }
    if (hctl.timed_out) {
      set_error("cd_batch_persistent: a CTA's wait for work gave up after the wait limit with no item completed");
      return fail(CD_ETIMEOUT);
    }
    for (int k = 0; k < nw; ++k) {
      const int i = members[k];
      if (hst[k].status != CD_OK || hst[k].type != kJobNone) {
        const int code = hst[k].status != CD_OK ? hst[k].status : CD_ETIMEOUT;
        std::string why = code == CD_ENOTPSD ? "matrix not PSD (pivot diagonal <= 0 or residual below -1e-10 max D)"
                          : code == CD_ENOMEM ? "number of vectors exceeds max_vectors = " + std::to_string(plan[i].Mcap)
                                              : "decomposition did not finish";
        set_error("cd_batch_persistent: system " + std::to_string(i) + ": " + why);
        return fail(code);
      }
    }
    for (int k = 0; k < nw; ++k) {
      const int i = members[k];
      const size_t N2 = (size_t)hd[k].N * hd[k].N;
      BP_CUDA(cudaMemcpy(J[i], hd[k].J, sizeof(double) * N2, cudaMemcpyDeviceToHost));
      BP_CUDA(cudaMemcpy(K[i], hd[k].Kx, sizeof(double) * N2, cudaMemcpyDeviceToHost));
      if (M_out) M_out[i] = hst[k].K;
    }
    for (int k = 0; k < kJobKinds; ++k) {
      sum.kind_ns[k] += hctl.kind_ns[k];
      sum.kind_ops[k] += hctl.kind_ops[k];
    }
    sum.idle_ns += hctl.idle_ns;
    for (int k = 0; k < 4; ++k) sum.tc_ns[k] += hctl.tc_ns[k];
    free_wave();
    launch_host_ms += now_ms() - tw1;
  }
  if (stats) {
    stats[0] = t_setup - t0;       // system set-up (host workers)
    stats[1] = upload_ms;          // descriptors and uploads, all waves
    stats[2] = device_ms;          // the graph launches (one persistent kernel each), device time
    stats[3] = launch_host_ms;     // launches, waits and read-back, host time
    stats[4] = (double)grid;
    stats[5] = (double)max_wave;   // bytes reserved (the largest wave's)
    // CTA-seconds per item kind: 1 select, 2 gather, 3 update, 4 step, 5 density, 6 v = L d,
    // 7 J_p = L^T v, 8 J unpack, 10 ERI columns, 13 B = L C, 14 partial K tiles, 15 K sum; 16 idle
    for (int k = 0; k < kJobKinds; ++k) stats[6 + k] = 0.0;
    const int kinds[][2] = {{1, kJobSelect}, {2, kJobCols}, {3, kJobUpdate}, {4, kJobStep}, {5, kJobJk1},
                            {6, kJobJk2}, {7, kJobJk3}, {8, kJobJk4}, {9, kJobSlice}, {10, kJobCols + 8},
                            {13, kJobJk1 + 8}, {14, kJobJk2 + 8}, {15, kJobJk3 + 8}};
    for (auto& kk : kinds) stats[6 + kk[0]] = (double)sum.kind_ns[kk[1]] * 1e-9;
    stats[6 + 16] = (double)sum.idle_ns * 1e-9;
    if (getenv("CDERI_DEBUG"))
      fprintf(stderr, "[cderi] tensor-core update items, thread-0 seconds: copies %.2f, MMA %.2f, drain %.2f, result %.2f\n",
              sum.tc_ns[0] * 1e-9, sum.tc_ns[1] * 1e-9, sum.tc_ns[2] * 1e-9, sum.tc_ns[3] * 1e-9);
    for (int k = 0; k < kJobKinds; ++k) stats[23 + k] = (double)sum.kind_ops[k];
    stats[39] = (double)waves.size();
  }
  cleanup();
  return CD_OK;
#undef BP_CUDA
}
