// ozaki.cu -- exact-slice GEMM on the tcgen05 tensor cores (see ozaki.cuh).
//
// CTA tile 128 (rows of A) x BN (rows of B; 64, or 32 for 7 slices), k-blocks
// of 32 BF16 (64-byte rows, 64-byte swizzle) staged by TMA in a STAGES-deep
// ring.  Two accumulator sets in tensor memory (when they fit) let the drain
// of one k-chunk overlap the MMAs of the next.  Warp roles: warps 0-3 drain
// tensor memory (one TMEM lane per thread), warp 4 issues the TMA loads, warp
// 5 allocates tensor memory and issues the MMAs.  Every mbarrier wait is
// bounded; on time-out the CTA stops, frees its tensor memory and sets the
// error flag.
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <atomic>
#include <mutex>
#include "internal.cuh"
#include "ozaki.cuh"
#include "tc.cuh"

namespace cd {
namespace {

constexpr int BM = 128, BK = 32;
constexpr int kThreads = 192;

template <int SA, int SB, int KEEP, int BN, int STAGES>
struct Cfg {
  static constexpr int G = KEEP - 1;                       // accumulator groups (s+t = 2..KEEP)
  static constexpr int A_BYTES = SA * BM * BK * 2;
  static constexpr int B_BYTES = SB * BN * BK * 2;
  static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int ACC_COLS = G * BN;                  // one accumulator set
  // two accumulator sets (double buffering) when they fit in the 512 columns
  static constexpr int NBUF = 2 * ACC_COLS <= 512 ? 2 : 1;
  static constexpr int NEED = NBUF * ACC_COLS;
  static constexpr int TMEM_COLS = NEED <= 32 ? 32 : (NEED <= 64 ? 64 : (NEED <= 128 ? 128 : (NEED <= 256 ? 256 : 512)));
  static constexpr int SMEM = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
  static_assert(ACC_COLS <= 512, "accumulators exceed tensor memory");
  static_assert(SB >= KEEP - 1, "the first A slice's MMA must cover every accumulator group");
  static_assert(SB * BN <= 256 && (BN % 16) == 0, "stacked B operand: N = SB*BN must be <= 256");
  static_assert(SMEM <= 232448, "shared memory over the per-CTA limit");
};

// BN = 32 tiles cap registers (two CTAs' worth) so that an FP64 kernel can share the SM
template <int SA, int SB, int KEEP, int BN, int STAGES>
__global__ void __launch_bounds__(kThreads, BN == 32 ? 2 : 1)
ozaki_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
             int64_t m_rows, int64_t n_rows, int nkb_total, int kb_per_split, int kcb, int F,
             unsigned long long* __restrict__ D, int64_t ldd, int* err, int sym, unsigned long long wait_ns,
             int a4d) {
  using C = Cfg<SA, SB, KEEP, BN, STAGES>;
  // symmetric product (A == B): tiles entirely below the diagonal are skipped
  if (sym && (int64_t)blockIdx.x * BN + BN <= (int64_t)blockIdx.y * BM) return;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + STAGES * C::STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;      // [2] accumulator set ready for the drain
  uint64_t* tempty = tfull + 2;          // [2] accumulator set drained
  uint64_t* mma_done = tempty + 2;       // MMAs of an aborted CTA completed
  uint32_t* tmem_slot = (uint32_t*)(mma_done + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // column tiles vary fastest so that the CTAs sharing a row tile of A run together (L2 reuse)
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int kb0 = blockIdx.z * kb_per_split;
  const int kb1 = min(nkb_total, kb0 + kb_per_split);
  const int nkb = kb1 - kb0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { tc::mbar_init(&tfull[b], 1); tc::mbar_init(&tempty[b], 4); }
    tc::mbar_init(mma_done, 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 5) tc::tmem_alloc<C::TMEM_COLS>(tmem_slot);
  if (warp == 4 && lane == 0) { tc::prefetch_tmap(&tmA); tc::prefetch_tmap(&tmB); }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int issued = 0;   // TMA stages issued (producer thread)
  if (nkb > 0) {
    if (warp == 4) {
      if (lane == 0) {
        // ---------------- TMA producer
        for (int i = 0; i < nkb; ++i) {
          const int s = i % STAGES;
          const uint32_t ph = (uint32_t)((i / STAGES) & 1);
          if (!tc::mbar_wait(&empty[s], ph ^ 1u, abort_flag, err, 2, wait_ns)) break;
          uint8_t* a = smem + s * C::STAGE_BYTES;
          uint8_t* b = a + C::A_BYTES;
          tc::mbar_arrive_expect_tx(&full[s], C::STAGE_BYTES);
          const int kx = (kb0 + i) * BK;
          if (a4d) tc::tma_load_4d(a, &tmA, 0, (int32_t)m0, 0, kb0 + i, &full[s]);   // chunk kb = 32 k-values
          else tc::tma_load_3d(a, &tmA, kx, (int32_t)m0, 0, &full[s]);
          tc::tma_load_3d(b, &tmB, kx, (int32_t)n0, 0, &full[s]);
          issued = i + 1;
        }
      }
    } else if (warp == 5) {
      if (lane == 0) {
        // ---------------- MMA issuer
        int chunk = 0;
        for (int i = 0; i < nkb; ++i) {
          const int s = i % STAGES;
          const uint32_t ph = (uint32_t)((i / STAGES) & 1);
          const bool chunk_start = (i % kcb) == 0;
          const int buf = C::NBUF == 2 ? (chunk & 1) : 0;
          if (chunk_start && chunk >= C::NBUF) {
            // the set about to be overwritten was filled by chunk - NBUF: wait for its drain
            const int prev = chunk - C::NBUF;
            if (!tc::mbar_wait(&tempty[buf], (uint32_t)((prev / C::NBUF) & 1), abort_flag, err, 8, wait_ns)) break;
            tc::tc_fence_after();
          }
          if (!tc::mbar_wait(&full[s], ph, abort_flag, err, 1, wait_ns)) break;
          tc::tc_fence_after();
          const uint32_t a = tc::smem_u32(smem + s * C::STAGE_BYTES);
          const uint32_t b = a + C::A_BYTES;
          const uint32_t acc = tmem + (uint32_t)(buf * C::ACC_COLS);
          // One MMA per A slice s: the B slices t = 1..nt are stacked in shared
          // memory (rows t*BN..), and the accumulator of group s+t sits at
          // column (s+t-2)*BN, so A_s x [B_1; ...; B_nt] lands every product
          // (s, t) in its group with a single N = nt*BN instruction.  The first
          // one of a chunk (s = 1, covering every group) overwrites.
#pragma unroll
          for (int sa = 0; sa < SA; ++sa) {
            const int nt = (SB < KEEP - 1 - sa) ? SB : KEEP - 1 - sa;
            if (nt <= 0) continue;
            const uint32_t idesc = tc::idesc_bf16_f32_n(BM, nt * BN);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint64_t ad = sdesc_k_sw64(a + sa * (BM * BK * 2) + kk * 32);
              const uint64_t bd = sdesc_k_sw64(b + kk * 32);
              tc::umma_bf16(acc + sa * BN, ad, bd, idesc, (chunk_start && sa == 0 && kk == 0) ? 0u : 1u);
            }
          }
          tc::umma_commit(&empty[s]);
          if ((i % kcb) == kcb - 1 || i == nkb - 1) {
            tc::umma_commit(&tfull[buf]);
            ++chunk;
          }
        }
      }
    } else {
      // ---------------- drain (warps 0-3): thread = TMEM lane = tile row
      const int row = warp * 32 + lane;
      long long run[BN];
#pragma unroll
      for (int c = 0; c < BN; ++c) run[c] = 0;
      const int nchunks = (nkb + kcb - 1) / kcb;
      bool ok = true;
      for (int ch = 0; ch < nchunks; ++ch) {
        const int buf = C::NBUF == 2 ? (ch & 1) : 0;
        if (!tc::mbar_wait(&tfull[buf], (uint32_t)((ch / C::NBUF) & 1), abort_flag, err, 4, wait_ns)) { ok = false; break; }
        tc::tc_fence_after();
        const uint32_t acc = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * C::ACC_COLS);
#pragma unroll
        for (int g = 0; g < KEEP - 1; ++g) {
          const int sh = F - 8 * (g + 2) + 2;  // weight of group g in units of 2^-F
#pragma unroll
          for (int cb = 0; cb < BN / 16; ++cb) {
            uint32_t v[16];
            tc::tmem_ld16(acc + g * BN + cb * 16, v);
            tc::tmem_ld_wait();
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const long long iv = exact_float_to_ll(__uint_as_float(v[c]));
              long long add;
              if (sh >= 0) add = iv << sh;
              else add = (iv + (1ll << (-sh - 1))) >> (-sh);
              run[cb * 16 + c] += add;
            }
          }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[buf]);
      }
      const int64_t m = m0 + row;
      if (ok && m < m_rows) {
#pragma unroll
        for (int c = 0; c < BN; ++c) {
          const int64_t n = n0 + c;
          if (n < n_rows && run[c] != 0) atomicAdd(D + n * ldd + m, (unsigned long long)run[c]);
        }
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  // Every role has left its loop, so the abort flag is final here.  After an
  // abort some issued work may still be in flight: the last STAGES TMA loads
  // (the MMA warp may have stopped before consuming them; each completes its
  // stage's phase) and MMAs the drain never waited for.  Both are waited for
  // (bounded) before the shared and tensor memory of the CTA are released.
  if (*abort_flag) {
    if (warp == 4 && lane == 0) {
      for (int i = issued > STAGES ? issued - STAGES : 0; i < issued; ++i)
        tc::mbar_settle(&full[i % STAGES], (uint32_t)((i / STAGES) & 1));
    } else if (warp == 5 && lane == 0) {
      tc::umma_commit(mma_done);   // arrives once every MMA this thread issued has completed
      tc::mbar_settle(mma_done, 0u);
    }
    tc::tc_fence_before();
    __syncthreads();
  }
  if (warp == 5) {
    tc::tc_fence_after();
    tc::tmem_dealloc<C::TMEM_COLS>(tmem);
  }
}

// ------------------------------------------------------------------ host ----
std::atomic<unsigned long long> g_wait_ns{tc::kWaitNsDefault};
unsigned long long wait_limit_ns() { return g_wait_ns.load(std::memory_order_relaxed); }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// 3D map over bf16 slices [S][rows][kpitch]; box {BK, box_rows, S}, 64-byte swizzle
int make_map(CUtensorMap* map, const void* base, int S, int64_t rows, int64_t kdim, int64_t kpitch, int box_rows) {
  auto enc = encode_fn();
  if (!enc) { set_error("cuTensorMapEncodeTiled unavailable"); return CD_ECUDA; }
  if (((uintptr_t)base & 15) || (kpitch * 2) % 16) { set_error("slice tensor not 16-byte aligned"); return CD_EINVAL; }
  cuuint64_t dims[3] = {(cuuint64_t)kdim, (cuuint64_t)rows, (cuuint64_t)S};
  cuuint64_t strides[2] = {(cuuint64_t)(kpitch * 2), (cuuint64_t)(kpitch * 2 * rows)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)S};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled failed: " + std::to_string((int)r)); return CD_EINVAL; }
  return CD_OK;
}

// 4D map over slices stored in k-chunks of 32: [chunks][S][rows][32] bf16; box {32, box_rows, S, 1}
int make_map_chunked(CUtensorMap* map, const void* base, int S, int64_t rows, int64_t kdim, int box_rows) {
  auto enc = encode_fn();
  if (!enc) { set_error("cuTensorMapEncodeTiled unavailable"); return CD_ECUDA; }
  if ((uintptr_t)base & 15) { set_error("slice tensor not 16-byte aligned"); return CD_EINVAL; }
  const int64_t chunks = (kdim + BK - 1) / BK;
  cuuint64_t dims[4] = {(cuuint64_t)BK, (cuuint64_t)rows, (cuuint64_t)S, (cuuint64_t)chunks};
  cuuint64_t strides[3] = {(cuuint64_t)(BK * 2), (cuuint64_t)(BK * 2 * rows), (cuuint64_t)(BK * 2 * rows * S)};
  cuuint32_t box[4] = {(cuuint32_t)BK, (cuuint32_t)box_rows, (cuuint32_t)S, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) { set_error("cuTensorMapEncodeTiled (chunked) failed: " + std::to_string((int)r)); return CD_EINVAL; }
  return CD_OK;
}

template <int SA, int SB, int KEEP, int BN, int STAGES>
int run(const CUtensorMap& ta, const CUtensorMap& tb, int64_t a_rows, int64_t b_rows, int nkb, int ksplit, int kcb,
        int F, unsigned long long* D, int64_t ldd, int* err, int sym, cudaStream_t st, int a4d) {
  using C = Cfg<SA, SB, KEEP, BN, STAGES>;
  auto k = ozaki_kernel<SA, SB, KEEP, BN, STAGES>;
  CD_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  const int per = (nkb + ksplit - 1) / ksplit;
  const int nsplit = (nkb + per - 1) / per;
  const int64_t row_tiles = (a_rows + BM - 1) / BM;
  if (row_tiles > 65535) { set_error("ozaki_gemm: too many row tiles"); return CD_EINVAL; }
  dim3 grid((unsigned)((b_rows + BN - 1) / BN), (unsigned)row_tiles, (unsigned)nsplit);
  k<<<grid, kThreads, C::SMEM, st>>>(ta, tb, a_rows, b_rows, nkb, per, kcb, F, D, ldd, err, sym, wait_limit_ns(), a4d);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

template <int S, bool CHUNKED>
__global__ void slice_rows_kernel(const double* __restrict__ src, int64_t src_rs, int64_t src_ks, int64_t rows,
                                  int64_t kcount, const int32_t* __restrict__ row_exp,
                                  __nv_bfloat16* __restrict__ dst, int64_t dst_rows, int64_t kpitch, int64_t k0) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * kcount) return;
  const int64_t r = t / kcount, k = t % kcount;
  // round(x 2^(8S-1-e)) from the bit pattern, then integer digits
  float a[S];
  fixed_digits<S>(scaled_double_to_ll(src[r * src_rs + k * src_ks], 8 * S - 1 - row_exp[r]), a);
  const int64_t kk = k0 + k;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int64_t at = CHUNKED ? (((kk / kSliceChunk) * S + s) * dst_rows + r) * kSliceChunk + kk % kSliceChunk
                               : ((int64_t)s * dst_rows + r) * kpitch + kk;
    dst[at] = __float2bfloat16_rn(a[s]);
  }
}

}  // namespace

int ozaki_gemm(const OzakiPlan& p, const void* As, int64_t a_rows, int64_t a_kpitch, const void* Bs, int64_t b_rows,
               int64_t b_kpitch, int64_t kdim, unsigned long long* D, int64_t ldd, int ksplit, int* err_dev,
               cudaStream_t st, bool sym, bool a_chunked) {
  const int symi = sym ? 1 : 0;
  if (kdim <= 0 || a_rows <= 0 || b_rows <= 0) return CD_OK;
  CUtensorMap ta, tb;
  // B tile rows: the stacked B slices (SB x bn <= 256) and two accumulator sets
  // (2 x groups x bn <= 512 TMEM columns) must fit; the widest tile that does
  // reads each A slice from shared memory for the most products
  const int bn = p.SA >= 7 ? 32 : (p.SA == 5 ? 48 : 64);
  if (a_chunked) CD_TRY(make_map_chunked(&ta, As, p.SA, a_rows, kdim, BM));
  else CD_TRY(make_map(&ta, As, p.SA, a_rows, kdim, a_kpitch, BM));
  const int a4d = a_chunked ? 1 : 0;
  CD_TRY(make_map(&tb, Bs, p.SB, b_rows, kdim, b_kpitch, bn));
  const int nkb = (int)((kdim + BK - 1) / BK);
  // exactness of the FP32 accumulation: (products sharing an accumulator) * kc * 129^2 <= 2^24
  const int maxg = std::min(p.KEEP - 1, std::min(p.SA, p.SB));
  int kc = (int)(16777216.0 / (std::max(1, maxg) * kSliceProdMax));
  int kcb = std::max(1, kc / BK);
  if (p.SA == 3 && p.SB == 3 && p.KEEP == 4) return run<3, 3, 4, 64, 5>(ta, tb, a_rows, b_rows, nkb, ksplit, kcb, p.F, D, ldd, err_dev, symi, st, a4d);
  if (p.SA == 5 && p.SB == 5 && p.KEEP == 6) return run<5, 5, 6, 48, 4>(ta, tb, a_rows, b_rows, nkb, ksplit, kcb, p.F, D, ldd, err_dev, symi, st, a4d);
  if (p.SA == 4 && p.SB == 4 && p.KEEP == 5) return run<4, 4, 5, 64, 4>(ta, tb, a_rows, b_rows, nkb, ksplit, kcb, p.F, D, ldd, err_dev, symi, st, a4d);
  if (p.SA == 7 && p.SB == 7 && p.KEEP == 8) return run<7, 7, 8, 32, 3>(ta, tb, a_rows, b_rows, nkb, ksplit, kcb, p.F, D, ldd, err_dev, symi, st, a4d);
  if (p.SA == 1 && p.SB == 1 && p.KEEP == 2) return run<1, 1, 2, 64, 4>(ta, tb, a_rows, b_rows, nkb, ksplit, kcb, p.F, D, ldd, err_dev, symi, st, a4d);
  set_error("ozaki_gemm: unsupported slice plan");
  return CD_EINVAL;
}

int launch_slice_rows_f64(const double* src, int64_t src_rs, int64_t src_ks, int64_t rows, int64_t kcount,
                          const int32_t* row_exp, int S, void* dst, int64_t dst_rows, int64_t kpitch, int64_t k0,
                          cudaStream_t st, bool chunked) {
  const int64_t tot = rows * kcount;
  if (tot <= 0) return CD_OK;
  const unsigned grid = (unsigned)((tot + 255) / 256);
  __nv_bfloat16* d = (__nv_bfloat16*)dst;
  if (chunked) {
    if (S != 7) { set_error("slice: the chunked layout holds 7 slices"); return CD_EINVAL; }
    slice_rows_kernel<7, true><<<grid, 256, 0, st>>>(src, src_rs, src_ks, rows, kcount, row_exp, d, dst_rows, kpitch, k0);
  }
  else if (S == 7) slice_rows_kernel<7, false><<<grid, 256, 0, st>>>(src, src_rs, src_ks, rows, kcount, row_exp, d, dst_rows, kpitch, k0);
  else if (S == 5) slice_rows_kernel<5, false><<<grid, 256, 0, st>>>(src, src_rs, src_ks, rows, kcount, row_exp, d, dst_rows, kpitch, k0);
  else if (S == 4) slice_rows_kernel<4, false><<<grid, 256, 0, st>>>(src, src_rs, src_ks, rows, kcount, row_exp, d, dst_rows, kpitch, k0);
  else if (S == 3) slice_rows_kernel<3, false><<<grid, 256, 0, st>>>(src, src_rs, src_ks, rows, kcount, row_exp, d, dst_rows, kpitch, k0);
  else if (S == 1) slice_rows_kernel<1, false><<<grid, 256, 0, st>>>(src, src_rs, src_ks, rows, kcount, row_exp, d, dst_rows, kpitch, k0);
  else { set_error("slice: unsupported slice count"); return CD_EINVAL; }
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

}  // namespace cd

// ---------------------------------------------------------------------------
// Stand-alone exact-slice product of two FP64 device matrices (C ABI
// cd_slice_matmul): out[i][j] = sum_k X[i][k] Y[j][k].
namespace cd {
namespace {
__global__ void row_exp_kernel(const double* __restrict__ X, int64_t ldx, int64_t rows, int64_t k,
                               int32_t* __restrict__ e) {
  const int64_t r = blockIdx.x;
  if (r >= rows) return;
  double m = 0.0;
  for (int64_t c = threadIdx.x; c < k; c += blockDim.x) m = fmax(m, fabs(X[r * ldx + c]));
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
    m = fmax(m, sh[0]);
    int ex = 0;
    if (m > 0.0) frexp(m, &ex);
    e[r] = ex;
  }
}
__global__ void fixed_to_f64_kernel(const unsigned long long* __restrict__ D, int64_t ldd, int64_t m, int64_t n,
                                    const int32_t* __restrict__ ex, const int32_t* __restrict__ ey, int F,
                                    double* __restrict__ out, int64_t ldo) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * n) return;
  const int64_t i = t / n, j = t % n;
  out[i * ldo + j] = ldexp((double)(long long)D[j * ldd + i], ex[i] + ey[j] - F);
}
}  // namespace
}  // namespace cd

extern "C" int cd_slice_matmul(const double* X, int64_t ldx, int64_t m, const double* Y, int64_t ldy, int64_t n,
                               int64_t k, int32_t slices, double* out, int64_t ldo, void* stream) {
  using namespace cd;
  if (!X || !Y || !out || m <= 0 || n <= 0 || k <= 0 || ldx < k || ldy < k || ldo < n) {
    set_error("cd_slice_matmul: bad argument");
    return CD_EINVAL;
  }
  if (slices != 1 && slices != 3 && slices != 4 && slices != 5 && slices != 7) {
    set_error("cd_slice_matmul: slices must be 1, 3, 4, 5 or 7");
    return CD_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t kp = (k + 7) / 8 * 8;
  OzakiPlan plan;
  plan.SA = plan.SB = slices;
  plan.KEEP = slices + 1;
  int lk = 1;
  while ((1ll << lk) < k) ++lk;
  plan.F = 61 - lk;
  void *As = nullptr, *Bs = nullptr;
  int32_t *ex = nullptr, *ey = nullptr;
  unsigned long long* D = nullptr;
  int* err = nullptr;
  int rc = CD_OK;
  auto fin = [&](int code) {
    cudaStreamSynchronize(st);
    cudaFree(As); cudaFree(Bs); cudaFree(ex); cudaFree(ey); cudaFree(D); cudaFree(err);
    return code;
  };
  if (cudaMalloc(&As, (size_t)slices * m * kp * 2) != cudaSuccess || cudaMalloc(&Bs, (size_t)slices * n * kp * 2) != cudaSuccess ||
      cudaMalloc(&ex, sizeof(int32_t) * m) != cudaSuccess || cudaMalloc(&ey, sizeof(int32_t) * n) != cudaSuccess ||
      cudaMalloc(&D, sizeof(unsigned long long) * m * n) != cudaSuccess || cudaMalloc(&err, sizeof(int)) != cudaSuccess) {
    set_error("cd_slice_matmul: allocation failed");
    return fin(CD_ENOMEM);
  }
  cudaMemsetAsync(As, 0, (size_t)slices * m * kp * 2, st);
  cudaMemsetAsync(Bs, 0, (size_t)slices * n * kp * 2, st);
  cudaMemsetAsync(D, 0, sizeof(unsigned long long) * m * n, st);
  cudaMemsetAsync(err, 0, sizeof(int), st);
  row_exp_kernel<<<(unsigned)m, 256, 0, st>>>(X, ldx, m, k, ex);
  count_launch();
  row_exp_kernel<<<(unsigned)n, 256, 0, st>>>(Y, ldy, n, k, ey);
  count_launch();
  if ((rc = launch_slice_rows_f64(X, ldx, 1, m, k, ex, slices, As, m, kp, 0, st)) != CD_OK) return fin(rc);
  if ((rc = launch_slice_rows_f64(Y, ldy, 1, n, k, ey, slices, Bs, n, kp, 0, st)) != CD_OK) return fin(rc);
  if ((rc = ozaki_gemm(plan, As, m, kp, Bs, n, kp, k, D, m, 1, err, st)) != CD_OK) return fin(rc);
  fixed_to_f64_kernel<<<(unsigned)((m * n + 255) / 256), 256, 0, st>>>(D, m, m, n, ex, ey, plan.F, out, ldo);
  count_launch();
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    set_error(std::string("cd_slice_matmul: CUDA failure: ") + cudaGetErrorString(cudaGetLastError()));
    return fin(CD_ECUDA);
  }
  if (herr) { set_error("cd_slice_matmul: tensor-core pipeline wait timed out"); return fin(CD_ETIMEOUT); }
  return fin(CD_OK);
}

namespace cd {
// registers of one CTA of the column-update GEMM (allocated per warp, 256 at a time)
int update_cta_registers(int* regs) {
  cudaFuncAttributes a;
  CD_CUDA(cudaFuncGetAttributes(&a, ozaki_kernel<7, 7, 8, 32, 3>));
  *regs = (kThreads / 32) * ((a.numRegs * 32 + 255) / 256 * 256);
  return CD_OK;
}
// the wall-clock limit of bounded device waits set by cd_set_wait_limit
unsigned long long device_wait_limit_ns() { return wait_limit_ns(); }
}  // namespace cd

extern "C" int cd_set_wait_limit(double seconds, double* previous) {
  using namespace cd;
  if (previous) *previous = (double)g_wait_ns.load() * 1e-9;
  if (!(seconds >= 0.0) || !(seconds <= 3600.0)) {
    set_error("cd_set_wait_limit: seconds must be in [0, 3600]");
    return CD_EINVAL;
  }
  g_wait_ns.store((unsigned long long)(seconds * 1e9));
  return CD_OK;
}

// ---------------------------------------------------------------------------
// Helpers of the sliced column update inside the decomposition.
namespace cd {
namespace {
// e_r with sqrt(d_r) < 2^e_r (frexp exponent); every Cholesky vector entry obeys
// |L^K_r| <= sqrt(D^K_r) <= sqrt(D^1_r), so 2^e_r is a fixed scale for row r.
__global__ void row_exp_sqrt_kernel(const double* __restrict__ d, int64_t n, int32_t* __restrict__ e) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  int ex = 0;
  const double v = d[r];
  if (v > 0.0) frexp(sqrt(v), &ex);
  e[r] = ex;
}
// Bs[s][j][k] = slice s of row rows[j], vector k, for valid[j] <= k < K, else 0
// (k < kfill); Ls holds the slices in k-chunks of 32: [k/32][S][n][32]
__global__ void gather_slices_kernel(const __nv_bfloat16* __restrict__ Ls, int64_t n,
                                     const int64_t* __restrict__ rows, const int64_t* __restrict__ valid, int nb,
                                     int S, int64_t K, int64_t kfill, __nv_bfloat16* __restrict__ Bs,
                                     int64_t bpitch) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)nb * kfill;
  if (t >= per * S) return;
  const int s = (int)(t / per);
  const int64_t rem = t % per;
  const int j = (int)(rem / kfill);
  const int64_t k = rem % kfill;
  __nv_bfloat16 v = __float2bfloat16(0.0f);
  if (k >= valid[j] && k < K)
    v = Ls[(((k / kSliceChunk) * S + s) * n + rows[j]) * kSliceChunk + k % kSliceChunk];
  Bs[((int64_t)s * nb + j) * bpitch + k] = v;
}
// cols[slot[j]][r] -= 2^(e_r + e_{row j} - F) * D[j][r]
__global__ void colupd_finalize_kernel(const unsigned long long* __restrict__ D, int64_t ldd, int64_t n, int nb,
                                       const int32_t* __restrict__ e, const int64_t* __restrict__ rows,
                                       const int32_t* __restrict__ slots, int F, double* __restrict__ cols,
                                       int64_t ld) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y;
  if (r >= n) return;
  const long long v = (long long)D[(int64_t)j * ldd + r];
  const int sc = e[r] + e[rows[j]] - F;
  cols[(int64_t)slots[j] * ld + r] -= ldexp((double)v, sc);
}
}  // namespace

int launch_row_exp_sqrt(const double* d, int64_t n, int32_t* e, cudaStream_t st) {
  if (n <= 0) return CD_OK;
  row_exp_sqrt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d, n, e);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_gather_slices(const void* Ls, int64_t n, const int64_t* rows, const int64_t* valid, int nb,
                         int S, int64_t K, void* Bs, int64_t bpitch, cudaStream_t st) {
  const int64_t kfill = (K + 31) / 32 * 32;
  const int64_t tot = (int64_t)S * nb * kfill;
  if (tot <= 0) return CD_OK;
  gather_slices_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>((const __nv_bfloat16*)Ls, n, rows, valid,
                                                                      nb, S, K, kfill, (__nv_bfloat16*)Bs, bpitch);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

int launch_colupd_finalize(const unsigned long long* D, int64_t ldd, int64_t n, int nb, const int32_t* e,
                           const int64_t* rows, const int32_t* slots, int F, double* cols, int64_t ld, cudaStream_t st) {
  if (n <= 0 || nb <= 0) return CD_OK;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)nb);
  colupd_finalize_kernel<<<grid, 256, 0, st>>>(D, ldd, n, nb, e, rows, slots, F, cols, ld);
  count_launch();
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

}  // namespace cd
