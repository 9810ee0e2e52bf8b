// eri.cu -- kernel (a) launches: ERI columns over the screened bra shell pairs
// against groups of ket function pairs, and the diagonal (row|row).  The
// integral arithmetic (Boys function, Obara-Saika / Head-Gordon-Pople
// recurrences) is in eri_dev.cuh.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include "internal.cuh"
#include "eri_dev.cuh"

namespace cd {
namespace {

// Without a work counter: grid x = tiles of 128 bra shell pairs of one class,
// y = ket groups.  With one (persistent): a grid of resident CTAs takes items
// (tile, group) from the counter, tile-major, so the heaviest bra tiles (the
// class is sorted by primitive pairs, descending) go first and the last items
// are the lightest: the launch ends with a short tail.
template <int LA, int LB>
__global__ void __launch_bounds__(128) eri_columns_kernel(PairSet bra, const int64_t* __restrict__ order, int64_t b0,
                                                          int64_t b1, PairSet ket,
                                                          const KetGroup* __restrict__ groups, double* __restrict__ out,
                                                          int64_t ld, const double* __restrict__ tab,
                                                          unsigned long long* __restrict__ op_count,
                                                          unsigned* __restrict__ work_counter, int ngroups) {
  unsigned long long ops = 0;
  if (!work_counter) {
    column_item<LA, LB>(bra, order, b0, b1, ket, groups, blockIdx.x, blockIdx.y, out, ld, tab, ops);
  } else {
    const int64_t ntiles = (b1 - b0 + 127) / 128;
    const unsigned long long nitems = (unsigned long long)ntiles * (unsigned long long)ngroups;
    __shared__ unsigned s_item;
    for (;;) {
      if (threadIdx.x == 0) s_item = atomicAdd(work_counter, 1u);
      __syncthreads();
      const unsigned long long it = s_item;
      __syncthreads();
      if (it >= nitems) break;
      column_item<LA, LB>(bra, order, b0, b1, ket, groups, (int64_t)(it / ngroups), (int)(it % ngroups), out, ld,
                          tab, ops);
    }
  }
  if (op_count) {  // warp sum, one atomic per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ops += __shfl_xor_sync(0xffffffffu, ops, o);
    if ((threadIdx.x & 31) == 0 && ops) atomicAdd(op_count, ops);
  }
}

// diagonal: thread = (shell pair, component c); ket = same shell pair, same component
template <int LA, int LB>
__global__ void __launch_bounds__(128) eri_diag_kernel(PairSet ps, int64_t s0, int64_t s1, double* __restrict__ diag,
                                                       const double* __restrict__ tab) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t sp = s0 + t / 9;
  const int c = (int)(t % 9);
  if (sp >= s1) return;
  const int32_t r = __ldg(ps.row + 9 * sp + c);
  if (r < 0) return;
  double v[1][9];
  const int kcs[1] = {c / 3}, kds[1] = {c % 3};
  const int ax[3] = {0, 1, 2};
  unsigned n_table = 0;
  quartet<LA, LB, LA, LB, 1>(ps, sp, ps, sp, kcs, kds, ax, tab, v, n_table);
  diag[r] = v[0][c];
}

}  // namespace

int launch_eri_columns(const PairSet& bra, const int64_t* bra_order, const int64_t* class_off,
                       const PairSet& ket, const KetGroup* kets_dev, int nket,
                       double* out, int64_t ld, const double* boys, cudaStream_t st,
                       unsigned long long* op_count, const EriStreams* es) {
  if (nket <= 0) return CD_OK;
  if (es) {
    CD_CUDA(cudaEventRecord(es->fork, st));
    CD_CUDA(cudaStreamWaitEvent(es->side[0], es->fork, 0));
    CD_CUDA(cudaStreamWaitEvent(es->side[1], es->fork, 0));
  }
  // persistent grids need one zeroed work counter per class
  if (es && es->counters) CD_CUDA(cudaMemsetAsync(es->counters, 0, 3 * sizeof(unsigned), st));
  if (es && es->counters && es->topup) {
    // beside the update: primary grids here, top-ups behind the update
    CD_CUDA(cudaEventRecord(es->counters_ready, st));
    CD_CUDA(cudaStreamWaitEvent(es->topup, es->counters_ready, 0));
    for (int pass = 0; pass < 2; ++pass) {
      cudaStream_t s = pass == 0 ? st : es->topup;
      for (int cls = 2; cls >= 0; --cls) {
        const int64_t b0 = class_off[cls], b1 = class_off[cls + 1];
        if (b1 <= b0) continue;
        const int per_sm = pass == 0 ? es->primary[cls] : es->resident[cls] - es->primary[cls];
        if (per_sm <= 0) continue;
        const int64_t items = (b1 - b0 + 127) / 128 * (int64_t)nket;
        dim3 grid((unsigned)std::min<int64_t>(items, (int64_t)per_sm * es->sms), 1);
        unsigned* ctr = es->counters + cls;
        if (cls == 0) eri_columns_kernel<0, 0><<<grid, 128, 0, s>>>(bra, bra_order, b0, b1, ket, kets_dev, out, ld, boys, op_count, ctr, nket);
        else if (cls == 1) eri_columns_kernel<1, 0><<<grid, 128, 0, s>>>(bra, bra_order, b0, b1, ket, kets_dev, out, ld, boys, op_count, ctr, nket);
        else eri_columns_kernel<1, 1><<<grid, 128, 0, s>>>(bra, bra_order, b0, b1, ket, kets_dev, out, ld, boys, op_count, ctr, nket);
        count_launch();
      }
    }
    CD_CUDA(cudaGetLastError());
    CD_CUDA(cudaEventRecord(es->topup_done, es->topup));
    CD_CUDA(cudaStreamWaitEvent(st, es->topup_done, 0));
    return CD_OK;
  }
  // the most expensive class (pp bra pairs) is launched first, on the calling stream
  for (int cls = 2; cls >= 0; --cls) {
    int64_t b0 = class_off[cls], b1 = class_off[cls + 1];
    if (b1 <= b0) continue;
    cudaStream_t s = es ? (cls == 2 ? st : es->side[cls]) : st;
    const int64_t ntiles = (b1 - b0 + 127) / 128;
    unsigned* ctr = (es && es->counters) ? es->counters + cls : nullptr;
    dim3 grid((unsigned)ntiles, (unsigned)nket);
    if (ctr) {
      // as many CTAs as are resident at once, or fewer when there are fewer items
      const int per_sm = es->resident[cls] > 0 ? es->resident[cls] : 2;
      const int64_t items = ntiles * (int64_t)nket;
      grid = dim3((unsigned)std::min<int64_t>(items, (int64_t)per_sm * es->sms), 1);
    }
    if (cls == 0) eri_columns_kernel<0, 0><<<grid, 128, 0, s>>>(bra, bra_order, b0, b1, ket, kets_dev, out, ld, boys, op_count, ctr, nket);
    else if (cls == 1) eri_columns_kernel<1, 0><<<grid, 128, 0, s>>>(bra, bra_order, b0, b1, ket, kets_dev, out, ld, boys, op_count, ctr, nket);
    else eri_columns_kernel<1, 1><<<grid, 128, 0, s>>>(bra, bra_order, b0, b1, ket, kets_dev, out, ld, boys, op_count, ctr, nket);
    count_launch();
  }
  CD_CUDA(cudaGetLastError());
  if (es) {
    for (int k = 0; k < 2; ++k) {
      CD_CUDA(cudaEventRecord(es->join[k], es->side[k]));
      CD_CUDA(cudaStreamWaitEvent(st, es->join[k], 0));
    }
  }
  return CD_OK;
}

int eri_resident_ctas(int* per_sm3, int* sms) {
  int dev = 0;
  CD_CUDA(cudaGetDevice(&dev));
  CD_CUDA(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  CD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm3[0], eri_columns_kernel<0, 0>, 128, 0));
  CD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm3[1], eri_columns_kernel<1, 0>, 128, 0));
  CD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm3[2], eri_columns_kernel<1, 1>, 128, 0));
  return CD_OK;
}

int eri_coresident_ctas(int regs, int* per_sm3) {
  int dev = 0;
  CD_CUDA(cudaGetDevice(&dev));
  int regs_sm = 0;
  CD_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  const void* k[3] = {(const void*)eri_columns_kernel<0, 0>, (const void*)eri_columns_kernel<1, 0>,
                      (const void*)eri_columns_kernel<1, 1>};
  for (int c = 0; c < 3; ++c) {
    // the SM's shared memory goes to the update's CTA: same carveout for both kernels
    CD_CUDA(cudaFuncSetAttribute(k[c], cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    cudaFuncAttributes a;
    CD_CUDA(cudaFuncGetAttributes(&a, k[c]));
    const int per_warp = (a.numRegs * 32 + 255) / 256 * 256;   // registers are allocated per warp, 256 at a time
    const int per_cta = per_warp * (128 / 32);
    per_sm3[c] = std::max(0, (regs_sm - regs) / per_cta);
  }
  return CD_OK;
}

int launch_eri_diag(const PairSet& ps, const int64_t* /*order*/, const int64_t* class_off,
                    double* diag, const double* boys, cudaStream_t st) {
  for (int cls = 0; cls < 3; ++cls) {
    int64_t s0 = class_off[cls], s1 = class_off[cls + 1];
    if (s1 <= s0) continue;
    int64_t nt = (s1 - s0) * 9;
    unsigned grid = (unsigned)((nt + 127) / 128);
    if (cls == 0) eri_diag_kernel<0, 0><<<grid, 128, 0, st>>>(ps, s0, s1, diag, boys);
    else if (cls == 1) eri_diag_kernel<1, 0><<<grid, 128, 0, st>>>(ps, s0, s1, diag, boys);
    else eri_diag_kernel<1, 1><<<grid, 128, 0, st>>>(ps, s0, s1, diag, boys);
    count_launch();
  }
  CD_CUDA(cudaGetLastError());
  return CD_OK;
}

}  // namespace cd

namespace cd {
// Algorithmic operation count of one primitive quartet (every add, multiply,
// fused multiply-add, reciprocal, square root and exponential is one
// operation), from the recurrences as written in the Obara-Saika /
// Head-Gordon-Pople scheme, with nothing shared between ket components:
//   set-up       PQ (3), |PQ|^2 (3), zeta+eta, 1/(zeta+eta), rho, T, prefactor (2): 12
//   Boys         F_L(T) from a tabulated Taylor series (8), exp(-T) (1), the
//                downward recursion (2 per order): 9 + 2L; scaled [0]^(m): L + 1
//   bra VRR      [e+1_i]^(m) = PA_i [e]^(m) + WP_i [e]^(m+1) (2) + N_i(e)/(2 zeta)
//                ([e-1_i]^(m) - rho/zeta [e-1_i]^(m+1)) (2 when N_i(e) > 0):
//                [p]^(m), m < L: 6L; [d]^(m), m < L-1: (3 x 4 + 3 x 2)(L-1)
//   ket VRR, per component, for every bra function e (NE of them: 1, 3 or 9):
//                [e|f+1_k]^(m) = QC_k [e|f]^(m) + WQ_k [e|f]^(m+1) (2)
//                + f-term (2 when f_k > 0) + N_k(e)/(2(zeta+eta)) [e-1_k|f]^(m+1)
//                (1 when N_k(e) > 0); level 1 for m < FK, level 2 for m = 0
//   contraction  one add per [e|f] result kept (NE per ket level needed)
// The horizontal recurrences run once per contracted integral (not per
// quartet) and are not counted.
double eri_alg_ops_per_quartet(int EB, int FK, int nc) {
  const int L = EB + FK;
  double ops = 12.0 + (9.0 + 2.0 * L) + (L + 1.0);
  if (EB >= 1) ops += 6.0 * L;
  if (EB == 2) ops += 18.0 * (L - 1);
  // bra functions e (s | p | s, p, d) and how many of them carry a given
  // Cartesian direction k (N_k(e) > 0): p: 1 of 3; d: 3 of 6 (e.g. x: xx, xy, xz)
  const int NE = EB == 0 ? 1 : (EB == 1 ? 3 : 9);
  const int withk = EB == 0 ? 0 : (EB == 1 ? 1 : 1 + 3);
  if (FK == 0) return ops + NE;
  double per = 0.0;
  // level 1 ([e|1_k]^(m), m < FK): 2 per value, + 1 where N_k(e) > 0
  per += FK * (2.0 * NE + withk);
  if (FK == 2) {
    // level 2 ([e|1_k + 1_l]^(0)): 2, + 2 for the f-term when k = l (1 of 3
    // components on average: counted as 2/3), + 1 where N_l(e) > 0
    per += 2.0 * NE + (2.0 / 3.0) * 2.0 * NE + withk;
    per += 2.0 * NE;   // contraction of the two ket levels the HRR needs
  } else {
    per += NE;         // contraction
  }
  return ops + nc * per;
}

std::vector<KetGroup> group_kets(const std::vector<KetDesc>& kets) {
  std::vector<KetDesc> k(kets);
  // same shell pair together, and within it the same kc (the level-1 recurrence is then shared)
  std::stable_sort(k.begin(), k.end(), [](const KetDesc& a, const KetDesc& b) {
    return a.sp < b.sp || (a.sp == b.sp && (a.kc < b.kc || (a.kc == b.kc && a.kd < b.kd)));
  });
  std::vector<KetGroup> out;
  for (size_t i = 0; i < k.size();) {
    size_t j = i;
    // (pp) ket shell pairs: up to all 9 components in one group (CDERI_PP_KET_GROUP
    // lowers the cap: fewer accumulators per thread, less sharing); others up to 3
    static const size_t pp_cap = [] {
      const char* e = getenv("CDERI_PP_KET_GROUP");
      const long v = e ? strtol(e, nullptr, 10) : (long)kMaxKetGroup;
      return (size_t)(v >= 1 && v <= kMaxKetGroup ? v : kMaxKetGroup);
    }();
    const size_t cap = (k[i].lc == 1 && k[i].ld == 1) ? pp_cap : 3;
    while (j < k.size() && k[j].sp == k[i].sp && j - i < cap) ++j;
    KetGroup g;
    std::memset(&g, 0, sizeof(g));
    g.sp = k[i].sp;
    g.lc = k[i].lc;
    g.ld = k[i].ld;
    g.nc = (int8_t)(j - i);
    for (size_t c = 0; c < j - i; ++c) {
      g.kc[c] = k[i + c].kc;
      g.kd[c] = k[i + c].kd;
      g.slot[c] = k[i + c].slot;
    }
    out.push_back(g);
    i = j;
  }
  return out;
}
}  // namespace cd
