// internal.cuh -- shared declarations of the CUDA translation units of libcderi.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <utility>
#include <vector>
#include "../../include/cderi.h"

namespace cd {

// ----- error handling -----------------------------------------------------
void set_error(const std::string& msg);
// process-wide count of kernel launches issued by the library
void count_launch(int n = 1);
long long launch_counter();
struct Status {
  int code = CD_OK;
};
#define CD_CUDA(call)                                                         \
  do {                                                                        \
    cudaError_t _e = (call);                                                  \
    if (_e != cudaSuccess) {                                                  \
      cudaGetLastError(); /* a non-sticky error must not leak into later calls */ \
      ::cd::set_error(std::string("CUDA: ") + cudaGetErrorString(_e) + " at " \
                      + __FILE__ + ":" + std::to_string(__LINE__));           \
      return CD_ECUDA;                                                        \
    }                                                                         \
  } while (0)
#define CD_TRY(call)                 \
  do {                               \
    int _rc = (call);                \
    if (_rc != CD_OK) return _rc;    \
  } while (0)

// ----- stream-ordered scratch memory ------------------------------------------
// Per-call scratch comes from the device's default memory pool through
// cudaMallocAsync / cudaFreeAsync on the call's stream, so concurrent calls on
// different streams never wait for each other in an implicit device-wide
// synchronisation.  The pool keeps freed memory (release threshold = max), so
// repeated calls do not remap it.  Long-lived objects (systems, factors) use
// cudaMalloc / cudaFree.
int scratch_alloc_bytes(void** p, size_t bytes, cudaStream_t st);
inline void scratch_free(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}
template <class T>
int scratch_alloc(T** p, size_t n, cudaStream_t st) {
  return scratch_alloc_bytes((void**)p, sizeof(T) * (n ? n : 1), st);
}

// ----- device arrays that grow in place (vmm.cu) ------------------------------
// A virtual address range reserved once; physical memory mapped into it in
// granules as the array grows.  The address never changes and growing copies
// nothing.  release() waits for the device (like cudaFree) before unmapping.
struct VmArray {
  void* base = nullptr;
  size_t reserved = 0;      // bytes of address space
  size_t mapped = 0;        // bytes backed by device memory (a multiple of gran)
  size_t gran = 0;
  int device = 0;
  struct Piece { size_t offset, size; unsigned long long handle; };
  std::vector<Piece> pieces;
  int reserve(size_t bytes);     // reserve address space (nothing mapped)
  int grow(size_t bytes);        // map memory so that [0, bytes) is usable
  void release();
  void swap(VmArray& o) {
    std::swap(base, o.base); std::swap(reserved, o.reserved); std::swap(mapped, o.mapped);
    std::swap(gran, o.gran); std::swap(device, o.device); pieces.swap(o.pieces);
  }
  VmArray() = default;
  VmArray(const VmArray&) = delete;
  VmArray& operator=(const VmArray&) = delete;
  ~VmArray() { release(); }
};

// ----- Boys function table (Taylor expansion about grid points) ------------
// Row k holds F_0..F_12 at T_k = k * kBoysStep and, in the last column,
// exp(-T_k).  Below kBoysTmax, F_L(T) and exp(-T) come from 8- and 9-term
// Taylor expansions about the nearest grid point (|T - T_k| <= 0.05) and the
// lower orders from the downward recursion; above it, F_0 = sqrt(pi / 4T)
// and the upward recursion with exp(-T) < 1e-26 dropped.
constexpr int kBoysMaxM = 4;            // l <= 1 per centre -> L <= 4
constexpr int kBoysTaylor = 8;          // Taylor terms for F_L
constexpr int kExpTaylor = 9;           // Taylor terms for exp(-T)
constexpr double kBoysStep = 0.1;
constexpr double kBoysTmax = 60.0;
constexpr int kBoysPoints = 602;
constexpr int kBoysFcols = kBoysMaxM + kBoysTaylor + 1;  // F_0..F_12
constexpr int kBoysCols = kBoysFcols + 1;                // + exp(-T_k)
// After the kBoysPoints x kBoysCols main table: for each L = 0..kBoysMaxM the
// Taylor coefficients of F_L about every grid point, c[L][k][j] = F_{L+j}(T_k) / j!
// (j < kBoysTaylor), so that F_L(T_k - d) is a plain Horner sum in d
constexpr int kBoysCoefOff = kBoysPoints * kBoysCols;
constexpr int kBoysTableSize = kBoysCoefOff + (kBoysMaxM + 1) * kBoysPoints * kBoysTaylor;
// bra primitive pairs with |Kp| below this are dropped.  The contribution of
// one such primitive pair to a contracted integral was measured on the N = 2000
// lattice system (30,000 dropped pairs with |Kp| in [1e-24, 1e-18) against
// same-centre kets, summed over the ket primitives): at most 3e-18 -- below the
// rounding of the integrals themselves; raising the threshold from 1e-24 cut
// the FP64 work of the ERI columns at N = 2000 by a tenth
constexpr double kPrimPrune = 1e-18;

// ----- shell-pair records (device, structure of arrays) -------------------
// A shell pair joins shells S1 >= S2 (shell index).  It is stored in canonical
// orientation: centre "A" carries the larger l (A = S1 on a tie).  Per
// primitive pair (a on A, b on B): zeta = a + b, P, PA = P - A, and
// Kp = sqrt(2) pi^{5/4} d_a d_b exp(-a b / zeta |A-B|^2) / zeta, so that the
// (ss|ss) prefactor of a primitive quartet is Kp_bra Kp_ket / sqrt(zeta + eta).
struct PairSet {
  int64_t n = 0;          // shell pairs
  int64_t npp = 0;        // primitive pairs
  // per shell pair
  int32_t* pp_off = nullptr;   // [n+1] first primitive pair
  int8_t*  la = nullptr;       // [n] canonical l of A
  int8_t*  lb = nullptr;       // [n]
  double*  AB = nullptr;       // [n][3] A - B (canonical)
  int32_t* row = nullptr;      // [n][9] output row of component (i on A)*3 + (j on B), -1 = none
  // per primitive pair
  double* zeta = nullptr;      // [npp]
  double* P = nullptr;         // [npp][3]
  double* PA = nullptr;        // [npp][3]
  double* Kp = nullptr;        // [npp]
  double* o2z = nullptr;       // [npp] 1 / (2 zeta)
};

// Host-side mirror used while building.
struct PairSetHost {
  std::vector<int32_t> pp_off, row;
  std::vector<int8_t> la, lb;
  std::vector<double> AB, zeta, P, PA, Kp, o2z;
  std::vector<int32_t> s1, s2;     // shell indices of the pair (S1 >= S2)
  std::vector<int8_t> swapped;     // 1 if A = S2
};

struct HostBasis {
  int nsh = 0, nbf = 0;
  std::vector<double> cen;        // [nsh][3]
  std::vector<int> l, nprim, pofs, bf0;
  std::vector<double> exps, dcoef;  // effective coefficients
  std::vector<int> bf_shell, bf_comp;
};

int validate_and_normalise(const cd_basis_t* b, HostBasis* hb);
void build_pairs(const HostBasis& hb, const std::vector<int32_t>& s1, const std::vector<int32_t>& s2,
                 PairSetHost* out, double prune = 0.0);
int upload_pairs(const PairSetHost& h, PairSet* d, cudaStream_t st);
void free_pairs(PairSet* d);
const double* boys_table_device(int* rc);   // per device, built once

// ket descriptor of one column: shell-pair index and canonical components
struct KetDesc {
  int32_t sp;      // shell pair index (in the pair set that holds it)
  int32_t slot;    // output column: out + slot * ld
  int8_t kc, kd;   // component on canonical C (0..2, or 0 for s) and D
  int8_t lc, ld;
};

// ket function pairs of one ket shell pair evaluated together (shared
// primitive set-up, Boys function, bra recurrence and, per distinct kc, the
// first ket level): up to 9 for a (pp) shell pair, up to 3 otherwise
constexpr int kMaxKetGroup = 9;
struct KetGroup {
  int32_t sp;        // shell pair index in `all`
  int8_t lc, ld;     // canonical class of the shell pair
  int8_t nc;         // components in the group
  int8_t pad;
  int8_t kc[kMaxKetGroup], kd[kMaxKetGroup];
  int16_t pad2;
  int32_t slot[kMaxKetGroup];   // output columns: out + slot * ld
};
// group ket descriptors of the same shell pair
std::vector<KetGroup> group_kets(const std::vector<KetDesc>& kets);

// Algorithmic FP64 operation count of one primitive quartet of a column
// block: bra shell pair of class EB = la + lb (all its components) against nc
// ket components of a ket shell pair of class FK = lc + ld, by a plain
// Obara-Saika / Head-Gordon-Pople evaluation (see eri.cu).  Independent of how
// the kernel shares work between components.
double eri_alg_ops_per_quartet(int EB, int FK, int nc);

// ERI kernels (eri.cu)
// out[slot * ld + row] = (bra rows | ket component) for every bra shell pair in `bra`
// bra_order: NULL (every bra shell pair; class c is [class_off[c], class_off[c+1]))
// or a device list of bra shell pairs grouped by class, class c being entries
// [class_off[c], class_off[c+1]) of the list.  Rows come from bra.row.
// Optional side streams for the ERI launches: the three bra classes (pp, ps,
// ss: different register budgets, so three kernels) run concurrently, the
// expensive pp class first on the calling stream and the others on side[0],
// side[1]; the calling stream then waits for both.  The last wave of each
// class kernel is thereby filled with the other classes' work.
struct EriStreams {
  cudaStream_t side[2] = {nullptr, nullptr};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[2] = {nullptr, nullptr};
  // persistent grids (optional): 3 device work counters (one per class), the
  // resident CTAs per SM of each class kernel and the SM count
  unsigned* counters = nullptr;
  int resident[3] = {0, 0, 0};
  int sms = 0;
  // Co-residence with the tensor-core column update (optional): when `topup` is
  // set, the update has been queued on it.  Each class then runs a primary
  // persistent grid on the calling stream that leaves room for one update CTA
  // on every SM (primary[c] CTAs per SM), and top-up grids queued on `topup`
  // behind the update take the rest of the same work counters once the update
  // is done.  The calling stream waits for the top-ups.
  cudaStream_t topup = nullptr;
  int primary[3] = {0, 0, 0};
  cudaEvent_t counters_ready = nullptr, topup_done = nullptr;
};
int eri_resident_ctas(int* per_sm3, int* sms);
// CTAs per SM of each class kernel that fit beside one CTA using `regs` registers
// and all of the shared memory, with the kernels' shared-memory carveout set to
// the maximum so that both can be resident together
int eri_coresident_ctas(int regs, int* per_sm3);
int launch_eri_columns(const PairSet& bra, const int64_t* bra_order, const int64_t* class_off,
                       const PairSet& ket, const KetGroup* groups_dev, int ngroups,
                       double* out, int64_t ld, const double* boys, cudaStream_t st,
                       unsigned long long* op_count = nullptr,   // FP64-pipe operation counter (optional)
                       const EriStreams* es = nullptr);
// diag[row] = (row|row) for every shell pair in `ps` (rows from ps.row)
int launch_eri_diag(const PairSet& ps, const int64_t* order, const int64_t* class_off,
                    double* diag, const double* boys, cudaStream_t st);

}  // namespace cd

// ----- opaque objects -------------------------------------------------------
struct cd_system {
  cd::HostBasis hb;
  cd::PairSet all;               // every shell pair (used for kets and the diagonal)
  cd::PairSet bra;               // screened shell pairs, sorted by class
  int64_t* bra_order = nullptr;  // unused (bra already sorted); kept for symmetry
  int64_t bra_class_off[4] = {0, 0, 0, 0};
  std::vector<int32_t> bra_to_all;          // bra shell pair -> index in `all`
  std::vector<int32_t> bra_row_h;           // host copy of bra.row ([n][9] row of each component, -1 = none)
  std::vector<int32_t> bra_npp_h;           // surviving primitive pairs of each bra shell pair
  std::vector<int32_t> all_npp_h;           // primitive pairs of each shell pair of `all`
  std::vector<int64_t> all_class_off_h;     // class offsets of `all` (sorted by class)
  int64_t all_class_off[4] = {0, 0, 0, 0};
  int64_t n_rows = 0, n_rows_pad = 0;
  std::vector<int64_t> row_packed;          // [n_rows]
  std::vector<double> row_diag;             // [n_rows]
  std::vector<int32_t> row_allsp;           // [n_rows] shell pair (in `all`) of the row
  std::vector<int8_t> row_kc, row_kd;       // canonical components of the row
  double* diag_dev = nullptr;               // [n_rows_pad] (row|row)
  int32_t* row_mu_dev = nullptr;            // [n_rows] mu of each row
  int32_t* row_nu_dev = nullptr;            // [n_rows] nu of each row
  const double* boys = nullptr;
  double schwarz = 0.0;
  double ms_setup = 0.0;
};

struct cd_factor {
  cd_system* sys = nullptr;
  bool owns_sys = false;
  int64_t M = 0, Mcap = 0, ld = 0, n = 0;
  double* L = nullptr;      // FP64 vectors [Mcap][ld] (the base of Lvm)
  cd::VmArray Lvm;          // their storage: grows in place as vectors are added
  float* L32 = nullptr;     // FP32 copy [M][ld] when requested
  int vec_precision = CD_FP64;
  std::vector<int64_t> piv;
  std::vector<double> gaps;
  std::vector<double> pivd;     // tracked residual diagonal of each pivot when it was taken
  std::vector<double> resid;
  double resid_max = 0.0;
  double stats[16] = {0};
  double eri_quartets = 0.0;   // primitive quartets of the ERI column kernels
  double eri_alg_ops = 0.0;    // their algorithmic FP64 operation count (eri_alg_ops_per_quartet)
  double mem_peak = 0.0;       // device bytes at the decomposition's peak (pool high-water mark + vector arrays)
  double mem_resident = 0.0;   // device bytes the factor keeps after the call
};
