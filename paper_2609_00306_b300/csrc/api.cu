// api.cu -- the C ABI (include/cderi.h): system set-up, the blocked pivoted
// decomposition driver, J/K, error reporting.
#include <math.h>
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <thread>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <unordered_map>
#include <vector>
#include "internal.cuh"
#include "pivot.cuh"
#include "ozaki.cuh"

namespace cd {
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launch_counter() { return g_launches.load(); }
int launch_to_fp32(const double* src, int64_t ld, int64_t M, int64_t n, float* dst, cudaStream_t st);
int mo_vectors_sliced(const float* L32, const double* L64, int64_t ld, int64_t P0, int64_t nP, int64_t n, int N,
                      int n_mo, const double* C_dev, const int32_t* mu, const int32_t* nu, int S, double* out_dev,
                      cudaStream_t st);
int jk_mixed(const float* L32, const double* L64, int64_t ld, int64_t M, int64_t n, int N, int O, const double* C_dev,
             const int32_t* mu, const int32_t* nu, double* J_dev, double* K_dev, bool wantJ, bool wantK,
             int S, cudaStream_t st);
}  // namespace cd

using namespace cd;

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <class T>
static int dalloc(T** p, size_t n) {
  *p = nullptr;
  if (n == 0) return CD_OK;
  cudaError_t e = cudaMalloc((void**)p, sizeof(T) * n);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error(std::string("cudaMalloc of ") + std::to_string(sizeof(T) * n) + " bytes failed: " + cudaGetErrorString(e));
    *p = nullptr;
    return CD_ENOMEM;
  }
  return CD_OK;
}

// ---------------------------------------------------------------- system ----
static void system_release(cd_system* s) {
  if (!s) return;
  free_pairs(&s->all);
  free_pairs(&s->bra);
  cudaFree(s->diag_dev);
  cudaFree(s->row_mu_dev);
  cudaFree(s->row_nu_dev);
  delete s;
}

static int system_create_impl(const cd_basis_t* basis, double schwarz, cudaStream_t st, cd_system** out) {
  double t0 = now_ms();
  if (!(schwarz >= 0.0) || !std::isfinite(schwarz)) { set_error("schwarz threshold must be finite and >= 0"); return CD_EINVAL; }
  cd_system* s = new cd_system();
  s->schwarz = schwarz;
  int rc = validate_and_normalise(basis, &s->hb);
  if (rc != CD_OK) { delete s; return rc; }
  const HostBasis& hb = s->hb;
  s->boys = boys_table_device(&rc);
  if (rc != CD_OK) { delete s; return rc; }
  const int nsh = hb.nsh, nbf = hb.nbf;
  // every shell pair S1 >= S2, grouped by canonical class (ss, ps, pp)
  std::vector<int32_t> cs1[3], cs2[3];
  for (int a = 0; a < nsh; ++a)
    for (int b = 0; b <= a; ++b) {
      int cls = hb.l[a] + hb.l[b];
      cs1[cls].push_back(a);
      cs2[cls].push_back(b);
    }
  std::vector<int32_t> s1, s2;
  for (int c = 0; c < 3; ++c) {
    s->all_class_off[c] = (int64_t)s1.size();
    s1.insert(s1.end(), cs1[c].begin(), cs1[c].end());
    s2.insert(s2.end(), cs2[c].begin(), cs2[c].end());
  }
  s->all_class_off[3] = (int64_t)s1.size();
  const bool dbg = getenv("CDERI_DEBUG") != nullptr;
  auto phase = [&](const char* what) {
    if (dbg) fprintf(stderr, "[cderi] system set-up: %-28s %8.1f ms\n", what, now_ms() - t0);
  };
  PairSetHost hall;
  build_pairs(hb, s1, s2, &hall);
  phase("all shell pairs built");
  rc = upload_pairs(hall, &s->all, st);
  if (rc != CD_OK) { system_release(s); return rc; }
  // diagonal of every packed pair (kernel a, diagonal mode)
  const int64_t npk = (int64_t)nbf * (nbf + 1) / 2;
  double* dall = nullptr;
  rc = scratch_alloc(&dall, (size_t)npk, st);
  if (rc != CD_OK) { system_release(s); return rc; }
  rc = launch_eri_diag(s->all, nullptr, s->all_class_off, dall, s->boys, st);
  std::vector<double> hd(npk);
  if (rc == CD_OK && cudaMemcpyAsync(hd.data(), dall, sizeof(double) * npk, cudaMemcpyDeviceToHost, st) != cudaSuccess) rc = CD_ECUDA;
  scratch_free(dall, st);
  if (rc == CD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = CD_ECUDA;
  if (rc != CD_OK) { if (rc == CD_ECUDA) set_error("diagonal pass failed"); system_release(s); return rc; }
  phase("diagonal on the device");
  for (int64_t p = 0; p < npk; ++p)
    if (!std::isfinite(hd[p])) { set_error("non-finite ERI diagonal"); system_release(s); return CD_EINVAL; }
  double dmax = 0.0;
  for (double v : hd) dmax = std::max(dmax, v);
  // shell-pair screening: keep (AB) iff sqrt(max_{mu nu in AB} D * max D) >= schwarz
  const int64_t nsp = (int64_t)s1.size();
  std::vector<char> keep(nsp, 0);
  std::vector<int32_t> ks1, ks2, kall;
  for (int64_t k = 0; k < nsp; ++k) {
    double m = 0.0;
    for (int c = 0; c < 9; ++c) {
      int32_t r = hall.row[9 * k + c];
      if (r >= 0) m = std::max(m, hd[r]);
    }
    if (sqrt(m * dmax) >= schwarz) {
      keep[k] = 1;
      ks1.push_back(s1[k]); ks2.push_back(s2[k]); kall.push_back((int32_t)k);
    }
  }
  for (int c = 0; c < 4; ++c) {
    int64_t off = 0;
    for (int64_t k = 0; k < s->all_class_off[c]; ++k) off += keep[k];
    s->bra_class_off[c] = off;
  }
  // rows: packed indices of the kept pairs, increasing
  std::vector<int64_t>& rows = s->row_packed;
  for (int64_t k = 0; k < nsp; ++k)
    if (keep[k])
      for (int c = 0; c < 9; ++c)
        if (hall.row[9 * k + c] >= 0) rows.push_back(hall.row[9 * k + c]);
  std::sort(rows.begin(), rows.end());
  const int64_t n = (int64_t)rows.size();
  s->n_rows = n;
  s->n_rows_pad = std::max<int64_t>(32, (n + 31) / 32 * 32);
  std::vector<int32_t> p2r(npk, -1);
  for (int64_t r = 0; r < n; ++r) p2r[rows[r]] = (int32_t)r;
  phase("screened rows");
  PairSetHost hbra;
  build_pairs(hb, ks1, ks2, &hbra, kPrimPrune);
  {
    // order the bra shell pairs of each class by surviving primitive pairs
    // (descending), then along a Morton curve through the pair midpoints: the
    // 32 lanes of a warp then run the same number of primitive quartets and
    // mostly the same Boys branch
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int a = 0; a < nsh; ++a)
      for (int x = 0; x < 3; ++x) {
        lo[x] = std::min(lo[x], hb.cen[3 * a + x]);
        hi[x] = std::max(hi[x], hb.cen[3 * a + x]);
      }
    const size_t nk = ks1.size();
    std::vector<uint64_t> key(nk);
    for (size_t k = 0; k < nk; ++k) {
      uint64_t m = 0;
      for (int x = 0; x < 3; ++x) {
        const double mid = 0.5 * (hb.cen[3 * ks1[k] + x] + hb.cen[3 * ks2[k] + x]);
        const double span = hi[x] - lo[x];
        const uint64_t q = span > 0 ? (uint64_t)std::min(1023.0, std::floor((mid - lo[x]) / span * 1024.0)) : 0;
        for (int bit = 0; bit < 10; ++bit) m |= ((q >> bit) & 1ull) << (3 * bit + x);
      }
      const uint64_t npp = (uint64_t)(hbra.pp_off[k + 1] - hbra.pp_off[k]);
      key[k] = ((63ull - std::min<uint64_t>(npp, 63)) << 32) | m;
    }
    std::vector<size_t> perm(nk);
    for (size_t k = 0; k < nk; ++k) perm[k] = k;
    for (int c = 0; c < 3; ++c)
      std::stable_sort(perm.begin() + s->bra_class_off[c], perm.begin() + s->bra_class_off[c + 1],
                       [&](size_t x, size_t y) { return key[x] < key[y]; });
    std::vector<int32_t> p1(nk), p2(nk), pa(nk);
    for (size_t k = 0; k < nk; ++k) { p1[k] = ks1[perm[k]]; p2[k] = ks2[perm[k]]; pa[k] = kall[perm[k]]; }
    ks1.swap(p1); ks2.swap(p2); kall.swap(pa);
    build_pairs(hb, ks1, ks2, &hbra, kPrimPrune);
  }
  phase("bra pairs ordered");
  for (auto& r : hbra.row)
    if (r >= 0) r = p2r[r];
  s->bra_to_all = kall;
  s->bra_row_h = hbra.row;
  s->bra_npp_h.resize(hbra.pp_off.empty() ? 0 : hbra.pp_off.size() - 1);
  for (size_t k = 0; k + 1 < hbra.pp_off.size(); ++k) s->bra_npp_h[k] = hbra.pp_off[k + 1] - hbra.pp_off[k];
  s->all_npp_h.resize(hall.pp_off.empty() ? 0 : hall.pp_off.size() - 1);
  for (size_t k = 0; k + 1 < hall.pp_off.size(); ++k) s->all_npp_h[k] = hall.pp_off[k + 1] - hall.pp_off[k];
  rc = upload_pairs(hbra, &s->bra, st);
  if (rc != CD_OK) { system_release(s); return rc; }
  // per-row data: diagonal, (mu, nu), ket descriptor pieces
  std::vector<int32_t> allidx((size_t)nsh * nsh, -1);
  for (int64_t k = 0; k < nsp; ++k) allidx[(size_t)s1[k] * nsh + s2[k]] = (int32_t)k;
  s->row_diag.resize(n);
  s->row_allsp.resize(n);
  s->row_kc.resize(n);
  s->row_kd.resize(n);
  std::vector<int32_t> rmu(n), rnu(n);
  for (int64_t r = 0; r < n; ++r) {
    int64_t p = rows[r];
    s->row_diag[r] = hd[p];
    int64_t mu = (int64_t)((sqrt(8.0 * (double)p + 1.0) - 1.0) / 2.0);
    while (mu * (mu + 1) / 2 > p) --mu;
    while ((mu + 1) * (mu + 2) / 2 <= p) ++mu;
    int64_t nu = p - mu * (mu + 1) / 2;
    rmu[r] = (int32_t)mu;
    rnu[r] = (int32_t)nu;
    int Sm = hb.bf_shell[mu], Sn = hb.bf_shell[nu];
    int32_t k = allidx[(size_t)Sm * nsh + Sn];
    s->row_allsp[r] = k;
    int cm = hb.bf_comp[mu], cn = hb.bf_comp[nu];
    if (hall.swapped[k]) { s->row_kc[r] = (int8_t)cn; s->row_kd[r] = (int8_t)cm; }
    else { s->row_kc[r] = (int8_t)cm; s->row_kd[r] = (int8_t)cn; }
  }
  rc = dalloc(&s->diag_dev, (size_t)s->n_rows_pad);
  if (rc == CD_OK) rc = dalloc(&s->row_mu_dev, (size_t)std::max<int64_t>(n, 1));
  if (rc == CD_OK) rc = dalloc(&s->row_nu_dev, (size_t)std::max<int64_t>(n, 1));
  if (rc != CD_OK) { system_release(s); return rc; }
  CD_CUDA(cudaMemsetAsync(s->diag_dev, 0, sizeof(double) * s->n_rows_pad, st));
  if (n > 0) {
    CD_CUDA(cudaMemcpyAsync(s->diag_dev, s->row_diag.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    CD_CUDA(cudaMemcpyAsync(s->row_mu_dev, rmu.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    CD_CUDA(cudaMemcpyAsync(s->row_nu_dev, rnu.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  }
  CD_CUDA(cudaStreamSynchronize(st));
  phase("row tables uploaded");
  s->ms_setup = now_ms() - t0;
  *out = s;
  return CD_OK;
}

static KetDesc ket_of_row(const cd_system* s, int64_t r, int32_t slot) {
  KetDesc k;
  int32_t sp = s->row_allsp[r];
  k.sp = sp;
  k.slot = slot;
  k.kc = s->row_kc[r];
  k.kd = s->row_kd[r];
  // canonical classes of `all`: [0, off1) ss, [off1, off2) ps, [off2, off3) pp
  if (sp < s->all_class_off[1]) { k.lc = 0; k.ld = 0; }
  else if (sp < s->all_class_off[2]) { k.lc = 1; k.ld = 0; }
  else { k.lc = 1; k.ld = 1; }
  return k;
}

// ---------------------------------------------------------------- factor ----
static void factor_release(cd_factor* f) {
  if (!f) return;
  f->Lvm.release();
  f->L = nullptr;
  cudaFree(f->L32);
  if (f->owns_sys) system_release(f->sys);
  delete f;
}

namespace {
constexpr int kSlices = 7;        // 8-bit slices per vector entry in the sliced update
constexpr int kSliceF = 60;       // fixed-point fraction bits of the update (|sum| < 1 per unit scale)

struct Work {  // scratch of one factorisation, freed (stream-ordered) at the end
  cudaStream_t st = nullptr;
  double* pool = nullptr;
  double* D0 = nullptr;
  double* D1 = nullptr;
  double* Bg = nullptr;
  int32_t* slots_dev = nullptr;
  int64_t* rows_dev = nullptr;
  int64_t* valid_dev = nullptr;
  KetGroup* kets_dev = nullptr;
  StepScratch* sc = nullptr;
  StepResult* res_dev = nullptr;
  // host mirrors: ordinary (pageable) memory -- the copies are followed by a
  // stream synchronisation anyway, and pinned-memory frees would synchronise
  // the whole device (concurrent batch workers)
  StepResult res_hv[1];
  double dp_hv[1];
  std::vector<double> dh;
  StepResult* res_h = res_hv;
  double* dp_h = dp_hv;
  // sliced update
  VmArray Lsvm;                     // slice store, grows in place
  void* Ls = nullptr;               // bf16 [kcap/32][kSlices][n][32] (the base of Lsvm)
  void* Bs = nullptr;               // bf16 [kSlices][b][kcap]
  unsigned long long* Dint = nullptr;  // int64 [b][ld]
  int32_t* erow = nullptr;          // [n]
  int* err = nullptr;
  unsigned long long* eri_ops = nullptr;   // FP64-pipe operations of the ERI column kernels
  int64_t kcap = 0;
  // candidate selection on the device
  SelectState* sel = nullptr;
  int64_t* cand_rows = nullptr;
  double* cand_vals = nullptr;
  std::vector<int64_t> cand_rows_h;
  std::vector<double> cand_vals_h;
  unsigned cand_count_h[1] = {0};
  // span policies: residual diagonals of the block's columns
  int64_t* slot_rows_dev = nullptr;  // [b] working row of each pool slot (-1 = empty)
  double* slot_vals_dev = nullptr;   // [b]
  std::vector<double> slot_vals_h;
  // two-step, first step: compacted rows
  int32_t* rowmap_dev = nullptr;     // [bra.n][9] working row of each bra component (-1 = dropped)
  int64_t* order_dev = nullptr;      // live bra shell pairs, grouped by class
  uint8_t* cand_dev = nullptr;       // [n] candidate mask (working rows)
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  EriStreams eri;                    // concurrent launches of the three ERI class kernels
  // device-driven pivot steps (full pivoting): state, slot map, pivots, and the
  // CUDA graph of b step launches (re-captured when its buffers move)
  DevStep* ds_dev = nullptr;
  DevStep ds_h;
  int32_t* slot_of_row = nullptr;
  int64_t* piv_dev = nullptr;
  double* pivd_dev = nullptr;
  int64_t* sm_rows = nullptr;
  int32_t* sm_slots = nullptr;
  std::vector<int64_t> piv_h;
  std::vector<double> pivd_h;
  cudaGraphExec_t step_exec = nullptr;
  const void* step_key[3] = {nullptr, nullptr, nullptr};   // L, pool, D buffers the graph was captured with
  // second stream for the sliced update, used only with CDERI_OVERLAP_UPDATE=1
  // (by default the update runs on the main stream before the ERI columns)
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_ready = nullptr, ev_gemm = nullptr, ev_g0 = nullptr, ev_g1 = nullptr;
  std::vector<int32_t> upd_slots;
  std::vector<int64_t> upd_rows, upd_valid;
  ~Work() {
    for (void* p : {(void*)pool, (void*)D0, (void*)D1, (void*)Bg, (void*)slots_dev, (void*)rows_dev,
                    (void*)valid_dev, (void*)kets_dev, (void*)sc, (void*)res_dev, Bs, (void*)Dint,
                    (void*)erow, (void*)err, (void*)sel, (void*)cand_rows, (void*)cand_vals, (void*)eri_ops,
                    (void*)slot_rows_dev, (void*)slot_vals_dev, (void*)rowmap_dev, (void*)order_dev,
                    (void*)cand_dev})
      scratch_free(p, st);

    for (auto& e : ev) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {eri.fork, eri.join[0], eri.join[1], eri.counters_ready, eri.topup_done})
      if (e) cudaEventDestroy(e);
    scratch_free(eri.counters, st);
    for (void* p : {(void*)ds_dev, (void*)slot_of_row, (void*)piv_dev, (void*)pivd_dev, (void*)sm_rows,
                    (void*)sm_slots})
      scratch_free(p, st);
    if (step_exec) cudaGraphExecDestroy(step_exec);
    for (cudaStream_t x : eri.side) if (x) cudaStreamDestroy(x);
    for (cudaEvent_t e : {ev_ready, ev_gemm, ev_g0, ev_g1}) if (e) cudaEventDestroy(e);
    if (st2) cudaStreamDestroy(st2);
  }
};
}  // namespace

// Bytes of one k-chunk (32 vectors) of the slice store over n rows.
static size_t slice_chunk_bytes(int64_t n) { return (size_t)kSlices * (size_t)std::max<int64_t>(n, 1) * 32 * 2; }

// Grow the vector store to `newcap` vectors, and the slice store with it: more
// memory is mapped behind the same addresses, nothing is copied.
static int grow_vectors(cd_factor* f, Work* w, bool slice, int b, int64_t newcap, int64_t K, cudaStream_t st) {
  (void)K;
  CD_TRY(f->Lvm.grow(sizeof(double) * (size_t)newcap * f->ld));
  if (slice) {
    const int64_t nk = (newcap + 31) / 32 * 32;
    CD_TRY(w->Lsvm.grow(slice_chunk_bytes(f->n) * (size_t)(nk / 32)));
    void* nBs = nullptr;   // the update's B operand is rebuilt for every block: no copy
    CD_TRY(scratch_alloc((uint16_t**)&nBs, (size_t)kSlices * b * nk, st));
    scratch_free(w->Bs, st);
    w->Bs = nBs;
    w->kcap = nk;
  }
  f->Mcap = newcap;
  return CD_OK;
}

// capacity after growth: what is needed, and at least 256 vectors more, in whole 32-vector chunks
static int64_t grown_capacity(int64_t need, int64_t cap, int64_t Mmax) {
  int64_t nc = std::max<int64_t>(need, cap + 256);
  nc = (nc + 31) / 32 * 32;
  return std::min<int64_t>(nc, Mmax);
}

// reduce = true: first step of the two-step scheme (rows below tau dropped and
// compacted; only f->piv, in system rows, is meaningful afterwards)
static int factor_impl(cd_system* s, const cd_opts_t* o, cudaStream_t st, cd_factor* f, bool reduce = false) {
  const double t_start = now_ms();
  const double tau = o->tau;
  if (!(tau > 0.0) || !std::isfinite(tau)) { set_error("tau must be finite and > 0"); return CD_EINVAL; }
  const int b = o->block ? o->block : 64;
  if (b < 1 || b > kMaxBlock) { set_error("block must be in [1, 256]"); return CD_EINVAL; }
  if (o->vec_precision != CD_FP64 && o->vec_precision != CD_VEC_FP32) { set_error("bad vec_precision"); return CD_EINVAL; }
  if (o->update != CD_UPDATE_SLICE && o->update != CD_UPDATE_FP64) { set_error("bad update mode"); return CD_EINVAL; }
  const bool slice = o->update == CD_UPDATE_SLICE;
  const bool forced = o->forced_pivots != nullptr;
  const int64_t nf = forced ? o->n_forced : 0;
  const bool span_mode = o->algorithm != CD_ALG_FULL;
  const double span = o->span > 0.0 ? o->span : 0.01;
  if (span_mode && !(span > 0.0 && span <= 1.0)) { set_error("span factor must be in (0, 1]"); return CD_EINVAL; }
  if (span_mode && forced) { set_error("forced pivots need CD_ALG_FULL"); return CD_EINVAL; }
  int64_t n = s->n_rows, ld = s->n_rows_pad;
  const int64_t N = s->hb.nbf;
  if (forced) {
    if (nf < 0) { set_error("n_forced < 0"); return CD_EINVAL; }
    for (int64_t k = 0; k < nf; ++k)
      if (o->forced_pivots[k] < 0 || o->forced_pivots[k] >= n) { set_error("forced pivot out of range"); return CD_EINVAL; }
  }
  int64_t Mmax = o->max_vectors > 0 ? std::min<int64_t>(o->max_vectors, n) : std::min<int64_t>(n, 16 * N);
  if (forced) Mmax = std::min<int64_t>(Mmax, std::max<int64_t>(nf, 1));
  Mmax = std::max<int64_t>(Mmax, 1);
  size_t freeb = 0, totb = 0;
  CD_CUDA(cudaMemGetInfo(&freeb, &totb));
  const double budget = o->mem_budget_gb > 0 ? o->mem_budget_gb * 1e9 : 0.9 * (double)freeb;
  // bytes per vector of capacity, and the fixed part
  const double per_vec = 8.0 * ld + (slice ? 2.0 * kSlices * (n + b) : 0.0);
  const double fixed = 8.0 * ld * (b + 2) + 8.0 * Mmax * b + (slice ? 8.0 * b * ld + 4.0 * n : 0.0);
  // the stores grow in place, so they start small (one vector per basis function)
  int64_t Mcap = std::min<int64_t>(Mmax, std::max<int64_t>(256, N));
  if (fixed + per_vec * Mcap > budget) {
    Mcap = (int64_t)((budget - fixed) / per_vec);
    if (Mcap < 1) { set_error("device memory budget too small for the decomposition"); return CD_ENOMEM; }
  }
  f->sys = s;
  f->n = n;
  f->ld = ld;
  f->vec_precision = o->vec_precision;
  // device-memory accounting: scratch comes from the default pool (its
  // high-water mark is reset here), the vector arrays from cudaMalloc
  cudaMemPool_t mpool = nullptr;
  uint64_t pool_used0 = 0;
  {
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&mpool, dev) == cudaSuccess) {
      uint64_t zero = 0;
      cudaMemPoolSetAttribute(mpool, cudaMemPoolAttrUsedMemHigh, &zero);
      cudaMemPoolGetAttribute(mpool, cudaMemPoolAttrUsedMemCurrent, &pool_used0);
    } else {
      mpool = nullptr;
      cudaGetLastError();
    }
  }
  Work w;
  w.st = st;
  CD_TRY(f->Lvm.reserve(sizeof(double) * (size_t)Mmax * ld));
  CD_TRY(f->Lvm.grow(sizeof(double) * (size_t)Mcap * ld));
  f->L = (double*)f->Lvm.base;
  f->Mcap = Mcap;
  CD_TRY(scratch_alloc(&w.pool, (size_t)b * ld, st));
  CD_TRY(scratch_alloc(&w.D0, (size_t)ld, st));
  CD_TRY(scratch_alloc(&w.D1, (size_t)ld, st));
  CD_TRY(scratch_alloc(&w.Bg, (size_t)Mmax * b, st));
  CD_TRY(scratch_alloc(&w.slots_dev, (size_t)b, st));
  CD_TRY(scratch_alloc(&w.rows_dev, (size_t)b, st));
  CD_TRY(scratch_alloc(&w.valid_dev, (size_t)b, st));
  CD_TRY(scratch_alloc(&w.kets_dev, (size_t)b, st));
  CD_TRY(scratch_alloc(&w.sc, 1, st));
  CD_TRY(scratch_alloc(&w.res_dev, 1, st));
  if (slice) {
    w.kcap = (Mcap + 31) / 32 * 32;
    CD_TRY(w.Lsvm.reserve(slice_chunk_bytes(n) * (size_t)((Mmax + 31) / 32)));
    CD_TRY(w.Lsvm.grow(slice_chunk_bytes(n) * (size_t)(w.kcap / 32)));
    w.Ls = w.Lsvm.base;
    CD_TRY(scratch_alloc((uint16_t**)&w.Bs, (size_t)kSlices * b * w.kcap, st));
    CD_TRY(scratch_alloc(&w.Dint, (size_t)b * ld, st));
    CD_TRY(scratch_alloc(&w.erow, (size_t)std::max<int64_t>(n, 1), st));
    CD_TRY(scratch_alloc(&w.err, 1, st));
    CD_CUDA(cudaMemsetAsync(w.err, 0, sizeof(int), st));
    CD_TRY(launch_row_exp_sqrt(s->diag_dev, n, w.erow, st));
  }
  const int cand_cap = 4 * b;
  // candidate mask (system rows).  The first step of the two-step scheme drops
  // the other rows at its first compaction and needs no mask afterwards.
  const uint8_t* cmask_h = o->candidates;
  const uint8_t* cmask = nullptr;
  if (cmask_h && n > 0) {
    CD_TRY(scratch_alloc(&w.cand_dev, (size_t)n, st));
    CD_CUDA(cudaMemcpyAsync(w.cand_dev, cmask_h, (size_t)n, cudaMemcpyHostToDevice, st));
    cmask = w.cand_dev;
  }
  if (span_mode) {
    CD_TRY(scratch_alloc(&w.slot_rows_dev, (size_t)b, st));
    CD_TRY(scratch_alloc(&w.slot_vals_dev, (size_t)b, st));
    w.slot_vals_h.resize(b);
  }
  CD_TRY(scratch_alloc(&w.sel, 1, st));
  CD_TRY(scratch_alloc(&w.eri_ops, 1, st));
  CD_CUDA(cudaMemsetAsync(w.eri_ops, 0, sizeof(unsigned long long), st));
  CD_TRY(scratch_alloc(&w.cand_rows, (size_t)cand_cap, st));
  CD_TRY(scratch_alloc(&w.cand_vals, (size_t)cand_cap, st));
  w.cand_rows_h.resize(cand_cap);
  w.cand_vals_h.resize(cand_cap);
  for (auto& e : w.ev) CD_CUDA(cudaEventCreate(&e));
  for (auto& x : w.eri.side) CD_CUDA(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  CD_TRY(scratch_alloc(&w.eri.counters, 3, st));
  CD_TRY(eri_resident_ctas(w.eri.resident, &w.eri.sms));
  // CDERI_OVERLAP_UPDATE=1 runs the sliced update beside the ERI columns.  Measured at
  // N = 2000 it is slower (12.5 s against 11.5 s per step: beside an ERI CTA the
  // update CTA runs at half speed, and the ERI grids at half occupancy), so the
  // default runs them in sequence
  const char* ov_env = getenv("CDERI_OVERLAP_UPDATE");
  const bool overlap = slice && ov_env && ov_env[0] == '1';
  if (overlap) {
    int upd_regs = 0;
    CD_TRY(update_cta_registers(&upd_regs));
    CD_TRY(eri_coresident_ctas(upd_regs, w.eri.primary));
    CD_CUDA(cudaEventCreateWithFlags(&w.eri.counters_ready, cudaEventDisableTiming));
    CD_CUDA(cudaEventCreateWithFlags(&w.eri.topup_done, cudaEventDisableTiming));
  }
  CD_CUDA(cudaEventCreateWithFlags(&w.eri.fork, cudaEventDisableTiming));
  for (auto& e : w.eri.join) CD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  // full pivoting runs the in-block steps on the device (CDERI_HOST_STEPS=1: one
  // host round trip per step instead)
  const bool dev_steps = !forced && !span_mode && !reduce && getenv("CDERI_HOST_STEPS") == nullptr;
  if (dev_steps) {
    CD_TRY(scratch_alloc(&w.ds_dev, 1, st));
    CD_TRY(scratch_alloc(&w.slot_of_row, (size_t)std::max<int64_t>(n, 1), st));
    CD_TRY(scratch_alloc(&w.piv_dev, (size_t)Mmax, st));
    CD_TRY(scratch_alloc(&w.pivd_dev, (size_t)Mmax, st));
    CD_TRY(scratch_alloc(&w.sm_rows, (size_t)b, st));
    CD_TRY(scratch_alloc(&w.sm_slots, (size_t)b, st));
    w.piv_h.resize(b);
    w.pivd_h.resize(b);
  }
  if (slice) {
    CD_CUDA(cudaStreamCreateWithFlags(&w.st2, cudaStreamNonBlocking));
    CD_CUDA(cudaEventCreateWithFlags(&w.ev_ready, cudaEventDisableTiming));
    CD_CUDA(cudaEventCreateWithFlags(&w.ev_gemm, cudaEventDisableTiming));
    CD_CUDA(cudaEventCreate(&w.ev_g0));
    CD_CUDA(cudaEventCreate(&w.ev_g1));
  }
  CD_CUDA(cudaMemsetAsync(w.sc, 0, sizeof(StepScratch), st));
  CD_CUDA(cudaMemsetAsync(w.pool, 0, sizeof(double) * b * ld, st));
  CD_CUDA(cudaMemsetAsync(w.D1, 0, sizeof(double) * ld, st));
  if (o->diag_shift != 0.0) {
    // test hook: the diagonal of A - shift I (host-made indefinite input)
    if (!std::isfinite(o->diag_shift)) { set_error("diag_shift must be finite"); return CD_EINVAL; }
    w.dh.assign(ld, 0.0);
    for (int64_t r = 0; r < n; ++r) w.dh[r] = s->row_diag[r] - o->diag_shift;
    CD_CUDA(cudaMemcpyAsync(w.D0, w.dh.data(), sizeof(double) * ld, cudaMemcpyHostToDevice, st));
    CD_CUDA(cudaStreamSynchronize(st));
  } else {
    CD_CUDA(cudaMemcpyAsync(w.D0, s->diag_dev, sizeof(double) * ld, cudaMemcpyDeviceToDevice, st));
  }
  double d1max = 0.0;
  for (double v : s->row_diag) d1max = std::max(d1max, v);
  const double neg_tol = -1e-10 * d1max;
  double* Dcur = w.D0;
  double* Dnext = w.D1;
  StepResult res;
  if (n > 0) {
    CD_TRY(launch_argmax(Dcur, n, w.sc, w.res_dev, st, cmask));
    CD_CUDA(cudaMemcpyAsync(w.res_h, w.res_dev, sizeof(StepResult), cudaMemcpyDeviceToHost, st));
    CD_CUDA(cudaStreamSynchronize(st));
    res = *w.res_h;
  } else {
    res.dmax = -1.0; res.idx = -1; res.bad = 0;
  }
  // ---- working rows.  All rows, or (two-step, first step) the rows whose
  // residual diagonal is still >= tau: a residual diagonal never increases, so a
  // row below tau can never be a pivot again and is dropped for good (Sec. 3);
  // every row-indexed buffer is then compacted to the live rows.
  std::vector<int64_t> grow;                  // working row -> system row (reduce)
  PairSet bra_v = s->bra;                     // bra shell pairs with rows mapped to working rows
  const int64_t* order_v = nullptr;
  int64_t cls_v[4] = {s->bra_class_off[0], s->bra_class_off[1], s->bra_class_off[2], s->bra_class_off[3]};
  auto sysrow = [&](int64_t r) -> int64_t { return reduce ? grow[r] : r; };
  std::vector<int64_t> slot_row(b, -1), slot_valid(b, 0);
  std::unordered_map<int64_t, int> row2slot;
  int64_t K = 0;
  // surviving bra primitive pairs per class (for the algorithmic ERI count);
  // recomputed from the live list after each compaction
  double bra_npp_cls[3] = {0.0, 0.0, 0.0};
  auto count_bra = [&](const std::vector<int64_t>* order_h) {
    for (int c = 0; c < 3; ++c) {
      bra_npp_cls[c] = 0.0;
      if (order_h) {
        for (int64_t i = cls_v[c]; i < cls_v[c + 1]; ++i) bra_npp_cls[c] += s->bra_npp_h[(*order_h)[i]];
      } else {
        for (int64_t k = s->bra_class_off[c]; k < s->bra_class_off[c + 1]; ++k) bra_npp_cls[c] += s->bra_npp_h[k];
      }
    }
  };
  count_bra(nullptr);
  // compacts when forced, or when fewer than 3/4 of the working rows are live
  auto compact_rows = [&](bool force) -> int {
    std::vector<double> dh(n);
    if (n > 0) CD_CUDA(cudaMemcpyAsync(dh.data(), Dcur, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    CD_CUDA(cudaStreamSynchronize(st));
    std::vector<int32_t> idx;
    for (int64_t r = 0; r < n; ++r)
      if (dh[r] >= tau && (!cmask_h || cmask_h[r])) idx.push_back((int32_t)r);
    const int64_t m = (int64_t)idx.size();
    if (!force && 4 * m >= 3 * n) return CD_OK;
    const int64_t ldm = std::max<int64_t>(32, (m + 31) / 32 * 32);
    int32_t* idx_dev = nullptr;
    CD_TRY(scratch_alloc(&idx_dev, (size_t)std::max<int64_t>(m, 1), st));
    if (m > 0) CD_CUDA(cudaMemcpyAsync(idx_dev, idx.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    VmArray nLvm;
    CD_TRY(nLvm.reserve(sizeof(double) * (size_t)Mmax * ldm));
    CD_TRY(nLvm.grow(sizeof(double) * (size_t)f->Mcap * ldm));
    double* nL = (double*)nLvm.base;
    CD_TRY(launch_compact_f64(f->L, ld, idx_dev, m, K, nL, ldm, st));
    double *npool = nullptr, *nD0 = nullptr, *nD1 = nullptr;
    CD_TRY(scratch_alloc(&npool, (size_t)b * ldm, st));
    CD_TRY(scratch_alloc(&nD0, (size_t)ldm, st));
    CD_TRY(scratch_alloc(&nD1, (size_t)ldm, st));
    CD_CUDA(cudaMemsetAsync(npool, 0, sizeof(double) * b * ldm, st));
    CD_CUDA(cudaMemsetAsync(nD0, 0, sizeof(double) * ldm, st));
    CD_CUDA(cudaMemsetAsync(nD1, 0, sizeof(double) * ldm, st));
    CD_TRY(launch_compact_f64(w.pool, ld, idx_dev, m, b, npool, ldm, st));
    CD_TRY(launch_compact_f64(Dcur, ld, idx_dev, m, 1, nD0, ldm, st));
    VmArray nLsvm;
    if (slice) {
      int32_t* nerow = nullptr;
      CD_TRY(nLsvm.reserve(slice_chunk_bytes(m) * (size_t)((Mmax + 31) / 32)));
      CD_TRY(nLsvm.grow(slice_chunk_bytes(m) * (size_t)(w.kcap / 32)));
      CD_TRY(scratch_alloc(&nerow, (size_t)std::max<int64_t>(m, 1), st));
      // every (chunk, slice) plane keeps the live rows, 64 bytes each
      CD_TRY(launch_compact_rows16(w.Ls, n, idx_dev, m, (int)((w.kcap / 32) * kSlices), 64, nLsvm.base, st));
      CD_TRY(launch_compact_i32(w.erow, idx_dev, m, nerow, st));
      scratch_free(w.erow, st);
      w.erow = nerow;
    }
    CD_CUDA(cudaStreamSynchronize(st));
    f->Lvm.swap(nLvm);        // the old stores are released when nLvm / nLsvm go out of scope
    f->L = (double*)f->Lvm.base;
    if (slice) {
      w.Lsvm.swap(nLsvm);
      w.Ls = w.Lsvm.base;
    }
    scratch_free(w.pool, st);
    scratch_free(w.D0, st);
    scratch_free(w.D1, st);
    scratch_free(idx_dev, st);
    w.pool = npool;
    w.D0 = Dcur = nD0;
    w.D1 = Dnext = nD1;
    // working <-> system rows, pool slots
    std::vector<int64_t> old2new(n, -1);
    for (int64_t i = 0; i < m; ++i) old2new[idx[i]] = i;
    std::vector<int64_t> ngrow(m);
    for (int64_t i = 0; i < m; ++i) ngrow[i] = grow.empty() ? idx[i] : grow[idx[i]];
    grow.swap(ngrow);
    row2slot.clear();
    for (int sl = 0; sl < b; ++sl) {
      if (slot_row[sl] < 0) continue;
      slot_row[sl] = old2new[slot_row[sl]];
      if (slot_row[sl] >= 0) row2slot[slot_row[sl]] = sl;
    }
    // bra components mapped to working rows; the shell pairs with a live row
    std::vector<int32_t> sys2w(s->n_rows, -1);
    for (int64_t i = 0; i < m; ++i) sys2w[grow[i]] = (int32_t)i;
    std::vector<int32_t> rmap(s->bra_row_h.size(), -1);
    std::vector<int64_t> order;
    int64_t co[4] = {0, 0, 0, 0};
    for (int c = 0; c < 3; ++c) {
      co[c] = (int64_t)order.size();
      for (int64_t k = s->bra_class_off[c]; k < s->bra_class_off[c + 1]; ++k) {
        bool any = false;
        for (int x = 0; x < 9; ++x) {
          const int32_t r = s->bra_row_h[9 * k + x];
          if (r >= 0 && sys2w[r] >= 0) { rmap[9 * k + x] = sys2w[r]; any = true; }
        }
        if (any) order.push_back(k);
      }
    }
    co[3] = (int64_t)order.size();
    scratch_free(w.rowmap_dev, st);
    scratch_free(w.order_dev, st);
    w.rowmap_dev = nullptr;
    w.order_dev = nullptr;
    CD_TRY(scratch_alloc(&w.rowmap_dev, std::max<size_t>(rmap.size(), 1), st));
    CD_TRY(scratch_alloc(&w.order_dev, std::max<size_t>(order.size(), 1), st));
    if (!rmap.empty())
      CD_CUDA(cudaMemcpyAsync(w.rowmap_dev, rmap.data(), sizeof(int32_t) * rmap.size(), cudaMemcpyHostToDevice, st));
    if (!order.empty())
      CD_CUDA(cudaMemcpyAsync(w.order_dev, order.data(), sizeof(int64_t) * order.size(), cudaMemcpyHostToDevice, st));
    bra_v.row = w.rowmap_dev;
    order_v = w.order_dev;
    for (int c = 0; c < 4; ++c) cls_v[c] = co[c];
    count_bra(&order);
    n = m;
    ld = ldm;
    f->n = n;
    f->ld = ld;
    cmask_h = nullptr;  // every working row is a candidate now
    cmask = nullptr;
    if (n > 0) {
      CD_TRY(launch_argmax(Dcur, n, w.sc, w.res_dev, st));
      CD_CUDA(cudaMemcpyAsync(w.res_h, w.res_dev, sizeof(StepResult), cudaMemcpyDeviceToHost, st));
    }
    CD_CUDA(cudaStreamSynchronize(st));
    if (n > 0) res = *w.res_h;
    else { res.dmax = -1.0; res.idx = -1; res.bad = 0; }
    return CD_OK;
  };
  if (reduce) CD_TRY(compact_rows(true));
  OzakiPlan plan;
  plan.SA = plan.SB = kSlices;
  plan.KEEP = kSlices + 1;
  plan.F = kSliceF;
  double t_eri = 0, t_upd = 0, t_sel = 0, t_steps = 0, upd_flops = 0, eri_ints = 0;
  int64_t nblocks = 0, ncols = 0;
  bool done = false;
  const bool dbg = getenv("CDERI_DEBUG") != nullptr;
  // The sliced update (tensor cores, HBM) and the ERI columns (FP64 pipe) use
  // different units: with `overlap` the update goes to the second stream and
  // the ERI grids are sized to leave every SM room for one update CTA (see
  // EriStreams); the ERI top-ups follow the update on that stream.  By default
  // the update runs on the main stream before the ERI columns.
  while (!done) {
    if (reduce && K > 0) CD_TRY(compact_rows(false));
    if (forced ? (K >= nf) : !(res.dmax >= tau)) break;
    // qualified threshold of this macro iteration (span policies)
    const double thr = span_mode ? std::max(span * res.dmax, tau) : tau;
    if (dbg) fprintf(stderr, "[cderi] block %lld K=%lld dmax=%.3e idx=%lld\n", (long long)nblocks, (long long)K,
                     res.dmax, (long long)res.idx);
    // ---- candidate block
    const double ts = now_ms();
    std::vector<int64_t> cand;
    if (forced) {
      for (int64_t k = K; k < nf && (int64_t)cand.size() < b; ++k)
        if (std::find(cand.begin(), cand.end(), o->forced_pivots[k]) == cand.end()) cand.push_back(o->forced_pivots[k]);
    } else {
      // the b largest residual diagonals >= tau (radix select on the device)
      CD_TRY(launch_select(Dcur, n, thr, b, w.sel, w.cand_rows, w.cand_vals, cand_cap, st, cmask));
      CD_CUDA(cudaMemcpyAsync(w.cand_count_h, &w.sel->count, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      CD_CUDA(cudaMemcpyAsync(w.cand_rows_h.data(), w.cand_rows, sizeof(int64_t) * cand_cap, cudaMemcpyDeviceToHost, st));
      CD_CUDA(cudaMemcpyAsync(w.cand_vals_h.data(), w.cand_vals, sizeof(double) * cand_cap, cudaMemcpyDeviceToHost, st));
      CD_CUDA(cudaStreamSynchronize(st));
      std::vector<std::pair<double, int64_t>> c;
      const unsigned cnt = *w.cand_count_h;
      if (cnt <= (unsigned)cand_cap) {
        for (unsigned i = 0; i < cnt; ++i) c.emplace_back(w.cand_vals_h[i], w.cand_rows_h[i]);
      } else {  // many exact ties at the threshold: full scan on the host
        w.dh.resize(n);
        CD_CUDA(cudaMemcpyAsync(w.dh.data(), Dcur, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
        CD_CUDA(cudaStreamSynchronize(st));
        for (int64_t r = 0; r < n; ++r)
          if (w.dh[r] >= thr && (!cmask_h || cmask_h[r])) c.emplace_back(w.dh[r], r);
      }
      auto cmp = [](const std::pair<double, int64_t>& x, const std::pair<double, int64_t>& y) {
        return x.first > y.first || (x.first == y.first && x.second < y.second);
      };
      if ((int64_t)c.size() > b) {
        std::nth_element(c.begin(), c.begin() + b, c.end(), cmp);
        c.resize(b);
      }
      std::sort(c.begin(), c.end(), cmp);
      for (auto& x : c) cand.push_back(x.second);
    }
    t_sel += now_ms() - ts;
    // ---- pool: keep columns still wanted, free the rest
    std::unordered_map<int64_t, int> want;
    for (size_t j = 0; j < cand.size(); ++j) want[cand[j]] = (int)j;
    for (int sl = 0; sl < b; ++sl)
      if (slot_row[sl] >= 0 && !want.count(slot_row[sl])) {
        row2slot.erase(slot_row[sl]);
        slot_row[sl] = -1;
      }
    std::vector<KetDesc> kets;
    int free_sl = 0;
    for (int64_t r : cand) {
      if (row2slot.count(r)) continue;
      while (slot_row[free_sl] >= 0) ++free_sl;
      slot_row[free_sl] = r;
      slot_valid[free_sl] = 0;
      row2slot[r] = free_sl;
      kets.push_back(ket_of_row(s, sysrow(r), free_sl));
    }
    ++nblocks;
    ncols += (int64_t)kets.size();
    // ---- sliced update of every pool column with vectors [valid, K): on the
    // second stream, overlapping the ERI columns below
    bool gemm_issued = false;
    int nb_upd = 0;
    if (slice) {
      w.upd_slots.clear(); w.upd_rows.clear(); w.upd_valid.clear();
      for (int x = 0; x < b; ++x)
        if (slot_row[x] >= 0 && slot_valid[x] < K) {
          w.upd_slots.push_back(x); w.upd_rows.push_back(slot_row[x]); w.upd_valid.push_back(slot_valid[x]);
        }
      nb_upd = (int)w.upd_slots.size();
      if (nb_upd > 0 && K > 0) {
        cudaStream_t s2 = overlap ? w.st2 : st;
        CD_CUDA(cudaEventRecord(w.ev_ready, st));      // slices of the last block are written
        CD_CUDA(cudaStreamWaitEvent(s2, w.ev_ready, 0));
        CD_CUDA(cudaEventRecord(w.ev_g0, s2));
        CD_CUDA(cudaMemcpyAsync(w.slots_dev, w.upd_slots.data(), sizeof(int32_t) * nb_upd, cudaMemcpyHostToDevice, s2));
        CD_CUDA(cudaMemcpyAsync(w.rows_dev, w.upd_rows.data(), sizeof(int64_t) * nb_upd, cudaMemcpyHostToDevice, s2));
        CD_CUDA(cudaMemcpyAsync(w.valid_dev, w.upd_valid.data(), sizeof(int64_t) * nb_upd, cudaMemcpyHostToDevice, s2));
        CD_TRY(launch_gather_slices(w.Ls, n, w.rows_dev, w.valid_dev, nb_upd, kSlices, K, w.Bs, w.kcap, s2));
        CD_CUDA(cudaMemsetAsync(w.Dint, 0, sizeof(unsigned long long) * nb_upd * ld, s2));
        CD_TRY(ozaki_gemm(plan, w.Ls, n, w.kcap, w.Bs, nb_upd, w.kcap, K, w.Dint, ld, 1, w.err, s2, false, true));
        CD_CUDA(cudaEventRecord(w.ev_g1, s2));
        CD_CUDA(cudaEventRecord(w.ev_gemm, s2));
        for (int x = 0; x < nb_upd; ++x) upd_flops += 2.0 * (double)n * (double)(K - w.upd_valid[x]);
        gemm_issued = true;
      }
    }
    CD_CUDA(cudaEventRecord(w.ev[0], st));
    std::vector<KetGroup> groups = group_kets(kets);
    if (!kets.empty()) {
      CD_CUDA(cudaMemcpyAsync(w.kets_dev, groups.data(), sizeof(KetGroup) * groups.size(), cudaMemcpyHostToDevice, st));
      w.eri.topup = (overlap && gemm_issued) ? w.st2 : nullptr;
      CD_TRY(launch_eri_columns(bra_v, order_v, cls_v, s->all, w.kets_dev, (int)groups.size(), w.pool, ld,
                                s->boys, st, w.eri_ops, getenv("CDERI_ERI_SERIAL") ? nullptr : &w.eri));
      eri_ints += (double)kets.size() * (double)n;
      // algorithmic work of the launch: per bra class, its primitive pairs x each group's ket primitive pairs
      for (const KetGroup& g : groups) {
        const double npk = (double)s->all_npp_h[g.sp];
        for (int c = 0; c < 3; ++c) {
          const double q = bra_npp_cls[c] * npk;
          f->eri_quartets += q;
          f->eri_alg_ops += q * eri_alg_ops_per_quartet(c, g.lc + g.ld, g.nc);
        }
      }
    }
    CD_CUDA(cudaEventRecord(w.ev[1], st));
    if (slice) {
      if (gemm_issued) {
        CD_CUDA(cudaStreamWaitEvent(st, w.ev_gemm, 0));
        CD_TRY(launch_colupd_finalize(w.Dint, ld, n, nb_upd, w.erow, w.rows_dev, w.slots_dev, plan.F, w.pool, ld, st));
        int herr_blk = 0;
        CD_CUDA(cudaMemcpyAsync(&herr_blk, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        CD_CUDA(cudaStreamSynchronize(st));  // host copies of the group vectors are complete
        if (herr_blk) {  // an incomplete update must not feed the pivot steps
          set_error("tensor-core update: a bounded pipeline wait timed out (wait bits " + std::to_string(herr_blk) + ")");
          return CD_ETIMEOUT;
        }
      }
    } else {
      std::unordered_map<int64_t, std::vector<int>> groups;
      for (int sl = 0; sl < b; ++sl)
        if (slot_row[sl] >= 0 && slot_valid[sl] < K) groups[slot_valid[sl]].push_back(sl);
      for (auto& g : groups) {
        const int64_t k0 = g.first;
        std::vector<int32_t> sl(g.second.begin(), g.second.end());
        std::vector<int64_t> rr;
        for (int x : sl) rr.push_back(slot_row[x]);
        const int nb = (int)sl.size();
        CD_CUDA(cudaMemcpyAsync(w.slots_dev, sl.data(), sizeof(int32_t) * nb, cudaMemcpyHostToDevice, st));
        CD_CUDA(cudaMemcpyAsync(w.rows_dev, rr.data(), sizeof(int64_t) * nb, cudaMemcpyHostToDevice, st));
        CD_TRY(launch_gather(f->L, ld, w.rows_dev, nb, k0, K, w.Bg, st));
        CD_TRY(launch_colupd(w.pool, ld, w.slots_dev, nb, f->L, k0, K, w.Bg, n, st));
        upd_flops += 2.0 * (double)n * nb * (double)(K - k0);
        CD_CUDA(cudaStreamSynchronize(st));
      }
    }
    CD_CUDA(cudaEventRecord(w.ev[2], st));
    for (int sl = 0; sl < b; ++sl)
      if (slot_row[sl] >= 0) slot_valid[sl] = K;
    const int64_t Kb = K;
    bool first = true;
    if (span_mode) {  // residual diagonals of the block's columns
      CD_CUDA(cudaMemcpyAsync(w.slot_rows_dev, slot_row.data(), sizeof(int64_t) * b, cudaMemcpyHostToDevice, st));
      CD_TRY(launch_gather_vals(Dcur, w.slot_rows_dev, b, w.slot_vals_dev, st));
      CD_CUDA(cudaMemcpyAsync(w.slot_vals_h.data(), w.slot_vals_dev, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
    }
    CD_CUDA(cudaStreamSynchronize(st));  // columns of this block are complete
    const double t_blk = now_ms();
    if (dev_steps) {
      // ---- the block's pivot steps on the device: one upload of the state,
      // one graph launch of b step kernels, one read-back
      std::vector<int64_t> srows;
      std::vector<int32_t> sslots;
      for (int sl = 0; sl < b; ++sl)
        if (slot_row[sl] >= 0) { srows.push_back(slot_row[sl]); sslots.push_back(sl); }
      const int nocc = (int)srows.size();
      if (K + nocc > f->Mcap && f->Mcap < Mmax) {
        int64_t nc = grown_capacity(K + nocc, f->Mcap, Mmax);
        if (fixed + per_vec * nc > budget) nc = (int64_t)((budget - fixed) / per_vec);
        if (nc > f->Mcap) CD_TRY(grow_vectors(f, &w, slice, b, nc, K, st));
      }
      if (nocc > 0) {
        CD_CUDA(cudaMemcpyAsync(w.sm_rows, srows.data(), sizeof(int64_t) * nocc, cudaMemcpyHostToDevice, st));
        CD_CUDA(cudaMemcpyAsync(w.sm_slots, sslots.data(), sizeof(int32_t) * nocc, cudaMemcpyHostToDevice, st));
      }
      CD_TRY(launch_slot_map(w.slot_of_row, n, w.sm_rows, w.sm_slots, nocc, st));
      w.ds_h.res = res;
      w.ds_h.K = K;
      w.ds_h.Kb = K;
      w.ds_h.Kcap = f->Mcap;
      w.ds_h.Dcur0 = Dcur;
      w.ds_h.Dnext0 = Dnext;
      w.ds_h.tau = tau;
      w.ds_h.done = 0;
      w.ds_h.reason = 0;
      CD_CUDA(cudaMemcpyAsync(w.ds_dev, &w.ds_h, sizeof(DevStep), cudaMemcpyHostToDevice, st));
      if (!w.step_exec || w.step_key[0] != f->L || w.step_key[1] != w.pool) {
        if (w.step_exec) { cudaGraphExecDestroy(w.step_exec); w.step_exec = nullptr; }
        CD_TRY(build_step_graph(&w.step_exec, b, w.ds_dev, w.slot_of_row, w.pool, f->L, ld, n, neg_tol, cmask,
                                w.piv_dev, w.pivd_dev, w.sc));
        w.step_key[0] = f->L;
        w.step_key[1] = w.pool;
      }
      CD_CUDA(cudaGraphLaunch(w.step_exec, st));
      count_launch(b);
      CD_CUDA(cudaMemcpyAsync(&w.ds_h, w.ds_dev, sizeof(DevStep), cudaMemcpyDeviceToHost, st));
      // at most min(nocc, Mcap - K) steps can have run (piv_dev holds Mmax >= Mcap entries)
      const int64_t ncopy = std::min<int64_t>(nocc, f->Mcap - K);
      if (ncopy > 0) {
        CD_CUDA(cudaMemcpyAsync(w.piv_h.data(), w.piv_dev + K, sizeof(int64_t) * ncopy, cudaMemcpyDeviceToHost, st));
        CD_CUDA(cudaMemcpyAsync(w.pivd_h.data(), w.pivd_dev + K, sizeof(double) * ncopy, cudaMemcpyDeviceToHost, st));
      }
      CD_CUDA(cudaStreamSynchronize(st));
      const int64_t Knew = w.ds_h.K;
      if (Knew < K || Knew > K + std::max<int64_t>(ncopy, 0)) {
        set_error("internal: device step count out of range");
        return CD_EINVAL;
      }
      for (int64_t k = K; k < Knew; ++k) {
        const int64_t p = w.piv_h[k - K];
        f->piv.push_back(p);
        f->gaps.push_back(0.0);
        f->pivd.push_back(w.pivd_h[k - K]);
        auto it = row2slot.find(p);
        if (it == row2slot.end()) { set_error("internal: device step took a row outside the block"); return CD_EINVAL; }
        slot_row[it->second] = -1;
        row2slot.erase(it);
      }
      if ((Knew - K) & 1) std::swap(Dcur, Dnext);
      res = w.ds_h.res;
      const bool stepped = Knew > K;
      K = Knew;
      if (stepped) {
        float a = 0, c = 0;
        cudaEventElapsedTime(&a, w.ev[0], w.ev[1]);
        if (slice) {
          if (gemm_issued) cudaEventElapsedTime(&c, w.ev_g0, w.ev_g1);
        } else {
          cudaEventElapsedTime(&c, w.ev[1], w.ev[2]);
        }
        t_eri += a;
        t_upd += c;
        first = false;
      }
      const int reason = w.ds_h.done ? w.ds_h.reason : 0;
      if (reason == kStepNotPsd) {
        if (res.bad) set_error("residual diagonal below -1e-10 max D (matrix not PSD) after step " + std::to_string(K));
        else set_error("pivot diagonal not positive (matrix not PSD) at step " + std::to_string(K));
        return CD_ENOTPSD;
      }
      if (reason == kStepCapacity) {
        if (f->Mcap >= Mmax) set_error("number of vectors exceeds max_vectors = " + std::to_string(Mmax));
        else set_error("device memory budget exhausted at M = " + std::to_string(K));
        return CD_ENOMEM;
      }
      if (reason == kStepConverged) done = true;
    } else
    // ---- serial pivot steps inside the block, one host round trip each
    for (;;) {
      int64_t p;
      double dp;
      if (forced) {
        if (K >= nf) { done = true; break; }
        p = o->forced_pivots[K];
      } else if (span_mode) {
        if (!(res.dmax >= tau)) { done = true; break; }
        // the largest residual diagonal among the block's unused columns (ties:
        // lowest row); the macro iteration ends when it is below the threshold
        int best = -1;
        for (int x = 0; x < b; ++x) {
          if (slot_row[x] < 0) continue;
          const double v = w.slot_vals_h[x];
          if (best < 0 || v > w.slot_vals_h[best] || (v == w.slot_vals_h[best] && slot_row[x] < slot_row[best]))
            best = x;
        }
        if (best < 0 || !(w.slot_vals_h[best] >= thr)) break;
        p = slot_row[best];
      } else {
        if (!(res.dmax >= tau)) { done = true; break; }
        p = res.idx;
      }
      auto it = row2slot.find(p);
      if (it == row2slot.end()) break;  // argmax outside the block: new block
      const int sl = it->second;
      if (forced) {
        CD_CUDA(cudaMemcpyAsync(w.dp_h, Dcur + p, sizeof(double), cudaMemcpyDeviceToHost, st));
        CD_CUDA(cudaStreamSynchronize(st));
        dp = *w.dp_h;
      } else if (span_mode) {
        dp = w.slot_vals_h[sl];
      } else {
        dp = res.dmax;
      }
      if (!(dp > 0.0)) {
        set_error("pivot diagonal not positive (matrix not PSD) at step " + std::to_string(K));
        return CD_ENOTPSD;
      }
      if (K >= f->Mcap) {
        if (f->Mcap >= Mmax) {
          set_error("number of vectors exceeds max_vectors = " + std::to_string(Mmax));
          return CD_ENOMEM;
        }
        int64_t nc = grown_capacity(K + 1, f->Mcap, Mmax);
        if (fixed + per_vec * nc > budget) nc = (int64_t)((budget - fixed) / per_vec);
        if (nc <= f->Mcap) { set_error("device memory budget exhausted at M = " + std::to_string(K)); return CD_ENOMEM; }
        CD_TRY(grow_vectors(f, &w, slice, b, nc, K, st));
      }
      const double gap = forced ? res.dmax - dp : 0.0;
      CD_TRY(launch_finalize(w.pool + (int64_t)sl * ld, f->L, ld, Kb, K, p, Dcur, Dnext, f->L + K * ld, n, neg_tol,
                             w.sc, w.res_dev, st, cmask));
      CD_CUDA(cudaMemcpyAsync(w.res_h, w.res_dev, sizeof(StepResult), cudaMemcpyDeviceToHost, st));
      if (span_mode) {
        CD_TRY(launch_gather_vals(Dnext, w.slot_rows_dev, b, w.slot_vals_dev, st));
        CD_CUDA(cudaMemcpyAsync(w.slot_vals_h.data(), w.slot_vals_dev, sizeof(double) * b, cudaMemcpyDeviceToHost, st));
      }
      CD_CUDA(cudaStreamSynchronize(st));
      if (first) {
        float a = 0, c = 0;
        cudaEventElapsedTime(&a, w.ev[0], w.ev[1]);
        if (slice) {
          if (gemm_issued) cudaEventElapsedTime(&c, w.ev_g0, w.ev_g1);
        } else {
          cudaEventElapsedTime(&c, w.ev[1], w.ev[2]);
        }
        t_eri += a;
        t_upd += c;
        first = false;
      }
      res = *w.res_h;
      std::swap(Dcur, Dnext);
      f->piv.push_back(sysrow(p));
      f->gaps.push_back(gap);
      f->pivd.push_back(dp);
      ++K;
      row2slot.erase(it);
      slot_row[sl] = -1;
      if (res.bad) {
        set_error("residual diagonal below -1e-10 max D (matrix not PSD) after step " + std::to_string(K));
        return CD_ENOTPSD;
      }
    }
    t_steps += now_ms() - t_blk;
    if (first && !done && !forced) {
      // the argmax row is always among the block's candidates; a block without a
      // step would repeat forever
      CD_CUDA(cudaStreamSynchronize(st));
      set_error("internal: candidate selection missed the pivot row " + std::to_string(res.idx) + " at step " +
                std::to_string(K));
      return CD_EINVAL;
    }
    if (first) {  // block ended without a step (only possible with a forced list)
      CD_CUDA(cudaStreamSynchronize(st));
      float a = 0, c = 0;
      cudaEventElapsedTime(&a, w.ev[0], w.ev[1]);
      if (slice) {
        if (gemm_issued) cudaEventElapsedTime(&c, w.ev_g0, w.ev_g1);
      } else {
        cudaEventElapsedTime(&c, w.ev[1], w.ev[2]);
      }
      t_eri += a;
      t_upd += c;
      if (forced && K < nf && !row2slot.count(o->forced_pivots[K])) {
        set_error("internal: forced pivot not in block");
        return CD_EINVAL;
      }
    }
    // slices of this block's vectors, for the next block's update
    if (slice && !done && K > Kb)
      CD_TRY(launch_slice_rows_f64(f->L + Kb * ld, 1, ld, n, K - Kb, w.erow, kSlices, w.Ls, n, w.kcap, Kb, st, true));
  }
  if (slice) {
    int herr = 0;
    CD_CUDA(cudaMemcpyAsync(&herr, w.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CD_CUDA(cudaStreamSynchronize(st));
    if (herr) {
      set_error("tensor-core update: a bounded pipeline wait timed out (wait bits " + std::to_string(herr) + ")");
      return CD_ETIMEOUT;
    }
  }
  f->M = K;
  f->resid_max = res.dmax;
  f->resid.resize(n);
  if (n > 0) {
    CD_CUDA(cudaMemcpyAsync(f->resid.data(), Dcur, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  }
  // the slice store is no longer needed: release it before the FP32 copy
  CD_CUDA(cudaStreamSynchronize(st));
  if (mpool) {
    uint64_t high = 0;
    cudaMemPoolGetAttribute(mpool, cudaMemPoolAttrUsedMemHigh, &high);
    // the slice and vector stores are both at their largest at the end of the loop
    f->mem_peak = (double)(high > pool_used0 ? high - pool_used0 : 0) + (double)f->Lvm.mapped + (double)w.Lsvm.mapped;
  }
  w.Lsvm.release();
  w.Ls = nullptr;
  scratch_free(w.Bs, st); w.Bs = nullptr;
  scratch_free(w.pool, st); w.pool = nullptr;
  if (f->vec_precision == CD_VEC_FP32 && K > 0) {
    // the stored vectors become FP32: the FP64 array is released once the copy is made
    CD_TRY(dalloc(&f->L32, (size_t)K * ld));
    CD_TRY(launch_to_fp32(f->L, ld, K, ld, f->L32, st));
    f->mem_peak = std::max(f->mem_peak, (double)f->Lvm.mapped + 4.0 * (double)K * ld);
    CD_CUDA(cudaStreamSynchronize(st));
    f->Lvm.release();
    f->L = nullptr;
  }
  f->mem_resident = (double)f->Lvm.mapped + (f->L32 ? 4.0 * (double)K * ld : 0.0);
  CD_CUDA(cudaStreamSynchronize(st));
  const double t_all = now_ms() - t_start;
  f->stats[0] = s->ms_setup;
  f->stats[1] = t_eri;
  f->stats[2] = t_upd;
  f->stats[3] = t_steps;
  f->stats[4] = t_sel;
  f->stats[5] = t_all;
  f->stats[6] = (double)nblocks;
  f->stats[7] = (double)ncols;
  f->stats[8] = upd_flops;
  f->stats[9] = eri_ints;
  f->stats[10] = (double)K;
  f->stats[11] = slice ? 1.0 : 0.0;
  {
    unsigned long long ops = 0;
    CD_CUDA(cudaMemcpy(&ops, w.eri_ops, sizeof(ops), cudaMemcpyDeviceToHost));
    f->stats[12] = (double)ops;
  }
  return CD_OK;
}

// ---------------------------------------------------------------- C ABI ----
extern "C" {

const char* cd_last_error(void) { return g_err.c_str(); }
const char* cd_version(void) { return "cderi 0.1 (sm_103a)"; }

int cd_system_create(const cd_basis_t* basis, double schwarz, void* stream, cd_system_t** out) {
  if (!out) { set_error("out is NULL"); return CD_EINVAL; }
  *out = nullptr;
  cd_system* s = nullptr;
  int rc = system_create_impl(basis, schwarz, (cudaStream_t)stream, &s);
  if (rc == CD_OK) *out = s;
  return rc;
}

void cd_system_free(cd_system_t* sys) { system_release(sys); }

int cd_system_info(const cd_system_t* s, int32_t* n_basis, int64_t* n_rows, int64_t* n_shell_pairs) {
  if (!s) { set_error("system is NULL"); return CD_EINVAL; }
  if (n_basis) *n_basis = s->hb.nbf;
  if (n_rows) *n_rows = s->n_rows;
  if (n_shell_pairs) *n_shell_pairs = s->bra.n;
  return CD_OK;
}

int cd_system_rows(const cd_system_t* s, int64_t* packed, double* diag) {
  if (!s) { set_error("system is NULL"); return CD_EINVAL; }
  if (packed) std::memcpy(packed, s->row_packed.data(), sizeof(int64_t) * s->n_rows);
  if (diag) std::memcpy(diag, s->row_diag.data(), sizeof(double) * s->n_rows);
  return CD_OK;
}

int cd_eri_columns(const cd_system_t* s, const int64_t* cols, int32_t ncols, double* out, int64_t ld, void* stream) {
  if (!s || !out || (ncols > 0 && !cols) || ncols < 0) { set_error("cd_eri_columns: bad argument"); return CD_EINVAL; }
  if (ld < s->n_rows) { set_error("cd_eri_columns: ld < n_rows"); return CD_EINVAL; }
  if (ncols == 0) return CD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<KetDesc> k(ncols);
  for (int j = 0; j < ncols; ++j) {
    if (cols[j] < 0 || cols[j] >= s->n_rows) { set_error("cd_eri_columns: column row out of range"); return CD_EINVAL; }
    k[j] = ket_of_row(s, cols[j], j);
  }
  std::vector<KetGroup> g = group_kets(k);
  KetGroup* kd = nullptr;
  CD_TRY(scratch_alloc(&kd, g.size(), st));
  int rc = CD_OK;
  if (cudaMemcpyAsync(kd, g.data(), sizeof(KetGroup) * g.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) rc = CD_ECUDA;
  if (rc == CD_OK) rc = launch_eri_columns(s->bra, nullptr, s->bra_class_off, s->all, kd, (int)g.size(), out, ld, s->boys, st);
  if (rc == CD_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = CD_ECUDA;
  if (rc == CD_ECUDA) set_error("cd_eri_columns: CUDA failure");
  scratch_free(kd, st);
  return rc;
}

int cd_eri_factor_sys(cd_system_t* sys, const cd_opts_t* opts, void* stream, cd_factor_t** out) {
  if (!out) { set_error("out is NULL"); return CD_EINVAL; }
  *out = nullptr;
  if (!sys || !opts) { set_error("system or opts is NULL"); return CD_EINVAL; }
  if (opts->algorithm < CD_ALG_FULL || opts->algorithm > CD_ALG_TWOSTEP) { set_error("bad algorithm"); return CD_EINVAL; }
  cd_factor* f = new cd_factor();
  int rc = CD_OK;
  if (opts->algorithm == CD_ALG_TWOSTEP) {
    // step 1: the Cholesky basis, by the span policy on the rows still >= tau
    const double t0 = now_ms();
    if (opts->forced_pivots) { set_error("forced pivots need CD_ALG_FULL"); delete f; return CD_EINVAL; }
    cd_factor* f1 = new cd_factor();
    cd_opts_t o1 = *opts;
    o1.algorithm = CD_ALG_SPAN;
    o1.vec_precision = CD_FP64;
    rc = factor_impl(sys, &o1, (cudaStream_t)stream, f1, true);
    std::vector<int64_t> basis = f1->piv;
    const double s1_blocks = f1->stats[6], s1_cols = f1->stats[7];
    cudaStreamSynchronize((cudaStream_t)stream);
    factor_release(f1);
    const double t1 = now_ms() - t0;
    // step 2: the vectors of that basis over every row, Eq. (CVsLT)
    if (rc == CD_OK) {
      cd_opts_t o2 = *opts;
      o2.algorithm = CD_ALG_FULL;
      o2.forced_pivots = basis.data();
      o2.n_forced = (int64_t)basis.size();
      rc = factor_impl(sys, &o2, (cudaStream_t)stream, f);
    }
    if (rc == CD_OK) {
      f->stats[5] += t1;
      f->stats[13] = t1;
      f->stats[14] = s1_blocks;
      f->stats[15] = s1_cols;
    }
  } else {
    rc = factor_impl(sys, opts, (cudaStream_t)stream, f);
  }
  if (rc != CD_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    factor_release(f);
    return rc;
  }
  *out = f;
  return CD_OK;
}

int cd_eri_factor(const cd_basis_t* basis, const cd_opts_t* opts, void* stream, cd_factor_t** out) {
  if (!out) { set_error("out is NULL"); return CD_EINVAL; }
  *out = nullptr;
  if (!opts) { set_error("opts is NULL"); return CD_EINVAL; }
  cd_system* s = nullptr;
  CD_TRY(cd_system_create(basis, opts->schwarz, stream, &s));
  cd_factor* f = nullptr;
  int rc = cd_eri_factor_sys(s, opts, stream, &f);
  if (rc != CD_OK) { system_release(s); return rc; }
  f->owns_sys = true;
  *out = f;
  return CD_OK;
}

void cd_factor_free(cd_factor_t* f) { factor_release(f); }

int cd_factor_info(const cd_factor_t* f, int64_t* M, int64_t* n_rows, int32_t* n_basis, double* resid) {
  if (!f) { set_error("factor is NULL"); return CD_EINVAL; }
  if (M) *M = f->M;
  if (n_rows) *n_rows = f->n;
  if (n_basis) *n_basis = f->sys->hb.nbf;
  if (resid) *resid = f->resid_max;
  return CD_OK;
}

int cd_factor_pivots(const cd_factor_t* f, int64_t* piv_rows, int64_t* piv_packed, double* gaps, double* resid_diag) {
  if (!f) { set_error("factor is NULL"); return CD_EINVAL; }
  for (int64_t k = 0; k < f->M; ++k) {
    if (piv_rows) piv_rows[k] = f->piv[k];
    if (piv_packed) piv_packed[k] = f->sys->row_packed[f->piv[k]];
    if (gaps) gaps[k] = f->gaps[k];
  }
  if (resid_diag && f->n > 0) std::memcpy(resid_diag, f->resid.data(), sizeof(double) * f->n);
  return CD_OK;
}

int cd_factor_eri_work(const cd_factor_t* f, double* quartets, double* algorithmic_ops) {
  if (!f) { set_error("cd_factor_eri_work: factor is NULL"); return CD_EINVAL; }
  if (quartets) *quartets = f->eri_quartets;
  if (algorithmic_ops) *algorithmic_ops = f->eri_alg_ops;
  return CD_OK;
}

int cd_factor_memory(const cd_factor_t* f, double* peak_bytes, double* resident_bytes) {
  if (!f) { set_error("cd_factor_memory: factor is NULL"); return CD_EINVAL; }
  if (peak_bytes) *peak_bytes = f->mem_peak;
  if (resident_bytes) *resident_bytes = f->mem_resident;
  return CD_OK;
}

int cd_factor_pivot_diag(const cd_factor_t* f, double* out) {
  if (!f || (f->M > 0 && !out)) { set_error("cd_factor_pivot_diag: bad argument"); return CD_EINVAL; }
  if (f->M > 0) std::memcpy(out, f->pivd.data(), sizeof(double) * f->M);
  return CD_OK;
}

int cd_factor_vectors(const cd_factor_t* f, double* L_host, const void** L_dev, int64_t* ld, int32_t* dtype) {
  if (!f) { set_error("factor is NULL"); return CD_EINVAL; }
  const bool f32 = f->vec_precision == CD_VEC_FP32 && f->L32;
  if (L_dev) *L_dev = f32 ? (const void*)f->L32 : (const void*)f->L;
  if (ld) *ld = f->ld;
  if (dtype) *dtype = f32 ? 1 : 0;
  if (L_host && f->M > 0) {
    if (f32) {
      std::vector<float> tmp((size_t)f->M * f->ld);
      CD_CUDA(cudaMemcpy(tmp.data(), f->L32, sizeof(float) * tmp.size(), cudaMemcpyDeviceToHost));
      for (int64_t k = 0; k < f->M; ++k)
        for (int64_t r = 0; r < f->n; ++r) L_host[k * f->n + r] = tmp[(size_t)k * f->ld + r];
    } else {
      CD_CUDA(cudaMemcpy2D(L_host, sizeof(double) * f->n, f->L, sizeof(double) * f->ld, sizeof(double) * f->n, f->M,
                           cudaMemcpyDeviceToHost));
    }
  }
  return CD_OK;
}

int cd_factor_gather(const cd_factor_t* f, const int64_t* rows, int32_t nrows, double* out) {
  if (!f || (nrows > 0 && (!rows || !out)) || nrows < 0) { set_error("cd_factor_gather: bad argument"); return CD_EINVAL; }
  if (nrows == 0 || f->M == 0) return CD_OK;
  for (int32_t j = 0; j < nrows; ++j)
    if (rows[j] < 0 || rows[j] >= f->n) { set_error("cd_factor_gather: row out of range"); return CD_EINVAL; }
  int64_t* rd = nullptr;
  double* od = nullptr;
  CD_TRY(dalloc(&rd, (size_t)nrows));
  int rc = dalloc(&od, (size_t)nrows * f->M);
  if (rc != CD_OK) { cudaFree(rd); return rc; }
  rc = CD_ECUDA;
  if (cudaMemcpy(rd, rows, sizeof(int64_t) * nrows, cudaMemcpyHostToDevice) == cudaSuccess &&
      (f->L ? launch_gather(f->L, f->ld, rd, nrows, 0, f->M, od, nullptr)
            : launch_gather(f->L32, f->ld, rd, nrows, 0, f->M, od, nullptr)) == CD_OK &&
      cudaMemcpy(out, od, sizeof(double) * nrows * f->M, cudaMemcpyDeviceToHost) == cudaSuccess)
    rc = CD_OK;
  if (rc != CD_OK) set_error("cd_factor_gather: CUDA failure");
  cudaFree(rd);
  cudaFree(od);
  return rc;
}

int cd_factor_stats(const cd_factor_t* f, double* stats16) {
  if (!f || !stats16) { set_error("cd_factor_stats: bad argument"); return CD_EINVAL; }
  std::memcpy(stats16, f->stats, sizeof(f->stats));
  return CD_OK;
}

long long cd_kernel_launches(void) { return cd::launch_counter(); }

int cd_jk(const cd_factor_t* f, const double* C_occ, int32_t n_occ, double* J, double* K, int32_t mode, void* stream) {
  if (!f || !C_occ || n_occ <= 0) { set_error("cd_jk: bad argument"); return CD_EINVAL; }
  const int m = mode & 0xff;
  const bool dev = (mode & CD_JK_DEVICE) != 0;
  const bool wantJ = !(mode & CD_JK_ONLY_K), wantK = !(mode & CD_JK_ONLY_J);
  if ((wantJ && !J) || (wantK && !K)) { set_error("cd_jk: J or K is NULL"); return CD_EINVAL; }
  if (m != CD_JK_FP64 && m != CD_JK_BF16X3 && m != CD_JK_BF16X4 && m != CD_JK_BF16X5) {
    set_error("cd_jk: unknown mode");
    return CD_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int N = f->sys->hb.nbf, O = n_occ;
  const int64_t n = f->n, M = f->M, ld = f->ld;
  double *dC = nullptr, *dJ = nullptr, *dK = nullptr, *d = nullptr, *v = nullptr, *Jp = nullptr;
  double *Lfull = nullptr, *B = nullptr;
  int rc = CD_OK;
  auto fail = [&](int code) {
    if (!dev) { scratch_free(dC, st); scratch_free(dJ, st); scratch_free(dK, st); }
    for (void* p : {(void*)d, (void*)v, (void*)Jp, (void*)Lfull, (void*)B}) scratch_free(p, st);
    cudaStreamSynchronize(st);
    return code;
  };
  if (dev) {
    dC = const_cast<double*>(C_occ);
    dJ = J;
    dK = K;
  } else {
    if ((rc = scratch_alloc(&dC, (size_t)N * O, st)) != CD_OK) return fail(rc);
    if (wantJ && (rc = scratch_alloc(&dJ, (size_t)N * N, st)) != CD_OK) return fail(rc);
    if (wantK && (rc = scratch_alloc(&dK, (size_t)N * N, st)) != CD_OK) return fail(rc);
    if (cudaMemcpyAsync(dC, C_occ, sizeof(double) * N * O, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_error("cd_jk: copy of C_occ failed");
      return fail(CD_ECUDA);
    }
  }
  if (m == CD_JK_BF16X3 || m == CD_JK_BF16X4 || m == CD_JK_BF16X5) {
    // the stored precision of the vectors decides what is sliced: the FP32 copy
    // when the factor keeps one, otherwise the FP64 vectors themselves
    const float* L32 = f->L32;
    float* tmp32 = nullptr;
    if (!L32 && (mode & CD_JK_VEC_FP32)) {  // FP32-rounded vectors requested: round on the fly
      if ((rc = scratch_alloc(&tmp32, (size_t)std::max<int64_t>(M, 1) * ld, st)) != CD_OK) return fail(rc);
      if ((rc = launch_to_fp32(f->L, ld, M, ld, tmp32, st)) != CD_OK) { scratch_free(tmp32, st); return fail(rc); }
      L32 = tmp32;
    }
    rc = jk_mixed(L32, L32 ? nullptr : f->L, ld, M, n, N, O, dC, f->sys->row_mu_dev, f->sys->row_nu_dev, dJ, dK,
                  wantJ, wantK, m == CD_JK_BF16X5 ? 5 : (m == CD_JK_BF16X4 ? 4 : 3), st);
    scratch_free(tmp32, st);
    if (rc != CD_OK) return fail(rc);
  } else {
    if (wantJ) {
      if ((rc = scratch_alloc(&d, (size_t)std::max<int64_t>(n, 1), st)) != CD_OK) return fail(rc);
      if ((rc = scratch_alloc(&v, (size_t)std::max<int64_t>(M, 1), st)) != CD_OK) return fail(rc);
      if ((rc = scratch_alloc(&Jp, (size_t)std::max<int64_t>(n, 1), st)) != CD_OK) return fail(rc);
      if ((rc = launch_density_packed(dC, N, O, f->sys->row_mu_dev, f->sys->row_nu_dev, n, d, st)) != CD_OK) return fail(rc);
      if (f->L) {
        if ((rc = launch_gemv_rows<double>(f->L, ld, M, n, d, v, st)) != CD_OK) return fail(rc);
        if ((rc = launch_gemv_cols<double>(f->L, ld, M, n, v, Jp, st)) != CD_OK) return fail(rc);
      } else {  // FP32-stored vectors, FP64 accumulation
        if ((rc = launch_gemv_rows<float>(f->L32, ld, M, n, d, v, st)) != CD_OK) return fail(rc);
        if ((rc = launch_gemv_cols<float>(f->L32, ld, M, n, v, Jp, st)) != CD_OK) return fail(rc);
      }
      if ((rc = launch_unpack_sym(Jp, f->sys->row_mu_dev, f->sys->row_nu_dev, n, N, dJ, st)) != CD_OK) return fail(rc);
    }
    if (wantK) {
      const double perP = 8.0 * ((double)N * N + (double)N * O);
      int Pc = (int)std::max<double>(1.0, std::min<double>((double)std::max<int64_t>(M, 1), 2.0e9 / perP));
      if ((rc = scratch_alloc(&Lfull, (size_t)Pc * N * N, st)) != CD_OK) return fail(rc);
      if ((rc = scratch_alloc(&B, (size_t)Pc * N * O, st)) != CD_OK) return fail(rc);
      if (cudaMemsetAsync(dK, 0, sizeof(double) * N * N, st) != cudaSuccess) return fail(CD_ECUDA);
      for (int64_t P0 = 0; P0 < M; P0 += Pc) {
        const int pc = (int)std::min<int64_t>(Pc, M - P0);
        rc = f->L ? launch_unpack_vectors<double, double>(f->L, ld, P0, pc, f->sys->row_mu_dev, f->sys->row_nu_dev, n,
                                                          N, Lfull, st)
                  : launch_unpack_vectors<float, double>(f->L32, ld, P0, pc, f->sys->row_mu_dev, f->sys->row_nu_dev,
                                                         n, N, Lfull, st);
        if (rc != CD_OK) return fail(rc);
        // B[p] = Lfull[p] (N x N) * C (N x O)
        if ((rc = launch_dgemm(N, O, N, pc, 1.0, Lfull, N, 1, (int64_t)N * N, dC, O, 1, 0, B, O, (int64_t)N * O, false, st)) != CD_OK) return fail(rc);
        // K += 2 sum_p B[p] B[p]^T
        if ((rc = launch_dgemm(N, N, O, pc, 2.0, B, O, 1, (int64_t)N * O, B, 1, O, (int64_t)N * O, dK, N, 0, true, st)) != CD_OK) return fail(rc);
      }
    }
  }
  if (!dev) {
    if (wantJ && cudaMemcpyAsync(J, dJ, sizeof(double) * N * N, cudaMemcpyDeviceToHost, st) != cudaSuccess) return fail(CD_ECUDA);
    if (wantK && cudaMemcpyAsync(K, dK, sizeof(double) * N * N, cudaMemcpyDeviceToHost, st) != cudaSuccess) return fail(CD_ECUDA);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("cd_jk: CUDA failure"); return fail(CD_ECUDA); }
  return fail(CD_OK);
}


int cd_mo_vectors(const cd_factor_t* f, const double* C, int32_t n_mo, int64_t P0, int64_t nP, int32_t slices,
                  double* out, int32_t flags, void* stream) {
  if (!f || !C || !out || n_mo <= 0 || P0 < 0 || nP < 0 || P0 + nP > f->M) {
    set_error("cd_mo_vectors: bad argument");
    return CD_EINVAL;
  }
  if (slices != 0 && slices != 3 && slices != 4 && slices != 5 && slices != 7) {
    set_error("cd_mo_vectors: slices must be 0 (FP64), 3, 4, 5 or 7");
    return CD_EINVAL;
  }
  if (nP == 0) return CD_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int N = f->sys->hb.nbf;
  const int64_t n = f->n, ld = f->ld;
  const bool dev = (flags & CD_JK_DEVICE) != 0;
  const size_t out_elems = (size_t)nP * n_mo * n_mo;
  double *dC = nullptr, *dOut = nullptr, *U = nullptr, *B = nullptr;
  auto done = [&](int code) {
    if (!dev) { scratch_free(dC, st); scratch_free(dOut, st); }
    scratch_free(U, st);
    scratch_free(B, st);
    cudaStreamSynchronize(st);
    return code;
  };
  int rc = CD_OK;
  if (dev) {
    dC = const_cast<double*>(C);
    dOut = out;
  } else {
    if ((rc = scratch_alloc(&dC, (size_t)N * n_mo, st)) != CD_OK) return done(rc);
    if ((rc = scratch_alloc(&dOut, out_elems, st)) != CD_OK) return done(rc);
    if (cudaMemcpyAsync(dC, C, sizeof(double) * N * n_mo, cudaMemcpyHostToDevice, st) != cudaSuccess) {
      set_error("cd_mo_vectors: copy of C failed");
      return done(CD_ECUDA);
    }
  }
  if (slices > 0) {
    rc = mo_vectors_sliced(f->L ? nullptr : f->L32, f->L, ld, P0, nP, n, N, n_mo, dC, f->sys->row_mu_dev,
                           f->sys->row_nu_dev, slices, dOut, st);
    if (rc != CD_OK) return done(rc);
  } else {
    // FP64: per chunk of vectors, U^P = unpack(L^P), B^P = U^P C, out^P = C^T B^P
    const double perP = 8.0 * ((double)N * N + (double)N * n_mo);
    const int Pc = (int)std::max<double>(1.0, std::min<double>((double)nP, 1.5e9 / perP));
    if ((rc = scratch_alloc(&U, (size_t)Pc * N * N, st)) != CD_OK) return done(rc);
    if ((rc = scratch_alloc(&B, (size_t)Pc * N * n_mo, st)) != CD_OK) return done(rc);
    for (int64_t Q0 = P0; Q0 < P0 + nP; Q0 += Pc) {
      const int pc = (int)std::min<int64_t>(Pc, P0 + nP - Q0);
      rc = f->L ? launch_unpack_vectors<double, double>(f->L, ld, Q0, pc, f->sys->row_mu_dev, f->sys->row_nu_dev, n, N,
                                                        U, st)
                : launch_unpack_vectors<float, double>(f->L32, ld, Q0, pc, f->sys->row_mu_dev, f->sys->row_nu_dev, n,
                                                       N, U, st);
      if (rc != CD_OK) return done(rc);
      if ((rc = launch_dgemm(N, n_mo, N, pc, 1.0, U, N, 1, (int64_t)N * N, dC, n_mo, 1, 0, B, n_mo,
                             (int64_t)N * n_mo, false, st)) != CD_OK)
        return done(rc);
      double* o = dOut + (Q0 - P0) * (int64_t)n_mo * n_mo;
      if ((rc = launch_dgemm(n_mo, n_mo, N, pc, 1.0, dC, 1, n_mo, 0, B, n_mo, 1, (int64_t)N * n_mo, o, n_mo,
                             (int64_t)n_mo * n_mo, false, st)) != CD_OK)
        return done(rc);
    }
  }
  if (!dev && cudaMemcpyAsync(out, dOut, sizeof(double) * out_elems, cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return done(CD_ECUDA);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("cd_mo_vectors: CUDA failure"); return done(CD_ECUDA); }
  return done(CD_OK);
}

// ---------------------------------------------------------------- batch ----
// Many independent systems: a pool of host workers, each driving its own
// non-blocking CUDA stream, takes systems from a shared queue (largest first)
// and runs set-up, decomposition and J/K for each.  Small systems do not fill
// the GPU on their own; running several at once on separate streams overlaps
// their kernels.  Per-call scratch is stream-ordered, so workers never wait
// on each other; objects are freed after every worker has finished.
int cd_batch_run(int32_t n_sys, const cd_basis_t* bases, const cd_opts_t* opts, const double* const* C_occ,
                 const int32_t* n_occ, double* const* J, double* const* K, int32_t jk_mode, int32_t workers,
                 void* stream) {
  if (n_sys < 0 || (n_sys > 0 && (!bases || !opts || !C_occ || !n_occ || !J || !K))) {
    set_error("cd_batch_run: bad argument");
    return CD_EINVAL;
  }
  if (n_sys == 0) return CD_OK;
  int dev = 0;
  CD_CUDA(cudaGetDevice(&dev));
  const int nw = std::max(1, std::min<int>(n_sys, workers > 0 ? workers : 8));
  // order: largest basis first
  std::vector<int> order(n_sys);
  std::vector<int64_t> size(n_sys, 0);
  for (int i = 0; i < n_sys; ++i) {
    order[i] = i;
    for (int sh = 0; sh < bases[i].n_shells; ++sh) size[i] += 2 * (bases[i].l ? bases[i].l[sh] : 0) + 1;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return size[a] > size[b]; });
  cudaEvent_t start;
  CD_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  CD_CUDA(cudaEventRecord(start, (cudaStream_t)stream));
  std::atomic<int> next{0};
  std::vector<int> rcs(n_sys, CD_OK);
  std::vector<std::string> msgs(n_sys);
  std::vector<cd_system*> systems(n_sys, nullptr);
  std::vector<cd_factor_t*> factors(n_sys, nullptr);
  std::vector<cudaStream_t> streams(nw, nullptr);
  std::vector<cudaEvent_t> done(nw, nullptr);
  for (int w = 0; w < nw; ++w) {
    CD_CUDA(cudaStreamCreateWithFlags(&streams[w], cudaStreamNonBlocking));
    CD_CUDA(cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming));
    CD_CUDA(cudaStreamWaitEvent(streams[w], start, 0));
  }
  auto work = [&](int w) {
    cudaSetDevice(dev);
    cudaStream_t st = streams[w];
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n_sys) break;
      const int i = order[k];
      int rc = cd_system_create(&bases[i], opts[i].schwarz, st, &systems[i]);
      if (rc == CD_OK) rc = cd_eri_factor_sys(systems[i], &opts[i], st, &factors[i]);
      if (rc == CD_OK) rc = cd_jk(factors[i], C_occ[i], n_occ[i], J[i], K[i], jk_mode, st);
      rcs[i] = rc;
      if (rc != CD_OK) msgs[i] = g_err;
    }
    cudaEventRecord(done[w], st);
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nw; ++w) th.emplace_back(work, w);
  work(0);
  for (auto& t : th) t.join();
  for (int w = 0; w < nw; ++w) cudaStreamWaitEvent((cudaStream_t)stream, done[w], 0);
  cudaStreamSynchronize((cudaStream_t)stream);
  for (int i = 0; i < n_sys; ++i) {
    if (factors[i]) factor_release(factors[i]);
    if (systems[i]) system_release(systems[i]);
  }
  for (int w = 0; w < nw; ++w) {
    cudaEventDestroy(done[w]);
    cudaStreamDestroy(streams[w]);
  }
  cudaEventDestroy(start);
  for (int i = 0; i < n_sys; ++i)
    if (rcs[i] != CD_OK) {
      set_error("cd_batch_run: system " + std::to_string(i) + ": " + msgs[i]);
      return rcs[i];
    }
  return CD_OK;
}

}  // extern "C"
