// basis.cu -- host-side preparation: validation, normalisation of contracted
// s/p functions, shell-pair / primitive-pair records, the Boys-function table.
#include <math.h>
#include <algorithm>
#include <map>
#include <mutex>
#include <thread>
#include "internal.cuh"

namespace cd {

static const double kPi = 3.14159265358979323846;

// Normalised primitives: s -> (2a/pi)^{3/4}; Cartesian p -> (2a/pi)^{3/4} (4a)^{1/2}.
// Contracted function rescaled to unit self-overlap using the same-centre
// overlaps (pi/(a+b))^{3/2} (s) and (pi/(a+b))^{3/2} / (2(a+b)) (p_x p_x).
int validate_and_normalise(const cd_basis_t* b, HostBasis* hb) {
  if (!b || b->n_shells <= 0 || !b->center || !b->l || !b->nprim || !b->exps || !b->coefs) {
    set_error("basis: null pointer or no shells");
    return CD_EINVAL;
  }
  hb->nsh = b->n_shells;
  hb->cen.assign(b->center, b->center + 3 * (size_t)b->n_shells);
  hb->l.resize(hb->nsh);
  hb->nprim.resize(hb->nsh);
  hb->pofs.resize(hb->nsh);
  hb->bf0.resize(hb->nsh);
  int np = 0, nbf = 0;
  for (int s = 0; s < hb->nsh; ++s) {
    int l = b->l[s], n = b->nprim[s];
    if (l < 0 || l > 1) { set_error("basis: shell " + std::to_string(s) + " has l outside {0,1}"); return CD_EINVAL; }
    if (n < 1 || n > CD_MAX_PRIM) { set_error("basis: shell " + std::to_string(s) + " has nprim outside [1,16]"); return CD_EINVAL; }
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(b->center[3 * s + k])) { set_error("basis: non-finite centre"); return CD_EINVAL; }
    hb->l[s] = l; hb->nprim[s] = n; hb->pofs[s] = np; hb->bf0[s] = nbf;
    np += n; nbf += 2 * l + 1;
  }
  if ((int64_t)nbf * (nbf + 1) / 2 > (int64_t)INT32_MAX) { set_error("basis: too many functions"); return CD_EINVAL; }
  hb->nbf = nbf;
  hb->exps.assign(b->exps, b->exps + np);
  hb->dcoef.resize(np);
  for (int i = 0; i < np; ++i) {
    if (!(b->exps[i] > 0.0) || !std::isfinite(b->exps[i])) { set_error("basis: exponent not positive/finite"); return CD_EINVAL; }
    if (!std::isfinite(b->coefs[i])) { set_error("basis: non-finite coefficient"); return CD_EINVAL; }
  }
  for (int s = 0; s < hb->nsh; ++s) {
    int o = hb->pofs[s], n = hb->nprim[s], l = hb->l[s];
    for (int i = 0; i < n; ++i) {
      double a = hb->exps[o + i];
      double nrm = pow(2.0 * a / kPi, 0.75) * (l == 1 ? sqrt(4.0 * a) : 1.0);
      hb->dcoef[o + i] = b->coefs[o + i] * nrm;
    }
    double S = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double ab = hb->exps[o + i] + hb->exps[o + j];
        double ov = pow(kPi / ab, 1.5) / (l == 1 ? 2.0 * ab : 1.0);
        S += hb->dcoef[o + i] * hb->dcoef[o + j] * ov;
      }
    if (!(S > 0.0)) { set_error("basis: contracted function with zero norm"); return CD_EINVAL; }
    double sc = 1.0 / sqrt(S);
    for (int i = 0; i < n; ++i) hb->dcoef[o + i] *= sc;
  }
  hb->bf_shell.resize(nbf);
  hb->bf_comp.resize(nbf);
  for (int s = 0; s < hb->nsh; ++s)
    for (int k = 0; k < 2 * hb->l[s] + 1; ++k) {
      hb->bf_shell[hb->bf0[s] + k] = s;
      hb->bf_comp[hb->bf0[s] + k] = k;
    }
  return CD_OK;
}

// Records for the shell pairs (s1[k], s2[k]), s1 >= s2, in the given order.
// row[] is filled with the packed pair index (callers remap it).
// run body(k) for k in [0, n) on the host's cores, in contiguous chunks
template <class F>
static void parallel_for(size_t n, F&& body) {
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nt = std::min<size_t>(hw, std::max<size_t>(1, n / 4096));
  if (nt <= 1) {
    for (size_t k = 0; k < n; ++k) body(k);
    return;
  }
  std::vector<std::thread> th;
  const size_t chunk = (n + nt - 1) / nt;
  for (size_t t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      const size_t k0 = t * chunk, k1 = std::min(n, k0 + chunk);
      for (size_t k = k0; k < k1; ++k) body(k);
    });
  for (auto& x : th) x.join();
}

void build_pairs(const HostBasis& hb, const std::vector<int32_t>& s1, const std::vector<int32_t>& s2,
                 PairSetHost* out, double prune) {
  const double c0 = sqrt(2.0) * pow(kPi, 1.25);
  size_t n = s1.size();
  out->pp_off.assign(n + 1, 0);
  out->la.resize(n); out->lb.resize(n); out->AB.resize(3 * n);
  out->row.assign(9 * n, -1);
  out->s1 = s1; out->s2 = s2;
  out->swapped.resize(n);
  // primitive-pair prefactor of primitives (i on A, j on B) of shell pair k
  auto kp_of = [&](int A, int B, int i, int j, double AB2) {
    const double a = hb.exps[hb.pofs[A] + i], b = hb.exps[hb.pofs[B] + j];
    const double z = a + b;
    return c0 * hb.dcoef[hb.pofs[A] + i] * hb.dcoef[hb.pofs[B] + j] * exp(-a * b / z * AB2) / z;
  };
  auto orient = [&](size_t k, int* A, int* B, double* AB2) {
    const int S1 = s1[k], S2 = s2[k];
    const int sw = hb.l[S1] < hb.l[S2];
    *A = sw ? S2 : S1;
    *B = sw ? S1 : S2;
    double d = 0.0;
    for (int x = 0; x < 3; ++x) d += (hb.cen[3 * *A + x] - hb.cen[3 * *B + x]) * (hb.cen[3 * *A + x] - hb.cen[3 * *B + x]);
    *AB2 = d;
    return sw;
  };
  // pass 1: surviving primitive pairs per shell pair, then their offsets
  std::vector<int32_t> cnt(n, 0);
  parallel_for(n, [&](size_t k) {
    int A, B;
    double AB2;
    orient(k, &A, &B, &AB2);
    int c = 0;
    for (int i = 0; i < hb.nprim[A]; ++i)
      for (int j = 0; j < hb.nprim[B]; ++j)
        if (!(prune > 0.0 && fabs(kp_of(A, B, i, j, AB2)) < prune)) ++c;
    cnt[k] = c;
  });
  size_t q = 0;
  for (size_t k = 0; k < n; ++k) { out->pp_off[k] = (int32_t)q; q += cnt[k]; }
  out->pp_off[n] = (int32_t)q;
  out->zeta.resize(q); out->P.resize(3 * q); out->PA.resize(3 * q); out->Kp.resize(q); out->o2z.resize(q);
  // pass 2: the records
  parallel_for(n, [&](size_t k) {
    int A, B;
    double AB2;
    const int sw = orient(k, &A, &B, &AB2);
    const int S1 = s1[k], S2 = s2[k];
    out->swapped[k] = (int8_t)sw;
    out->la[k] = (int8_t)hb.l[A];
    out->lb[k] = (int8_t)hb.l[B];
    const double* cA = &hb.cen[3 * A];
    const double* cB = &hb.cen[3 * B];
    for (int x = 0; x < 3; ++x) out->AB[3 * k + x] = cA[x] - cB[x];
    size_t w = (size_t)out->pp_off[k];
    for (int i = 0; i < hb.nprim[A]; ++i)
      for (int j = 0; j < hb.nprim[B]; ++j) {
        const double kp = kp_of(A, B, i, j, AB2);
        if (prune > 0.0 && fabs(kp) < prune) continue;
        const double a = hb.exps[hb.pofs[A] + i], b = hb.exps[hb.pofs[B] + j];
        const double z = a + b;
        out->zeta[w] = z;
        for (int x = 0; x < 3; ++x) {
          const double P = (a * cA[x] + b * cB[x]) / z;
          out->P[3 * w + x] = P;
          out->PA[3 * w + x] = P - cA[x];
        }
        out->Kp[w] = kp;
        out->o2z[w] = 0.5 / z;
        ++w;
      }
    // components: i on A, j on B
    const int nA = 2 * hb.l[A] + 1, nB = 2 * hb.l[B] + 1;
    for (int i = 0; i < nA; ++i)
      for (int j = 0; j < nB; ++j) {
        const int fA = hb.bf0[A] + i, fB = hb.bf0[B] + j;
        if (S1 == S2 && fA < fB) continue;  // same shell: keep mu >= nu only
        const int64_t mu = std::max(fA, fB), nu = std::min(fA, fB);
        out->row[9 * k + 3 * i + j] = (int32_t)(mu * (mu + 1) / 2 + nu);
      }
  });
}

template <class T>
static int up(T** dst, const std::vector<T>& v, cudaStream_t st) {
  if (v.empty()) { *dst = nullptr; return CD_OK; }
  CD_CUDA(cudaMalloc((void**)dst, sizeof(T) * v.size()));
  CD_CUDA(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return CD_OK;
}

int upload_pairs(const PairSetHost& h, PairSet* d, cudaStream_t st) {
  d->n = (int64_t)h.la.size();
  d->npp = (int64_t)h.zeta.size();
  CD_TRY(up(&d->pp_off, h.pp_off, st));
  CD_TRY(up(&d->la, h.la, st));
  CD_TRY(up(&d->lb, h.lb, st));
  CD_TRY(up(&d->AB, h.AB, st));
  CD_TRY(up(&d->row, h.row, st));
  CD_TRY(up(&d->zeta, h.zeta, st));
  CD_TRY(up(&d->P, h.P, st));
  CD_TRY(up(&d->PA, h.PA, st));
  CD_TRY(up(&d->Kp, h.Kp, st));
  CD_TRY(up(&d->o2z, h.o2z, st));
  return CD_OK;
}

void free_pairs(PairSet* d) {
  cudaFree(d->pp_off); cudaFree(d->la); cudaFree(d->lb); cudaFree(d->AB); cudaFree(d->row);
  cudaFree(d->zeta); cudaFree(d->P); cudaFree(d->PA); cudaFree(d->Kp); cudaFree(d->o2z);
  *d = PairSet();
}

// F_m(T) = exp(-T) sum_i (2T)^i / prod_{k=0..i} (2m+2k+1), evaluated in long
// double (all terms positive, no cancellation) for the table points.
static long double boys_series(int m, long double T) {
  long double term = 1.0L / (2 * m + 1), sum = term;
  for (int i = 1; i < 4000; ++i) {
    term *= 2.0L * T / (2 * m + 2 * i + 1);
    sum += term;
    if (term < 1e-22L * sum) break;
  }
  return expl(-T) * sum;
}

int scratch_alloc_bytes(void** p, size_t bytes, cudaStream_t st) {
  static std::mutex mu;
  static std::map<int, bool> configured;
  *p = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { set_error("cudaGetDevice failed"); return CD_ECUDA; }
  {
    std::lock_guard<std::mutex> g(mu);
    if (!configured[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      configured[dev] = true;
    }
  }
  cudaError_t e = cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("device scratch allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    return CD_ENOMEM;
  }
  return CD_OK;
}

const double* boys_table_device(int* rc) {
  static std::mutex mu;
  static std::map<int, double*> tables;
  std::lock_guard<std::mutex> g(mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { *rc = CD_ECUDA; set_error("cudaGetDevice failed"); return nullptr; }
  auto it = tables.find(dev);
  if (it != tables.end()) { *rc = CD_OK; return it->second; }
  std::vector<double> h((size_t)kBoysTableSize);
  for (int k = 0; k < kBoysPoints; ++k) {
    const long double T = (long double)k * (long double)kBoysStep;
    long double F[kBoysFcols];
    for (int m = 0; m < kBoysFcols; ++m) {
      F[m] = boys_series(m, T);
      h[(size_t)k * kBoysCols + m] = (double)F[m];
    }
    h[(size_t)k * kBoysCols + kBoysFcols] = (double)expl(-T);
    for (int L = 0; L <= kBoysMaxM; ++L) {
      long double fact = 1.0L;
      for (int j = 0; j < kBoysTaylor; ++j) {
        if (j > 0) fact *= (long double)j;
        h[(size_t)kBoysCoefOff + ((size_t)L * kBoysPoints + k) * kBoysTaylor + j] = (double)(F[L + j] / fact);
      }
    }
  }
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * h.size()) != cudaSuccess ||
      cudaMemcpy(d, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    set_error("Boys table upload failed");
    *rc = CD_ECUDA;
    return nullptr;
  }
  tables[dev] = d;
  *rc = CD_OK;
  return d;
}

}  // namespace cd
