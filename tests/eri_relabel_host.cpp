// Host build of the ERI device code (paper_2609_00306_b300/csrc/eri_dev.cuh):
// for every bra class (ss, ps, pp) and every single ket component of a (ps)
// or (pp) ket shell pair, the relabelled-axis evaluation (ket direction moved
// to axis 0, compile-time Kronecker deltas) must give the same contracted
// integrals as the general evaluation with runtime ket directions, on random
// primitive-pair data.  Both read the same Boys table, so any smooth table
// serves: the check is of the recurrence bookkeeping, not of the Boys values.
// Exit status 0 when every case agrees to 1e-13 of its largest integral.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>
// device intrinsics the header uses, as plain host functions
template <typename T> static inline T __ldg(const T* p) { return *p; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
static inline int __double2int_rn(double x) { return (int)std::nearbyint(x); }
static struct { unsigned x; } threadIdx;
#include "../paper_2609_00306_b300/csrc/eri_dev.cuh"
using namespace cd;

namespace {

struct HostPairs {
  std::vector<int32_t> pp_off, row;
  std::vector<int8_t> la, lb;
  std::vector<double> AB, zeta, P, PA, Kp, o2z;
  PairSet view() {
    PairSet s;
    s.n = (int64_t)la.size();
    s.npp = (int64_t)zeta.size();
    s.pp_off = pp_off.data();
    s.la = la.data();
    s.lb = lb.data();
    s.AB = AB.data();
    s.row = row.data();
    s.zeta = zeta.data();
    s.P = P.data();
    s.PA = PA.data();
    s.Kp = Kp.data();
    s.o2z = o2z.data();
    return s;
  }
};

// shell pairs with 2-3 x 2-3 primitives, exponents log-uniform in [0.15, 20],
// centres within a few bohr; every component gets its own output row
HostPairs make_pairs(std::mt19937_64& g, int npairs, int la, int lb) {
  std::uniform_real_distribution<double> U(0.0, 1.0);
  HostPairs h;
  h.pp_off.push_back(0);
  for (int s = 0; s < npairs; ++s) {
    double A[3], B[3];
    for (int x = 0; x < 3; ++x) {
      A[x] = 6 * U(g) - 3;
      B[x] = A[x] + 3 * U(g) - 1.5;
    }
    const int na = 2 + (int)(U(g) * 2), nb = 2 + (int)(U(g) * 2);
    for (int i = 0; i < na; ++i)
      for (int j = 0; j < nb; ++j) {
        const double a = std::exp(std::log(0.15) + U(g) * std::log(20 / 0.15));
        const double b = std::exp(std::log(0.15) + U(g) * std::log(20 / 0.15));
        const double z = a + b;
        h.zeta.push_back(z);
        h.o2z.push_back(0.5 / z);
        double ab2 = 0;
        for (int x = 0; x < 3; ++x) {
          const double P = (a * A[x] + b * B[x]) / z;
          h.P.push_back(P);
          h.PA.push_back(P - A[x]);
          ab2 += (A[x] - B[x]) * (A[x] - B[x]);
        }
        h.Kp.push_back(std::exp(-a * b / z * ab2) * (0.5 + U(g)));
      }
    h.pp_off.push_back((int32_t)h.zeta.size());
    h.la.push_back((int8_t)la);
    h.lb.push_back((int8_t)lb);
    for (int x = 0; x < 3; ++x) h.AB.push_back(A[x] - B[x]);
    for (int c = 0; c < 9; ++c) h.row.push_back(s * 9 + c);
  }
  return h;
}

template <int LA, int LB, int LC, int LD, int KD>
double check(std::mt19937_64& g, const double* tab, int kc, int kd) {
  constexpr int kBra = 16;
  HostPairs bh = make_pairs(g, kBra, LA, LB), kh = make_pairs(g, 3, LC, LD);
  PairSet bra = bh.view(), ket = kh.view();
  KetGroup kg;
  std::memset(&kg, 0, sizeof(kg));
  kg.sp = 1;
  kg.lc = LC;
  kg.ld = LD;
  kg.nc = 1;
  kg.kc[0] = (int8_t)kc;
  kg.kd[0] = (int8_t)kd;
  kg.slot[0] = 0;
  const int64_t ld = kBra * 9;
  std::vector<double> general(ld, 0.0), relabelled(ld, 0.0);
  unsigned long long ops_general = 0, ops_relabelled = 0;
  for (int sb = 0; sb < kBra; ++sb) {
    column_block<LA, LB, LC, LD, 1>(bra, sb, ket, kg, general.data(), ld, tab, ops_general);
    column_block<LA, LB, LC, LD, 1, 0, KD>(bra, sb, ket, kg, relabelled.data(), ld, tab, ops_relabelled);
  }
  double mx = 0, worst = 0;
  int nonzero = 0;
  for (int64_t r = 0; r < ld; ++r) {
    mx = std::max(mx, std::fabs(general[r]));
    worst = std::max(worst, std::fabs(general[r] - relabelled[r]));
    nonzero += general[r] != 0.0;
  }
  std::printf("bra (%d%d) ket (%d%d) component (%d,%d): %d integrals, max %.3e, max diff %.3e, ops %llu -> %llu\n",
              LA, LB, LC, LD, kc, kd, nonzero, mx, worst, ops_general, ops_relabelled);
  if (nonzero == 0 || ops_relabelled > ops_general) return 1.0;
  return worst / mx;
}

}  // namespace

int main() {
  std::vector<double> tab(kBoysTableSize);
  for (int k = 0; k < kBoysPoints; ++k)
    for (int c = 0; c < kBoysCols; ++c) tab[k * kBoysCols + c] = std::exp(-0.005 * k) / (2 * c + 1 + 0.1 * k);
  for (int i = kBoysCoefOff; i < kBoysTableSize; ++i) tab[i] = 1.0 / (1.0 + (i % 97) * 0.37);
  std::mt19937_64 g(12345);
  const double* t = tab.data();
  double w = 0;
  for (int kc = 0; kc < 3; ++kc) {
    w = std::max(w, check<0, 0, 1, 0, 0>(g, t, kc, 0));
    w = std::max(w, check<1, 0, 1, 0, 0>(g, t, kc, 0));
    w = std::max(w, check<1, 1, 1, 0, 0>(g, t, kc, 0));
    for (int kd = 0; kd < 3; ++kd) {
      if (kd == kc) {
        w = std::max(w, check<0, 0, 1, 1, 0>(g, t, kc, kd));
        w = std::max(w, check<1, 0, 1, 1, 0>(g, t, kc, kd));
        w = std::max(w, check<1, 1, 1, 1, 0>(g, t, kc, kd));
      } else {
        w = std::max(w, check<0, 0, 1, 1, 1>(g, t, kc, kd));
        w = std::max(w, check<1, 0, 1, 1, 1>(g, t, kc, kd));
        w = std::max(w, check<1, 1, 1, 1, 1>(g, t, kc, kd));
      }
    }
  }
  std::printf("worst relative difference %.3e\n", w);
  return w < 1e-13 ? 0 : 1;
}
