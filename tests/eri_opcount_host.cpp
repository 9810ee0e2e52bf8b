// Host build of the ERI device code with an operation-counting FP64 type: for
// one primitive quartet of every bra class against a single (ps) or (pp) ket
// component, the number of FP64 operations the relabelled-axis path saves
// over the general path, counted at the source level (adds, multiplies, FMAs,
// conversions), must equal the saving that the kernel's executed-operation
// counter (fixed_ops in eri_dev.cuh) books.  The counter's absolute numbers
// model FMA contraction and are compared with hardware counters elsewhere; the
// difference between the two paths removes only whole FMAs and adds, so it
// is the same at both levels.  Exit status 0 when every difference agrees.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>
#include <cuda_runtime.h>
#include "../paper_2609_00306_b300/csrc/internal.cuh"

static long long g_ops = 0;
struct Counted {
  double v;
  constexpr Counted() : v(0) {}
  constexpr Counted(double x) : v(x) {}  // loads and literals: no operation
  explicit Counted(float x) : v(x) { ++g_ops; }
  explicit Counted(int x) : v(x) { ++g_ops; }
  explicit operator float() const {
    ++g_ops;
    return (float)v;
  }
};
static inline Counted operator+(Counted a, Counted b) { ++g_ops; return Counted(a.v + b.v); }
static inline Counted operator-(Counted a, Counted b) { ++g_ops; return Counted(a.v - b.v); }
static inline Counted operator*(Counted a, Counted b) { ++g_ops; return Counted(a.v * b.v); }
static inline Counted operator-(Counted a) { return Counted(-a.v); }  // an operand modifier
static inline Counted& operator+=(Counted& a, Counted b) { ++g_ops; a.v += b.v; return a; }
static inline bool operator<(Counted a, Counted b) { return a.v < b.v; }
static inline Counted fma(Counted a, Counted b, Counted c) { ++g_ops; return Counted(std::fma(a.v, b.v, c.v)); }
template <typename T> static inline T __ldg(const T* p) { return *p; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
static inline int __double2int_rn(Counted x) { ++g_ops; return (int)std::nearbyint(x.v); }
static struct { unsigned x; } threadIdx;
// the device header's FP64 arithmetic in the counting type (the pair data stay double)
#define double Counted
#include "../paper_2609_00306_b300/csrc/eri_dev.cuh"
#undef double
using namespace cd;

namespace {

// one bra and one ket primitive pair; the values only need to be finite
std::vector<int32_t> g_off = {0, 1}, g_row = {0, 1, 2, 3, 4, 5, 6, 7, 8};
std::vector<int8_t> g_l = {1};
std::vector<double> g_ab = {0.3, -0.2, 0.5}, g_zeta = {1.3}, g_pa = {0.05, -0.1, 0.2}, g_kp = {0.7},
                    g_o2z = {1.0 / 2.6}, g_pbra = {0.1, 0.2, 0.3}, g_pket = {1.1, -0.4, 0.9};

PairSet pairs(std::vector<double>& P) {
  PairSet s;
  s.n = 1;
  s.npp = 1;
  s.pp_off = g_off.data();
  s.la = s.lb = g_l.data();
  s.AB = g_ab.data();
  s.row = g_row.data();
  s.zeta = g_zeta.data();
  s.P = P.data();
  s.PA = g_pa.data();
  s.Kp = g_kp.data();
  s.o2z = g_o2z.data();
  return s;
}

template <int LA, int LB, int LC, int LD, int KD>
bool check(const Counted* tab) {
  PairSet bra = pairs(g_pbra), ket = pairs(g_pket);
  const int kcs[1] = {0}, kds[1] = {KD}, ax[3] = {0, 1, 2};
  Counted out[1][9];
  unsigned nt = 0;
  g_ops = 0;
  quartet<LA, LB, LC, LD, 1>(bra, 0, ket, 0, kcs, kds, ax, tab, out, nt);
  const long long general = g_ops;
  g_ops = 0;
  quartet<LA, LB, LC, LD, 1, 0, KD>(bra, 0, ket, 0, kcs, kds, ax, tab, out, nt);
  const long long relabelled = g_ops;
  const long long booked = (long long)fixed_ops<LA + LB, LC + LD, 1>(1) - (long long)fixed_ops<LA + LB, LC + LD, 1, 0, KD>(1);
  std::printf("bra (%d%d) ket (%d%d) KD %d: source %lld -> %lld (saves %lld), counter saves %lld\n", LA, LB, LC, LD,
              KD, general, relabelled, general - relabelled, booked);
  return general - relabelled == booked;
}

}  // namespace

int main() {
  std::vector<Counted> tab(kBoysTableSize, Counted(0.01));
  const Counted* t = tab.data();
  bool ok = true;
  ok &= check<0, 0, 1, 0, 0>(t);
  ok &= check<1, 0, 1, 0, 0>(t);
  ok &= check<1, 1, 1, 0, 0>(t);
  ok &= check<0, 0, 1, 1, 0>(t);
  ok &= check<1, 0, 1, 1, 0>(t);
  ok &= check<1, 1, 1, 1, 0>(t);
  ok &= check<0, 0, 1, 1, 1>(t);
  ok &= check<1, 0, 1, 1, 1>(t);
  ok &= check<1, 1, 1, 1, 1>(t);
  std::printf(ok ? "all savings agree\n" : "MISMATCH\n");
  return ok ? 0 : 1;
}
