// eri_dev.cuh -- device code of kernel (a), the contracted s/p electron-repulsion
// integrals in FP64, shared by the column kernels (eri.cu) and the persistent
// batch kernel (batch.cu).
//
// One thread evaluates one (bra shell pair | ket function pair) combination:
// all bra components (up to 9) against one ket component, looping over the
// primitive quartets.  Per primitive quartet the Boys function comes from a
// Taylor table (F_L and exp(-T)) plus downward recursion, and 1/(p+q) and its
// square root from one FP32 seed refined by Newton steps in FP64 (the FP64
// pipe is the bound, so no library division, sqrt or exp); the vertical recurrence of
// Obara and Saika, in the two-electron form of Head-Gordon and Pople, builds
// [e0|f0] (e <= 2 on the bra, f <= 2 on the ket); after contraction the
// horizontal recurrences (a,b+1_j| = (a+1_j,b| + AB_j (a,b| and
// |c,d+1_l) = |c+1_l,d) + CD_l |c,d) give the requested components.
// Bra shell pairs are sorted by angular class, so warps run one class.
#pragma once
#include "internal.cuh"

namespace cd {
namespace {

constexpr double kSqrtPiOver4 = 0.88622692545275801365;  // sqrt(pi)/2

template <int L>
__device__ __forceinline__ void boys_fm(double T, double (&F)[L + 1], const double* __restrict__ tab) {
  if (T < kBoysTmax) {
    const int k = __double2int_rn(T * (1.0 / kBoysStep));
    const double d = (double)k * kBoysStep - T;  // F_L(T) = sum_j F_{L+j}(T_k) d^j / j!
    const double* __restrict__ row = tab + k * kBoysCols;
    // Horner sum of the pre-divided coefficients F_{L+j}(T_k) / j!
    const double* __restrict__ c = tab + kBoysCoefOff + (L * kBoysPoints + k) * kBoysTaylor;
    double f = __ldg(c + kBoysTaylor - 1);
#pragma unroll
    for (int j = kBoysTaylor - 2; j >= 0; --j) f = fma(f, d, __ldg(c + j));
    F[L] = f;
    if constexpr (L == 1) {
      // F_0 by its own Horner sum: cheaper than exp(-T) and one downward step
      const double* __restrict__ c0 = tab + kBoysCoefOff + k * kBoysTaylor;
      double f0 = __ldg(c0 + kBoysTaylor - 1);
#pragma unroll
      for (int j = kBoysTaylor - 2; j >= 0; --j) f0 = fma(f0, d, __ldg(c0 + j));
      F[0] = f0;
    } else if constexpr (L > 1) {
      // exp(-T) = exp(-T_k) exp(d), exp(d) by Horner with constant coefficients 1/j!
      constexpr double inv_fact[kExpTaylor] = {1.0, 1.0, 1.0 / 2, 1.0 / 6, 1.0 / 24, 1.0 / 120, 1.0 / 720,
                                               1.0 / 5040, 1.0 / 40320};
      double e = inv_fact[kExpTaylor - 1];
#pragma unroll
      for (int j = kExpTaylor - 2; j >= 0; --j) e = fma(e, d, inv_fact[j]);
      const double emT = __ldg(row + kBoysFcols) * e;
#pragma unroll
      for (int m = L - 1; m >= 0; --m) F[m] = fma(2.0 * T, F[m + 1], emT) * (1.0 / (2 * m + 1));
    }
  } else {
    // r = 1/sqrt(T): FP32 seed, two FP64 Newton steps; F_0 = sqrt(pi)/2 r, F_{m+1} = (2m+1) F_m r^2 / 2
    double r = (double)rsqrtf((float)T);
    r = r * fma(-0.5 * T, r * r, 1.5);
    r = r * fma(-0.5 * T, r * r, 1.5);
    F[0] = kSqrtPiOver4 * r;
    const double h = 0.5 * r * r;
#pragma unroll
    for (int m = 0; m < L; ++m) F[m + 1] = (double)(2 * m + 1) * F[m] * h;
  }
}

__host__ __device__ constexpr int didx(int i, int j) {
  // (i <= j): xx 0, xy 1, xz 2, yy 3, yz 4, zz 5
  return i == 0 ? j : (i == 1 ? 2 + j : 5);
}
__device__ __forceinline__ double sel3(const double (&v)[3], int k) {
  return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]);
}

// Contracted bra-shell-pair x NC ket-function-pair block (the NC ket pairs
// belong to one ket shell pair).  out[c][i*3+j] receives (a_i b_j | c_kc d_kd)
// for ket component c and the bra components (i on A, j on B).  The primitive
// set-up, Boys function and bra recurrence are shared by the NC components.
//
// KC >= 0 (one ket component, NC = 1): the Cartesian axes are relabelled,
// axis x of the computation being axis ax[x] of the input, so that the ket
// component is (c_KC d_KD) with KC = 0 and KD = 0 (c = d) or 1 (c != d).  The
// Gaussians are isotropic and the recurrences the same along every axis, so
// the integrals of the relabelled frame are those of the input with the
// component indices mapped through ax.  With the ket directions known at
// compile time the terms of the recurrences that carry a Kronecker delta
// (N_k(e) / 2s, delta_kl / 2q) exist only where they are non-zero.  out is then
// indexed in the relabelled frame.
template <int LA, int LB, int LC, int LD, int NC, int KC = -1, int KD = -1>
__device__ __forceinline__ void quartet(const PairSet& bra, int64_t sb, const PairSet& ket, int64_t sk,
                                        const int (&kcs)[NC], const int (&kds)[NC], const int (&ax)[3],
                                        const double* __restrict__ tab, double (&out)[NC][9], unsigned& n_table) {
  constexpr bool SPEC = KC >= 0;
  static_assert(!SPEC || (NC == 1 && KC == 0 && (KD == 0 || KD == 1) && LC + LD >= 1), "bad ket specialisation");
  // input offsets of the three axes (0, 1, 2 unless relabelled)
  const int x0 = SPEC ? ax[0] : 0, x1 = SPEC ? ax[1] : 1, x2 = SPEC ? ax[2] : 2;
  constexpr int EB = LA + LB;
  constexpr int FK = LC + LD;
  constexpr int L = EB + FK;
  constexpr int NE = EB == 0 ? 1 : (EB == 1 ? 3 : 9);  // s | p | p + d
  constexpr int NF = FK == 2 ? 2 : 1;
  double acc[NC][NE][NF];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int e = 0; e < NE; ++e)
#pragma unroll
      for (int f = 0; f < NF; ++f) acc[c][e][f] = 0.0;

  const int b0 = __ldg(bra.pp_off + sb), b1 = __ldg(bra.pp_off + sb + 1);
  const int k0 = __ldg(ket.pp_off + sk), k1 = __ldg(ket.pp_off + sk + 1);
  for (int ib = b0; ib < b1; ++ib) {
    const double p = __ldg(bra.zeta + ib);
    const double Px = __ldg(bra.P + 3 * ib + x0), Py = __ldg(bra.P + 3 * ib + x1), Pz = __ldg(bra.P + 3 * ib + x2);
    double PA[3];
    PA[0] = __ldg(bra.PA + 3 * ib + x0); PA[1] = __ldg(bra.PA + 3 * ib + x1); PA[2] = __ldg(bra.PA + 3 * ib + x2);
    const double Kb = __ldg(bra.Kp + ib);
    for (int ik = k0; ik < k1; ++ik) {
      const double q = __ldg(ket.zeta + ik);
      double PQ[3];
      PQ[0] = Px - __ldg(ket.P + 3 * ik + x0);
      PQ[1] = Py - __ldg(ket.P + 3 * ik + x1);
      PQ[2] = Pz - __ldg(ket.P + 3 * ik + x2);
      const double s = p + q;
      // y = 1/sqrt(s): FP32 seed (rel. error < 2^-22), two Newton steps in FP64 (error < 2^-88)
      double y = (double)rsqrtf((float)s);
      y = y * fma(-0.5 * s, y * y, 1.5);
      y = y * fma(-0.5 * s, y * y, 1.5);
      const double is = y * y;
      const double rho = p * q * is;
      const double T = rho * (PQ[0] * PQ[0] + PQ[1] * PQ[1] + PQ[2] * PQ[2]);
      const double base = Kb * __ldg(ket.Kp + ik) * y;
      double F[L + 1];
      n_table += (T < kBoysTmax) ? 1u : 0u;
      boys_fm<L>(T, F, tab);
      double S0[L + 1];
#pragma unroll
      for (int m = 0; m <= L; ++m) S0[m] = base * F[m];
      // ---- bra vertical recurrence: [p|0]^(m), [d|0]^(m)  (shared by the ket components)
      double WP[3], e1[3][L > 0 ? L : 1], e2[6][L > 1 ? L - 1 : 1];
      if constexpr (EB >= 1) {
        const double c = -q * is;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          WP[i] = c * PQ[i];
#pragma unroll
          for (int m = 0; m < L; ++m) e1[i][m] = fma(PA[i], S0[m], WP[i] * S0[m + 1]);
        }
      }
      if constexpr (EB == 2) {
        const double o2p = __ldg(bra.o2z + ib), rp = q * is;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = i; j < 3; ++j)
#pragma unroll
            for (int m = 0; m < L - 1; ++m) {
              double v = fma(PA[j], e1[i][m], WP[j] * e1[i][m + 1]);
              if (i == j) v = fma(o2p, fma(-rp, S0[m + 1], S0[m]), v);
              e2[didx(i, j)][m] = v;
            }
      }
      if constexpr (FK == 0) {
        if constexpr (EB == 0) acc[0][0][0] += S0[0];
        if constexpr (EB >= 1) {
#pragma unroll
          for (int i = 0; i < 3; ++i) acc[0][i][0] += e1[i][0];
        }
        if constexpr (EB == 2) {
#pragma unroll
          for (int t = 0; t < 6; ++t) acc[0][3 + t][0] += e2[t][0];
        }
      } else {
        const double pis = p * is;
        double QC[3];
        QC[0] = __ldg(ket.PA + 3 * ik + x0); QC[1] = __ldg(ket.PA + 3 * ik + x1); QC[2] = __ldg(ket.PA + 3 * ik + x2);
        double WQ3[3] = {pis * PQ[0], pis * PQ[1], pis * PQ[2]};
        const double o2s = 0.5 * is;
        constexpr int MF = FK;
        double f1s[MF], f1p[3][MF], f1d[6][MF];
        // ---- ket vertical recurrence, level f = 1_kc (m <= FK-1)
        auto level1 = [&](int kc) {
          const double QCk = sel3(QC, kc), WQk = sel3(WQ3, kc);
#pragma unroll
          for (int m = 0; m < MF; ++m) {
            f1s[m] = fma(QCk, S0[m], WQk * S0[m + 1]);
            if constexpr (EB >= 1) {
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                double v = fma(QCk, e1[i][m], WQk * e1[i][m + 1]);
                if (i == kc) v = fma(o2s, S0[m + 1], v);
                f1p[i][m] = v;
              }
            }
            if constexpr (EB == 2) {
#pragma unroll
              for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j) {
                  double v = fma(QCk, e2[didx(i, j)][m], WQk * e2[didx(i, j)][m + 1]);
                  if constexpr (SPEC) {
                    if (i == KC && j == KC) v = fma(o2s, e1[i][m + 1] + e1[j][m + 1], v);
                    else if (i == KC) v = fma(o2s, e1[j][m + 1], v);
                    else if (j == KC) v = fma(o2s, e1[i][m + 1], v);
                  } else {
                    double lower = (i == kc ? e1[j][m + 1] : 0.0) + (j == kc ? e1[i][m + 1] : 0.0);
                    v = fma(o2s, lower, v);
                  }
                  f1d[didx(i, j)][m] = v;
                }
            }
          }
        };
        // ---- accumulate ket component cc from level 1 (and level 2 for a (pp) ket)
        auto accumulate = [&](int cc, int kc, int kd) {
          if constexpr (FK == 1) {
            if constexpr (EB == 0) acc[cc][0][0] += f1s[0];
            if constexpr (EB >= 1) {
#pragma unroll
              for (int i = 0; i < 3; ++i) acc[cc][i][0] += f1p[i][0];
            }
            if constexpr (EB == 2) {
#pragma unroll
              for (int t = 0; t < 6; ++t) acc[cc][3 + t][0] += f1d[t][0];
            }
          } else {
            const double QCl = sel3(QC, kd), WQl = sel3(WQ3, kd);
            // d_kl / 2q: a runtime factor, or (relabelled frame) present only when KC == KD
            constexpr bool DKL = !SPEC || KC == KD;
            const double o2q = DKL ? __ldg(ket.o2z + ik) : 0.0, rq = pis;
            const double dkl = SPEC ? o2q : ((kc == kd) ? o2q : 0.0);
            // [e|1k+1l] = QC_l [e|1k]^0 + WQ_l [e|1k]^1 + d_kl/(2q)([e|0]^0 - rho/q [e|0]^1) + e_l/(2s) [e-1_l|1k]^1
            if constexpr (EB == 0) {
              double v = fma(QCl, f1s[0], WQl * f1s[1]);
              if constexpr (DKL) v = fma(dkl, fma(-rq, S0[1], S0[0]), v);
              acc[cc][0][0] += v;
              acc[cc][0][1] += f1s[0];
            }
            if constexpr (EB >= 1) {
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                double v = fma(QCl, f1p[i][0], WQl * f1p[i][1]);
                if constexpr (DKL) v = fma(dkl, fma(-rq, e1[i][1], e1[i][0]), v);
                if (i == kd) v = fma(o2s, f1s[1], v);
                acc[cc][i][0] += v;
                acc[cc][i][1] += f1p[i][0];
              }
            }
            if constexpr (EB == 2) {
#pragma unroll
              for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = i; j < 3; ++j) {
                  const int t = didx(i, j);
                  double v = fma(QCl, f1d[t][0], WQl * f1d[t][1]);
                  if constexpr (DKL) v = fma(dkl, fma(-rq, e2[t][1], e2[t][0]), v);
                  if constexpr (SPEC) {
                    if (i == KD && j == KD) v = fma(o2s, f1p[i][1] + f1p[j][1], v);
                    else if (i == KD) v = fma(o2s, f1p[j][1], v);
                    else if (j == KD) v = fma(o2s, f1p[i][1], v);
                  } else {
                    double lower = (i == kd ? f1p[j][1] : 0.0) + (j == kd ? f1p[i][1] : 0.0);
                    v = fma(o2s, lower, v);
                  }
                  acc[cc][3 + t][0] += v;
                  acc[cc][3 + t][1] += f1d[t][0];
                }
            }
          }
        };
        if constexpr (FK == 2 && NC > 1) {
          // level 1 depends only on kc: computed once per distinct kc of the group
#pragma unroll
          for (int kcv = 0; kcv < 3; ++kcv) {
            bool any = false;
#pragma unroll
            for (int cc = 0; cc < NC; ++cc) any = any || (kcs[cc] == kcv);
            if (!any) continue;
            level1(kcv);
#pragma unroll
            for (int cc = 0; cc < NC; ++cc)
              if (kcs[cc] == kcv) accumulate(cc, kcv, kds[cc]);
          }
        } else {
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) {
            level1(SPEC ? KC : kcs[cc]);
            accumulate(cc, SPEC ? KC : kcs[cc], SPEC ? KD : kds[cc]);
          }
        }
      }
    }
  }
  double CD3[3] = {0.0, 0.0, 0.0};
  if constexpr (FK == 2) {
    CD3[0] = __ldg(ket.AB + 3 * sk + x0); CD3[1] = __ldg(ket.AB + 3 * sk + x1); CD3[2] = __ldg(ket.AB + 3 * sk + x2);
  }
  double AB3[3] = {0.0, 0.0, 0.0};
  if constexpr (LB == 1) {
    AB3[0] = __ldg(bra.AB + 3 * sb + x0); AB3[1] = __ldg(bra.AB + 3 * sb + x1); AB3[2] = __ldg(bra.AB + 3 * sb + x2);
  }
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    // ---- ket horizontal recurrence
    double val[NE];
    if constexpr (FK == 2) {
      const double CDl = sel3(CD3, SPEC ? KD : kds[cc]);
#pragma unroll
      for (int e = 0; e < NE; ++e) val[e] = fma(CDl, acc[cc][e][1], acc[cc][e][0]);
    } else {
#pragma unroll
      for (int e = 0; e < NE; ++e) val[e] = acc[cc][e][0];
    }
    // ---- bra horizontal recurrence
#pragma unroll
    for (int c = 0; c < 9; ++c) out[cc][c] = 0.0;
    if constexpr (EB == 0) {
      out[cc][0] = val[0];
    } else if constexpr (LB == 0) {
#pragma unroll
      for (int i = 0; i < 3; ++i) out[cc][3 * i] = val[i];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const int t = i <= j ? didx(i, j) : didx(j, i);
          out[cc][3 * i + j] = fma(AB3[j], val[i], val[3 + t]);
        }
    }
  }
}

// FP64-pipe operations (DFMA, DMUL, DADD, FP64 conversions) per primitive
// quartet, counted from the code above, for the roofline of this kernel:
//   set-up 22; Boys tabulated branch 12 (+ 7 for L = 1, + 10 + 2L for L > 1), asymptotic
//   branch 12 + 2L, both + (L+1) for S0; bra recurrence 4 + 6L (p) and
//   1 + 18(L-1) more (d); ket: 5, level 1 per distinct kc FK x (2 | 9 | 33),
//   per component NE adds (ket ss), NE adds (level 1 only) or 6 | 19 | 67 (pp).
//   Relabelled frame (KC = 0): level 1 FK x (2 | 9 | 25); (pp) components
//   6 | 19 | 59 when KD = KC, 4 | 13 | 41 when KD != KC.
template <int EB, int FK, int NC, int KC = -1, int KD = -1>
__device__ __forceinline__ unsigned fixed_ops(int n_level1) {
  constexpr int L = EB + FK;
  constexpr int NE = EB == 0 ? 1 : (EB == 1 ? 3 : 9);
  constexpr bool SPEC = KC >= 0;
  int ops = 22 + (L + 1);
  if (EB >= 1) ops += 4 + 6 * L;
  if (EB == 2) ops += 1 + 18 * (L - 1);
  if (FK == 0) {
    ops += NE;
  } else {
    const int lvl1 = FK * (EB == 0 ? 2 : (EB == 1 ? 9 : (SPEC ? 25 : 33)));
    int acc = FK == 1 ? NE : (EB == 0 ? 6 : (EB == 1 ? 19 : 67));
    if (SPEC && FK == 2) acc = KC == KD ? (EB == 0 ? 6 : (EB == 1 ? 19 : 59)) : (EB == 0 ? 4 : (EB == 1 ? 13 : 41));
    ops += 5 + n_level1 * lvl1 + NC * acc;
  }
  return (unsigned)ops;
}

// KC >= 0: one ket component, evaluated in the relabelled frame of quartet()
// (KD = 0 for c = d, 1 otherwise); the results are written back to the bra
// rows of the input components.
template <int LA, int LB, int LC, int LD, int NC, int KC = -1, int KD = -1>
__device__ __forceinline__ void column_block(const PairSet& bra, int64_t sb, const PairSet& ket, const KetGroup& kg,
                                             double* __restrict__ out, int64_t ld, const double* __restrict__ tab,
                                             unsigned long long& ops) {
  int kcs[NC], kds[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    kcs[c] = c < kg.nc ? kg.kc[c] : kg.kc[0];
    kds[c] = c < kg.nc ? kg.kd[c] : kg.kd[0];
  }
  // relabelled axes: computation axis x is input axis ax[x]; axis 0 carries the
  // ket's c component and, for c != d, axis 1 its d component
  int ax[3] = {0, 1, 2};
  if constexpr (KC >= 0) {
    const int c0 = kcs[0], d0 = kds[0];
    ax[0] = c0;
    ax[1] = (LC + LD == 2 && d0 != c0) ? d0 : (c0 == 2 ? 0 : c0 + 1);
    ax[2] = 3 - ax[0] - ax[1];
  }
  double v[NC][9];
  unsigned n_table = 0;
  quartet<LA, LB, LC, LD, NC, KC, KD>(bra, sb, ket, kg.sp, kcs, kds, ax, tab, v, n_table);
  {
    constexpr int L = LA + LB + LC + LD;
    int n_level1 = NC;
    if (LC + LD == 2 && NC > 1) {  // distinct kc values (level 1 shared per kc)
      n_level1 = 0;
      for (int kcv = 0; kcv < 3; ++kcv) {
        bool any = false;
        for (int cc = 0; cc < NC; ++cc) any = any || (kcs[cc] == kcv);
        n_level1 += any ? 1 : 0;
      }
    }
    const unsigned long long nq = (unsigned long long)(__ldg(bra.pp_off + sb + 1) - __ldg(bra.pp_off + sb)) *
                                  (unsigned long long)(__ldg(ket.pp_off + kg.sp + 1) - __ldg(ket.pp_off + kg.sp));
    ops += nq * fixed_ops<LA + LB, LC + LD, NC, KC, KD>(n_level1) + (unsigned long long)n_table * (12 + (L == 1 ? 7 : (L > 1 ? 10 + 2 * L : 0))) +
           (nq - n_table) * (12 + 2 * L);
  }
  const int32_t* rw = bra.row + 9 * sb;
#pragma unroll
  for (int cc = 0; cc < NC; ++cc) {
    if (cc >= kg.nc) break;
    double* o = out + (int64_t)kg.slot[cc] * ld;
#pragma unroll
    for (int c = 0; c < 9; ++c) {
      if (LA == 0 && c != 0) continue;
      if (LA == 1 && LB == 0 && (c % 3) != 0) continue;
      // component c = 3 i + j of the computation frame is (ax[i], ax[j]) of the input
      const int ci = KC < 0 ? c : (LA == 0 ? 0 : (LB == 0 ? 3 * ax[c / 3] : 3 * ax[c / 3] + ax[c % 3]));
      const int32_t r = __ldg(rw + ci);
      if (r >= 0) o[r] = v[cc][c];
    }
  }
}

// One work item: bra shell pairs [b0 + 128 tile, +128) of one class against ket group g.
template <int LA, int LB>
__device__ __forceinline__ void column_item(const PairSet& bra, const int64_t* __restrict__ order, int64_t b0,
                                            int64_t b1, const PairSet& ket, const KetGroup* __restrict__ groups,
                                            int64_t tile, int g, double* __restrict__ out, int64_t ld,
                                            const double* __restrict__ tab, unsigned long long& ops) {
  const KetGroup kg = groups[g];
  const int64_t ib = b0 + tile * 128 + threadIdx.x;
  if (ib < b1) {
    // bra shell pair: the ib-th of the class range, or the ib-th entry of a subset list
    const int64_t sb = order ? __ldg(order + ib) : ib;
    const int cls = kg.lc * 2 + kg.ld;
    if (cls == 0) column_block<LA, LB, 0, 0, 1>(bra, sb, ket, kg, out, ld, tab, ops);
    else if (cls == 2) {
      // single ket components in the relabelled frame (ket direction on axis 0)
      if (kg.nc == 1) column_block<LA, LB, 1, 0, 1, 0, 0>(bra, sb, ket, kg, out, ld, tab, ops);
      else column_block<LA, LB, 1, 0, 3>(bra, sb, ket, kg, out, ld, tab, ops);
    } else {
      if (kg.nc == 1) {
        if (kg.kc[0] == kg.kd[0]) column_block<LA, LB, 1, 1, 1, 0, 0>(bra, sb, ket, kg, out, ld, tab, ops);
        else column_block<LA, LB, 1, 1, 1, 0, 1>(bra, sb, ket, kg, out, ld, tab, ops);
      } else if (kg.nc <= 3) column_block<LA, LB, 1, 1, 3>(bra, sb, ket, kg, out, ld, tab, ops);
      else column_block<LA, LB, 1, 1, kMaxKetGroup>(bra, sb, ket, kg, out, ld, tab, ops);
    }
  }
}

}  // namespace
}  // namespace cd
