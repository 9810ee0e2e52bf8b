/*
 * cdoracle.c -- plain, slow FP64 CPU oracle for the Cholesky-decomposed ERI path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this file's library.  It shares no code, header,
 * table or constant with the CUDA path.
 *
 * What it computes, each piece written out from its definition:
 *   - Boys function F_m(T) (series + downward recursion; asymptotic form and
 *     upward recursion for large T) -- the standard textbook construction
 *     (Helgaker, Jorgensen, Olsen, "Molecular Electronic-Structure Theory",
 *     sec. 9.8).
 *   - Primitive Cartesian ERIs by the four-centre Obara-Saika recurrence
 *     (Obara & Saika, J. Chem. Phys. 84, 3963 (1986)), recursing on the first
 *     centre that still carries angular momentum.
 *   - Contracted, normalised s and Cartesian p functions.
 *   - Schwarz screening at shell-pair level (the paper only says integrals are
 *     prescreened, Sec. 1).
 *   - Fully pivoted, threshold-truncated Cholesky decomposition of the ERI
 *     matrix over composite pair indices (Sec. 2: D^1, argmax pivot, Eq. (subtr),
 *     Eq. (diag), stop when max D < tau), with a forced-pivot mode.
 *   - The exact ERI matrix over a list of pair indices (for J/K from exact
 *     integrals and for the dense checks in the tests).
 *   - Span-factor (partially pivoted) basis selection, with or without the
 *     discarding of rows below tau (Koch's one-step algorithm; the first step
 *     of the two-step scheme of Sec. 3), and the second step: the metric's
 *     Cholesky factor and the triangular solve of Eq. (CVsLT).
 *
 * Pair index convention: functions are numbered shell by shell (s; then p as
 * x, y, z); a composite pair (mu, nu) with mu >= nu has packed index
 * mu*(mu+1)/2 + nu.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt, for m = 0..mmax.     */
/* For T < 35: F_mmax from the convergent series                              */
/*   F_m(T) = exp(-T) sum_{i>=0} (2T)^i / [(2m+1)(2m+3)...(2m+2i+1)]          */
/* then the downward recursion F_m = (2T F_{m+1} + exp(-T)) / (2m+1).         */
/* For T >= 35: F_0 = (1/2) sqrt(pi/T) (erf(sqrt T) = 1 to double precision   */
/* there) and the upward recursion F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T).   */
/* ------------------------------------------------------------------------- */
void or_boys(int mmax, double T, double* F)
{
    double emT = exp(-T);
    if (T < 35.0) {
        double term = 1.0 / (2 * mmax + 1), sum = term;
        for (int i = 1; i < 2000; ++i) {
            term *= 2.0 * T / (2 * mmax + 2 * i + 1);
            sum += term;
            if (term < 1e-18 * sum) break;
        }
        F[mmax] = emT * sum;
        for (int m = mmax - 1; m >= 0; --m) F[m] = (2.0 * T * F[m + 1] + emT) / (2 * m + 1);
    } else {
        F[0] = 0.5 * sqrt(OR_PI / T);
        for (int m = 0; m < mmax; ++m) F[m + 1] = ((2 * m + 1) * F[m] - emT) / (2.0 * T);
    }
}

/* ------------------------------------------------------------------------- */
/* Obara-Saika recurrence for one primitive quartet.                         */
/* ------------------------------------------------------------------------- */
typedef struct {
    double PA[3], PB[3], QC[3], QD[3], WP[3], WQ[3];
    double o2p, o2q, o2pq;   /* 1/(2p), 1/(2q), 1/(2(p+q)) */
    double rp, rq;           /* rho/p, rho/q, rho = pq/(p+q) */
    double base;             /* 2 pi^{5/2} / (p q sqrt(p+q)) exp(-mu_ab AB^2) exp(-mu_cd CD^2) */
    double F[32];
} osq_t;

static int lsum(const int* a) { return a[0] + a[1] + a[2]; }

static double os_rec(const osq_t* s, const int* a, const int* b, const int* c, const int* d, int m)
{
    int la = lsum(a), lb = lsum(b), lc = lsum(c), ld = lsum(d);
    if (la + lb + lc + ld == 0) return s->base * s->F[m];
    int a1[3], b1[3], c1[3], d1[3], t[3];
    memcpy(a1, a, sizeof a1); memcpy(b1, b, sizeof b1);
    memcpy(c1, c, sizeof c1); memcpy(d1, d, sizeof d1);
    double v;
    if (la > 0 || lb > 0) {
        /* electron 1: lower the bra centre that carries angular momentum */
        int onA = la > 0;
        const int* x = onA ? a : b;
        int i = x[0] ? 0 : (x[1] ? 1 : 2);
        const double* PX = onA ? s->PA : s->PB;
        int* xr = onA ? a1 : b1;        /* the lowered function */
        xr[i] -= 1;
        const int* A = onA ? xr : a1;   /* (A B| after lowering */
        const int* B = onA ? b1 : xr;
        v = PX[i] * os_rec(s, A, B, c, d, m) + s->WP[i] * os_rec(s, A, B, c, d, m + 1);
        if (A[i] > 0) {  /* N_i(a)/(2p) [ (a-1_i b|cd)^m - rho/p (a-1_i b|cd)^{m+1} ] */
            memcpy(t, A, sizeof t); t[i] -= 1;
            v += A[i] * s->o2p * (os_rec(s, t, B, c, d, m) - s->rp * os_rec(s, t, B, c, d, m + 1));
        }
        if (B[i] > 0) {
            memcpy(t, B, sizeof t); t[i] -= 1;
            v += B[i] * s->o2p * (os_rec(s, A, t, c, d, m) - s->rp * os_rec(s, A, t, c, d, m + 1));
        }
        if (c[i] > 0) {  /* N_i(c)/(2(p+q)) (ab|c-1_i d)^{m+1} */
            memcpy(t, c, sizeof t); t[i] -= 1;
            v += c[i] * s->o2pq * os_rec(s, A, B, t, d, m + 1);
        }
        if (d[i] > 0) {
            memcpy(t, d, sizeof t); t[i] -= 1;
            v += d[i] * s->o2pq * os_rec(s, A, B, c, t, m + 1);
        }
        return v;
    }
    /* electron 2: lower the ket centre that carries angular momentum */
    int onC = lc > 0;
    const int* x = onC ? c : d;
    int i = x[0] ? 0 : (x[1] ? 1 : 2);
    const double* QX = onC ? s->QC : s->QD;
    int* xr = onC ? c1 : d1;
    xr[i] -= 1;
    const int* C = onC ? xr : c1;
    const int* D = onC ? d1 : xr;
    v = QX[i] * os_rec(s, a, b, C, D, m) + s->WQ[i] * os_rec(s, a, b, C, D, m + 1);
    if (C[i] > 0) {
        memcpy(t, C, sizeof t); t[i] -= 1;
        v += C[i] * s->o2q * (os_rec(s, a, b, t, D, m) - s->rq * os_rec(s, a, b, t, D, m + 1));
    }
    if (D[i] > 0) {
        memcpy(t, D, sizeof t); t[i] -= 1;
        v += D[i] * s->o2q * (os_rec(s, a, b, C, t, m) - s->rq * os_rec(s, a, b, C, t, m + 1));
    }
    /* bra sides are already zero here (la = lb = 0), so no cross terms */
    return v;
}

static void os_setup(osq_t* s, double ea, const double* A, double eb, const double* B,
                     double ec, const double* C, double ed, const double* D, int L)
{
    double p = ea + eb, q = ec + ed, pq = p + q;
    double P[3], Q[3], W[3], AB2 = 0, CD2 = 0, PQ2 = 0;
    for (int k = 0; k < 3; ++k) {
        P[k] = (ea * A[k] + eb * B[k]) / p;
        Q[k] = (ec * C[k] + ed * D[k]) / q;
        W[k] = (p * P[k] + q * Q[k]) / pq;
        AB2 += (A[k] - B[k]) * (A[k] - B[k]);
        CD2 += (C[k] - D[k]) * (C[k] - D[k]);
        PQ2 += (P[k] - Q[k]) * (P[k] - Q[k]);
        s->PA[k] = P[k] - A[k]; s->PB[k] = P[k] - B[k];
        s->QC[k] = Q[k] - C[k]; s->QD[k] = Q[k] - D[k];
        s->WP[k] = W[k] - P[k]; s->WQ[k] = W[k] - Q[k];
    }
    double rho = p * q / pq;
    s->o2p = 0.5 / p; s->o2q = 0.5 / q; s->o2pq = 0.5 / pq;
    s->rp = rho / p; s->rq = rho / q;
    s->base = 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(pq)) * exp(-ea * eb / p * AB2) * exp(-ec * ed / q * CD2);
    or_boys(L, rho * PQ2, s->F);
}

/* Primitive ERI of unnormalised Cartesian Gaussians x^a... exp(-ea r^2) etc. */
double or_eri_prim(const int* a, double ea, const double* A, const int* b, double eb, const double* B,
                   const int* c, double ec, const double* C, const int* d, double ed, const double* D)
{
    osq_t s;
    int L = lsum(a) + lsum(b) + lsum(c) + lsum(d);
    if (L > 30) return NAN;
    os_setup(&s, ea, A, eb, B, ec, C, ed, D, L);
    return os_rec(&s, a, b, c, d, 0);
}

/* ------------------------------------------------------------------------- */
/* Basis: contracted, normalised s and Cartesian p functions.                */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nsh, nbf;
    double* cen;     /* [nsh][3] */
    int* l;          /* [nsh] */
    int* nprim;      /* [nsh] */
    int* pofs;       /* [nsh] first primitive */
    double* exps;    /* [nprim_total] */
    double* dcoef;   /* [nprim_total] coefficient x primitive norm x contraction norm */
    int* bf_shell;   /* [nbf] */
    int* bf_cart;    /* [nbf][3] */
    int* sh_bf0;     /* [nsh] first function of the shell */
} obasis_t;

/* Normalised primitive: s -> (2a/pi)^{3/4}, Cartesian p -> (2a/pi)^{3/4} (4a)^{1/2}.
 * Same-centre overlaps of unnormalised primitives: s.s -> (pi/(a+b))^{3/2},
 * p_x.p_x -> (pi/(a+b))^{3/2} / (2(a+b)).  The contracted function is then
 * rescaled to unit self-overlap. */
void* or_basis_new(int nsh, const double* cen, const int* l, const int* nprim,
                   const double* exps, const double* coefs)
{
    obasis_t* b = (obasis_t*)calloc(1, sizeof(obasis_t));
    b->nsh = nsh;
    int np = 0, nbf = 0;
    for (int s = 0; s < nsh; ++s) {
        if (l[s] < 0 || l[s] > 1 || nprim[s] <= 0) { free(b); return NULL; }
        np += nprim[s];
        nbf += 2 * l[s] + 1;
    }
    b->nbf = nbf;
    b->cen = (double*)malloc(sizeof(double) * 3 * nsh);
    b->l = (int*)malloc(sizeof(int) * nsh);
    b->nprim = (int*)malloc(sizeof(int) * nsh);
    b->pofs = (int*)malloc(sizeof(int) * nsh);
    b->sh_bf0 = (int*)malloc(sizeof(int) * nsh);
    b->exps = (double*)malloc(sizeof(double) * np);
    b->dcoef = (double*)malloc(sizeof(double) * np);
    b->bf_shell = (int*)malloc(sizeof(int) * nbf);
    b->bf_cart = (int*)calloc(3 * nbf, sizeof(int));
    memcpy(b->cen, cen, sizeof(double) * 3 * nsh);
    memcpy(b->l, l, sizeof(int) * nsh);
    memcpy(b->nprim, nprim, sizeof(int) * nsh);
    memcpy(b->exps, exps, sizeof(double) * np);
    int po = 0, fo = 0;
    for (int s = 0; s < nsh; ++s) {
        b->pofs[s] = po;
        b->sh_bf0[s] = fo;
        for (int k = 0; k < 2 * l[s] + 1; ++k) {
            b->bf_shell[fo + k] = s;
            if (l[s] == 1) b->bf_cart[3 * (fo + k) + k] = 1;
        }
        /* primitive norms */
        for (int i = 0; i < nprim[s]; ++i) {
            double a = exps[po + i];
            double n = pow(2.0 * a / OR_PI, 0.75);
            if (l[s] == 1) n *= sqrt(4.0 * a);
            b->dcoef[po + i] = coefs[po + i] * n;
        }
        /* contraction norm: <chi|chi> over same-centre primitive overlaps */
        double S = 0.0;
        for (int i = 0; i < nprim[s]; ++i)
            for (int j = 0; j < nprim[s]; ++j) {
                double ab = exps[po + i] + exps[po + j];
                double ov = pow(OR_PI / ab, 1.5);
                if (l[s] == 1) ov /= 2.0 * ab;
                S += b->dcoef[po + i] * b->dcoef[po + j] * ov;
            }
        for (int i = 0; i < nprim[s]; ++i) b->dcoef[po + i] /= sqrt(S);
        po += nprim[s];
        fo += 2 * l[s] + 1;
    }
    return b;
}

void or_basis_free(void* h)
{
    obasis_t* b = (obasis_t*)h;
    if (!b) return;
    free(b->cen); free(b->l); free(b->nprim); free(b->pofs); free(b->sh_bf0);
    free(b->exps); free(b->dcoef); free(b->bf_shell); free(b->bf_cart); free(b);
}

int or_nbf(void* h) { return ((obasis_t*)h)->nbf; }

/* effective coefficients (c_i x N_i / sqrt<chi|chi>) of one shell */
void or_shell_coefs(void* h, int s, double* out)
{
    obasis_t* b = (obasis_t*)h;
    for (int i = 0; i < b->nprim[s]; ++i) out[i] = b->dcoef[b->pofs[s] + i];
}

/* Contracted ERI (i j | k l) over normalised functions. */
double or_eri(void* h, int i, int j, int k, int l)
{
    obasis_t* b = (obasis_t*)h;
    int f[4] = {i, j, k, l};
    int sh[4]; const int* cart[4]; const double* cen[4];
    for (int t = 0; t < 4; ++t) {
        sh[t] = b->bf_shell[f[t]];
        cart[t] = b->bf_cart + 3 * f[t];
        cen[t] = b->cen + 3 * sh[t];
    }
    int L = lsum(cart[0]) + lsum(cart[1]) + lsum(cart[2]) + lsum(cart[3]);
    double sum = 0.0;
    osq_t s;
    for (int pa = 0; pa < b->nprim[sh[0]]; ++pa)
        for (int pb = 0; pb < b->nprim[sh[1]]; ++pb)
            for (int pc = 0; pc < b->nprim[sh[2]]; ++pc)
                for (int pd = 0; pd < b->nprim[sh[3]]; ++pd) {
                    int ia = b->pofs[sh[0]] + pa, ib = b->pofs[sh[1]] + pb;
                    int ic = b->pofs[sh[2]] + pc, id = b->pofs[sh[3]] + pd;
                    os_setup(&s, b->exps[ia], cen[0], b->exps[ib], cen[1],
                             b->exps[ic], cen[2], b->exps[id], cen[3], L);
                    double v = os_rec(&s, cart[0], cart[1], cart[2], cart[3], 0);
                    sum += b->dcoef[ia] * b->dcoef[ib] * b->dcoef[ic] * b->dcoef[id] * v;
                }
    return sum;
}

static void unpack_pair(int64_t p, int* mu, int* nu)
{
    int64_t m = (int64_t)((sqrt(8.0 * (double)p + 1.0) - 1.0) / 2.0);
    while (m * (m + 1) / 2 > p) --m;
    while ((m + 1) * (m + 2) / 2 <= p) ++m;
    *mu = (int)m;
    *nu = (int)(p - m * (m + 1) / 2);
}

/* ERI matrix A[r][c] = (rows[r] | cols[c]) for packed pair indices. */
void or_eri_matrix(void* h, const int64_t* rows, int nr, const int64_t* cols, int nc, double* out)
{
    #pragma omp parallel for schedule(dynamic, 4)
    for (int r = 0; r < nr; ++r) {
        int i, j; unpack_pair(rows[r], &i, &j);
        for (int c = 0; c < nc; ++c) {
            int k, l; unpack_pair(cols[c], &k, &l);
            out[(int64_t)r * nc + c] = or_eri(h, i, j, k, l);
        }
    }
}

/* Diagonal (mu nu|mu nu) over all N(N+1)/2 packed pairs. */
void or_diag_all(void* h, double* out)
{
    obasis_t* b = (obasis_t*)h;
    int64_t np = (int64_t)b->nbf * (b->nbf + 1) / 2;
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < np; ++p) {
        int i, j; unpack_pair(p, &i, &j);
        out[p] = or_eri(h, i, j, i, j);
    }
}

/* Shell-pair Schwarz screening.  diag: the full packed diagonal.  A shell pair
 * (SA >= SB) is kept iff sqrt(max over its function pairs of D * max_all D) >= thr.
 * Writes the kept packed pair indices in increasing order; returns their count. */
int64_t or_screen(void* h, const double* diag, double thr, int64_t* rows_out)
{
    obasis_t* b = (obasis_t*)h;
    int64_t np = (int64_t)b->nbf * (b->nbf + 1) / 2;
    double dmax = 0.0;
    for (int64_t p = 0; p < np; ++p) if (diag[p] > dmax) dmax = diag[p];
    /* per shell pair maximum */
    int nsh = b->nsh;
    double* spmax = (double*)calloc((size_t)nsh * nsh, sizeof(double));
    for (int64_t p = 0; p < np; ++p) {
        int i, j; unpack_pair(p, &i, &j);
        int si = b->bf_shell[i], sj = b->bf_shell[j];
        double* x = &spmax[(size_t)si * nsh + sj];
        if (diag[p] > *x) *x = diag[p];
    }
    int64_t n = 0;
    for (int64_t p = 0; p < np; ++p) {
        int i, j; unpack_pair(p, &i, &j);
        int si = b->bf_shell[i], sj = b->bf_shell[j];
        if (sqrt(spmax[(size_t)si * nsh + sj] * dmax) >= thr) rows_out[n++] = p;
    }
    free(spmax);
    return n;
}

/* ------------------------------------------------------------------------- */
/* Memory order of the Eq. (subtr) sums.                                     */
/*                                                                           */
/* Every element of a new column is                                          */
/*     col_r = (r|p) - L^0_r L^0_p - L^1_r L^1_p - ... - L^{K-1}_r L^{K-1}_p  */
/* evaluated left to right.  Vectors are stored row-major [K][npairs], so a   */
/* loop over J for one r walks memory with a stride of npairs.  The default   */
/* order takes the rows in chunks (or_chunk_len) and runs J outermost        */
/* inside a chunk: each L^J is then read contiguously, and every element      */
/* still sees the same operations in the same order (J ascending), so both    */
/* orders give bit-identical results.  The plain per-element order and the    */
/* chunk length are selectable (or_set_order) so that a test can check that   */
/* identity with several chunks and a ragged last one.                       */
/* ------------------------------------------------------------------------- */
static int or_plain_order = 0;
static int64_t or_chunk_set = 0;   /* 0 = automatic */
void or_set_order(int plain, int chunk)
{
    or_plain_order = plain ? 1 : 0;
    or_chunk_set = chunk > 0 ? chunk : 0;
}
/* chunk length for npairs rows: at most 2048 (the working set of a chunk stays
 * in cache), and small enough to give every thread several chunks */
static int64_t or_chunk_len(int64_t npairs)
{
    if (or_chunk_set > 0) return or_chunk_set;
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    int64_t c = (npairs + 4 * (int64_t)nt - 1) / (4 * (int64_t)nt);
    c = (c + 7) / 8 * 8;
    if (c > 2048) c = 2048;
    if (c < 64) c = 64;
    return c;
}

/* out[r] = (r | k l) - sum_{J<K} L[J][r] * w[J * wstride] for r in [r0, r1),
 * J ascending for every r (the Eq. (subtr) sum with a strided weight list). */
static void or_subtr_rows(void* h, const int* ri, const int* rj, int64_t r0, int64_t r1, int k, int l,
                          const double* L, int64_t npairs, int K, const double* w, int64_t wstride,
                          double* out)
{
    if (or_plain_order) {
        for (int64_t r = r0; r < r1; ++r) {
            double col = or_eri(h, ri[r], rj[r], k, l);
            for (int J = 0; J < K; ++J) col -= L[(int64_t)J * npairs + r] * w[(int64_t)J * wstride];
            out[r] = col;
        }
        return;
    }
    for (int64_t r = r0; r < r1; ++r) out[r] = or_eri(h, ri[r], rj[r], k, l);
    for (int J = 0; J < K; ++J) {
        const double* LJ = L + (int64_t)J * npairs;
        const double wj = w[(int64_t)J * wstride];
        for (int64_t r = r0; r < r1; ++r) out[r] -= LJ[r] * wj;
    }
}

/* ------------------------------------------------------------------------- */
/* Fully pivoted incomplete Cholesky decomposition (Sec. 2).                  */
/*                                                                           */
/*   D^1_r = (r|r)                                   over the screened rows   */
/*   loop K = 0, 1, ...                                                       */
/*     Dmax = max_r D_r, p = argmax (ties -> lowest row)                      */
/*     stop when Dmax < tau                                                   */
/*     col_r = (r|p) - sum_{J<K} L^J_r L^J_p                  Eq. (subtr)     */
/*     L^K_r = col_r / sqrt(D_p)                              Eq. (subtr)     */
/*     D_r  -= (L^K_r)^2                                      Eq. (diag)      */
/*                                                                           */
/* Forced mode (nforced >= 0): the pivot of step K is forced[K] instead of    */
/* the argmax, for K < nforced, and the run stops after nforced steps; gap[K] */
/* records Dmax - D_forced at each step.                                      */
/* Candidate mask (cand != NULL): only rows with cand[r] != 0 may be pivots,  */
/* and Dmax, the argmax and the stop test run over those rows; the vectors    */
/* still cover every row.  This is the restriction of the Cholesky basis to  */
/* one block of the matrix (the (LL|LL) diagonals in the spin-free            */
/* relativistic case of Sec. 6.2, where no (SS|SS) diagonals are then needed).  */
/* L is row-major [mcap][npairs].  Returns M >= 0, or                         */
/*   -1 if M would exceed mcap, -2 if a pivot diagonal is not positive or a   */
/*   residual diagonal is below -1e-10 * max D^1 (matrix not PSD).            */
/* ------------------------------------------------------------------------- */
int or_cd(void* h, const int64_t* rows, int64_t npairs, double tau,
          const int64_t* forced, int nforced, int mcap,
          int64_t* piv_out, double* L, double* D, double* gap, double* pivD,
          const unsigned char* cand)
{
    int* ri = (int*)malloc(sizeof(int) * npairs);
    int* rj = (int*)malloc(sizeof(int) * npairs);
    for (int64_t r = 0; r < npairs; ++r) unpack_pair(rows[r], &ri[r], &rj[r]);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < npairs; ++r) D[r] = or_eri(h, ri[r], rj[r], ri[r], rj[r]);
    double d1max = 0.0;
    for (int64_t r = 0; r < npairs; ++r) if (D[r] > d1max) d1max = D[r];

    int K = 0, status = 0;
    for (;;) {
        double dmax = -INFINITY; int64_t am = -1;
        for (int64_t r = 0; r < npairs; ++r)
            if ((!cand || cand[r]) && D[r] > dmax) { dmax = D[r]; am = r; }
        int64_t p;
        if (nforced >= 0) {
            if (K >= nforced) break;
            p = forced[K];
            if (p < 0 || p >= npairs) { status = -3; break; }
        } else {
            if (!(dmax >= tau)) break;
            p = am;
        }
        if (K >= mcap) { status = -1; break; }
        if (!(D[p] > 0.0)) { status = -2; break; }
        if (gap) gap[K] = dmax - D[p];
        if (pivD) pivD[K] = D[p];
        double sq = sqrt(D[p]);
        int k = ri[p], l = rj[p];
        double* LK = L + (int64_t)K * npairs;
        const int64_t CH = or_chunk_len(npairs);
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r0 = 0; r0 < npairs; r0 += CH) {
            int64_t r1 = r0 + CH < npairs ? r0 + CH : npairs;
            or_subtr_rows(h, ri, rj, r0, r1, k, l, L, npairs, K, L + p, npairs, LK);
            for (int64_t r = r0; r < r1; ++r) LK[r] = LK[r] / sq;
        }
        int bad = 0;
        for (int64_t r = 0; r < npairs; ++r) {
            D[r] -= LK[r] * LK[r];
            if (D[r] < -1e-10 * d1max) bad = 1;
        }
        piv_out[K] = p;
        ++K;
        if (bad) { status = -2; break; }
    }
    free(ri); free(rj);
    return status < 0 ? status : K;
}

/* ------------------------------------------------------------------------- */
/* Span-factor (partially pivoted) selection of the Cholesky basis: Koch's    */
/* partially pivoted decomposition (Koch, Sanchez de Meras, Pedersen, J.      */
/* Chem. Phys. 118, 9481 (2003), cited in Sec. 3) and the first step of the   */
/* two-step scheme of Sec. 3 (sets of Table "two-step": B chosen basis, D     */
/* diagonals >= tau, Q qualified diagonals, C columns already used in the     */
/* current micro iteration).                                                  */
/*                                                                           */
/* One macro iteration:                                                       */
/*     Dmax = max_{r in D} D_r;  stop when Dmax < tau                         */
/*     thr  = max(span * Dmax, tau)                                           */
/*     Q    = rows r in D with D_r >= thr, largest first (ties: lowest row),  */
/*            at most qmax of them                                            */
/*     col_q = (r|q) - sum_{J<K} L^J_r L^J_q   for q in Q, r in D  Eq. (subtr)*/
/*     micro iterations, C = {}:                                              */
/*         q = argmax_{Q \ C} D_q (ties: lowest row); stop if D_q < thr       */
/*         L^K_r = col_q,r / sqrt(D_q)                  Eq. (subtr)           */
/*         col_q',r -= L^K_r L^K_q'   for q' in Q \ C                          */
/*         D_r -= (L^K_r)^2                              Eq. (diag)            */
/*         B += q, C += q, K += 1                                             */
/*     reduce = 1: D = {r in D : D_r >= tau}  (rows below tau are dropped for */
/*                 good: D_r never increases, Sec. 3)                         */
/* With reduce = 0 the rows are never dropped and L^K covers every row: that  */
/* is Koch's one-step algorithm and L is the final factor.  With reduce = 1   */
/* only the basis B (the pivots) is the result; the vectors then come from    */
/* or_cd_from_basis (second step).  The paper keeps the integrals of unused   */
/* qualified columns between macro iterations; this oracle recomputes them,   */
/* which changes the cost, not the result.  With span = 1 every macro         */
/* iteration takes exactly the argmax, i.e. full pivoting (or_cd).            */
/*                                                                           */
/* L is row-major [mcap][npairs]; entries of dropped rows are left at 0.      */
/* macro_start[i] = K at the start of macro iteration i (optional).           */
/* cand: candidate mask as for or_cd (NULL = every row); with reduce = 1 the  */
/* rows outside it are not carried through the first step at all.            */
/* Returns M >= 0, or -1 if M would exceed mcap, -2 if a pivot diagonal is    */
/* not positive or a residual below -1e-10 max D^1 (matrix not PSD).          */
/* ------------------------------------------------------------------------- */
int or_cd_span(void* h, const int64_t* rows, int64_t npairs, double tau, double span, int qmax, int reduce,
               int mcap, int64_t* piv_out, double* L, double* D, int* macro_start, int* n_macro,
               const unsigned char* cand)
{
    int* ri = (int*)malloc(sizeof(int) * npairs);
    int* rj = (int*)malloc(sizeof(int) * npairs);
    char* live = (char*)malloc(npairs);
    for (int64_t r = 0; r < npairs; ++r) unpack_pair(rows[r], &ri[r], &rj[r]);
    #pragma omp parallel for schedule(dynamic, 64)
    for (int64_t r = 0; r < npairs; ++r) D[r] = or_eri(h, ri[r], rj[r], ri[r], rj[r]);
    double d1max = 0.0;
    for (int64_t r = 0; r < npairs; ++r) if (D[r] > d1max) d1max = D[r];
    /* with a candidate mask and reduce = 1 the other rows are not needed at all */
    for (int64_t r = 0; r < npairs; ++r)
        live[r] = reduce ? (D[r] >= tau && (!cand || cand[r])) : 1;
    if (qmax < 1) qmax = 1;
    int64_t* Q = (int64_t*)malloc(sizeof(int64_t) * qmax);
    char* used = (char*)malloc(qmax);
    double* col = (double*)malloc(sizeof(double) * (size_t)qmax * npairs);

    int K = 0, status = 0, nm = 0;
    for (;;) {
        double dmax = -INFINITY;
        for (int64_t r = 0; r < npairs; ++r)
            if (live[r] && (!cand || cand[r]) && D[r] > dmax) dmax = D[r];
        if (!(dmax >= tau)) break;
        double thr = span * dmax;
        if (thr < tau) thr = tau;
        /* Q: the qmax largest D_r >= thr, by repeated selection */
        int nq = 0;
        while (nq < qmax) {
            int64_t best = -1;
            for (int64_t r = 0; r < npairs; ++r) {
                if (!live[r] || (cand && !cand[r]) || !(D[r] >= thr)) continue;
                int taken = 0;
                for (int i = 0; i < nq; ++i) if (Q[i] == r) { taken = 1; break; }
                if (taken) continue;
                if (best < 0 || D[r] > D[best]) best = r;
            }
            if (best < 0) break;
            Q[nq++] = best;
        }
        if (macro_start) macro_start[nm] = K;
        ++nm;
        /* columns of Q over the live rows, minus all previous vectors */
        for (int i = 0; i < nq; ++i) {
            int64_t q = Q[i];
            double* c = col + (size_t)i * npairs;
            int k = ri[q], l = rj[q];
            /* live rows only; a dropped row keeps 0 in every vector */
            const int64_t CH = or_chunk_len(npairs);
            #pragma omp parallel for schedule(dynamic, 1)
            for (int64_t r0 = 0; r0 < npairs; r0 += CH) {
                int64_t r1 = r0 + CH < npairs ? r0 + CH : npairs;
                for (int64_t a = r0; a < r1;) {
                    if (!live[a]) { c[a++] = 0.0; continue; }
                    int64_t e = a;
                    while (e < r1 && live[e]) ++e;
                    or_subtr_rows(h, ri, rj, a, e, k, l, L, npairs, K, L + q, npairs, c);
                    a = e;
                }
            }
            used[i] = 0;
        }
        /* micro iterations */
        for (;;) {
            int bi = -1;
            for (int i = 0; i < nq; ++i) {
                if (used[i]) continue;
                if (bi < 0 || D[Q[i]] > D[Q[bi]] || (D[Q[i]] == D[Q[bi]] && Q[i] < Q[bi])) bi = i;
            }
            if (bi < 0 || !(D[Q[bi]] >= thr)) break;
            int64_t q = Q[bi];
            if (K >= mcap) { status = -1; break; }
            if (!(D[q] > 0.0)) { status = -2; break; }
            double sq = sqrt(D[q]);
            double* LK = L + (int64_t)K * npairs;
            const double* cq = col + (size_t)bi * npairs;
            for (int64_t r = 0; r < npairs; ++r) LK[r] = live[r] ? cq[r] / sq : 0.0;
            used[bi] = 1;
            for (int i = 0; i < nq; ++i) {
                if (used[i]) continue;
                double* c = col + (size_t)i * npairs;
                double f = LK[Q[i]];
                for (int64_t r = 0; r < npairs; ++r) if (live[r]) c[r] -= LK[r] * f;
            }
            int bad = 0;
            for (int64_t r = 0; r < npairs; ++r) {
                if (!live[r]) continue;
                D[r] -= LK[r] * LK[r];
                if (D[r] < -1e-10 * d1max) bad = 1;
            }
            piv_out[K] = q;
            ++K;
            if (bad) { status = -2; break; }
        }
        if (status < 0) break;
        if (reduce)
            for (int64_t r = 0; r < npairs; ++r) if (live[r] && !(D[r] >= tau)) live[r] = 0;
    }
    if (n_macro) *n_macro = nm;
    free(ri); free(rj); free(live); free(Q); free(used); free(col);
    return status < 0 ? status : K;
}

/* ------------------------------------------------------------------------- */
/* Second step of the two-step scheme (Sec. 3, Eqs. (DF), (CVsLT)): given the */
/* Cholesky basis B = piv[0..M), the metric S_{JK} = (B_J|B_K) is factored as */
/* S = M M^T (plain Cholesky, no pivoting) and the vectors solve              */
/*     L^K_r = sum_P (r|B_P) (M^{-T})_{PK},                                   */
/* i.e. row by row, by forward substitution with the lower triangle of M:     */
/*     L^K_r = ((r|B_K) - sum_{J<K} L^J_r M_{KJ}) / M_{KK}.                    */
/* L is row-major [M][npairs].  Returns 0, or -2 if the metric is not         */
/* positive definite.                                                          */
/* ------------------------------------------------------------------------- */
int or_cd_from_basis(void* h, const int64_t* rows, int64_t npairs, const int64_t* piv, int M, double* L)
{
    int* ri = (int*)malloc(sizeof(int) * npairs);
    int* rj = (int*)malloc(sizeof(int) * npairs);
    for (int64_t r = 0; r < npairs; ++r) unpack_pair(rows[r], &ri[r], &rj[r]);
    double* S = (double*)calloc((size_t)M * M, sizeof(double));
    for (int J = 0; J < M; ++J)
        for (int K = 0; K <= J; ++K)
            S[(size_t)J * M + K] = or_eri(h, ri[piv[J]], rj[piv[J]], ri[piv[K]], rj[piv[K]]);
    /* S = M M^T, lower triangle in place (Cholesky-Banachiewicz) */
    int status = 0;
    for (int J = 0; J < M && status == 0; ++J) {
        for (int K = 0; K <= J; ++K) {
            double s = S[(size_t)J * M + K];
            for (int P = 0; P < K; ++P) s -= S[(size_t)J * M + P] * S[(size_t)K * M + P];
            if (K == J) {
                if (!(s > 0.0)) { status = -2; break; }
                S[(size_t)J * M + J] = sqrt(s);
            } else {
                S[(size_t)J * M + K] = s / S[(size_t)K * M + K];
            }
        }
    }
    if (status == 0) {
        const int64_t CH = or_chunk_len(npairs);
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t r0 = 0; r0 < npairs; r0 += CH) {
            int64_t r1 = r0 + CH < npairs ? r0 + CH : npairs;
            for (int K = 0; K < M; ++K) {
                double* LK = L + (int64_t)K * npairs;
                or_subtr_rows(h, ri, rj, r0, r1, ri[piv[K]], rj[piv[K]], L, npairs, K, S + (size_t)K * M, 1, LK);
                for (int64_t r = r0; r < r1; ++r) LK[r] = LK[r] / S[(size_t)K * M + K];
            }
        }
    }
    free(S); free(ri); free(rj);
    return status;
}
