/*
 * cderi.h -- C ABI of the B300 Cholesky-decomposed ERI library (libcderi.so).
 *
 * The library computes, on one GPU (sm_103a):
 *   1. the threshold-truncated, fully pivoted Cholesky decomposition of the
 *      atomic-orbital electron-repulsion matrix over composite pair indices,
 *      (mu nu|sigma rho) ~ sum_P L^P_{mu nu} L^P_{sigma rho}, with the ERI
 *      columns computed on demand (arXiv 2609.00306, Sec. 2: diagonal D^1,
 *      argmax pivot, Eq. (subtr), Eq. (diag), stop when max D < tau);
 *   2. the Coulomb and exchange matrices J, K of a closed-shell density
 *      D = 2 C C^T from those vectors (Sec. 4.1: J at O(N^2 M), K at O(O N^2 M)).
 *
 * Conventions used by every entry point
 *   - Basis functions are numbered shell by shell; a Cartesian p shell holds
 *     x, y, z in that order.  A composite pair (mu, nu), mu >= nu, has packed
 *     index mu*(mu+1)/2 + nu.  The *rows* of a factor are the screened pairs in
 *     increasing packed index; every Cholesky vector has one entry per row.
 *   - Matrices are row-major.  "Host" pointers are ordinary CPU memory;
 *     "device" pointers are CUDA global memory of the current device.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Entry points that return results to host memory synchronise that stream.
 *   - Every entry point returns CD_OK (0) or a negative CD_E* code; the message
 *     of the last failure on the calling thread is returned by cd_last_error().
 *     On failure nothing is allocated and output handles are set to NULL.
 *   - Ownership: the caller owns every buffer it passes in; objects created by
 *     the library (cd_system_t, cd_factor_t) are freed with their *_free call.
 */
#ifndef CDERI_H
#define CDERI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define CD_OK        0
#define CD_EINVAL   -1   /* malformed argument (NaN, l > 1, bad size, ...) */
#define CD_ENOMEM   -2   /* device footprint over the budget or allocation failed */
#define CD_ENOTPSD  -3   /* pivot diagonal <= 0 while max D >= tau, or D < -1e-10 max D^1 */
#define CD_ETIMEOUT -4   /* a bounded device wait gave up */
#define CD_ECUDA    -5   /* CUDA runtime error */

/* ---- precision / mode flags --------------------------------------------- */
#define CD_FP64          0  /* vectors stored FP64; J/K in FP64 */
#define CD_VEC_FP32      1  /* after the (FP64) factorisation, vectors rounded once to FP32 and kept
                               * only in FP32 (the FP64 array is released: half the memory); every
                               * consumer reads the FP32 values, accumulating in FP64 */

#define CD_JK_FP64       0  /* J and K contractions in FP64 */
#define CD_JK_BF16X3     1  /* FP32 vectors; BF16 tensor-core products of 3 exact 8-bit slices per operand row */
#define CD_JK_BF16X4     2  /* as CD_JK_BF16X3 with 4 slices (32-bit fixed point below each row maximum) */
#define CD_JK_BF16X5     3  /* as CD_JK_BF16X3 with 5 slices (40-bit fixed point below each row maximum) */
#define CD_JK_DEVICE     0x100 /* flag: C_occ, J, K are device pointers (else host) */
#define CD_JK_ONLY_J     0x200 /* flag: compute J only (K may be NULL) */
#define CD_JK_ONLY_K     0x400 /* flag: compute K only (J may be NULL) */
#define CD_JK_VEC_FP32   0x800 /* flag (mixed modes): contract FP32-rounded vectors even if FP64 ones are stored */

/* ---- inputs --------------------------------------------------------------- */
/* Basis of contracted Cartesian Gaussian shells (all host pointers, read-only,
 * caller-owned).  Coefficients multiply normalised primitives; the library
 * rescales each contracted function to unit self-overlap. */
typedef struct {
  int32_t n_shells;
  const double*  center;   /* [n_shells][3], bohr */
  const int32_t* l;        /* [n_shells], 0 = s, 1 = p (x, y, z) */
  const int32_t* nprim;    /* [n_shells], 1 .. CD_MAX_PRIM */
  const double*  exps;     /* [sum nprim], > 0 */
  const double*  coefs;    /* [sum nprim] */
} cd_basis_t;

#define CD_MAX_PRIM 16

typedef struct {
  double  tau;          /* decomposition threshold: stop when max residual diagonal < tau (Sec. 2) */
  double  schwarz;      /* shell-pair screening threshold (0 keeps every pair) */
  int32_t vec_precision;/* CD_FP64 or CD_VEC_FP32 */
  int32_t block;        /* speculative column block b (0 = default 64; 1 .. 256) */
  int64_t max_vectors;  /* cap on M (0 = min(rows, 16 N)); CD_ENOMEM when exceeded */
  double  mem_budget_gb;/* device footprint cap for the factor (0 = 90% of free memory) */
  const int64_t* forced_pivots; /* test hook: host list of pivot rows to follow (NULL = argmax) */
  int64_t n_forced;
  int32_t update;       /* column update of Eq. (subtr): CD_UPDATE_SLICE (default) or CD_UPDATE_FP64 */
  int32_t algorithm;    /* pivot policy: CD_ALG_FULL (default), CD_ALG_SPAN or CD_ALG_TWOSTEP (below) */
  double  span;         /* span factor eta in (0, 1] of CD_ALG_SPAN / CD_ALG_TWOSTEP (0 = 0.01) */
  const uint8_t* candidates; /* host [n_rows] (system row order), nonzero = the row may be a pivot;
                              * NULL = every row.  The Cholesky basis is then chosen from that
                              * block of the matrix only (Sec. 6.2: the (LL|LL) diagonals of the
                              * spin-free relativistic matrix); the stop test max D < tau runs over
                              * the candidate rows, the vectors still cover every row, and rows
                              * outside the block carry no tau guarantee.  With CD_ALG_TWOSTEP the
                              * first step never touches the other rows. */
  double  diag_shift;   /* test hook: decompose with every starting diagonal lowered by this amount,
                         * i.e. the diagonal of A - shift I, indefinite once shift exceeds the
                         * smallest diagonal; the decomposition must then stop with CD_ENOTPSD
                         * (0 = off) */
} cd_opts_t;

/* Pivot policies.
 *  CD_ALG_FULL    fully pivoted recursion of Sec. 2: every step takes the global
 *                 argmax of the residual diagonal (the block of b columns is
 *                 speculative and only decides which integrals are computed).
 *  CD_ALG_SPAN    partially pivoted decomposition with a span factor (Sec. 3,
 *                 Koch et al. 2003): each macro iteration takes the qualified
 *                 set Q = the b largest residual diagonals >= max(eta * Dmax,
 *                 tau), computes their columns, and then takes vectors inside Q
 *                 (largest residual first, ties to the lowest row) while the
 *                 largest one left is >= that threshold.  Vectors over all rows.
 *  CD_ALG_TWOSTEP the two-step scheme of Sec. 3: step 1 is CD_ALG_SPAN on the
 *                 rows whose residual diagonal is >= tau only (rows that fall
 *                 below tau are dropped for good, the kept rows compacted), and
 *                 gives the Cholesky basis B; step 2 computes the vectors of B
 *                 over all rows, L = (.|B) M^-T with S = M M^T the metric on B
 *                 (Eq. (CVsLT)), by the blocked recursion over B in order --
 *                 the same numbers as a forward substitution with the metric's
 *                 Cholesky factor.  stats[13] = step-1 ms, stats[14] = step-1
 *                 macro iterations, stats[15] = step-1 ERI columns.
 * With eta = 1 (or b = 1) both span policies reduce to full pivoting. */
#define CD_ALG_FULL     0
#define CD_ALG_SPAN     1
#define CD_ALG_TWOSTEP  2

#define CD_UPDATE_SLICE  0  /* exact-slice BF16 tensor-core GEMM, 7 slices (56-bit fixed point per row) */
#define CD_UPDATE_FP64   1  /* register-tiled FP64 DFMA GEMM */

typedef struct cd_system cd_system_t;   /* basis + screened pair list on the device */
typedef struct cd_factor cd_factor_t;   /* Cholesky basis and vectors on the device */

/* ---- system (basis, screening) ------------------------------------------ */
/* Validate and normalise the basis, compute the diagonal D^1 = (mu nu|mu nu)
 * of every pair on the GPU (Sec. 2, the starting diagonal of the recursion;
 * kernel: ERI diagonal) and keep the shell pairs (AB) with
 * sqrt(max_{mu nu in AB} D_{mu nu} * max D) >= schwarz (the integral
 * prescreening of Sec. 1, read at shell-pair granularity).  *out receives a
 * library-owned object (free with cd_system_free).  Errors: CD_EINVAL on a
 * malformed basis (NaN, exponent <= 0, l > 1, nprim out of range), CD_ECUDA,
 * CD_ENOMEM; *out is NULL then. */
int cd_system_create(const cd_basis_t* basis, double schwarz, void* stream, cd_system_t** out);
/* Frees a system and its device memory (NULL is ignored).  A factor made on
 * it with cd_eri_factor_sys must be freed first. */
void cd_system_free(cd_system_t* sys);
/* n_basis, number of rows (screened pairs), number of kept shell pairs
 * (each output may be NULL).  CD_EINVAL if sys is NULL. */
int cd_system_info(const cd_system_t* sys, int32_t* n_basis, int64_t* n_rows, int64_t* n_shell_pairs);
/* Host copies, caller-owned arrays of n_rows entries: packed index of each row
 * (may be NULL) and the row's diagonal D^1 = (row|row) of Sec. 2 (may be
 * NULL).  CD_EINVAL if sys is NULL. */
int cd_system_rows(const cd_system_t* sys, int64_t* packed, double* diag);

/* ERI columns (kernel a, column mode): out[j][r] = (row r | row cols[j]) for
 * j < ncols, r < n_rows -- the integral column (.|K) that opens Eq. (subtr)
 * of Sec. 2.  cols: host array of row indices.  out: caller-owned device
 * pointer, row-major with leading dimension ld >= n_rows (doubles).  Runs on
 * `stream` and synchronises it.  CD_EINVAL on a row out of range or
 * ld < n_rows, CD_ECUDA. */
int cd_eri_columns(const cd_system_t* sys, const int64_t* cols, int32_t ncols,
                   double* out, int64_t ld, void* stream);

/* ---- factorisation -------------------------------------------------------- */
/* Full pipeline: cd_system_create + the pivoted decomposition (Sec. 2).
 * Blocked speculative scheme: the b largest candidates' ERI columns are computed
 * at once (kernel a) and brought up to date by one GEMM against the existing
 * vectors (kernel c, FP64); each step then takes the global argmax of the
 * residual diagonal (kernel b) -- so the pivot sequence is the one of the plain
 * recursion -- and finalises the vector from its column if it is in the block,
 * otherwise starts a new block.  *out is NULL on failure. */
int cd_eri_factor(const cd_basis_t* basis, const cd_opts_t* opts, void* stream, cd_factor_t** out);
/* Same on an existing system (the factor keeps a reference; free the factor
 * before the system). */
int cd_eri_factor_sys(cd_system_t* sys, const cd_opts_t* opts, void* stream, cd_factor_t** out);
/* Frees a factor, its vectors and (for cd_eri_factor) its system; NULL is
 * ignored. */
void cd_factor_free(cd_factor_t* f);
/* M (vectors), number of rows, N, and the residual max diagonal at exit, which
 * is < tau after a completed decomposition (the truncation of Sec. 2: every
 * element of the residual matrix is then bounded by it).  Outputs may be NULL. */
int cd_factor_info(const cd_factor_t* f, int64_t* M, int64_t* n_rows, int32_t* n_basis, double* max_resid_diag);
/* The Cholesky basis {|K)} of Sec. 2 -- the pivots in the order taken -- as
 * host copies: row indices [M] and packed pair indices [M] (either may be
 * NULL), gaps [M] (max D - D_pivot when each pivot was taken; 0 unless forced;
 * may be NULL), and the final residual diagonal [n_rows] (may be NULL).  All
 * arrays caller-owned.  The pivots are int64 row indices (rows index the
 * screened pairs) and the pairs are packed indices mu(mu+1)/2 + nu rather
 * than (mu, nu) tuples: both are one integer per pivot, and the packed index
 * is the pair index of the paper's MN(N+1)/2 storage (Sec. 4.1). */
int cd_factor_pivots(const cd_factor_t* f, int64_t* piv_rows, int64_t* piv_packed, double* gaps, double* resid_diag);
/* The tracked residual diagonal D_{K} of every pivot when it was taken -- the
 * divisor of Eq. (subtr) -- into out [M] (host, caller-owned).  Two correct
 * runs can order near-tied pivots differently; comparing these values at the
 * first difference tells a near-tie (|dD| < 1e-12) from an error. */
int cd_factor_pivot_diag(const cd_factor_t* f, double* out);
/* The vectors L^K_{mu nu} (Sec. 2; stored in core, M x N(N+1)/2 words in the
 * paper's Sec. 4.1, here M x n_rows over the screened pairs).  If L_host !=
 * NULL it receives [M][n_rows] doubles (caller-owned; converted from FP32 when
 * stored so).  *L_dev (may be NULL) receives the library-owned device pointer
 * of the stored array (valid until cd_factor_free), leading dimension *ld
 * (elements), *dtype 0 = FP64, 1 = FP32. */
int cd_factor_vectors(const cd_factor_t* f, double* L_host, const void** L_dev, int64_t* ld, int32_t* dtype);
/* Entries of every vector on selected rows: out[K][j] = L^K_{rows[j]} (FP64,
 * host, caller-owned [M][nrows]); rows: host array of row indices.  With
 * these, (p|q) ~ sum_K L^K_p L^K_q (Sec. 2) can be checked on any sample of
 * pairs.  Synchronous.  CD_EINVAL on a row out of range. */
int cd_factor_gather(const cd_factor_t* f, const int64_t* rows, int32_t nrows, double* out);
/* Measurement record (the paper has no counterpart; its tables report
 * wall times and vector counts per run).  Statistics of the factorisation,
 * 16 doubles into a caller-owned array: [0] system set-up ms (host
 * clock), [1] ERI-column kernels ms, [2] column-update kernels ms (CUDA
 * events; the update runs on the calling stream before the ERI columns of each
 * block), [3] pivot steps ms (host clock), [4] candidate selection
 * ms, [5] total ms;
 * [6] blocks, [7] ERI columns computed, [8] column-update flops (2 x rows x
 * columns x vectors applied), [9] ERI column entries computed, [10] M;
 * [11] 1 if the sliced tensor-core update ran; [12] FP64-pipe operations of
 * the ERI column kernels (counted by the kernels from per-primitive-quartet
 * operation counts of their recurrences); [13] first-step ms, [14] first-step
 * macro iterations, [15] first-step ERI columns of CD_ALG_TWOSTEP (0 otherwise). */
int cd_factor_stats(const cd_factor_t* f, double* stats16);
/* Work of the ERI column kernels (measurement; no counterpart in the paper):
 * primitive quartets evaluated, and their algorithmic FP64 operation count --
 * a plain Obara-Saika / Head-Gordon-Pople evaluation per quartet and class,
 * every add, multiply, fused multiply-add, reciprocal, square root and
 * exponential counted once, nothing shared between ket components -- the
 * numerator of the ERI kernel's roofline.  Either output may be NULL. */
int cd_factor_eri_work(const cd_factor_t* f, double* quartets, double* algorithmic_ops);
/* Device memory of the decomposition (measurement; the paper reports the
 * memory of its runs, e.g. the CV storage of Sec. 4.1): *peak_bytes = the
 * scratch pool's high-water mark during the call (residual diagonals, column
 * pool, BF16 slices of the vectors, ...) plus the vector array at its final
 * capacity -- both are largest together, at the end of the pivot loop; in a
 * batch the pool figure includes the systems running at the same time.
 * *resident_bytes = what the factor keeps afterwards (vectors, and their FP32
 * copy with CD_VEC_FP32).  Either output may be NULL. */
int cd_factor_memory(const cd_factor_t* f, double* peak_bytes, double* resident_bytes);
/* Number of CUDA kernel launches issued by this library in this process
 * (measurement; no counterpart in the paper). */
long long cd_kernel_launches(void);

/* ---- J and K (Sec. 4.1) ------------------------------------------------- */
/* J_{mu nu} = sum_P L^P_{mu nu} sum_{sigma rho} L^P_{sigma rho} D_{sigma rho},
 * K_{mu nu} = sum_P sum_{sigma rho} L^P_{mu sigma} D_{sigma rho} L^P_{rho nu},
 * D = 2 C_occ C_occ^T.  C_occ [N][n_occ], J, K [N][N], row-major; host pointers
 * unless CD_JK_DEVICE.  mode: CD_JK_FP64, CD_JK_BF16X3, _X4 or _X5 (mixed:
 * the stored vectors -- FP32 when the factor was made with CD_VEC_FP32, else
 * FP64 -- are cut into 3, 4 or 5 exact 8-bit slices per row and contracted on
 * the BF16 tensor cores; the FP32 storage itself limits K to ~1e-7 relative).  J (kernel d): two streamed GEMVs
 * over the vectors.  K (kernel e): B^P = L^P C_occ, K = 2 sum_P B^P B^P^T. */
int cd_jk(const cd_factor_t* f, const double* C_occ, int32_t n_occ,
          double* J, double* K, int32_t mode, void* stream);

/* ---- Cholesky vectors in the MO basis (Sec. 4.1: CASSCF, CC) --------------- */
/* out[P - P0][i][j] = sum_{mu nu} C[mu][i] L^P_{mu nu} C[nu][j] for
 * P0 <= P < P0 + nP and i, j < n_mo, with L^P the symmetric N x N unpacking of
 * vector P (zero on screened-out pairs).  C [N][n_mo] row-major; out
 * [nP][n_mo][n_mo] row-major, caller-owned; host pointers unless flags has
 * CD_JK_DEVICE.  slices: 0 = FP64 GEMMs (FP64 pipe), 3 / 4 / 5 / 7 = exact
 * 8-bit-slice GEMMs on the BF16 tensor cores, B^P = L^P C then C^T B^P
 * (7 slices: 56-bit fixed point per row, FP64-equivalent).  The work is done in
 * chunks of vectors; O(N^3) per vector.  Errors: CD_EINVAL (bad range or
 * slices), CD_ECUDA, CD_ETIMEOUT (bounded tensor-core pipeline wait). */
int cd_mo_vectors(const cd_factor_t* f, const double* C, int32_t n_mo, int64_t P0, int64_t nP, int32_t slices,
                  double* out, int32_t flags, void* stream);

/* ---- batches of independent systems ---------------------------------------- */
/* The paper has no counterpart: it factors one molecule at a time.  Batching
 * many small independent systems is a throughput pattern of this library.
 * For i < n_sys: cd_system_create(bases[i], opts[i].schwarz), the
 * decomposition with opts[i], and cd_jk(C_occ[i], n_occ[i], J[i], K[i],
 * jk_mode).  `workers` host threads (0 = 8), each with its own CUDA stream,
 * take systems from a shared queue (largest first) so that the kernels of
 * small systems overlap on the GPU.  Work starts after what is queued on
 * `stream` and `stream` waits for all of it; the call returns when done.
 * Returns the first failing system's code (message names the system). */
int cd_batch_run(int32_t n_sys, const cd_basis_t* bases, const cd_opts_t* opts, const double* const* C_occ,
                 const int32_t* n_occ, double* const* J, double* const* K, int32_t jk_mode, int32_t workers,
                 void* stream);

/* The same computation (no paper counterpart either), FP64 and FP64-equivalent,
 * with the decompositions and J/K builds of all systems in ONE persistent
 * kernel launch recorded in a CUDA graph.  Per system: the fully pivoted
 * decomposition of Sec. 2 (blocked, b = opts[i].block <= 64, 0 = 64; FP64 ERI
 * columns and pivot steps on the device; the column update of Eq. (subtr) as
 * exact 7-slice BF16 products on the tensor cores, opts[i].update =
 * CD_UPDATE_SLICE, the default, with the vectors kept as slices, or as FP64
 * DFMA tiles, CD_UPDATE_FP64; a batch with any CD_UPDATE_SLICE system runs
 * the tensor-core build for all), then J and K of Sec. 4.1 in FP64 with
 * D = 2 C_occ C_occ^T.  Set-up (screening, diagonal) runs first on host
 * workers.  Work items (a block's ERI columns, update tiles, the rows
 * of a pivot step, J/K tiles) are claimed by the CTAs from per-system job
 * words; the CTA that completes a job's last item publishes the next job.
 * Inputs: bases, opts (tau, schwarz, block, max_vectors: vector capacity per
 * system, 0 = 8 N; update; opts[0].mem_budget_gb caps the device buffer of a wave, 0 =
 * 90% of free memory; CD_ALG_FULL only, no forced pivots, mask or shift), C_occ[i]
 * host [N_i][n_occ[i]] row-major.  Outputs (host, caller-owned): J[i], K[i]
 * [N_i][N_i]; M_out[i] the vector counts (may be NULL); stats (may be NULL,
 * 40 entries): [0] set-up ms, [1] upload ms, [2] device ms of the launches, [3]
 * host ms of the launches and read-back, [4] CTAs, [5] bytes reserved, [6 + k]
 * CTA-seconds spent in items of kind k (1 select, 2 gather, 3 update, 4 step,
 * 5 density, 6 v = L d, 7 J_p = L^T v, 8 J unpack, 9 slicing, 10 ERI columns, 13 B = L C,
 * 14 partial K tiles, 15 K sums), [22] CTA-seconds spent looking for work,
 * [23 + k] FP64-pipe operations of the items of kind k (one per FMA as the
 * algorithm counts them; for ERI columns the kernel's executed operations),
 * [39] waves.  Waves: when the buffers of all systems together exceed the
 * budget, the systems (largest first) go into the first wave that still fits
 * it, and the waves run one after another, each as its own graph launch on one
 * device buffer the size of the largest wave.  All device memory is
 * allocated for the call and freed before it returns; `stream` is waited for
 * before the work starts.  Errors: CD_EINVAL (arguments, names the system),
 * CD_ENOMEM (one system alone over the budget, or a system needing more than
 * its max_vectors), CD_ENOTPSD, CD_ETIMEOUT (a CTA waited longer than the wait
 * limit of cd_set_wait_limit with no item completed anywhere; the launch
 * then stops cleanly), CD_ECUDA. */
int cd_batch_persistent(int32_t n_sys, const cd_basis_t* bases, const cd_opts_t* opts,
                        const double* const* C_occ, const int32_t* n_occ, double* const* J, double* const* K,
                        int64_t* M_out, double* stats, void* stream);

/* ---- building block: exact-slice tensor-core product ------------------------ */
/* out[i][j] = sum_k X[i][k] Y[j][k] for FP64 device matrices X [m][k] (leading
 * dimension ldx) and Y [n][k] (ldy); out FP64 device [m][n] (ldo).  Each row is
 * scaled by a power of two to |x| <= 1 and split into `slices` BF16 integer
 * slices (1, 3 or 7; 8 bits each), the slice products with s + t <= slices + 1
 * run on the tcgen05 tensor cores with exact FP32 accumulation over chunks of
 * k, and are summed in 64-bit fixed point (error-free splitting of Ozaki et
 * al., Numer. Algorithms 59 (2012) 95).  Error <= ~2^-(8 slices - 1) of
 * sum_k |x||y| scaled back.  This is the kernel behind the column update
 * (Eq. (subtr), 7 slices) and the mixed-precision exchange build (3 slices).
 * Allocates its own scratch; synchronises `stream`.  CD_ETIMEOUT if a bounded
 * pipeline wait gave up. */
int cd_slice_matmul(const double* X, int64_t ldx, int64_t m, const double* Y, int64_t ldy, int64_t n,
                    int64_t k, int32_t slices, double* out, int64_t ldo, void* stream);

/* ---- bounded device waits ------------------------------------------------------ */
/* Failure detection (no counterpart in the paper).  The tensor-core pipelines
 * (column update, mixed J/K, MO vectors, cd_slice_matmul) wait on mbarriers
 * with a wall-clock limit (default 2 s); a wait that runs out makes every CTA
 * of the launch stop issuing work, let its in-flight copies and MMAs finish,
 * free its tensor memory and return, and the entry point returns CD_ETIMEOUT
 * with the device still usable.  This sets the limit for launches issued from
 * now on (process-wide; seconds in [0, 3600], 0 = give up at the first wait
 * whose phase is not already complete) and returns the previous limit in *previous
 * (may be NULL).  Meant for tests of that error path and for tuning. */
int cd_set_wait_limit(double seconds, double* previous);

/* ---- errors ---------------------------------------------------------------- */
/* Message of the last failure on the calling thread (library-owned string,
 * valid until the thread's next failing call). */
const char* cd_last_error(void);
/* Library version string. */
const char* cd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CDERI_H */
