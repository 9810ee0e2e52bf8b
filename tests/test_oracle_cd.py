"""Pins for the oracle's Cholesky decomposition and J/K, against facts fixed
outside it:

* LAPACK's complete-pivoting Cholesky (dpstrf) on the same ERI matrix: same
  pivots (up to near-ties), same rank, same factor.
* The truncation bound of Sec. 2: once max D < tau, every element of the
  residual A - L L^T is bounded by tau (Cauchy-Schwarz on a PSD residual).
* The density-fitting form of the same vectors, Eq. (CVsLT): L = (.|P) M^-T
  with S = M M^T the metric on the pivots, by numpy Cholesky + triangular solve.
* Eckart-Young / Ky Fan: tr(A - L L^T) >= sum of the discarded eigenvalues.
* J and K from the vectors against J and K from the exact ERI tensor, within
  the tau bound, and to 1e-10 when tau is pushed to 1e-13.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack

import oracle
import synth


def _full(name):
    s = synth.make_workload(name)
    o = oracle.Oracle(s.basis)
    N = o.nbf
    rows = o.screen(s.schwarz)
    A = o.eri_matrix(rows)
    return s, o, rows, A


@pytest.fixture(scope="module")
def s40():
    s, o, rows, A = _full("s40")
    r = o.cd(rows, s.tau)
    return s, o, rows, A, r


@pytest.fixture(scope="module")
def sp8():
    s, o, rows, A = _full("sp8")
    r = o.cd(rows, s.tau)
    return s, o, rows, A, r


def test_cd_matches_lapack_dpstrf(s40):
    s, o, rows, A, r = s40
    c, piv, rank, info = scipy.linalg.lapack.dpstrf(A.copy(), lower=1, tol=s.tau)
    piv = piv - 1
    # dpstrf stops when the pivot is <= tol, the oracle when max D < tau: equal away from equality
    assert rank == r.M
    Lf = np.tril(c)[:, :rank]  # A[piv][:, piv] ~= Lf Lf^T
    # same pivot sequence, except where two candidate diagonals are within 1e-12
    same = piv[:rank] == r.piv
    if not np.all(same):
        # a divergence is allowed only at a near-tie: the residual diagonal after
        # the first k vectors (recomputed from A, not from the oracle's tracked D)
        # must be within 1e-12 at the two pivots
        k = int(np.argmin(same))
        Dk = np.diag(A) - np.sum(r.L[:k] ** 2, axis=0)
        assert abs(Dk[r.piv[k]] - Dk[piv[k]]) < 1e-12
    else:
        Lo = r.L[:, piv].T  # rows in dpstrf order
        assert np.max(np.abs(Lo - Lf)) < 1e-10 * np.max(np.abs(Lf))


def test_residual_bounded_by_tau(s40, sp8):
    for s, o, rows, A, r in (s40, sp8):
        R = A - r.L.T @ r.L
        dmax = r.D.max()
        assert dmax < s.tau
        assert np.max(np.abs(R)) <= dmax + 1e-13
        # the tracked residual diagonal is the diagonal of the residual matrix
        assert np.max(np.abs(np.diag(R) - r.D)) < 1e-13
        # every residual diagonal only loses a square per step (fl(D - L^2) <= D), so the
        # pivot diagonals, the running maxima, never increase, exactly; the last is >= tau
        assert np.all(r.pivD > 0)
        assert np.all(np.diff(r.pivD) <= 0.0)
        assert r.pivD[-1] >= s.tau > dmax


def test_density_fitting_route(s40, sp8):
    for s, o, rows, A, r in (s40, sp8):
        S = A[np.ix_(r.piv, r.piv)]
        M = np.linalg.cholesky(S)
        LDF = scipy.linalg.solve_triangular(M, A[:, r.piv].T, lower=True)  # M^-1 (P|.) = (L^T M^-T)^T
        assert np.max(np.abs(LDF - r.L)) < 1e-9 * np.max(np.abs(r.L))


def test_eckart_young_trace_bound(s40, sp8):
    for s, o, rows, A, r in (s40, sp8):
        w = np.linalg.eigvalsh(A)[::-1]
        tr_res = np.sum(r.D)
        assert tr_res >= np.sum(w[r.M:]) - 1e-12


def test_full_decomposition_reconstructs(sp8):
    s, o, rows, A, _ = sp8
    r = o.cd(rows, 1e-13)
    assert np.max(np.abs(A - r.L.T @ r.L)) < 1e-12


def test_forced_mode_replays_free_run(s40):
    s, o, rows, A, r = s40
    f = o.cd(rows, s.tau, forced=r.piv)
    assert f.M == r.M
    assert np.array_equal(f.piv, r.piv)
    assert np.max(np.abs(f.gap)) == 0.0
    assert np.array_equal(f.L, r.L)


def test_screening_keeps_everything_at_zero_threshold():
    s = synth.make_workload("sp8")
    o = oracle.Oracle(s.basis)
    N = o.nbf
    assert o.screen(0.0).shape[0] == N * (N + 1) // 2


def test_screening_drops_far_pairs():
    s = synth.make_lattice((4, 1, 1), seed=41, n_occ=2, tau=1e-5)
    o = oracle.Oracle(s.basis)
    d = o.diag_all()
    rows = o.screen(1e-3, d)
    mu, nu = oracle.unpack_pair(rows)
    # every kept function pair's shell pair has sqrt(max D_shellpair * max D) >= thr; check directly
    dmax = d.max()
    N = o.nbf
    shell_of = np.repeat(np.arange(s.basis.n_shells), 2 * s.basis.l + 1)
    allp = np.arange(d.shape[0])
    amu, anu = oracle.unpack_pair(allp)
    key = shell_of[amu] * 1000 + shell_of[anu]
    spmax = {}
    for k, v in zip(key, d):
        spmax[k] = max(spmax.get(k, 0.0), v)
    kept = set(rows.tolist())
    for p in allp:
        want = np.sqrt(spmax[key[p]] * dmax) >= 1e-3
        assert (p in kept) == want
    assert len(kept) < d.shape[0]


@pytest.mark.parametrize("name", ["s40", "sp8"])
def test_jk_cd_vs_exact_integrals(name):
    s = synth.make_workload(name)
    o = oracle.Oracle(s.basis)
    rows = o.screen(s.schwarz)
    r = o.cd(rows, s.tau)
    T = o.eri_tensor()
    Je, Ke = oracle.jk_exact(T, s.C_occ)
    J, K = oracle.jk_from_vectors(r.L, rows, s.C_occ)
    Dm = oracle.density(s.C_occ)
    bound = r.D.max() * np.sum(np.abs(Dm)) + 1e-12
    assert np.max(np.abs(J - Je)) <= bound
    assert np.max(np.abs(K - Ke)) <= bound
    # symmetric, and tr(DK) > 0 (K is PSD-weighted for a PSD density)
    assert np.allclose(J, J.T, atol=1e-13) and np.allclose(K, K.T, atol=1e-13)
    assert np.sum(Dm * K) > 0
    # nearly exact decomposition -> nearly exact J and K
    r2 = o.cd(rows, 1e-13)
    J2, K2 = oracle.jk_from_vectors(r2.L, rows, s.C_occ)
    assert np.max(np.abs(J2 - Je)) < 1e-10 * np.max(np.abs(Je))
    assert np.max(np.abs(K2 - Ke)) < 1e-10 * np.max(np.abs(Ke))


def test_jk_exact_closed_form_single_s():
    # one normalised s primitive: J = (ss|ss) D, K = (ss|ss) D with D = 2 c^2
    b = synth.Basis(center=np.zeros((1, 3)), l=np.zeros(1, np.int32), nprim=np.ones(1, np.int32),
                    exps=np.array([0.8]), coefs=np.array([1.0]))
    o = oracle.Oracle(b)
    T = o.eri_tensor()
    C = np.ones((1, 1))
    J, K = oracle.jk_exact(T, C)
    # (ss|ss) for one normalised primitive with exponent a: 2 sqrt(a) sqrt(2/pi) ... = sqrt(4a/pi)*... use closed form
    a = 0.8
    ssss = 2 * np.pi ** 2.5 / (2 * a * 2 * a * np.sqrt(4 * a)) * (2 * a / np.pi) ** 3.0
    assert abs(J[0, 0] - 2 * ssss) < 1e-13 and abs(K[0, 0] - 2 * ssss) < 1e-13


@pytest.mark.parametrize("name,chunk", [("s40", 97), ("sp8", 50), ("sp18", 700)])
def test_loop_order_is_bit_identical(name, chunk):
    """The chunked, vector-outer memory order of the Eq. (subtr) sums gives the
    same bits as the plain per-element loop: free and forced decompositions, the
    span-factor selection with and without dropped rows, and the second step."""
    s = synth.make_workload(name)
    o = oracle.Oracle(s.basis)
    rows = o.screen(s.schwarz)
    assert rows.shape[0] % chunk != 0  # several chunks and a ragged last one
    out = {}
    try:
        for plain in (True, False):
            oracle.set_loop_order(plain=plain, chunk=chunk)
            r = o.cd(rows, s.tau)
            sp = o.cd_span(rows, s.tau, span=0.05, qmax=16, reduce=False)
            sr = o.cd_span(rows, s.tau, span=0.05, qmax=16, reduce=True)
            fb = o.cd_from_basis(rows, sr.piv)
            out[plain] = (r, sp, sr, fb)
    finally:
        oracle.set_loop_order()
    (r0, sp0, sr0, fb0), (r1, sp1, sr1, fb1) = out[True], out[False]
    assert np.array_equal(r0.piv, r1.piv) and np.array_equal(r0.L, r1.L) and np.array_equal(r0.D, r1.D)
    assert np.array_equal(sp0.piv, sp1.piv) and np.array_equal(sp0.L, sp1.L)
    assert np.array_equal(sr0.piv, sr1.piv) and np.array_equal(sr0.L, sr1.L)
    assert np.array_equal(fb0, fb1)
