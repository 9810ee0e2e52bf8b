"""Pins for the oracle's span-factor selection (Koch's partially pivoted
decomposition) and the two-step scheme of Sec. 3, against facts fixed outside
the code under test:

* span = 1, or a qualified set of one column, is full pivoting: the pivots are
  LAPACK dpstrf's (complete-pivoting Cholesky) on the same ERI matrix.
* The second step, Eq. (CVsLT), against numpy's Cholesky of the basis metric and
  scipy's triangular solve.
* For any span, the residual A - L L^T of the final vectors is PSD with every
  element bounded by tau (Sec. 2 truncation bound), over ALL rows, including the
  rows the first step discarded.
* The selection rule itself, recomputed from the final vectors: the first pivot
  of each macro iteration is the argmax of the residual diagonal, every pivot's
  residual diagonal is >= max(span * Dmax, tau) of its macro iteration, and no
  residual diagonal is >= tau at the end.
* Discarding rows below tau (two-step) does not change the basis chosen on the
  full rows (Koch), since a residual diagonal never increases.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack

import oracle
import synth


def _setup(name):
    s = synth.make_workload(name)
    o = oracle.Oracle(s.basis)
    rows = o.screen(s.schwarz)
    A = o.eri_matrix(rows)
    return s, o, rows, A


@pytest.fixture(scope="module")
def s40():
    return _setup("s40")


@pytest.fixture(scope="module")
def sp8():
    return _setup("sp8")


def _dpstrf_pivots(A, tau):
    c, piv, rank, info = scipy.linalg.lapack.dpstrf(A.copy(), lower=1, tol=tau)
    return (piv - 1)[:rank]


@pytest.mark.parametrize("reduce", [False, True])
def test_span_one_is_full_pivoting(s40, sp8, reduce):
    for s, o, rows, A in (s40, sp8):
        ref = _dpstrf_pivots(A, s.tau)
        r = o.cd_span(rows, s.tau, span=1.0, qmax=64, reduce=reduce)
        assert r.M == ref.shape[0]
        k = np.flatnonzero(r.piv != ref)
        if k.size:  # only a near-tie may reorder the sequence
            k = int(k[0])
            Dk = np.diag(A) - np.sum(r.L[:k] ** 2, axis=0)
            assert abs(Dk[r.piv[k]] - Dk[ref[k]]) < 1e-12
        # one pivot per macro iteration
        assert np.array_equal(r.macro_start, np.arange(r.M))


def test_single_qualified_column_is_full_pivoting(s40):
    s, o, rows, A = s40
    ref = _dpstrf_pivots(A, s.tau)
    r = o.cd_span(rows, s.tau, span=1e-3, qmax=1, reduce=True)
    assert r.M == ref.shape[0] and np.array_equal(r.piv, ref)


@pytest.mark.parametrize("span", [0.5, 0.05, 1e-3])
def test_second_step_against_numpy(s40, sp8, span):
    for s, o, rows, A in (s40, sp8):
        r = o.cd_span(rows, s.tau, span=span, qmax=32, reduce=True)
        L = o.cd_from_basis(rows, r.piv)
        S = A[np.ix_(r.piv, r.piv)]
        Mf = np.linalg.cholesky(S)
        Lref = scipy.linalg.solve_triangular(Mf, A[:, r.piv].T, lower=True)
        assert np.max(np.abs(L - Lref)) < 1e-10 * np.max(np.abs(Lref))


@pytest.mark.parametrize("span", [0.5, 0.05, 1e-3])
def test_residual_bounded_by_tau_on_all_rows(s40, sp8, span):
    for s, o, rows, A in (s40, sp8):
        r = o.cd_span(rows, s.tau, span=span, qmax=32, reduce=True)
        L = o.cd_from_basis(rows, r.piv)
        R = A - L.T @ L
        d = np.diag(R)
        assert d.max() < s.tau
        assert np.max(np.abs(R)) <= d.max() + 1e-13
        assert np.linalg.eigvalsh(R).min() > -1e-12


@pytest.mark.parametrize("span", [0.5, 0.05, 1e-3])
def test_selection_rule_recomputed(s40, sp8, span):
    for s, o, rows, A in (s40, sp8):
        r = o.cd_span(rows, s.tau, span=span, qmax=32, reduce=False)
        diag = np.diag(A)
        starts = list(r.macro_start) + [r.M]
        for i in range(len(starts) - 1):
            k0, k1 = starts[i], starts[i + 1]
            D0 = diag - np.sum(r.L[:k0] ** 2, axis=0)
            dmax = D0.max()
            thr = max(span * dmax, s.tau)
            assert D0[r.piv[k0]] >= dmax - 1e-12  # macro iteration opens with the argmax
            for k in range(k0, k1):
                Dk = diag - np.sum(r.L[:k] ** 2, axis=0)
                assert Dk[r.piv[k]] >= thr - 1e-12
        Dend = diag - np.sum(r.L ** 2, axis=0)
        assert Dend.max() < s.tau


@pytest.mark.parametrize("span", [0.3, 0.01])
def test_discarding_rows_keeps_the_basis(s40, sp8, span):
    for s, o, rows, A in (s40, sp8):
        koch = o.cd_span(rows, s.tau, span=span, qmax=16, reduce=False)
        two = o.cd_span(rows, s.tau, span=span, qmax=16, reduce=True)
        assert np.array_equal(koch.piv, two.piv)
        assert np.array_equal(koch.macro_start, two.macro_start)
        # Koch's vectors are the second step's vectors of the same basis
        L2 = o.cd_from_basis(rows, two.piv)
        assert np.max(np.abs(L2 - koch.L)) < 1e-12 * np.max(np.abs(koch.L))


def test_smaller_span_fewer_macro_iterations(s40):
    s, o, rows, A = s40
    n = [len(o.cd_span(rows, s.tau, span=sp, qmax=64, reduce=True).macro_start) for sp in (1.0, 0.1, 1e-3)]
    assert n[0] > n[1] > n[2]
