"""Pins for the oracle's candidate-restricted decomposition (the Cholesky basis
chosen from one block of the matrix only: the (LL|LL) diagonals of the
spin-free relativistic case, Sec. 6.2):

* The residual diagonals of candidate rows depend only on the candidate block
  A[C, C] (they are its Schur complements), so the restricted pivot sequence is
  LAPACK dpstrf's on A[C, C], mapped back to rows.
* The vectors on all rows are the density-fitting form of that basis,
  L = (.|B) M^-T with S = M M^T on the basis (numpy Cholesky + scipy solve).
* Every candidate residual diagonal ends below tau; rows outside the block carry
  no such guarantee (and in these systems some end above it).
* The span policies obey the same restriction: every pivot is a candidate and
  the first step of the two-step scheme picks the same basis as Koch's.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.linalg.lapack

import oracle
import synth


def _masks(s, rows):
    """Two candidate blocks: pairs of two s functions ('LL'-like), and pairs on one centre."""
    b = s.basis
    shell_of_bf = []
    for sh in range(b.n_shells):
        shell_of_bf += [sh] * (1 if b.l[sh] == 0 else 3)
    shell_of_bf = np.array(shell_of_bf)
    is_s = np.array([b.l[sh] == 0 for sh in shell_of_bf])
    cen = np.array([tuple(b.center[sh]) for sh in shell_of_bf])
    mu, nu = oracle.unpack_pair(rows)
    ss = is_s[mu] & is_s[nu]
    same = np.all(cen[mu] == cen[nu], axis=1)
    return {"ss": ss, "same_centre": same}


@pytest.fixture(scope="module", params=["sp8", "sp18"])
def case(request):
    s = synth.make_workload(request.param)
    o = oracle.Oracle(s.basis)
    rows = o.screen(s.schwarz)
    A = o.eri_matrix(rows)
    return s, o, rows, A, _masks(s, rows)


@pytest.mark.parametrize("which", ["ss", "same_centre"])
def test_restricted_pivots_are_dpstrf_on_the_block(case, which):
    s, o, rows, A, masks = case
    m = masks[which]
    C = np.flatnonzero(m)
    r = o.cd(rows, s.tau, candidates=m)
    c, piv, rank, info = scipy.linalg.lapack.dpstrf(A[np.ix_(C, C)].copy(), lower=1, tol=s.tau)
    ref = C[piv[:rank] - 1]
    assert r.M == rank
    k = np.flatnonzero(r.piv != ref)
    if k.size:
        k = int(k[0])
        Dk = np.diag(A) - np.sum(r.L[:k] ** 2, axis=0)
        assert abs(Dk[r.piv[k]] - Dk[ref[k]]) < 1e-12
    assert np.all(m[r.piv])


@pytest.mark.parametrize("which", ["ss", "same_centre"])
def test_restricted_vectors_and_bound(case, which):
    s, o, rows, A, masks = case
    m = masks[which]
    r = o.cd(rows, s.tau, candidates=m)
    S = A[np.ix_(r.piv, r.piv)]
    Mf = np.linalg.cholesky(S)
    Lref = scipy.linalg.solve_triangular(Mf, A[:, r.piv].T, lower=True)
    assert np.max(np.abs(r.L - Lref)) < 1e-9 * np.max(np.abs(Lref))
    d = np.diag(A - r.L.T @ r.L)
    assert d[m].max() < s.tau
    assert np.max(np.abs(d - r.D)) < 1e-13


def test_restriction_leaves_rows_above_tau(case):
    s, o, rows, A, masks = case
    r = o.cd(rows, s.tau, candidates=masks["ss"])
    assert r.D[~masks["ss"]].max() >= s.tau  # the guarantee is only on the block


@pytest.mark.parametrize("which", ["ss", "same_centre"])
def test_span_policies_respect_the_block(case, which):
    s, o, rows, A, masks = case
    m = masks[which]
    koch = o.cd_span(rows, s.tau, 0.05, qmax=16, reduce=False, candidates=m)
    two = o.cd_span(rows, s.tau, 0.05, qmax=16, reduce=True, candidates=m)
    assert np.all(m[koch.piv])
    assert np.array_equal(koch.piv, two.piv)
    L2 = o.cd_from_basis(rows, two.piv)
    d = np.diag(A - L2.T @ L2)
    assert d[m].max() < s.tau
    # span = 1: the restricted full-pivoting sequence
    full = o.cd(rows, s.tau, candidates=m)
    one = o.cd_span(rows, s.tau, 1.0, qmax=16, reduce=True, candidates=m)
    assert np.array_equal(one.piv, full.piv)
