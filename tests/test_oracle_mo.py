"""Pins for the oracle's MO transformation of the Cholesky vectors (Sec. 4.1):

* C = identity returns the unpacked vectors themselves.
* MO integrals rebuilt from the MO vectors, sum_P L^P_pq L^P_rs, against the MO
  transformation of the exact ERI tensor, within the truncation bound: every
  element of the AO residual is at most max D < tau, so an MO element is off by
  at most max D * (sum |C_mu p C_nu q|) * (sum |C_sigma r C_rho s|).
* An orthogonal C leaves sum_P ||L^P||_F^2 unchanged (Frobenius invariance).
* Every MO vector is symmetric.
"""
import numpy as np
import pytest

import oracle
import synth


@pytest.fixture(scope="module", params=["s40", "sp8"])
def case(request):
    s = synth.make_workload(request.param)
    o = oracle.Oracle(s.basis)
    rows = o.screen(s.schwarz)
    r = o.cd(rows, s.tau)
    return s, o, rows, r


def test_identity_gives_unpacked_vectors(case):
    s, o, rows, r = case
    N = o.nbf
    X = oracle.mo_vectors(r.L, rows, np.eye(N))
    assert np.array_equal(X, oracle.unpack_vectors(r.L, rows, N))


def test_mo_integrals_within_truncation_bound(case):
    s, o, rows, r = case
    N = o.nbf
    C = s.C_occ[:, :6]
    X = oracle.mo_vectors(r.L, rows, C)
    eri_cd = np.einsum("Ppq,Prs->pqrs", X, X)
    eri_ex = oracle.mo_eri(o.eri_tensor(), C)
    w = np.einsum("ap,bq->pq", np.abs(C), np.abs(C))  # sum |C_mu p C_nu q|
    bound = r.D.max() * np.einsum("pq,rs->pqrs", w, w)
    assert np.all(np.abs(eri_cd - eri_ex) <= bound + 1e-13)
    # and the vectors are not trivially small: the integrals themselves are O(1)
    assert np.max(np.abs(eri_ex)) > 0.1


def test_orthogonal_transform_keeps_frobenius_norm(case):
    s, o, rows, r = case
    N = o.nbf
    Q, _ = np.linalg.qr(np.random.default_rng(7).standard_normal((N, N)))
    X = oracle.mo_vectors(r.L, rows, Q)
    U = oracle.unpack_vectors(r.L, rows, N)
    assert abs(np.sum(X * X) - np.sum(U * U)) <= 1e-11 * np.sum(U * U)
    assert np.max(np.abs(X - np.transpose(X, (0, 2, 1)))) <= 1e-13 * np.max(np.abs(X))
