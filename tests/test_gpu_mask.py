"""Candidate-restricted decompositions on the GPU (cd_opts_t.candidates: the
Cholesky basis chosen from one block of the matrix, Sec. 6.2) against the
oracle's ``cd(candidates=...)`` / ``cd_span(candidates=...)``.

Same bar as the other parity tests: identical basis and vector count except at
a near-tie (the oracle's own residual diagonals of the two choices within
1e-12), vectors to 1e-10 x max |L|, every candidate residual below tau.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_00306_b300 import build
    build.build()
    import paper_2609_00306_b300 as cd
    cd.load()


def _masks(s, rows):
    b = s.basis
    shell_of_bf = []
    for sh in range(b.n_shells):
        shell_of_bf += [sh] * (1 if b.l[sh] == 0 else 3)
    shell_of_bf = np.array(shell_of_bf)
    is_s = b.l[shell_of_bf] == 0
    cen = b.center[shell_of_bf]
    mu, nu = oracle.unpack_pair(rows)
    return {"ss": is_s[mu] & is_s[nu], "same_centre": np.all(cen[mu] == cen[nu], axis=1)}


_cache = {}


def _setup(name):
    if name not in _cache:
        s = synth.make_workload(name)
        o = oracle.Oracle(s.basis)
        rows = o.screen(s.schwarz)
        _cache[name] = (s, o, rows, _masks(s, rows))
    return _cache[name]


def _same_sequence(o, rows, s, got, ref, m):
    k = np.flatnonzero(got[: ref.shape[0]] != ref[: got.shape[0]])
    if k.size:
        k = int(k[0])
        Dk = o.cd(rows, s.tau, forced=ref[:k]).D
        assert abs(Dk[got[k]] - Dk[ref[k]]) < 1e-12
        # the basis size does not depend on how a near-tie was broken
        assert got.shape[0] == ref.shape[0], (got.shape[0], ref.shape[0])
        return False
    assert got.shape[0] == ref.shape[0]
    return True


@pytest.mark.parametrize("which", ["ss", "same_centre"])
@pytest.mark.parametrize("name", ["sp8", "sp18", "sp27"])
def test_full_pivoting_on_a_block(name, which):
    import paper_2609_00306_b300 as cd
    s, o, rows, masks = _setup(name)
    m = masks[which]
    ref = o.cd(rows, s.tau, candidates=m)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, block=16, candidates=m)
    prow, ppk, gaps, resid = f.pivots()
    assert np.all(m[prow])
    assert f.max_resid < s.tau and resid[m].max() < s.tau
    if _same_sequence(o, rows, s, prow, ref.piv, m):
        L = f.vectors_host()
        assert np.max(np.abs(L - ref.L)) <= 1e-10 * np.max(np.abs(ref.L))


@pytest.mark.parametrize("alg", ["span", "twostep"])
@pytest.mark.parametrize("name", ["sp18", "sp27"])
def test_span_policies_on_a_block(name, alg):
    import paper_2609_00306_b300 as cd
    s, o, rows, masks = _setup(name)
    m = masks["ss"]
    ref = o.cd_span(rows, s.tau, 0.05, qmax=16, reduce=(alg == "twostep"), candidates=m)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, block=16, span=0.05, candidates=m,
                         algorithm=cd.CD_ALG_SPAN if alg == "span" else cd.CD_ALG_TWOSTEP)
    prow, ppk, gaps, resid = f.pivots()
    assert np.all(m[prow])
    assert resid[m].max() < s.tau
    if _same_sequence(o, rows, s, prow, ref.piv, m):
        Lref = ref.L if alg == "span" else o.cd_from_basis(rows, ref.piv)
        L = f.vectors_host()
        assert np.max(np.abs(L - Lref)) <= 1e-10 * np.max(np.abs(Lref))
