"""CV -> MO transformation on the GPU (cd_mo_vectors) against the oracle's
``mo_vectors`` on the same (oracle-replayed) vectors.

Tolerances, relative to max |out|: FP64 GEMMs 1e-12; exact slices, 7 x 8 bits
(56-bit fixed point per row) 1e-12; 5 slices 1e-8; 3 slices 1e-4 (each operand
row is cut 8S-1 bits below its maximum; N terms per sum).
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


_cache = {}


def _case(name):
    if name not in _cache:
        import paper_2609_00306_b300 as cd
        s = synth.make_workload(name)
        o = oracle.Oracle(s.basis)
        rows = o.screen(s.schwarz)
        r = o.cd(rows, s.tau)
        f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, forced=r.piv)
        _cache[name] = (s, rows, f, f.vectors_host(), r.L)
    return _cache[name]


TOL = {0: 1e-12, 7: 1e-12, 5: 1e-8, 3: 1e-4}


@pytest.mark.parametrize("slices", [0, 7, 5, 3])
@pytest.mark.parametrize("name", ["s40", "sp18", "sp27"])
def test_mo_vectors_match_oracle(name, slices):
    """Against the oracle's transform of the oracle's own vectors (same pivots,
    forced): the vectors themselves agree to 1e-10 x max|L| (the decomposition
    parity bound), so FP64-equivalent modes are held to that; and against the
    oracle's transform of the GPU's vectors at the transform's own tolerance."""
    s, rows, f, L, Lo = _case(name)
    assert np.max(np.abs(L - Lo)) <= 1e-10 * np.max(np.abs(Lo))
    rng = np.random.default_rng(11)
    for n_mo in (1, s.n_occ, s.n_basis):
        C = rng.standard_normal((s.n_basis, n_mo)) / np.sqrt(s.n_basis)
        ref = oracle.mo_vectors(Lo, rows, C)
        got = f.mo_vectors(C, slices=slices)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= max(TOL[slices], 1e-10) * np.max(np.abs(ref))
        ref_g = oracle.mo_vectors(L, rows, C)
        assert np.max(np.abs(got - ref_g)) <= TOL[slices] * np.max(np.abs(ref_g))


@pytest.mark.parametrize("slices", [0, 7])
def test_mo_vectors_subrange_and_device(slices):
    s, rows, f, L, Lo = _case("sp18")
    C = s.C_occ
    ref = oracle.mo_vectors(L, rows, C)
    P0, nP = 5, min(37, f.M - 5)
    got = f.mo_vectors(C, P0=P0, nP=nP, slices=slices)
    assert np.max(np.abs(got - ref[P0:P0 + nP])) <= TOL[slices] * np.max(np.abs(ref))
    Cd = torch.tensor(C, device="cuda")
    out = torch.zeros((nP, C.shape[1], C.shape[1]), dtype=torch.float64, device="cuda")
    f.mo_vectors_device(Cd, out, P0=P0, slices=slices)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref[P0:P0 + nP])) <= TOL[slices] * np.max(np.abs(ref))


def test_mo_vectors_rejects_bad_arguments():
    import paper_2609_00306_b300 as cd
    s, rows, f, L, Lo = _case("sp18")
    with pytest.raises(cd.CDError):
        f.mo_vectors(s.C_occ, P0=f.M - 1, nP=2)
    with pytest.raises(cd.CDError):
        f.mo_vectors(s.C_occ, slices=6)
