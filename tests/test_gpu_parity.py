"""GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (FP64 throughout on both sides):
* ERI values: 1e-12 x max |column| + 1e-15 (different but exact-in-theory
  recurrences; the Boys table is accurate to ~1e-15 relative).
* Pivot sequence: identical, except where the oracle's own gap between the
  pivot and the runner-up diagonal is below 1e-12 (near-tie: the two sides may
  break it differently); vector count M identical.
* Forced replay of the oracle's pivots: vectors to 1e-10 x max |L|, gaps < 1e-12.
* J, K (FP64): 1e-11 relative to max |J|, max |K|.
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


def oracle_run(name):
    if name not in _cache:
        s = synth.make_workload(name)
        o = oracle.Oracle(s.basis)
        diag = o.diag_all()
        rows = o.screen(s.schwarz, diag)
        r = o.cd(rows, s.tau)
        J, K = oracle.jk_from_vectors(r.L, rows, s.C_occ)
        _cache[name] = (s, o, diag, rows, r, J, K)
    return _cache[name]


SMALL = ["s40", "sp8", "sp18", "sp27"]


@pytest.mark.parametrize("name", SMALL)
def test_screened_rows_and_diagonal(name):
    import paper_2609_00306_b300 as cd
    s, o, diag, rows, r, J, K = oracle_run(name)
    sysm = cd.System(s.basis, s.schwarz)
    packed, d = sysm.rows()
    assert np.array_equal(packed, rows)
    ref = diag[rows]
    assert np.max(np.abs(d - ref)) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("name", SMALL)
def test_eri_columns(name):
    import paper_2609_00306_b300 as cd
    s, o, diag, rows, r, J, K = oracle_run(name)
    sysm = cd.System(s.basis, s.schwarz)
    rng = np.random.default_rng(3)
    n = rows.shape[0]
    cols = np.unique(np.concatenate([r.piv[:20], rng.integers(0, n, 24), [0, n - 1]]))
    got = sysm.eri_columns(cols).cpu().numpy()
    ref = o.eri_matrix(rows[cols], rows)  # [ncols, n]
    scale = np.max(np.abs(ref), axis=1, keepdims=True)
    err = np.abs(got - ref) / (scale + 1e-300)
    assert np.max(err) <= 1e-12, float(np.max(err))


UPDATES = {"slice": 0, "fp64": 1}


@pytest.mark.parametrize("update", ["slice", "fp64"])
@pytest.mark.parametrize("name", SMALL)
def test_factor_free_run_matches_oracle(name, update):
    import paper_2609_00306_b300 as cd
    s, o, diag, rows, r, J, K = oracle_run(name)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, block=16, update=UPDATES[update])
    prow, ppk, gaps, resid = f.pivots()
    assert f.M == r.M
    assert np.array_equal(ppk, rows[prow])
    assert f.max_resid < s.tau
    assert np.max(resid) < s.tau
    diverge = np.nonzero(prow != r.piv)[0]
    if diverge.size:
        k = int(diverge[0])
        # replay the oracle up to step k and check the two choices were within 1e-12
        fr = o.cd(rows, s.tau, forced=r.piv[:k])
        Dk = fr.D
        assert abs(Dk[prow[k]] - Dk[r.piv[k]]) < 1e-12, (k, Dk[prow[k]], Dk[r.piv[k]])
    else:
        L = f.vectors_host()
        assert np.max(np.abs(L - r.L)) <= 1e-10 * np.max(np.abs(r.L))


@pytest.mark.parametrize("update", ["slice", "fp64"])
@pytest.mark.parametrize("name", SMALL)
@pytest.mark.parametrize("block", [1, 7, 64, 200])
def test_factor_forced_replay(name, block, update):
    import paper_2609_00306_b300 as cd
    s, o, diag, rows, r, J, K = oracle_run(name)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, block=block, forced=r.piv, update=UPDATES[update])
    prow, ppk, gaps, resid = f.pivots()
    assert f.M == r.M
    assert np.array_equal(prow, r.piv)
    assert np.max(np.abs(gaps)) < 1e-12
    L = f.vectors_host()
    assert np.max(np.abs(L - r.L)) <= 1e-10 * np.max(np.abs(r.L))
    assert np.max(np.abs(resid - r.D)) < 1e-12
    assert np.max(resid) < s.tau


@pytest.mark.parametrize("name", SMALL)
def test_jk_fp64_matches_oracle(name):
    import paper_2609_00306_b300 as cd
    s, o, diag, rows, r, J, K = oracle_run(name)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, forced=r.piv)
    Jg, Kg = f.jk(s.C_occ, cd.CD_JK_FP64)
    assert np.max(np.abs(Jg - J)) <= 1e-11 * np.max(np.abs(J))
    assert np.max(np.abs(Kg - K)) <= 1e-11 * np.max(np.abs(K))


def test_jk_device_buffers_match_host():
    import paper_2609_00306_b300 as cd
    s, o, diag, rows, r, J, K = oracle_run("sp18")
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, forced=r.piv)
    C = torch.tensor(s.C_occ, device="cuda")
    N = s.n_basis
    Jd = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    Kd = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    f.jk_device(C, Jd, Kd)
    torch.cuda.synchronize()
    Jh, Kh = f.jk(s.C_occ)
    # J is reduced with FP64 atomics (order not fixed): equal to rounding
    assert np.allclose(Jd.cpu().numpy(), Jh, rtol=0, atol=1e-14 * np.max(np.abs(Jh)))
    assert np.allclose(Kd.cpu().numpy(), Kh, rtol=0, atol=1e-14 * np.max(np.abs(Kh)))


def test_bad_options_are_rejected():
    import paper_2609_00306_b300 as cd
    s = synth.make_workload("sp8")
    for kw in [dict(tau=0.0), dict(tau=float("nan")), dict(tau=1e-6, block=1000), dict(tau=1e-6, forced=[10 ** 9])]:
        with pytest.raises(cd.CDError) as e:
            cd.cd_eri_factor(s.basis, **kw)
        assert e.value.code == -1


def test_max_vectors_cap_is_enomem():
    import paper_2609_00306_b300 as cd
    s = synth.make_workload("sp8")
    with pytest.raises(cd.CDError) as e:
        cd.cd_eri_factor(s.basis, 1e-6, max_vectors=5)
    assert e.value.code == -2


@pytest.mark.parametrize("vec,mode,tol", [("fp64", "bf16x3", 3e-6), ("fp64", "bf16x4", 2e-7),
                                          ("fp64", "bf16x5", 1e-8),
                                          ("fp32", "bf16x3", 3e-6), ("fp32", "bf16x4", 3e-7)])
@pytest.mark.parametrize("name", SMALL)
def test_jk_mixed_vs_oracle(name, vec, mode, tol):
    """Mixed path: the stored vectors (FP64, or rounded once to FP32) cut into
    3 or 4 exact 8-bit slices per row, products on the BF16 tensor cores with
    exact FP32 accumulation.  Error sources: the 8S-bit fixed point below each
    row maximum, and the FP32 rounding of L when the vectors are FP32 (2^-24
    per entry, ~1e-7 of max |K|).  Asserted bound on max|dX|/max|X|."""
    import paper_2609_00306_b300 as cd
    s, o, diag, rows, r, J, K = oracle_run(name)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, forced=r.piv,
                         vec_precision=cd.CD_VEC_FP32 if vec == "fp32" else cd.CD_FP64)
    m = {"bf16x3": cd.CD_JK_BF16X3, "bf16x4": cd.CD_JK_BF16X4, "bf16x5": cd.CD_JK_BF16X5}[mode]
    Jm, Km = f.jk(s.C_occ, m)
    eJ = np.max(np.abs(Jm - J)) / np.max(np.abs(J))
    eK = np.max(np.abs(Km - K)) / np.max(np.abs(K))
    Dm = oracle.density(s.C_occ)
    etJ = abs(np.sum(Dm * Jm) - np.sum(Dm * J)) / abs(np.sum(Dm * J))
    etK = abs(np.sum(Dm * Km) - np.sum(Dm * K)) / abs(np.sum(Dm * K))
    print(f"{name} {vec} {mode}: max|dJ|/max|J|={eJ:.2e} max|dK|/max|K|={eK:.2e} dtr(DJ)={etJ:.2e} dtr(DK)={etK:.2e}")
    assert eJ < (1e-7 if vec == "fp32" else 1e-12) and eK < tol
    assert np.array_equal(Km, Km.T)
