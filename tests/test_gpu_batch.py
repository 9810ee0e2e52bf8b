"""Batched decomposition + J/K of independent systems (cd_batch_run): every
system's result equals the one of a plain single-system call (same kernels,
same pivot order; J differs only by the order of FP64 atomic additions), and
two of them are checked against the CPU oracle."""
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


def _small_batch():
    # uneven sizes, tau alternating as in the 64-system workload, small enough for the oracle
    out = []
    for i, dims in enumerate([(2, 2, 2), (3, 2, 1), (3, 3, 2), (2, 2, 1), (3, 3, 1), (4, 2, 2)]):
        out.append(synth.make_lattice(dims, seed=7000 + i, n_occ=max(1, 4 * dims[0] * dims[1] * dims[2] // 8),
                                      tau=1e-4 if i % 2 == 0 else 1e-5, name=f"b{i}"))
    return out


@pytest.mark.parametrize("workers", [1, 3])
def test_batch_equals_single_calls(workers):
    import paper_2609_00306_b300 as cd
    systems = _small_batch()
    Jb, Kb = cd.batch_run(systems, jk_mode=cd.CD_JK_FP64, workers=workers)
    for s, J, K in zip(systems, Jb, Kb):
        f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz)
        J1, K1 = f.jk(s.C_occ, cd.CD_JK_FP64)
        assert np.max(np.abs(J - J1)) <= 1e-13 * np.max(np.abs(J1))
        assert np.max(np.abs(K - K1)) <= 1e-13 * np.max(np.abs(K1))


def test_batch_vs_oracle():
    import paper_2609_00306_b300 as cd
    systems = _small_batch()[:2]
    Jb, Kb = cd.batch_run(systems, jk_mode=cd.CD_JK_FP64, workers=2)
    for s, J, K in zip(systems, Jb, Kb):
        o = oracle.Oracle(s.basis)
        rows = o.screen(s.schwarz)
        r = o.cd(rows, s.tau)
        Jo, Ko = oracle.jk_from_vectors(r.L, rows, s.C_occ)
        assert np.max(np.abs(J - Jo)) <= 1e-11 * np.max(np.abs(Jo))
        assert np.max(np.abs(K - Ko)) <= 1e-11 * np.max(np.abs(Ko))


def test_batch_mixed_mode():
    import paper_2609_00306_b300 as cd
    systems = _small_batch()[2:5]
    Jb, Kb = cd.batch_run(systems, jk_mode=cd.CD_JK_BF16X5, workers=3)
    for s, J, K in zip(systems, Jb, Kb):
        f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz)
        J1, K1 = f.jk(s.C_occ, cd.CD_JK_FP64)
        assert np.max(np.abs(K - K1)) <= 1e-8 * np.max(np.abs(K1))
        assert np.max(np.abs(J - J1)) <= 1e-7 * np.max(np.abs(J1))


def test_batch_reports_failing_system():
    import paper_2609_00306_b300 as cd
    systems = _small_batch()[:2]
    systems[1].tau = -1.0
    with pytest.raises(cd.CDError) as e:
        cd.batch_run(systems, workers=2)
    assert "system 1" in str(e.value)
