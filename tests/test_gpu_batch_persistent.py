"""Batch of independent systems in one persistent kernel launch
(cd_batch_persistent): every system's vector count and J/K equal those of a
plain single-system FP64 call (same recursion, Sec. 2; J/K of Sec. 4.1 summed
in another order), all seven are checked against the CPU oracle, and the
error paths (M = 0, vector capacity, bad arguments, the bounded wait for
work) return their codes without disturbing the device.  A memory budget below
the batch's buffers splits it into waves with the same results."""
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


def _uneven_batch():
    # uneven sizes, tau alternating as in the 64-system workload, small enough for the oracle
    out = []
    for i, dims in enumerate([(2, 2, 2), (3, 2, 1), (3, 3, 2), (2, 2, 1), (3, 3, 1), (4, 2, 2), (4, 3, 2)]):
        out.append(synth.make_lattice(dims, seed=7100 + i, n_occ=max(1, 4 * dims[0] * dims[1] * dims[2] // 8),
                                      tau=1e-4 if i % 2 == 0 else 1e-5, name=f"p{i}"))
    return out


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("block,update", [(0, "slice"), (16, "slice"), (48, "slice"), (0, "fp64"), (16, "fp64")])
def test_persistent_equals_single_calls(block, update):
    import paper_2609_00306_b300 as cd
    systems = _uneven_batch()
    upd = cd.CD_UPDATE_SLICE if update == "slice" else cd.CD_UPDATE_FP64
    Jb, Kb, Mb, info = cd.batch_persistent(systems, blocks=[block] * len(systems), update=upd)
    assert info["ctas"] > 0 and info["launch_device_ms"] > 0
    for s, J, K, M in zip(systems, Jb, Kb, Mb):
        f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, update=cd.CD_UPDATE_FP64)
        J1, K1 = f.jk(s.C_occ, cd.CD_JK_FP64)
        assert M == f.M
        assert _rel(J, J1) <= 1e-12
        assert _rel(K, K1) <= 1e-12
        assert np.array_equal(J, J.T) and np.array_equal(K, K.T)
        f.free()


@pytest.mark.parametrize("update", ["slice", "fp64"])
def test_persistent_vs_oracle(update):
    # all seven uneven systems (N = 16-96, tau 1e-4 / 1e-5) against the oracle's decomposition and J/K
    import paper_2609_00306_b300 as cd
    systems = _uneven_batch()
    pick = list(range(len(systems)))
    upd = cd.CD_UPDATE_SLICE if update == "slice" else cd.CD_UPDATE_FP64
    Jb, Kb, Mb, _ = cd.batch_persistent([systems[i] for i in pick], update=upd)
    for k, i in enumerate(pick):
        s = systems[i]
        o = oracle.Oracle(s.basis)
        rows = o.screen(s.schwarz)
        r = o.cd(rows, s.tau)
        Jo, Ko = oracle.jk_from_vectors(r.L, rows, s.C_occ)
        assert Mb[k] == r.L.shape[0]
        assert _rel(Jb[k], Jo) <= 1e-11
        assert _rel(Kb[k], Ko) <= 1e-11


def test_persistent_zero_vectors():
    # tau above every diagonal: M = 0, J = K = 0 exactly, next to a normal system
    import paper_2609_00306_b300 as cd
    systems = _uneven_batch()[:2]
    systems[0].tau = 1e6
    Jb, Kb, Mb, _ = cd.batch_persistent(systems)
    assert Mb[0] == 0
    assert not np.any(Jb[0]) and not np.any(Kb[0])
    f = cd.cd_eri_factor(systems[1].basis, systems[1].tau, systems[1].schwarz, update=cd.CD_UPDATE_FP64)
    J1, K1 = f.jk(systems[1].C_occ, cd.CD_JK_FP64)
    assert Mb[1] == f.M and _rel(Kb[1], K1) <= 1e-12


def test_persistent_capacity_and_arguments():
    import paper_2609_00306_b300 as cd
    systems = _uneven_batch()[:3]
    with pytest.raises(cd.CDError) as e:
        cd.batch_persistent(systems, max_vectors=[0, 3, 0])
    assert e.value.code == cd.CD_ENOMEM and "system 1" in str(e.value)
    with pytest.raises(cd.CDError) as e:
        cd.batch_persistent(systems, blocks=[0, 0, 65])
    assert e.value.code == cd.CD_EINVAL and "system 2" in str(e.value)
    systems[0].tau = -1.0
    with pytest.raises(cd.CDError) as e:
        cd.batch_persistent(systems)
    assert e.value.code == cd.CD_EINVAL and "system 0" in str(e.value)


@pytest.mark.parametrize("update", ["slice", "fp64"])
def test_persistent_waves_under_a_small_budget(update):
    # a budget below the whole batch's buffers: the systems run in several
    # waves, one launch each on one reused device buffer (not cleared between
    # waves), with the same vector counts and J/K as in one wave
    import paper_2609_00306_b300 as cd
    systems = _uneven_batch()
    upd = cd.CD_UPDATE_SLICE if update == "slice" else cd.CD_UPDATE_FP64
    J1, K1, M1, info1 = cd.batch_persistent(systems, update=upd)
    assert info1["waves"] == 1
    # the largest system (N = 96) holds about half of the bytes (they grow as N^3)
    budget = 0.7 * info1["bytes"]
    Jw, Kw, Mw, infow = cd.batch_persistent(systems, update=upd, mem_budget_gb=budget / 1e9)
    assert infow["waves"] >= 2 and infow["bytes"] <= budget
    assert Mw == M1
    for k in range(len(systems)):
        assert _rel(Jw[k], J1[k]) <= 1e-12 and _rel(Kw[k], K1[k]) <= 1e-12
    # one system alone over the budget: CD_ENOMEM naming the system, before any device work
    with pytest.raises(cd.CDError) as e:
        cd.batch_persistent(systems, update=upd, mem_budget_gb=1e-6)
    assert e.value.code == cd.CD_ENOMEM and "system" in str(e.value) and "budget" in str(e.value)


def test_persistent_wait_limit_times_out_then_recovers():
    # wait limit 0: the first CTA that finds no work gives up at once; the
    # launch stops cleanly and the next call on the same device succeeds
    import paper_2609_00306_b300 as cd
    systems = _uneven_batch()[:3]
    prev = cd.set_wait_limit(0.0)
    try:
        with pytest.raises(cd.CDError) as e:
            cd.batch_persistent(systems)
        assert e.value.code == cd.CD_ETIMEOUT
    finally:
        cd.set_wait_limit(prev)
    Jb, Kb, Mb, _ = cd.batch_persistent(systems)
    f = cd.cd_eri_factor(systems[2].basis, systems[2].tau, systems[2].schwarz, update=cd.CD_UPDATE_FP64)
    assert Mb[2] == f.M
