"""The seeded input generator against the workload recipes it states: sizes,
thresholds, value ranges, geometry, orthonormal occupied block, and
reproducibility from the seed."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("name,N,n_occ,tau,schwarz", [
    ("s40", 40, 10, 1e-6, 0.0), ("sp400", 400, 50, 1e-5, 1e-12), ("sp1200", 1200, 150, 1e-5, 1e-12),
    ("sp2000", 2000, 250, 1e-4, 1e-12)])
def test_named_workloads(name, N, n_occ, tau, schwarz):
    s = synth.make_workload(name)
    assert s.n_basis == N and s.C_occ.shape == (N, n_occ)
    assert s.tau == tau and s.schwarz == schwarz
    b = s.basis
    assert b.exps.shape == b.coefs.shape == (int(b.nprim.sum()),)
    assert np.all((b.coefs >= 0.2) & (b.coefs <= 1.0))
    lo, hi = (0.1, 10.0) if name == "s40" else (0.15, 20.0)
    assert np.all((b.exps >= lo) & (b.exps <= hi))
    # orthonormal occupied columns
    assert np.max(np.abs(s.C_occ.T @ s.C_occ - np.eye(n_occ))) < 1e-12


def test_s40_geometry():
    s = synth.make_workload("s40")
    c = s.basis.center
    assert np.all(s.basis.l == 0) and np.all(s.basis.nprim == 3)
    assert np.all((c >= 0.0) & (c <= 8.0))
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2) + np.eye(len(c)) * 1e9
    assert d.min() >= 1.5


@pytest.mark.parametrize("name,dims", [("sp400", (5, 5, 4)), ("sp2000", (10, 10, 5))])
def test_lattice_geometry(name, dims):
    s = synth.make_workload(name)
    b = s.basis
    # one s shell (3 primitives) and one p shell (2 primitives) per centre, same centre for both
    assert np.array_equal(b.l, np.tile([0, 1], len(b.l) // 2))
    assert np.array_equal(b.nprim, np.tile([3, 2], len(b.l) // 2))
    cen = b.center[0::2]
    assert np.array_equal(cen, b.center[1::2])
    sites = np.array([(i, j, k) for i in range(dims[0]) for j in range(dims[1]) for k in range(dims[2])], float)
    assert np.max(np.abs(cen - 2.6 * sites)) <= 0.3


def test_reproducible_from_seed():
    a, b = synth.make_workload("sp400"), synth.make_workload("sp400")
    for x, y in ((a.basis.center, b.basis.center), (a.basis.exps, b.basis.exps), (a.C_occ, b.C_occ)):
        assert np.array_equal(x, y)
    assert not np.array_equal(a.basis.exps, synth.make_workload("sp1200").basis.exps[: a.basis.exps.shape[0]])


def test_batch_recipe():
    systems = synth.make_batch()
    assert len(systems) == 64
    Ns = np.array([s.n_basis for s in systems])
    assert Ns.min() >= 60 and Ns.max() <= 600
    assert [s.tau for s in systems[:4]] == [1e-4, 1e-5, 1e-4, 1e-5]
    for s in systems:
        assert s.C_occ.shape[1] == max(1, s.n_basis // 8)
