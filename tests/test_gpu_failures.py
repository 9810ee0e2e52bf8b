"""Error paths and degenerate inputs on the GPU, made on the host (no GPU fault):

* CD_ETIMEOUT: the tensor-core pipeline's bounded waits, with their limit set
  to 0 through cd_set_wait_limit (give up at the first wait whose phase is not
  already complete), give up; every CTA lets its in-flight
  copies and MMAs finish, frees its tensor memory and returns, and the call
  reports CD_ETIMEOUT.  The same process then runs a normal product on the
  same device and checks it.
* CD_ENOTPSD: the decomposition of A - shift I (the diag_shift test hook with
  shift above the smallest diagonal of the ERI matrix A) meets a residual
  diagonal below -1e-10 max D^1 after its first step (Sec. 2: a PSD matrix
  never produces one).
* CD_ENOMEM: a device-memory budget too small for the vectors is refused
  before anything is allocated.
* M = 0: tau above every diagonal gives no vector; J and K are then exactly
  zero through every J/K path (FP64, mixed, and the allocation-free Coulomb
  build is covered in its own file).
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_00306_b300 import build
    build.build()


def test_bounded_wait_times_out_and_device_stays_usable():
    import paper_2609_00306_b300 as cd
    from paper_2609_00306_b300.cderi import slice_matmul
    rng = np.random.default_rng(3)
    X = torch.tensor(rng.standard_normal((1024, 2048)), device="cuda")
    Y = torch.tensor(rng.standard_normal((256, 2048)), device="cuda")
    prev = cd.set_wait_limit(0.0)
    try:
        with pytest.raises(cd.CDError) as e:
            slice_matmul(X, Y, 7)
        assert e.value.code == cd.CD_ETIMEOUT
    finally:
        cd.set_wait_limit(prev)
    assert prev == pytest.approx(2.0)
    torch.cuda.synchronize()
    got = slice_matmul(X, Y, 7).cpu().numpy()
    ref = X.cpu().numpy() @ Y.cpu().numpy().T
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_bounded_wait_timeout_inside_the_decomposition():
    """The sliced column update of the decomposition runs the same pipeline: a
    wait that runs out ends the factorisation with CD_ETIMEOUT, and a normal
    factorisation follows on the same device."""
    import paper_2609_00306_b300 as cd
    s = synth.make_workload("sp18")
    prev = cd.set_wait_limit(0.0)
    try:
        with pytest.raises(cd.CDError) as e:
            cd.cd_eri_factor(s.basis, s.tau, s.schwarz)
        assert e.value.code == cd.CD_ETIMEOUT
    finally:
        cd.set_wait_limit(prev)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz)
    assert f.M > 0 and f.max_resid < s.tau


def test_wait_limit_rejects_bad_values():
    import paper_2609_00306_b300 as cd
    with pytest.raises(cd.CDError):
        cd.set_wait_limit(-1.0)
    assert cd.set_wait_limit(2.0) == pytest.approx(2.0)


def test_indefinite_input_is_enotpsd():
    import paper_2609_00306_b300 as cd
    s = synth.make_workload("sp8")
    sysm = cd.System(s.basis, s.schwarz)
    _, diag = sysm.rows()
    shift = 0.5 * (np.min(diag) + np.max(diag))   # A - shift I has negative diagonal entries
    for update in (cd.CD_UPDATE_SLICE, cd.CD_UPDATE_FP64):
        with pytest.raises(cd.CDError) as e:
            cd.cd_eri_factor(s.basis, s.tau, s.schwarz, diag_shift=shift, update=update)
        assert e.value.code == cd.CD_ENOTPSD
    # a shift below every diagonal keeps the matrix's diagonal positive: no error from the hook itself
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz, diag_shift=1e-3 * float(np.min(diag)))
    assert f.M > 0


def test_memory_budget_is_enomem_before_allocation():
    import paper_2609_00306_b300 as cd
    s = synth.make_workload("sp18")
    free0 = torch.cuda.mem_get_info()[0]
    with pytest.raises(cd.CDError) as e:
        cd.cd_eri_factor(s.basis, s.tau, s.schwarz, mem_budget_gb=1e-6)
    assert e.value.code == cd.CD_ENOMEM
    torch.cuda.synchronize()
    # nothing kept after the refusal (the system set-up before it is freed again)
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)


@pytest.mark.parametrize("name", ["sp8", "sp18"])
def test_no_vectors_gives_zero_j_and_k(name):
    import paper_2609_00306_b300 as cd
    s = synth.make_workload(name)
    sysm = cd.System(s.basis, s.schwarz)
    _, diag = sysm.rows()
    tau = 2.0 * float(np.max(diag))
    for vec in (cd.CD_FP64, cd.CD_VEC_FP32):
        f = cd.cd_eri_factor(s.basis, tau, s.schwarz, vec_precision=vec)
        assert f.M == 0 and f.max_resid < tau
        prow, ppk, gaps, resid = f.pivots()
        assert prow.shape == (0,) and np.array_equal(resid, diag)
        for mode in (cd.CD_JK_FP64, cd.CD_JK_BF16X3, cd.CD_JK_BF16X5):
            J, K = f.jk(s.C_occ, mode)
            assert np.array_equal(J, np.zeros_like(J)) and np.array_equal(K, np.zeros_like(K))
            N = s.n_basis
            # device buffers pre-filled with NaN must come back exactly zero
            Jd = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
            Kd = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
            f.jk_device(torch.tensor(s.C_occ, device="cuda"), Jd, Kd, mode)
            torch.cuda.synchronize()
            assert torch.count_nonzero(Jd).item() == 0 and torch.count_nonzero(Kd).item() == 0
