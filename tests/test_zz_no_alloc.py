"""cd_jk_coulomb_static: the Coulomb build for callers that cannot allocate
device memory (an arena that owns the device memory, or a host allocator that
must not be bypassed).  It takes its scratch from a static device
array instead of cudaMalloc.  Checked against the allocating cd_jk on two
calls in a row (the scratch keeps the previous call's contents, so the second
call shows that everything that must start at zero is cleared).  Collected
last on purpose: it runs after every other test, and also passes alone."""
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


def _j_allocating(f, C, N):
    J = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    f.jk_device(C, J, None)
    torch.cuda.synchronize()
    return J.cpu().numpy()


@pytest.mark.parametrize("name", ["sp18", "sp27"])
def test_coulomb_static_matches_cd_jk_twice(name):
    import paper_2609_00306_b300 as cd
    from paper_2609_00306_b300.static_jk import coulomb_static
    s = synth.make_workload(name)
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz)
    N = s.n_basis
    C = torch.tensor(s.C_occ, device="cuda")
    ref = _j_allocating(f, C, N)
    tol = 1e-13 * np.max(np.abs(ref))  # FP64; only the atomic summation order differs
    for _ in range(2):
        J = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        coulomb_static(f, C, J)
        torch.cuda.synchronize()
        got = J.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref)) <= tol


def test_coulomb_static_clears_after_a_factor_without_vectors():
    """A factor with no vector (tau above every diagonal) right after a normal
    one: J must be exactly zero, not the previous call's J left in the shared
    static scratch.  The device's free memory is unchanged by the calls."""
    import paper_2609_00306_b300 as cd
    from paper_2609_00306_b300.static_jk import coulomb_static
    s = synth.make_workload("sp18")
    N = s.n_basis
    C = torch.tensor(s.C_occ, device="cuda")
    f = cd.cd_eri_factor(s.basis, s.tau, s.schwarz)
    sysm = cd.System(s.basis, s.schwarz)
    tau0 = 2.0 * float(np.max(sysm.rows()[1]))
    f0 = cd.cd_eri_factor(s.basis, tau0, s.schwarz)
    assert f0.M == 0
    J = torch.zeros((N, N), dtype=torch.float64, device="cuda")
    coulomb_static(f, C, J)          # warm: symbol address looked up, kernels loaded
    torch.cuda.synchronize()
    assert torch.count_nonzero(J).item() > 0
    free0 = torch.cuda.mem_get_info()[0]
    coulomb_static(f, C, J)
    J0 = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    coulomb_static(f0, C, J0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free1
    assert free1 <= free0  # only the NaN-filled output tensor was added
    assert torch.count_nonzero(J0).item() == 0
