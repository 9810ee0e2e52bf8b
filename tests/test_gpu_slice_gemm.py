"""Exact-slice tensor-core GEMM (cd_slice_matmul) against FP64 matmul.

Error model: each row is scaled by 2^e (|x| <= 1) and cut into S slices of 8
bits, so a represented element is off by at most 2^-(8S) 2^e; the dropped
slice products (s + t > S + 1) and the 2^-F fixed-point rounding add less than
that.  Bound used: |err_ij| <= 4 k 2^-(8S-1) 2^(e_i + f_j).
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_00306_b300 import build
    build.build()


def _exps(X):
    m = np.max(np.abs(X), axis=1)
    return np.array([math.frexp(v)[1] if v > 0 else 0 for v in m])


@pytest.mark.parametrize("S", [1, 3, 4, 5, 7])
@pytest.mark.parametrize("shape", [(128, 64, 32), (300, 130, 777), (129, 65, 3001), (1000, 64, 96)])
def test_slice_matmul_error_bound(S, shape):
    from paper_2609_00306_b300.cderi import slice_matmul
    m, n, k = shape
    rng = np.random.default_rng(m * 7 + n + k + S)
    X = rng.standard_normal((m, k)) * np.exp(rng.uniform(-6, 6, (m, 1)))
    Y = rng.standard_normal((n, k)) * np.exp(rng.uniform(-6, 6, (n, 1)))
    X[rng.random((m, k)) < 0.1] *= 1e-5
    ref = X @ Y.T
    got = slice_matmul(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), S).cpu().numpy()
    ex, ey = _exps(X), _exps(Y)
    bound = 4.0 * k * 2.0 ** (-(8 * S - 1)) * np.exp2(ex[:, None] + ey[None, :])
    err = np.abs(got - ref)
    assert np.all(err <= bound + 1e-300), float(np.max(err / bound))
    if S == 7:
        # FP64-level: within a few ulps of sum |x||y|
        mag = np.abs(X) @ np.abs(Y).T
        assert np.max(err / mag) < 1e-14


def test_slice_matmul_integer_exact():
    from paper_2609_00306_b300.cderi import slice_matmul
    rng = np.random.default_rng(1)
    m, n, k = 256, 128, 2048
    # integers in [-127, 127] with a row max of exactly 127 or 128: one slice is exact
    X = rng.integers(-127, 128, (m, k)).astype(np.float64)
    Y = rng.integers(-127, 128, (n, k)).astype(np.float64)
    X[:, 0] = 127.0
    Y[:, 0] = -127.0
    got = slice_matmul(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), 1).cpu().numpy()
    assert np.array_equal(got, X @ Y.T)


def test_slice_matmul_zero_and_tiny_rows():
    from paper_2609_00306_b300.cderi import slice_matmul
    rng = np.random.default_rng(2)
    X = rng.standard_normal((130, 70))
    Y = rng.standard_normal((66, 70))
    X[5] = 0.0
    Y[3] = 1e-300 * rng.standard_normal(70)
    got = slice_matmul(torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda"), 7).cpu().numpy()
    ref = X @ Y.T
    assert np.all(got[5] == 0.0)
    assert np.max(np.abs(got - ref) / (np.abs(X) @ np.abs(Y).T + 1e-320)) < 1e-13
