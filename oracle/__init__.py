"""Plain FP64 CPU oracle for the Cholesky-decomposed ERI path.

TEST INFRASTRUCTURE ONLY: tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library itself never
does.  It shares no code with the CUDA path (see ``cdoracle.c`` for the C part).

What each function follows (the paper, arXiv 2609.00306, Sec. 2 and 4.1):

* ``Oracle.cd``  -- the fully pivoted Cholesky recursion of Sec. 2: diagonal
  D^1, argmax pivot, Eq. (subtr) for the new vector, Eq. (diag) for the
  diagonal update, truncation when max D < tau.  Implemented in C (``or_cd``).
* ``jk_from_vectors`` -- Coulomb and exchange matrices from the Cholesky
  vectors (Sec. 4.1): (mu nu|sigma rho) ~ sum_P L^P_{mu nu} L^P_{sigma rho},
  J_{mu nu} = sum_{sigma rho} (mu nu|sigma rho) D_{sigma rho},
  K_{mu nu} = sum_{sigma rho} (mu sigma|nu rho) D_{sigma rho} = sum_P (L^P D L^P)_{mu nu}.
* ``jk_exact``  -- the same J and K from the exact four-index ERI tensor.
* ``Oracle.cd_span`` -- partially pivoted selection with a span factor (Sec. 3
  and its Table of sets; Koch et al. 2003): qualified diagonals >= span * max D,
  micro iterations inside the qualified set, optional discarding of rows below
  tau (first step of the two-step scheme).  ``Oracle.cd_from_basis`` -- second
  step: Cholesky factor of the basis metric and the triangular solve of
  Eq. (CVsLT).  Both in C (``or_cd_span``, ``or_cd_from_basis``).
* ``mo_vectors`` -- the vectors in the MO basis used by CASSCF and CC (Sec.
  4.1), C^T L^P C for every P; ``mo_eri`` the MO integrals from the exact tensor.

Readings taken where the paper is silent (each one is listed with the design
notes): packed mu >= nu pair indices, strict ``< tau`` stop, ties to the lowest
pair index, division by the tracked diagonal, shell-pair Schwarz screening,
D = 2 C C^T.

Parity pins for this oracle live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cdoracle.c")
_LIB = os.path.join(_HERE, "_build", "libcdoracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        D, I, P = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
        I64 = ctypes.c_int64
        lib.or_boys.argtypes = [I, D, P]
        lib.or_eri_prim.restype = D
        lib.or_eri_prim.argtypes = [P, D, P, P, D, P, P, D, P, P, D, P]
        lib.or_basis_new.restype = P
        lib.or_basis_new.argtypes = [I, P, P, P, P, P]
        lib.or_basis_free.argtypes = [P]
        lib.or_nbf.restype = I
        lib.or_nbf.argtypes = [P]
        lib.or_shell_coefs.argtypes = [P, I, P]
        lib.or_eri.restype = D
        lib.or_eri.argtypes = [P, I, I, I, I]
        lib.or_eri_matrix.argtypes = [P, P, I, P, I, P]
        lib.or_diag_all.argtypes = [P, P]
        lib.or_screen.restype = I64
        lib.or_screen.argtypes = [P, P, D, P]
        lib.or_cd.restype = I
        lib.or_cd.argtypes = [P, P, I64, D, P, I, I, P, P, P, P, P, P]
        lib.or_cd_span.restype = I
        lib.or_cd_span.argtypes = [P, P, I64, D, D, I, I, I, P, P, P, P, P, P]
        lib.or_cd_from_basis.restype = I
        lib.or_cd_from_basis.argtypes = [P, P, I64, P, I, P]
        lib.or_set_order.argtypes = [I, I]
        _lib = lib
    return _lib


def set_loop_order(plain: bool = False, chunk: int = 2048) -> None:
    """Memory order of the Eq. (subtr) sums in the C decompositions: the plain
    per-element loop (``plain=True``) or row chunks of ``chunk`` with the vector
    index outermost (default).  Both give bit-identical results."""
    _load().or_set_order(int(bool(plain)), int(chunk))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def boys(mmax: int, T: float) -> np.ndarray:
    """F_0(T) .. F_mmax(T)."""
    F = np.zeros(mmax + 1)
    _load().or_boys(mmax, float(T), _ptr(F))
    return F


def eri_prim(a, ea, A, b, eb, B, c, ec, C, d, ed, D) -> float:
    """Primitive ERI of unnormalised Cartesian Gaussians (Obara-Saika)."""
    args = []
    for cart, e, cen in ((a, ea, A), (b, eb, B), (c, ec, C), (d, ed, D)):
        ci = np.ascontiguousarray(cart, dtype=np.int32)
        cc = np.ascontiguousarray(cen, dtype=np.float64)
        args += [ci, float(e), cc]
    keep = [x for x in args if isinstance(x, np.ndarray)]
    call = [(_ptr(x) if isinstance(x, np.ndarray) else x) for x in args]
    v = _load().or_eri_prim(*call)
    del keep
    return v


def pair_index(mu, nu):
    mu, nu = np.maximum(mu, nu), np.minimum(mu, nu)
    return mu * (mu + 1) // 2 + nu


def unpack_pair(p):
    p = np.asarray(p, dtype=np.int64)
    mu = ((np.sqrt(8.0 * p + 1.0) - 1.0) // 2).astype(np.int64)
    mu = np.where(mu * (mu + 1) // 2 > p, mu - 1, mu)
    mu = np.where((mu + 1) * (mu + 2) // 2 <= p, mu + 1, mu)
    return mu, p - mu * (mu + 1) // 2


@dataclasses.dataclass
class CDResult:
    rows: np.ndarray      # [npairs] packed pair index of each vector row
    piv: np.ndarray       # [M] pivot rows (indices into rows)
    L: np.ndarray         # [M, npairs] Cholesky vectors
    D: np.ndarray         # [npairs] residual diagonal after the last vector
    gap: np.ndarray       # [M] max D - D_pivot at each step (0 in free mode)
    pivD: np.ndarray      # [M] tracked diagonal of each pivot when chosen

    @property
    def M(self) -> int:
        return int(self.piv.shape[0])

    @property
    def piv_packed(self) -> np.ndarray:
        return self.rows[self.piv]


@dataclasses.dataclass
class SpanResult:
    rows: np.ndarray         # [npairs] packed pair index of each vector row
    piv: np.ndarray          # [M] chosen basis (pivot rows), in order
    L: np.ndarray            # [M, npairs] vectors (dropped rows left at 0 when rows were reduced)
    D: np.ndarray            # [npairs] residual diagonal (live rows)
    macro_start: np.ndarray  # [n_macro] vector count at the start of each macro iteration

    @property
    def M(self) -> int:
        return int(self.piv.shape[0])


class Oracle:
    """Oracle bound to one basis (``synth.Basis``)."""

    def __init__(self, basis):
        self._lib = _load()
        self._keep = [np.ascontiguousarray(basis.center, dtype=np.float64),
                      np.ascontiguousarray(basis.l, dtype=np.int32),
                      np.ascontiguousarray(basis.nprim, dtype=np.int32),
                      np.ascontiguousarray(basis.exps, dtype=np.float64),
                      np.ascontiguousarray(basis.coefs, dtype=np.float64)]
        cen, l, npr, ex, co = self._keep
        self._h = self._lib.or_basis_new(int(l.shape[0]), _ptr(cen), _ptr(l), _ptr(npr), _ptr(ex), _ptr(co))
        if not self._h:
            raise ValueError("invalid basis (l must be 0 or 1, nprim > 0)")
        self.nbf = self._lib.or_nbf(self._h)
        self.basis = basis

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_basis_free(self._h)
            self._h = None

    # -- integrals ---------------------------------------------------------
    def shell_coefs(self, s: int) -> np.ndarray:
        out = np.zeros(int(self.basis.nprim[s]))
        self._lib.or_shell_coefs(self._h, s, _ptr(out))
        return out

    def eri(self, i, j, k, l) -> float:
        return self._lib.or_eri(self._h, int(i), int(j), int(k), int(l))

    def eri_matrix(self, rows, cols=None) -> np.ndarray:
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cols = rows if cols is None else np.ascontiguousarray(cols, dtype=np.int64)
        out = np.zeros((rows.shape[0], cols.shape[0]))
        self._lib.or_eri_matrix(self._h, _ptr(rows), rows.shape[0], _ptr(cols), cols.shape[0], _ptr(out))
        return out

    def diag_all(self) -> np.ndarray:
        n = self.nbf * (self.nbf + 1) // 2
        out = np.zeros(n)
        self._lib.or_diag_all(self._h, _ptr(out))
        return out

    def eri_tensor(self) -> np.ndarray:
        """Full N^4 tensor (small N only) from the packed ERI matrix."""
        N = self.nbf
        allp = np.arange(N * (N + 1) // 2, dtype=np.int64)
        A = self.eri_matrix(allp)
        mu, nu = unpack_pair(allp)
        full = np.zeros((N, N, N, N))
        idx = np.zeros((N, N), dtype=np.int64)
        idx[mu, nu] = allp
        idx[nu, mu] = allp
        full[:] = A[idx[:, :, None, None], idx[None, None, :, :]]
        return full

    # -- screening ---------------------------------------------------------
    def screen(self, thr: float, diag: Optional[np.ndarray] = None) -> np.ndarray:
        """Packed indices of the function pairs of the kept shell pairs."""
        if diag is None:
            diag = self.diag_all()
        diag = np.ascontiguousarray(diag, dtype=np.float64)
        out = np.zeros(diag.shape[0], dtype=np.int64)
        n = self._lib.or_screen(self._h, _ptr(diag), float(thr), _ptr(out))
        return out[:n].copy()

    # -- Cholesky decomposition -------------------------------------------
    def cd(self, rows, tau: float, forced=None, mcap: Optional[int] = None,
           max_steps: Optional[int] = None, candidates=None, copy: bool = True) -> CDResult:
        """Run the decomposition; ``max_steps`` stops after that many vectors
        (a bounded sample of a large run; the result is then partial).
        ``candidates``: boolean mask over ``rows`` of the rows that may be pivots
        (None = all); the stop test then runs over those rows only.
        ``copy=False`` returns views into the work arrays instead of trimmed
        copies (for runs whose vectors fill most of the host memory)."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cand = None if candidates is None else np.ascontiguousarray(candidates, dtype=np.uint8)
        if max_steps is not None:
            mcap = int(max_steps)
        n = rows.shape[0]
        if forced is not None:
            forced = np.ascontiguousarray(forced, dtype=np.int64)
            nf = forced.shape[0]
        else:
            nf = -1
        mcap = mcap or (nf if nf >= 0 else min(n, max(64, 4 * self.nbf)))
        while True:
            piv = np.zeros(max(mcap, 1), dtype=np.int64)
            L = np.zeros((max(mcap, 1), n))
            D = np.zeros(n)
            gap = np.zeros(max(mcap, 1))
            pivD = np.zeros(max(mcap, 1))
            M = self._lib.or_cd(self._h, _ptr(rows), n, float(tau),
                                _ptr(forced) if forced is not None else None, nf, mcap,
                                _ptr(piv), _ptr(L), _ptr(D), _ptr(gap), _ptr(pivD),
                                _ptr(cand) if cand is not None else None)
            if M == -1 and max_steps is not None:
                M = int(max_steps)
            elif M == -1 and mcap < n:
                mcap = min(n, 2 * mcap)
                continue
            if M == -2:
                raise ArithmeticError("ERI matrix not positive semidefinite within tolerance")
            if M < 0:
                raise RuntimeError(f"oracle CD failed with status {M}")
            if not copy:
                return CDResult(rows, piv[:M], L[:M], D, gap[:M], pivD[:M])
            return CDResult(rows, piv[:M].copy(), L[:M].copy(), D, gap[:M].copy(), pivD[:M].copy())

    # -- span-factor selection and the two-step scheme --------------------
    def cd_span(self, rows, tau: float, span: float, qmax: int = 64, reduce: bool = False,
                mcap: Optional[int] = None, candidates=None) -> SpanResult:
        """Partially pivoted decomposition with span factor ``span`` (C ``or_cd_span``).

        ``reduce=False``: Koch's one-step algorithm, ``L`` is the factor.
        ``reduce=True``: first step of the two-step scheme (rows whose residual
        diagonal drops below tau are discarded); only ``piv`` is meaningful and
        the vectors come from :meth:`cd_from_basis`.
        """
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        cand = None if candidates is None else np.ascontiguousarray(candidates, dtype=np.uint8)
        n = rows.shape[0]
        mcap = mcap or min(n, max(64, 4 * self.nbf))
        while True:
            piv = np.zeros(max(mcap, 1), dtype=np.int64)
            L = np.zeros((max(mcap, 1), n))
            D = np.zeros(n)
            ms = np.zeros(max(mcap, 1) + 1, dtype=np.int32)
            nm = ctypes.c_int(0)
            M = self._lib.or_cd_span(self._h, _ptr(rows), n, float(tau), float(span), int(qmax), int(bool(reduce)),
                                     mcap, _ptr(piv), _ptr(L), _ptr(D), _ptr(ms), ctypes.byref(nm),
                                     _ptr(cand) if cand is not None else None)
            if M == -1 and mcap < n:
                mcap = min(n, 2 * mcap)
                continue
            if M == -2:
                raise ArithmeticError("ERI matrix not positive semidefinite within tolerance")
            if M < 0:
                raise RuntimeError(f"oracle span CD failed with status {M}")
            return SpanResult(rows, piv[:M].copy(), L[:M].copy(), D, ms[:nm.value].copy())

    def cd_from_basis(self, rows, piv) -> np.ndarray:
        """Second step of the two-step scheme: vectors [M, npairs] from the metric
        Cholesky factor of the basis ``piv`` and a triangular solve (``or_cd_from_basis``)."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        piv = np.ascontiguousarray(piv, dtype=np.int64)
        M = int(piv.shape[0])
        L = np.zeros((max(M, 1), rows.shape[0]))
        st = self._lib.or_cd_from_basis(self._h, _ptr(rows), rows.shape[0], _ptr(piv), M, _ptr(L))
        if st == -2:
            raise ArithmeticError("metric of the Cholesky basis is not positive definite")
        return L[:M].copy()


def density(C_occ: np.ndarray) -> np.ndarray:
    """D = 2 C C^T (closed-shell density of the occupied block)."""
    return 2.0 * C_occ @ C_occ.T


def unpack_vectors(L: np.ndarray, rows: np.ndarray, N: int) -> np.ndarray:
    """[M, npairs] packed vectors -> [M, N, N] symmetric matrices."""
    mu, nu = unpack_pair(rows)
    out = np.zeros((L.shape[0], N, N))
    out[:, mu, nu] = L
    out[:, nu, mu] = L
    return out


def jk_from_vectors(L: np.ndarray, rows: np.ndarray, C_occ: np.ndarray, want_j: bool = True, want_k: bool = True):
    """J and K from Cholesky vectors, written from the definitions (Sec. 4.1).

    J_{mu nu} = sum_P L^P_{mu nu} sum_{sigma rho} L^P_{sigma rho} D_{sigma rho}
    K_{mu nu} = sum_P sum_{sigma rho} L^P_{mu sigma} D_{sigma rho} L^P_{rho nu}
    with L^P the full symmetric N x N matrix of vector P and D = 2 C C^T.
    ``want_j`` / ``want_k`` skip the other matrix (returned as None).
    """
    N = C_occ.shape[0]
    Dm = density(C_occ)
    J = np.zeros((N, N)) if want_j else None
    K = np.zeros((N, N)) if want_k else None
    for P in range(L.shape[0]):
        LP = unpack_vectors(L[P:P + 1], rows, N)[0]
        if want_j:
            J += LP * np.sum(LP * Dm)
        if want_k:
            K += LP @ Dm @ LP
    return J, K


def jk_exact(tensor: np.ndarray, C_occ: np.ndarray):
    """J and K from the exact ERI tensor (mu nu|sigma rho)."""
    Dm = density(C_occ)
    J = np.einsum("mnsr,sr->mn", tensor, Dm)
    K = np.einsum("msnr,sr->mn", tensor, Dm)
    return J, K


def mo_vectors(L: np.ndarray, rows: np.ndarray, C: np.ndarray) -> np.ndarray:
    """Cholesky vectors in the MO basis (Sec. 4.1, CASSCF / CC): for every vector P,
    L^P_{pq} = sum_{mu nu} C_{mu p} L^P_{mu nu} C_{nu q}, L^P the symmetric N x N
    unpacking of the packed vector.  Returns [M, n_mo, n_mo]."""
    N = C.shape[0]
    U = unpack_vectors(L, rows, N)             # [M, N, N]
    return np.einsum("mp,Pmn,nq->Ppq", C, U, C, optimize=True)


def mo_eri(tensor: np.ndarray, C: np.ndarray) -> np.ndarray:
    """(pq|rs) = sum C_{mu p} C_{nu q} C_{sigma r} C_{rho s} (mu nu|sigma rho), from the exact tensor."""
    return np.einsum("ap,bq,cr,ds,abcd->pqrs", C, C, C, C, tensor, optimize=True)
