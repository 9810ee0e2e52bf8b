"""Checks of an oracle library build against facts fixed outside it, for the
mutation test (tests/test_oracle_mutants.py).  Run as a script on one shared
library; prints a JSON object {check name: passed} and never raises on a
failed check, so that a build with a planted mistake is reported, not fatal.

The references: the Boys function from the regularised incomplete gamma
function (scipy); the (ss|ss) closed form; p-type integrals as centre
derivatives of that closed form (central finite differences); normalised
integrals with the textbook primitive norms and the analytic self-overlap of a
contracted s function; the pivoted Cholesky against LAPACK dpstrf.
"""
import ctypes
import json
import math
import sys

import numpy as np
import scipy.linalg.lapack
import scipy.special

PI = math.pi


def boys_ref(m, T):
    if T == 0.0:
        return 1.0 / (2 * m + 1)
    a = m + 0.5
    return scipy.special.gammainc(a, T) * scipy.special.gamma(a) / (2.0 * T ** a)


def ssss(a, A, b, B, c, C, d, D):
    """(ss|ss) of unnormalised primitives, closed form with F_0 from erf."""
    A, B, C, D = map(np.asarray, (A, B, C, D))
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    T = p * q / (p + q) * float(np.sum((P - Q) ** 2))
    F0 = 1.0 if T == 0 else 0.5 * math.sqrt(PI / T) * math.erf(math.sqrt(T))
    return (2 * PI ** 2.5 / (p * q * math.sqrt(p + q)) * math.exp(-a * b / p * np.sum((A - B) ** 2))
            * math.exp(-c * d / q * np.sum((C - D) ** 2)) * F0)


def run(path):
    lib = ctypes.CDLL(path)
    P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    lib.or_boys.argtypes = [I, D, P]
    lib.or_eri_prim.restype = D
    lib.or_eri_prim.argtypes = [P, D, P, P, D, P, P, D, P, P, D, P]
    lib.or_basis_new.restype = P
    lib.or_basis_new.argtypes = [I, P, P, P, P, P]
    lib.or_eri.restype = D
    lib.or_eri.argtypes = [P, I, I, I, I]
    out = {}

    # Boys
    ok = True
    F = np.zeros(8)
    for T in (0.0, 0.3, 5.0, 20.0, 40.0, 80.0):
        lib.or_boys(4, T, F.ctypes.data_as(P))
        for m in range(5):
            ref = boys_ref(m, T)
            ok &= abs(F[m] - ref) <= 1e-12 * abs(ref)
    out["boys"] = bool(ok)

    def prim(la, ea, A, lb, eb, B, lc, ec, C, ld, ed, Dd):
        arr = [np.array(v, dtype=np.int32) for v in (la, lb, lc, ld)]
        cen = [np.array(v, dtype=np.float64) for v in (A, B, C, Dd)]
        ptr = [x.ctypes.data_as(P) for x in arr + cen]
        return lib.or_eri_prim(ptr[0], ea, ptr[4], ptr[1], eb, ptr[5], ptr[2], ec, ptr[6], ptr[3], ed, ptr[7])

    s0 = [0, 0, 0]
    ex = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    a, b, c, d = 0.9, 0.4, 1.3, 0.7
    A, B, C, Dd = [0.0, 0.1, -0.2], [1.1, -0.3, 0.4], [-0.5, 0.9, 1.2], [0.6, 0.2, -0.8]
    ref = ssss(a, A, b, B, c, C, d, Dd)
    out["ssss"] = bool(abs(prim(s0, a, A, s0, b, B, s0, c, C, s0, d, Dd) - ref) <= 1e-12 * abs(ref))

    h = 1e-4

    def shifted(X, i, t):
        Y = list(X)
        Y[i] += t
        return Y

    def d1(which, i):  # d/dX_i of the closed form, X = A, B, C or D
        args = [A, B, C, Dd]
        lo, hi = list(args), list(args)
        lo[which], hi[which] = shifted(args[which], i, -h), shifted(args[which], i, h)
        return (ssss(a, hi[0], b, hi[1], c, hi[2], d, hi[3]) - ssss(a, lo[0], b, lo[1], c, lo[2], d, lo[3])) / (2 * h)

    def d2(w1, i, w2, j):
        args = [A, B, C, Dd]
        tot = 0.0
        for s1, s2 in ((1, 1), (1, -1), (-1, 1), (-1, -1)):
            X = [list(v) for v in args]
            X[w1] = shifted(X[w1], i, s1 * h)
            X[w2] = shifted(X[w2], j, s2 * h)
            tot += s1 * s2 * ssss(a, X[0], b, X[1], c, X[2], d, X[3])
        return tot / (4 * h * h)

    exps = [a, b, c, d]
    scale = abs(ref)
    ok = True
    for which in range(4):
        for i in range(3):
            ls = [s0, s0, s0, s0]
            ls[which] = ex[i]
            got = prim(ls[0], a, A, ls[1], b, B, ls[2], c, C, ls[3], d, Dd)
            ok &= abs(got - d1(which, i) / (2 * exps[which])) <= 1e-6 * scale
    out["p_first_derivatives"] = bool(ok)
    ok = True
    # two p functions on different centres: d^2/dX_i dY_j of the closed form / (4 x y)
    for (w1, w2) in ((0, 1), (0, 2), (1, 3), (2, 3)):
        for (i, j) in ((0, 0), (1, 2), (2, 2)):
            ls = [s0, s0, s0, s0]
            ls[w1], ls[w2] = ex[i], ex[j]
            got = prim(ls[0], a, A, ls[1], b, B, ls[2], c, C, ls[3], d, Dd)
            ok &= abs(got - d2(w1, i, w2, j) / (4 * exps[w1] * exps[w2])) <= 1e-5 * scale
    out["p_second_derivatives"] = bool(ok)

    # normalised contracted functions: s and p shells with 2 primitives each, at A and B
    sa, sc_ = np.array([0.8, 0.25]), np.array([0.6, 0.5])
    pa, pc_ = np.array([0.55, 1.7]), np.array([0.7, 0.4])
    cen = np.array([A, B], dtype=np.float64)
    lsh = np.array([0, 1], dtype=np.int32)
    npr = np.array([2, 2], dtype=np.int32)
    exv = np.array([sa[0], sa[1], pa[0], pa[1]])
    cov = np.array([sc_[0], sc_[1], pc_[0], pc_[1]])
    hdl = lib.or_basis_new(2, cen.ctypes.data_as(P), lsh.ctypes.data_as(P), npr.ctypes.data_as(P),
                           exv.ctypes.data_as(P), cov.ctypes.data_as(P))
    Ns = (2 * sa / PI) ** 0.75
    S = sum(sc_[i] * sc_[j] * Ns[i] * Ns[j] * (PI / (sa[i] + sa[j])) ** 1.5 for i in range(2) for j in range(2))
    cs = sc_ * Ns / math.sqrt(S)
    # p_x primitive norm from its self-overlap (pi/2a)^{3/2} / (4a); contracted
    # p_x self-overlap from the overlaps (pi/(a+b))^{3/2} / (2(a+b))
    Npr = (2 * pa / PI) ** 0.75 * np.sqrt(4 * pa)
    Sp = sum(pc_[i] * pc_[j] * Npr[i] * Npr[j] * (PI / (pa[i] + pa[j])) ** 1.5 / (2 * (pa[i] + pa[j]))
             for i in range(2) for j in range(2))
    cp = pc_ * Npr / math.sqrt(Sp)
    ref_ss = sum(cs[i] * cs[j] * cs[k] * cs[l] * ssss(sa[i], A, sa[j], A, sa[k], A, sa[l], A)
                 for i in range(2) for j in range(2) for k in range(2) for l in range(2))
    out["normalised_s"] = bool(abs(lib.or_eri(hdl, 0, 0, 0, 0) - ref_ss) <= 1e-12 * abs(ref_ss))
    # (s p_x | s s): derivative of the closed form in B_x
    ref_sp = 0.0
    for i in range(2):
        for j in range(2):
            for k in range(2):
                for l in range(2):
                    f = lambda Bx: ssss(sa[i], A, pa[j], [Bx, B[1], B[2]], sa[k], A, sa[l], A)  # noqa: E731
                    ref_sp += (cs[i] * cp[j] * cs[k] * cs[l] * (f(B[0] + h) - f(B[0] - h)) / (2 * h)
                               / (2 * pa[j]))
    out["normalised_p"] = bool(abs(lib.or_eri(hdl, 0, 1, 0, 0) - ref_sp) <= 1e-7 * abs(ref_sp))
    return out


def run_cd(path, center, l, nprim, exps, coefs, tau):
    """The library's pivoted Cholesky on its own ERI matrix of a small basis,
    against LAPACK dpstrf on that same matrix: same rank, same pivots (away
    from near-ties), same factor."""
    lib = ctypes.CDLL(path)
    P, D, I, I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    lib.or_basis_new.restype = P
    lib.or_basis_new.argtypes = [I, P, P, P, P, P]
    lib.or_nbf.restype = I
    lib.or_nbf.argtypes = [P]
    lib.or_eri_matrix.argtypes = [P, P, I, P, I, P]
    lib.or_cd.restype = I
    lib.or_cd.argtypes = [P, P, I64, D, P, I, I, P, P, P, P, P, P]
    arrs = [np.ascontiguousarray(center, np.float64), np.ascontiguousarray(l, np.int32),
            np.ascontiguousarray(nprim, np.int32), np.ascontiguousarray(exps, np.float64),
            np.ascontiguousarray(coefs, np.float64)]
    h = lib.or_basis_new(len(arrs[1]), *[x.ctypes.data_as(P) for x in arrs])
    N = lib.or_nbf(h)
    rows = np.arange(N * (N + 1) // 2, dtype=np.int64)
    n = rows.shape[0]
    A = np.zeros((n, n))
    lib.or_eri_matrix(h, rows.ctypes.data_as(P), n, rows.ctypes.data_as(P), n, A.ctypes.data_as(P))
    mcap = n
    piv = np.zeros(mcap, dtype=np.int64)
    L = np.zeros((mcap, n))
    Dg = np.zeros(n)
    gap = np.zeros(mcap)
    pivD = np.zeros(mcap)
    M = lib.or_cd(h, rows.ctypes.data_as(P), n, tau, None, -1, mcap, piv.ctypes.data_as(P), L.ctypes.data_as(P),
                  Dg.ctypes.data_as(P), gap.ctypes.data_as(P), pivD.ctypes.data_as(P), None)
    c, p2, rank, info = scipy.linalg.lapack.dpstrf(A.copy(), lower=1, tol=tau)
    if M != rank:
        return False
    perm = p2 - 1                      # dpstrf's full row permutation
    if not np.array_equal(piv[:M], perm[:rank]):
        return False
    Lf = np.tril(c)[:, :rank]          # A[perm][:, perm] ~= Lf Lf^T
    return bool(np.max(np.abs(L[:M][:, perm].T - Lf)) < 1e-10 * np.max(np.abs(Lf)))


if __name__ == "__main__":
    res = run(sys.argv[1])
    if len(sys.argv) > 2:
        spec = json.loads(open(sys.argv[2]).read())
        res["cd_vs_dpstrf"] = run_cd(sys.argv[1], spec["center"], spec["l"], spec["nprim"], spec["exps"],
                                     spec["coefs"], spec["tau"])
    print(json.dumps(res))
