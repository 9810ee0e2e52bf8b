"""Pins for the oracle's integral layer, against facts fixed outside it.

* Boys function: the erf closed form of F_0, the value F_m(0) = 1/(2m+1), and
  adaptive quadrature of its integral definition.
* (ss|ss): the textbook closed form for four s Gaussians.
* p-type integrals: centre derivatives of that closed form, taken
  symbolically (an unnormalised Cartesian p Gaussian on A is (1/2a) d/dA_i of
  the s Gaussian), evaluated in 30-digit arithmetic.
* Rotation covariance of p functions, 8-fold permutational symmetry, and the
  positive semidefiniteness of the ERI matrix.
* Normalisation: unit self-overlap by radial quadrature.
* A printed textbook value set (H2/STO-3G, tests/golden/h2_sto3g.txt).
"""
import math
import os

import numpy as np
import pytest
import scipy.integrate
import scipy.special

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Boys -----
@pytest.mark.parametrize("T", [0.0, 1e-12, 1e-6, 0.05, 0.5, 1.0, 2.7, 7.3, 12.0, 20.0,
                               29.9, 34.99, 35.0, 35.01, 50.0, 120.0, 1e4])
def test_boys_f0_closed_form(T):
    F = oracle.boys(4, T)
    if T == 0.0:
        ref = 1.0
    elif T < 1e-10:
        ref = 1.0 - T / 3.0
    else:
        ref = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    assert abs(F[0] - ref) <= 2e-15 * max(1.0, abs(ref))


def test_boys_zero_argument():
    F = oracle.boys(8, 0.0)
    for m in range(9):
        assert abs(F[m] - 1.0 / (2 * m + 1)) < 1e-15


@pytest.mark.parametrize("m", [0, 1, 2, 3, 4, 6])
@pytest.mark.parametrize("T", [0.3, 3.0, 11.0, 26.0, 34.0, 36.0, 60.0])
def test_boys_quadrature(m, T):
    F = oracle.boys(m, T)
    import mpmath
    mpmath.mp.dps = 30
    val = float(mpmath.quad(lambda t: t ** (2 * m) * mpmath.exp(-T * t * t), [0, 0.25, 0.5, 1]))
    assert abs(F[m] - val) <= 1e-13 * val


# --------------------------------------------------------- closed forms ----
def _ssss_closed(a, A, b, B, c, C, d, D):
    A, B, C, D = (np.asarray(x, float) for x in (A, B, C, D))
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    rho = p * q / (p + q)
    T = rho * np.sum((P - Q) ** 2)
    F0 = 1.0 if T == 0 else 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
    return (2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q))
            * math.exp(-a * b / p * np.sum((A - B) ** 2))
            * math.exp(-c * d / q * np.sum((C - D) ** 2)) * F0)


def test_ssss_closed_form_random():
    rng = np.random.default_rng(11)
    z = np.zeros(3, dtype=np.int32)
    for _ in range(200):
        ex = np.exp(rng.uniform(math.log(0.1), math.log(30.0), 4))
        cen = rng.uniform(-3, 3, (4, 3))
        if rng.random() < 0.2:
            cen[1] = cen[0]
        if rng.random() < 0.1:
            cen[:] = cen[0]
        v = oracle.eri_prim(z, ex[0], cen[0], z, ex[1], cen[1], z, ex[2], cen[2], z, ex[3], cen[3])
        ref = _ssss_closed(ex[0], cen[0], ex[1], cen[1], ex[2], cen[2], ex[3], cen[3])
        assert abs(v - ref) <= 1e-13 * abs(ref), (v, ref)


# ------------------------------------------- p functions by derivatives ----
def _symbolic_ssss():
    import sympy as sp
    Ax, Ay, Az, Bx, By, Bz, Cx, Cy, Cz, Dx, Dy, Dz = sp.symbols("Ax Ay Az Bx By Bz Cx Cy Cz Dx Dy Dz", real=True)
    a, b, c, d = sp.symbols("a b c d", positive=True)
    A = sp.Matrix([Ax, Ay, Az]); B = sp.Matrix([Bx, By, Bz])
    C = sp.Matrix([Cx, Cy, Cz]); D = sp.Matrix([Dx, Dy, Dz])
    p, q = a + b, c + d
    P, Q = (a * A + b * B) / p, (c * C + d * D) / q
    rho = p * q / (p + q)
    T = rho * (P - Q).dot(P - Q)
    F0 = sp.sqrt(sp.pi) / 2 * sp.erf(sp.sqrt(T)) / sp.sqrt(T)
    expr = (2 * sp.pi ** sp.Rational(5, 2) / (p * q * sp.sqrt(p + q))
            * sp.exp(-a * b / p * (A - B).dot(A - B)) * sp.exp(-c * d / q * (C - D).dot(C - D)) * F0)
    syms = {"A": (Ax, Ay, Az), "B": (Bx, By, Bz), "C": (Cx, Cy, Cz), "D": (Dx, Dy, Dz)}
    return sp, expr, syms, (a, b, c, d)


@pytest.mark.parametrize("case", [
    # (cart per centre as axis index or None)
    (0, None, None, None),
    (None, 2, None, None),
    (None, None, 1, None),
    (None, None, None, 0),
    (0, 0, None, None),
    (0, 1, None, None),
    (2, None, 2, None),
    (1, None, None, 2),
    (0, 1, 2, None),
    (1, 1, 1, 1),
    (0, 2, 1, 0),
])
def test_p_integrals_match_centre_derivatives(case):
    sp, expr, syms, (a, b, c, d) = _symbolic_ssss()
    import mpmath
    mpmath.mp.dps = 30
    rng = np.random.default_rng(sum((k if k is not None else 7) * 10 ** i for i, k in enumerate(case)))
    ex = np.exp(rng.uniform(math.log(0.2), math.log(8.0), 4))
    cen = rng.uniform(-1.5, 1.5, (4, 3))
    e = expr
    scale = 1.0
    for k, (name, ax) in enumerate(zip("ABCD", case)):
        if ax is not None:
            e = sp.diff(e, syms[name][ax])
            scale /= 2.0 * ex[k]
    subs = {a: sp.Float(ex[0], 30), b: sp.Float(ex[1], 30), c: sp.Float(ex[2], 30), d: sp.Float(ex[3], 30)}
    for k, name in enumerate("ABCD"):
        for ax in range(3):
            subs[syms[name][ax]] = sp.Float(cen[k, ax], 30)
    ref = float(e.evalf(30, subs=subs)) * scale
    carts = []
    for ax in case:
        v = np.zeros(3, dtype=np.int32)
        if ax is not None:
            v[ax] = 1
        carts.append(v)
    val = oracle.eri_prim(carts[0], ex[0], cen[0], carts[1], ex[1], cen[1],
                          carts[2], ex[2], cen[2], carts[3], ex[3], cen[3])
    assert abs(val - ref) <= 1e-12 * max(abs(ref), 1e-3), (val, ref)


# ---------------------------------------------------- symmetry, PSD ---------
def test_eightfold_symmetry_sp():
    s = synth.make_workload("sp8")
    o = oracle.Oracle(s.basis)
    rng = np.random.default_rng(5)
    N = o.nbf
    for _ in range(60):
        i, j, k, l = (int(x) for x in rng.integers(0, N, 4))
        v = o.eri(i, j, k, l)
        for perm in [(j, i, k, l), (i, j, l, k), (j, i, l, k), (k, l, i, j), (l, k, i, j), (k, l, j, i), (l, k, j, i)]:
            assert abs(o.eri(*perm) - v) <= 1e-14 * max(1.0, abs(v))


@pytest.mark.parametrize("name", ["s40", "sp8"])
def test_eri_matrix_psd(name):
    s = synth.make_workload(name)
    o = oracle.Oracle(s.basis)
    N = o.nbf
    A = o.eri_matrix(np.arange(N * (N + 1) // 2))
    assert np.allclose(A, A.T, rtol=0, atol=1e-14)
    w = np.linalg.eigvalsh(A)
    assert w[0] >= -1e-12 * w[-1]


def _rot(axis, ang):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


def test_rotation_covariance_p():
    s = synth.make_lattice((2, 2, 1), seed=77, n_occ=2)
    b = s.basis
    R = _rot([0.3, -0.5, 0.8], 0.9)
    b2 = synth.Basis(center=b.center @ R.T, l=b.l, nprim=b.nprim, exps=b.exps, coefs=b.coefs)
    o1, o2 = oracle.Oracle(b), oracle.Oracle(b2)
    N = o1.nbf
    # transformation of each function under the rotation: s invariant, p_i -> sum_j R_ji p_j
    T = np.zeros((N, N))
    f = 0
    for l in b.l:
        if l == 0:
            T[f, f] = 1.0
            f += 1
        else:
            T[f:f + 3, f:f + 3] = R
            f += 3
    # full tensors (N = 16 here)
    t1 = o1.eri_tensor()
    t2 = o2.eri_tensor()
    t1r = np.einsum("ai,bj,ck,dl,ijkl->abcd", T, T, T, T, t1)
    assert np.max(np.abs(t1r - t2)) < 1e-12


# ------------------------------------------------------- normalisation -----
def test_unit_self_overlap_radial_quadrature():
    s = synth.make_lattice((1, 1, 2), seed=31, n_occ=1)
    o = oracle.Oracle(s.basis)
    pofs = np.concatenate([[0], np.cumsum(s.basis.nprim)])
    for sh in range(s.basis.n_shells):
        ex = s.basis.exps[pofs[sh]:pofs[sh + 1]]
        dc = o.shell_coefs(sh)
        l = int(s.basis.l[sh])

        def radial(r):
            g = np.sum(dc * np.exp(-ex * r * r))
            return g * g * r ** (2 + 2 * l) * 4 * math.pi / (3.0 if l == 1 else 1.0)
        val, _ = scipy.integrate.quad(radial, 0, np.inf, epsabs=0, epsrel=1e-13, limit=400)
        assert abs(val - 1.0) < 1e-12


# ------------------------------------------------------ textbook values ----
def test_h2_sto3g_szabo_ostlund():
    lines = [ln.split() for ln in open(os.path.join(GOLDEN, "h2_sto3g.txt")) if ln.strip() and not ln.startswith("#")]
    cen = np.array([[float(x) for x in ln[1:]] for ln in lines if ln[0] == "center"])
    exps = np.array([float(x) for x in next(ln for ln in lines if ln[0] == "exps")[1:]])
    coefs = np.array([float(x) for x in next(ln for ln in lines if ln[0] == "coefs")[1:]])
    basis = synth.Basis(center=cen, l=np.zeros(2, np.int32), nprim=np.full(2, 3, np.int32),
                        exps=np.concatenate([exps, exps]), coefs=np.concatenate([coefs, coefs]))
    o = oracle.Oracle(basis)
    for ln in lines:
        if ln[0] == "eri":
            i, j, k, l = (int(x) for x in ln[1:5])
            assert abs(o.eri(i, j, k, l) - float(ln[5])) < 6e-5, ln
