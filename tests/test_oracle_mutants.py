"""Mutation test of the oracle's pins: each plausible mistake below is planted
in a copy of the oracle's C source (never in the oracle itself), the copy is
built, and the independent checks of ``tests/_mutant_checks.py`` must reject
it.  The unmodified source must pass every check.  A mutant runs in a child
process, so that one that misbehaves cannot take the test run down with it.
"""
import json
import os
import subprocess
import sys

import pytest

import synth

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "oracle", "cdoracle.c")

# (name, text in the source, planted replacement); the first occurrence is replaced
MUTANTS = [
    ("boys downward recursion sign", "(2.0 * T * F[m + 1] + emT) / (2 * m + 1)",
     "(2.0 * T * F[m + 1] - emT) / (2 * m + 1)"),
    ("boys series denominator", "term *= 2.0 * T / (2 * mmax + 2 * i + 1);",
     "term *= 2.0 * T / (2 * mmax + 2 * i + 3);"),
    ("boys asymptotic prefactor", "F[0] = 0.5 * sqrt(OR_PI / T);", "F[0] = sqrt(OR_PI / T);"),
    ("bra recurrence W-P sign", "v = PX[i] * os_rec(s, A, B, c, d, m) + s->WP[i] * os_rec(s, A, B, c, d, m + 1);",
     "v = PX[i] * os_rec(s, A, B, c, d, m) - s->WP[i] * os_rec(s, A, B, c, d, m + 1);"),
    ("bra recurrence dropped rho/p term",
     "v += B[i] * s->o2p * (os_rec(s, A, t, c, d, m) - s->rp * os_rec(s, A, t, c, d, m + 1));",
     "v += B[i] * s->o2p * os_rec(s, A, t, c, d, m);"),
    ("cross term Boys order", "v += c[i] * s->o2pq * os_rec(s, A, B, t, d, m + 1);",
     "v += c[i] * s->o2pq * os_rec(s, A, B, t, d, m);"),
    ("ket recurrence Q-C sign", "v = QX[i] * os_rec(s, a, b, C, D, m) + s->WQ[i] * os_rec(s, a, b, C, D, m + 1);",
     "v = -QX[i] * os_rec(s, a, b, C, D, m) + s->WQ[i] * os_rec(s, a, b, C, D, m + 1);"),
    ("prefactor sqrt(p+q)", "s->base = 2.0 * pow(OR_PI, 2.5) / (p * q * sqrt(pq))",
     "s->base = 2.0 * pow(OR_PI, 2.5) / (p * q * pq)"),
    ("W transposed", "W[k] = (p * P[k] + q * Q[k]) / pq;", "W[k] = (q * P[k] + p * Q[k]) / pq;"),
    # (a constant factor in the p primitive norm would cancel in the contraction norm;
    # a wrong power of the exponent does not)
    ("p primitive norm", "if (l[s] == 1) n *= sqrt(4.0 * a);", "if (l[s] == 1) n *= 4.0 * a;"),
    ("s primitive norm power", "double n = pow(2.0 * a / OR_PI, 0.75);", "double n = pow(2.0 * a / OR_PI, 0.5);"),
    ("p contraction overlap", "if (l[s] == 1) ov /= 2.0 * ab;", "if (l[s] == 1) ov /= ab;"),
    # Eq. (subtr) in the oracle's default (row-chunked, J-outer) loop order
    ("cd update sign", "for (int64_t r = r0; r < r1; ++r) out[r] -= LJ[r] * wj;",
     "for (int64_t r = r0; r < r1; ++r) out[r] += LJ[r] * wj;"),
    ("cd divides by D not sqrt(D)", "double sq = sqrt(D[p]);", "double sq = D[p];"),
    ("cd diagonal update", "D[r] -= LK[r] * LK[r];", "D[r] -= 0.5 * LK[r] * LK[r];"),
]


def _build(tmp, name, text):
    src = os.path.join(tmp, name + ".c")
    lib = os.path.join(tmp, name + ".so")
    with open(src, "w") as fh:
        fh.write(text)
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", lib, src, "-lm"])
    return lib


def _checks(lib, spec):
    r = subprocess.run([sys.executable, os.path.join(HERE, "_mutant_checks.py"), lib, spec],
                       capture_output=True, text=True, timeout=300)
    if r.returncode != 0:  # a crash or an error is a rejection too
        return {"ran": False}
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def spec(tmp_path_factory):
    # s functions only: p components on one centre have exactly equal diagonals, and
    # dpstrf breaks such ties in its own way
    s = synth.make_workload("s40")
    b = s.basis
    path = tmp_path_factory.mktemp("spec") / "s40.json"
    path.write_text(json.dumps({"center": b.center.tolist(), "l": b.l.tolist(), "nprim": b.nprim.tolist(),
                                "exps": b.exps.tolist(), "coefs": b.coefs.tolist(), "tau": s.tau}))
    return str(path)


@pytest.fixture(scope="module")
def source():
    with open(SRC) as fh:
        return fh.read()


def test_unmodified_oracle_passes_every_check(tmp_path, source, spec):
    res = _checks(_build(str(tmp_path), "orig", source), spec)
    assert res.get("ran", True) and all(res.values()), res
    assert set(res) >= {"boys", "ssss", "p_first_derivatives", "p_second_derivatives", "normalised_s",
                        "normalised_p", "cd_vs_dpstrf"}


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, source, spec, name, old, new):
    assert source.count(old) >= 1, f"mutation site not found: {old}"
    mutant = source.replace(old, new, 1)
    res = _checks(_build(str(tmp_path), "mutant", mutant), spec)
    failed = [k for k, v in res.items() if not v]
    assert failed, f"no check caught the planted mistake '{name}': {res}"
