"""Properties of the stored oracle runs at N = 400, 1200 and 2000
(tests/golden/*_oracle.npz, written by make_golden.py from the oracle alone)
that the fully pivoted recursion of Sec. 2 fixes at any size, so that the
stored M and pivot list are checked against more than a re-run of the oracle:

* the pivot diagonals are the running maxima of residual diagonals that only
  lose squares, so they never increase, exactly;
* the stop rule: every pivot diagonal is >= tau, the final maximum residual
  diagonal is < tau, and M is the number of pivots;
* the pivots are distinct screened rows;
* D = 2 C C^T is PSD and K = 2 sum_P B^P B^P^T is PSD, so K has a non-negative
  diagonal and tr(D K) >= 0; J and K are symmetric on the sampled rows.
"""
import json
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden")


@pytest.mark.parametrize("name", ["sp400", "sp1200", "sp2000"])
def test_stored_oracle_run_obeys_the_recursion(name):
    g = np.load(os.path.join(GOLDEN, f"{name}_oracle.npz"))
    meta = json.loads(str(g["meta"]))
    tau, M = meta["tau"], meta["M"]
    pivD, piv = g["pivD"], g["piv_packed"]
    assert len(pivD) == M and len(piv) == M
    assert np.all(np.diff(pivD) <= 0.0)
    assert pivD[-1] >= tau > float(g["max_resid"])
    assert len(np.unique(piv)) == M
    N = meta["N"]
    assert np.all((piv >= 0) & (piv < N * (N + 1) // 2))
    assert np.all(g["K_diag"] >= 0.0)
    assert float(g["trDK"]) >= 0.0
    # sampled rows of J and K against their own transposes where both entries were stored
    rows = g["jkrows"]
    for X in ("J", "K"):
        block = g[f"{X}_rows"][:, rows]
        assert np.max(np.abs(block - block.T)) <= 1e-12 * np.max(np.abs(g[f"{X}_rows"]))
        assert np.array_equal(np.diag(block), g[f"{X}_diag"][rows])
