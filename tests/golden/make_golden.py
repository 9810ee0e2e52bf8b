"""Write the oracle's reference results for the large synthetic systems.

    python tests/golden/make_golden.py sp1200 [sp2000 ...] [--threads T]

For each named workload (``synth.make_workload``) this runs the CPU oracle
(``oracle/``) end to end -- screening, the fully pivoted decomposition of
Sec. 2 until max D < tau, and J, K from the vectors by their definitions
(Sec. 4.1) -- and stores what a GPU run can be compared with:

* M, the pivots (packed pair indices), the tracked residual diagonal of every
  pivot when it was taken (``pivD``), the final max residual diagonal;
* the vectors on 32 sampled rows (``L_rows`` [M, 32]) and the final residual
  diagonal there;
* J and K (FP64) on 48 sampled rows (full rows of the N x N matrices), their
  diagonals, tr(DJ), tr(DK), max|J|, max|K|, and J X, K X for 4 seeded
  Gaussian columns X (a projection that sees every element);
* the oracle's wall times (screening, decomposition, J alone, K alone) and the
  OpenMP thread count, so the file doubles as a measured CPU baseline.

Every number comes from ``oracle`` on inputs from ``synth``; nothing here
reads GPU results.  Output: ``tests/golden/<name>_oracle.npz`` plus a short
``<name>_oracle.txt`` summary.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

N_LROWS = 32      # sampled rows of the vectors
N_JKROWS = 48     # sampled rows of J and K
N_PROJ = 4        # Gaussian projection columns


def sample_indices(name: str, n_rows: int, N: int):
    """Seeded sample positions (the same seeds in the tests that read the file)."""
    rng = np.random.default_rng(20260 + sum(map(ord, name)))
    lrows = np.sort(rng.choice(n_rows, N_LROWS, replace=False))
    jkrows = np.sort(rng.choice(N, N_JKROWS, replace=False))
    X = rng.standard_normal((N, N_PROJ))
    return lrows, jkrows, X


def run(name: str, threads: int | None, mcap: int | None = None) -> str:
    import oracle
    import synth
    if threads:
        os.environ["OMP_NUM_THREADS"] = str(threads)
    s = synth.make_workload(name)
    o = oracle.Oracle(s.basis)
    N = o.nbf
    t0 = time.perf_counter()
    rows = o.screen(s.schwarz)
    t_screen = time.perf_counter() - t0
    n = rows.shape[0]
    print(f"[{name}] N={N} rows={n} tau={s.tau} screening {t_screen:.1f}s", flush=True)
    t0 = time.perf_counter()
    # vector capacity: large enough for the run (M/N is 5-7 for these systems);
    # the work array is zero-filled lazily, so only the vectors made use memory
    mcap = min(n, mcap or 8 * N)
    r = o.cd(rows, s.tau, mcap=mcap, copy=False)
    t_cd = time.perf_counter() - t0
    print(f"[{name}] M={r.M} max D={r.D.max():.6e} decomposition {t_cd:.1f}s", flush=True)
    t0 = time.perf_counter()
    J, _ = oracle.jk_from_vectors(r.L, rows, s.C_occ, want_k=False)
    t_j = time.perf_counter() - t0
    t0 = time.perf_counter()
    _, K = oracle.jk_from_vectors(r.L, rows, s.C_occ, want_j=False)
    t_k = time.perf_counter() - t0
    print(f"[{name}] J {t_j:.1f}s K {t_k:.1f}s", flush=True)
    Dm = oracle.density(s.C_occ)
    lrows, jkrows, X = sample_indices(name, n, N)
    meta = {
        "workload": name, "N": N, "n_rows": int(n), "tau": s.tau, "schwarz": s.schwarz,
        "n_occ": int(s.C_occ.shape[1]), "M": r.M, "max_resid": float(r.D.max()),
        "t_screen_s": t_screen, "t_cd_s": t_cd, "t_j_s": t_j, "t_k_s": t_k,
        "omp_threads": int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)),
        "host_cores": os.cpu_count(),
        "command": "python tests/golden/make_golden.py " + name,
    }
    out = os.path.join(HERE, f"{name}_oracle.npz")
    np.savez_compressed(
        out,
        meta=np.array(json.dumps(meta)),
        piv_packed=rows[r.piv], pivD=np.array(r.pivD), max_resid=np.array(r.D.max()),
        lrows=lrows, L_rows=np.ascontiguousarray(r.L[:, lrows]), D_rows=r.D[lrows],
        jkrows=jkrows, J_rows=J[jkrows], K_rows=K[jkrows],
        J_diag=np.diag(J).copy(), K_diag=np.diag(K).copy(),
        trDJ=np.array(np.sum(Dm * J)), trDK=np.array(np.sum(Dm * K)),
        maxJ=np.array(np.max(np.abs(J))), maxK=np.array(np.max(np.abs(K))),
        X=X, JX=J @ X, KX=K @ X,
    )
    with open(os.path.join(HERE, f"{name}_oracle.txt"), "w") as fh:
        fh.write(f"Oracle reference for {name} (Sec. 2 decomposition, Sec. 4.1 J/K), written by\n")
        fh.write(f"  {meta['command']}\n")
        for k in ("N", "n_rows", "tau", "n_occ", "M", "max_resid", "t_screen_s", "t_cd_s", "t_j_s", "t_k_s",
                  "omp_threads", "host_cores"):
            fh.write(f"{k}: {meta[k]}\n")
    print(f"[{name}] wrote {out}", flush=True)
    return out


def run_twostep(name: str, span: float, qmax: int, threads: int | None) -> str:
    """The two-step scheme of Sec. 3 on one workload: the first step's Cholesky
    basis (span-factor selection on the rows still >= tau, rows below tau
    dropped; ``Oracle.cd_span(reduce=True)``), then the second step's vectors
    of that basis over every row (metric Cholesky + triangular solve of
    Eq. (CVsLT); ``Oracle.cd_from_basis``), and J, K from them.  Writes
    ``<name>_twostep_oracle.npz``."""
    import oracle
    import synth
    if threads:
        os.environ["OMP_NUM_THREADS"] = str(threads)
    s = synth.make_workload(name)
    o = oracle.Oracle(s.basis)
    N = o.nbf
    rows = o.screen(s.schwarz)
    n = rows.shape[0]
    t0 = time.perf_counter()
    sp = o.cd_span(rows, s.tau, span, qmax=qmax, reduce=True, mcap=min(n, 8 * N))
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    L = o.cd_from_basis(rows, sp.piv)
    t2 = time.perf_counter() - t0
    diag = o.diag_all()[rows]
    resid = diag - np.einsum("kr,kr->r", L, L)
    J, K = oracle.jk_from_vectors(L, rows, s.C_occ)
    Dm = oracle.density(s.C_occ)
    lrows, jkrows, X = sample_indices(name, n, N)
    print(f"[{name} two-step] M={sp.M} macro={sp.macro_start.shape[0]} max resid={resid.max():.6e} "
          f"step1 {t1:.1f}s step2 {t2:.1f}s", flush=True)
    meta = {"workload": name, "scheme": "twostep", "span": span, "qmax": qmax, "N": N, "n_rows": int(n),
            "tau": s.tau, "M": sp.M, "n_macro": int(sp.macro_start.shape[0]), "max_resid": float(resid.max()),
            "t_step1_s": t1, "t_step2_s": t2,
            "command": f"python tests/golden/make_golden.py {name} --twostep"}
    out = os.path.join(HERE, f"{name}_twostep_oracle.npz")
    np.savez_compressed(
        out, meta=np.array(json.dumps(meta)), piv_packed=rows[sp.piv], max_resid=np.array(resid.max()),
        lrows=lrows, L_rows=np.ascontiguousarray(L[:, lrows]), D_rows=resid[lrows],
        jkrows=jkrows, J_rows=J[jkrows], K_rows=K[jkrows], J_diag=np.diag(J).copy(), K_diag=np.diag(K).copy(),
        trDJ=np.array(np.sum(Dm * J)), trDK=np.array(np.sum(Dm * K)),
        maxJ=np.array(np.max(np.abs(J))), maxK=np.array(np.max(np.abs(K))), X=X, JX=J @ X, KX=K @ X)
    print(f"[{name} two-step] wrote {out}", flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="+")
    ap.add_argument("--threads", type=int, default=None)
    ap.add_argument("--mcap", type=int, default=None, help="vector capacity (default 8 N)")
    ap.add_argument("--twostep", action="store_true",
                    help="the two-step scheme (span 0.01, qualified set of 64) instead of full pivoting")
    a = ap.parse_args()
    for name in a.names:
        if a.twostep:
            run_twostep(name, 0.01, 64, a.threads)
        else:
            run(name, a.threads, a.mcap)


if __name__ == "__main__":
    main()
