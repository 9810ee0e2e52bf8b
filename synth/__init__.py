"""Seeded synthetic inputs for the Cholesky-ERI hot path.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no normalisation, no integrals, no screening).  Both the
CPU oracle (``oracle/``) and the CUDA path consume its output, which is why it
lives in a module of its own.

A *system* is a basis of contracted Cartesian Gaussian shells (s, or s plus p
per center) together with an occupied-orbital block ``C_occ`` (orthonormal
columns).  Raw contraction coefficients are returned: each consumer normalises
the contracted functions itself.

Workloads (the paper has no public benchmark for this path; these synthetic
systems stand in for its molecules):

* ``s40``      -- 40 s-type functions: 40 centers uniform in an 8-bohr cube
  (minimum separation 1.5 bohr, rejection of whole centers), one s shell of 3
  primitives each, exponents log-uniform in [0.1, 10], coefficients uniform
  [0.2, 1]; tau 1e-6; n_occ 10; no Schwarz screening.
* ``lattice`` -- s+p systems: centers on a jittered cubic lattice (spacing 2.6
  bohr, jitter uniform +-0.3 bohr per coordinate), one s shell (3 primitives)
  and one Cartesian p shell (2 primitives) per center, exponents log-uniform in
  [0.15, 20], coefficients uniform [0.2, 1].  Named sizes: N=400 (5x5x4),
  N=1200 (10x10x3), N=2000 (10x10x5), plus small test lattices.
* ``batch64`` -- 64 lattice systems with center counts uniform in [15, 150]
  (first n sites of a near-cubic lattice), tau alternating 1e-4 / 1e-5,
  n_occ = N/8.

Draw order for one system (numpy PCG64, seed = 1000*config + system): center
positions (or lattice jitter), then per center: s exponents, s coefficients,
p exponents, p coefficients; then a Gaussian N x n_occ matrix whose QR factor
gives ``C_occ``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = ["Basis", "System", "make_s_cube", "make_lattice", "make_workload",
           "make_batch", "WORKLOADS"]


@dataclasses.dataclass
class Basis:
    """Shell list: one row per shell, primitives concatenated in shell order."""
    center: np.ndarray   # [n_shells, 3] float64, bohr
    l: np.ndarray        # [n_shells] int32, 0 = s, 1 = p (x, y, z)
    nprim: np.ndarray    # [n_shells] int32
    exps: np.ndarray     # [sum nprim] float64
    coefs: np.ndarray    # [sum nprim] float64, raw (consumer normalises)

    @property
    def n_shells(self) -> int:
        return int(self.l.shape[0])

    @property
    def n_basis(self) -> int:
        return int(np.sum(2 * self.l + 1))  # s -> 1, Cartesian p -> 3


@dataclasses.dataclass
class System:
    name: str
    basis: Basis
    C_occ: np.ndarray    # [N, n_occ] float64, orthonormal columns
    tau: float
    schwarz: float
    seed: int

    @property
    def n_basis(self) -> int:
        return self.basis.n_basis

    @property
    def n_occ(self) -> int:
        return int(self.C_occ.shape[1])


def _loguniform(rng: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))


def _c_occ(rng: np.random.Generator, n: int, n_occ: int) -> np.ndarray:
    g = rng.standard_normal((n, n_occ))
    q, r = np.linalg.qr(g)
    # fix the sign convention so the draw is reproducible across LAPACKs
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return np.ascontiguousarray(q * s[None, :])


def _assemble(centers: np.ndarray, shells_per_center: List[List[tuple]]) -> Basis:
    cen, ls, nps, ex, co = [], [], [], [], []
    for c, shells in zip(centers, shells_per_center):
        for (l, e, k) in shells:
            cen.append(c)
            ls.append(l)
            nps.append(len(e))
            ex.extend(e)
            co.extend(k)
    return Basis(center=np.asarray(cen, dtype=np.float64).reshape(-1, 3),
                 l=np.asarray(ls, dtype=np.int32),
                 nprim=np.asarray(nps, dtype=np.int32),
                 exps=np.asarray(ex, dtype=np.float64),
                 coefs=np.asarray(co, dtype=np.float64))


def make_s_cube(seed: int = 1000, n_centers: int = 40, box: float = 8.0,
                min_sep: float = 1.5, n_occ: int = 10, tau: float = 1e-6,
                nprim: int = 3, exp_range=(0.1, 10.0)) -> System:
    """s-only system: centers uniform in a cube with a minimum separation."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts: List[np.ndarray] = []
    while len(pts) < n_centers:
        c = rng.uniform(0.0, box, size=3)
        if all(np.linalg.norm(c - q) >= min_sep for q in pts):
            pts.append(c)
    shells = []
    for _ in range(n_centers):
        e = _loguniform(rng, exp_range[0], exp_range[1], nprim)
        k = rng.uniform(0.2, 1.0, size=nprim)
        shells.append([(0, e, k)])
    basis = _assemble(np.asarray(pts), shells)
    C = _c_occ(rng, basis.n_basis, n_occ)
    return System(f"s{n_centers}", basis, C, tau, 0.0, seed)


def _lattice_sites(dims, n_sites: Optional[int] = None) -> np.ndarray:
    nx, ny, nz = dims
    sites = [(i, j, k) for i in range(nx) for j in range(ny) for k in range(nz)]
    if n_sites is not None:
        sites = sites[:n_sites]
    return np.asarray(sites, dtype=np.float64)


def make_lattice(dims=(5, 5, 4), seed: int = 2000, spacing: float = 2.6,
                 jitter: float = 0.3, n_occ: int = 50, tau: float = 1e-5,
                 schwarz: float = 1e-12, n_sites: Optional[int] = None,
                 s_prims: int = 3, p_prims: int = 2, exp_range=(0.15, 20.0),
                 name: Optional[str] = None) -> System:
    """s+p system on a jittered cubic lattice."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sites = _lattice_sites(dims, n_sites)
    centers = sites * spacing + rng.uniform(-jitter, jitter, size=sites.shape)
    shells = []
    for _ in range(len(centers)):
        se = _loguniform(rng, exp_range[0], exp_range[1], s_prims)
        sk = rng.uniform(0.2, 1.0, size=s_prims)
        pe = _loguniform(rng, exp_range[0], exp_range[1], p_prims)
        pk = rng.uniform(0.2, 1.0, size=p_prims)
        shells.append([(0, se, sk), (1, pe, pk)])
    basis = _assemble(centers, shells)
    C = _c_occ(rng, basis.n_basis, n_occ)
    nm = name or f"lattice{dims[0]}x{dims[1]}x{dims[2]}"
    return System(nm, basis, C, tau, schwarz, seed)


def make_batch(n_sys: int = 64, config: int = 4) -> List[System]:
    """Uneven batch: center counts uniform in [15, 150], tau alternating."""
    out = []
    sizes = np.random.Generator(np.random.PCG64(1000 * config)).integers(15, 151, size=n_sys)
    for s, n in enumerate(sizes):
        n = int(n)
        side = int(math.ceil(n ** (1.0 / 3.0)))
        N = 4 * n
        out.append(make_lattice(dims=(side, side, side), seed=1000 * config + s + 1,
                                n_occ=max(1, N // 8), tau=1e-4 if s % 2 == 0 else 1e-5,
                                n_sites=n, name=f"batch{s}_n{N}"))
    return out


# Named workloads.  Config numbering follows the workload list above.
WORKLOADS = {
    # tiny test systems (not benchmark lines)
    "sp8":    lambda: make_lattice((2, 2, 2), seed=9001, n_occ=4, tau=1e-6, name="sp8"),
    "sp18":   lambda: make_lattice((3, 3, 2), seed=9002, n_occ=9, tau=1e-5, name="sp18"),
    "sp27":   lambda: make_lattice((3, 3, 3), seed=9003, n_occ=13, tau=1e-5, name="sp27"),
    # named workloads
    "s40":    lambda: make_s_cube(seed=1000),
    "sp400":  lambda: make_lattice((5, 5, 4), seed=2000, n_occ=50, tau=1e-5, name="sp400"),
    "sp1200": lambda: make_lattice((10, 10, 3), seed=3000, n_occ=150, tau=1e-5, name="sp1200"),
    "sp2000": lambda: make_lattice((10, 10, 5), seed=5000, n_occ=250, tau=1e-4, name="sp2000"),
}


def make_workload(name: str) -> System:
    return WORKLOADS[name]()
