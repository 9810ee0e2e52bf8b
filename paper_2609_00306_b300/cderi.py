"""Thin ctypes binding of libcderi.so (include/cderi.h).

Argument marshalling only: every step of the decomposition and of J/K runs in
the library's CUDA kernels.  PyTorch supplies device buffers and the current
stream.  There is no CPU fallback: if the shared library is missing or no GPU
is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcderi.so")

CD_OK, CD_EINVAL, CD_ENOMEM, CD_ENOTPSD, CD_ETIMEOUT, CD_ECUDA = 0, -1, -2, -3, -4, -5
CD_FP64, CD_VEC_FP32 = 0, 1
CD_JK_FP64, CD_JK_BF16X3, CD_JK_BF16X4, CD_JK_BF16X5 = 0, 1, 2, 3
CD_JK_DEVICE, CD_JK_ONLY_J, CD_JK_ONLY_K, CD_JK_VEC_FP32 = 0x100, 0x200, 0x400, 0x800
CD_MAX_PRIM = 16
CD_UPDATE_SLICE, CD_UPDATE_FP64 = 0, 1
CD_ALG_FULL, CD_ALG_SPAN, CD_ALG_TWOSTEP = 0, 1, 2

_ERRNAMES = {CD_EINVAL: "CD_EINVAL", CD_ENOMEM: "CD_ENOMEM", CD_ENOTPSD: "CD_ENOTPSD",
             CD_ETIMEOUT: "CD_ETIMEOUT", CD_ECUDA: "CD_ECUDA"}

# every symbol declared in include/cderi.h
EXPORTS = ["cd_system_create", "cd_system_free", "cd_system_info", "cd_system_rows", "cd_eri_columns",
           "cd_eri_factor", "cd_eri_factor_sys", "cd_factor_free", "cd_factor_info", "cd_factor_pivots",
           "cd_factor_vectors", "cd_factor_pivot_diag", "cd_factor_memory", "cd_factor_eri_work", "cd_factor_gather", "cd_factor_stats", "cd_kernel_launches", "cd_jk", "cd_mo_vectors", "cd_batch_run", "cd_batch_persistent", "cd_slice_matmul", "cd_set_wait_limit", "cd_last_error", "cd_version"]


class CDError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


class cd_basis_t(ctypes.Structure):
    _fields_ = [("n_shells", ctypes.c_int32), ("center", ctypes.c_void_p), ("l", ctypes.c_void_p),
                ("nprim", ctypes.c_void_p), ("exps", ctypes.c_void_p), ("coefs", ctypes.c_void_p)]


class cd_opts_t(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double), ("schwarz", ctypes.c_double), ("vec_precision", ctypes.c_int32),
                ("block", ctypes.c_int32), ("max_vectors", ctypes.c_int64), ("mem_budget_gb", ctypes.c_double),
                ("forced_pivots", ctypes.c_void_p), ("n_forced", ctypes.c_int64),
                ("update", ctypes.c_int32), ("algorithm", ctypes.c_int32), ("span", ctypes.c_double),
                ("candidates", ctypes.c_void_p), ("diag_shift", ctypes.c_double)]


_lib = None


def load(path: Optional[str] = None):
    """Load libcderi.so (built by paper_2609_00306_b300/build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with `python -m paper_2609_00306_b300.build`")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "cd_system_create": (ctypes.c_int, [P, D, P, P]),
        "cd_system_free": (None, [P]),
        "cd_system_info": (ctypes.c_int, [P, P, P, P]),
        "cd_system_rows": (ctypes.c_int, [P, P, P]),
        "cd_eri_columns": (ctypes.c_int, [P, P, I32, P, I64, P]),
        "cd_eri_factor": (ctypes.c_int, [P, P, P, P]),
        "cd_eri_factor_sys": (ctypes.c_int, [P, P, P, P]),
        "cd_factor_free": (None, [P]),
        "cd_factor_info": (ctypes.c_int, [P, P, P, P, P]),
        "cd_factor_pivots": (ctypes.c_int, [P, P, P, P, P]),
        "cd_factor_vectors": (ctypes.c_int, [P, P, P, P, P]),
        "cd_factor_pivot_diag": (ctypes.c_int, [P, P]),
        "cd_factor_memory": (ctypes.c_int, [P, P, P]),
        "cd_factor_eri_work": (ctypes.c_int, [P, P, P]),
        "cd_set_wait_limit": (ctypes.c_int, [D, P]),
        "cd_factor_stats": (ctypes.c_int, [P, P]),
        "cd_factor_gather": (ctypes.c_int, [P, P, I32, P]),
        "cd_jk": (ctypes.c_int, [P, P, I32, P, P, I32, P]),
        "cd_mo_vectors": (ctypes.c_int, [P, P, I32, I64, I64, I32, P, I32, P]),
        "cd_kernel_launches": (ctypes.c_longlong, []),
        "cd_batch_run": (ctypes.c_int, [I32, P, P, P, P, P, P, I32, I32, P]),
        "cd_batch_persistent": (ctypes.c_int, [I32, P, P, P, P, P, P, P, P, P]),
        "cd_slice_matmul": (ctypes.c_int, [P, I64, I64, P, I64, I64, I64, I32, P, I64, P]),
        "cd_last_error": (ctypes.c_char_p, []),
        "cd_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int):
    if rc != CD_OK:
        raise CDError(rc, load().cd_last_error().decode())


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class _BasisArgs:
    """Keeps the numpy arrays of a cd_basis_t alive."""

    def __init__(self, basis):
        self.center = np.ascontiguousarray(basis.center, dtype=np.float64)
        self.l = np.ascontiguousarray(basis.l, dtype=np.int32)
        self.nprim = np.ascontiguousarray(basis.nprim, dtype=np.int32)
        self.exps = np.ascontiguousarray(basis.exps, dtype=np.float64)
        self.coefs = np.ascontiguousarray(basis.coefs, dtype=np.float64)
        self.s = cd_basis_t(int(self.l.shape[0]), self.center.ctypes.data, self.l.ctypes.data,
                            self.nprim.ctypes.data, self.exps.ctypes.data, self.coefs.ctypes.data)


def make_opts(tau: float, schwarz: float = 0.0, vec_precision: int = CD_FP64, block: int = 0,
              max_vectors: int = 0, mem_budget_gb: float = 0.0, forced: Optional[Sequence[int]] = None,
              update: int = CD_UPDATE_SLICE, algorithm: int = CD_ALG_FULL, span: float = 0.0,
              candidates=None, diag_shift: float = 0.0):
    o = cd_opts_t(float(tau), float(schwarz), int(vec_precision), int(block), int(max_vectors),
                  float(mem_budget_gb), None, 0, int(update), int(algorithm), float(span), None,
                  float(diag_shift))
    keep = []
    if forced is not None:
        f = np.ascontiguousarray(forced, dtype=np.int64)
        o.forced_pivots = f.ctypes.data
        o.n_forced = int(f.shape[0])
        keep.append(f)
    if candidates is not None:
        c = np.ascontiguousarray(candidates, dtype=np.uint8)
        o.candidates = c.ctypes.data
        keep.append(c)
    return o, keep


class System:
    """cd_system_t: normalised basis and Schwarz-screened pair rows on the GPU."""

    def __init__(self, basis, schwarz: float = 0.0, stream=None):
        lib = load()
        self._args = _BasisArgs(basis)
        h = ctypes.c_void_p()
        _check(lib.cd_system_create(ctypes.byref(self._args.s), float(schwarz), _stream(stream), ctypes.byref(h)))
        self._h = h
        nb, nr, nsp = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.cd_system_info(h, ctypes.byref(nb), ctypes.byref(nr), ctypes.byref(nsp)))
        self.n_basis, self.n_rows, self.n_shell_pairs = nb.value, nr.value, nsp.value

    def rows(self):
        packed = np.zeros(self.n_rows, dtype=np.int64)
        diag = np.zeros(self.n_rows)
        _check(load().cd_system_rows(self._h, _p(packed), _p(diag)))
        return packed, diag

    def eri_columns(self, cols, out=None, stream=None):
        """out[j, r] = (row r | row cols[j]) as a torch float64 CUDA tensor."""
        import torch
        cols = np.ascontiguousarray(cols, dtype=np.int64)
        if out is None:
            out = torch.zeros((cols.shape[0], self.n_rows), dtype=torch.float64, device="cuda")
        assert out.dtype == torch.float64 and out.is_cuda and out.is_contiguous()
        _check(load().cd_eri_columns(self._h, _p(cols), int(cols.shape[0]), ctypes.c_void_p(out.data_ptr()),
                                     int(out.shape[1]), _stream(stream)))
        return out

    def free(self):
        if getattr(self, "_h", None):
            load().cd_system_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Factor:
    """cd_factor_t: pivots and Cholesky vectors on the GPU."""

    def __init__(self, h, system: Optional[System] = None):
        self._h = h
        self._system = system  # keep alive
        lib = load()
        M, nr, nb, res = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        _check(lib.cd_factor_info(h, ctypes.byref(M), ctypes.byref(nr), ctypes.byref(nb), ctypes.byref(res)))
        self.M, self.n_rows, self.n_basis, self.max_resid = M.value, nr.value, nb.value, res.value

    def pivots(self):
        rows = np.zeros(self.M, dtype=np.int64)
        packed = np.zeros(self.M, dtype=np.int64)
        gaps = np.zeros(self.M)
        resid = np.zeros(self.n_rows)
        _check(load().cd_factor_pivots(self._h, _p(rows), _p(packed), _p(gaps), _p(resid)))
        return rows, packed, gaps, resid

    def pivot_diag(self) -> np.ndarray:
        """Tracked residual diagonal of each pivot when it was taken [M]."""
        out = np.zeros(self.M)
        _check(load().cd_factor_pivot_diag(self._h, _p(out)))
        return out

    def eri_work(self) -> dict:
        """Primitive quartets of the ERI column kernels and their algorithmic FP64 operations."""
        q, a = ctypes.c_double(), ctypes.c_double()
        _check(load().cd_factor_eri_work(self._h, ctypes.byref(q), ctypes.byref(a)))
        return {"quartets": q.value, "algorithmic_ops": a.value}

    def memory(self) -> dict:
        """Device bytes at the decomposition's peak and kept by the factor."""
        pk, rs = ctypes.c_double(), ctypes.c_double()
        _check(load().cd_factor_memory(self._h, ctypes.byref(pk), ctypes.byref(rs)))
        return {"peak_bytes": pk.value, "resident_bytes": rs.value}

    def vectors_host(self) -> np.ndarray:
        L = np.zeros((self.M, self.n_rows))
        _check(load().cd_factor_vectors(self._h, _p(L), None, None, None))
        return L

    def gather(self, rows) -> np.ndarray:
        """[M, len(rows)] FP64 entries of every vector on the given rows."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((self.M, rows.shape[0]))
        _check(load().cd_factor_gather(self._h, _p(rows), int(rows.shape[0]), _p(out)))
        return out

    def vectors_device(self):
        ptr, ld, dt = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int32()
        _check(load().cd_factor_vectors(self._h, None, ctypes.byref(ptr), ctypes.byref(ld), ctypes.byref(dt)))
        return ptr.value, ld.value, dt.value

    def stats(self) -> dict:
        s = np.zeros(16)
        _check(load().cd_factor_stats(self._h, _p(s)))
        keys = ["ms_system", "ms_eri", "ms_colupd", "ms_steps", "ms_select", "ms_total", "blocks", "eri_columns",
                "colupd_flops", "eri_entries", "M", "sliced", "eri_fp64_ops", "step1_ms", "step1_blocks",
                "step1_eri_columns"]
        return dict(zip(keys, s.tolist()))

    def jk(self, C_occ, mode: int = CD_JK_FP64, stream=None, want=("J", "K")):
        """J, K as numpy arrays (host path: copies inside the call)."""
        C = np.ascontiguousarray(C_occ, dtype=np.float64)
        N = self.n_basis
        J = np.zeros((N, N)) if "J" in want else None
        K = np.zeros((N, N)) if "K" in want else None
        flags = mode
        if J is None:
            flags |= CD_JK_ONLY_K
        if K is None:
            flags |= CD_JK_ONLY_J
        _check(load().cd_jk(self._h, _p(C), int(C.shape[1]), _p(J) if J is not None else None,
                            _p(K) if K is not None else None, int(flags), _stream(stream)))
        return J, K

    def mo_vectors(self, C, P0: int = 0, nP: Optional[int] = None, slices: int = 7, stream=None) -> np.ndarray:
        """[nP, n_mo, n_mo] Cholesky vectors in the MO basis C [N, n_mo] (C ABI cd_mo_vectors)."""
        C = np.ascontiguousarray(C, dtype=np.float64)
        nP = self.M - P0 if nP is None else int(nP)
        out = np.zeros((max(nP, 0), C.shape[1], C.shape[1]))
        _check(load().cd_mo_vectors(self._h, _p(C), int(C.shape[1]), int(P0), int(nP), int(slices), _p(out), 0,
                                    _stream(stream)))
        return out

    def mo_vectors_device(self, C_dev, out_dev, P0: int = 0, slices: int = 7, stream=None):
        """Same, with torch CUDA tensors C [N, n_mo] and out [nP, n_mo, n_mo] (float64)."""
        assert C_dev.is_cuda and out_dev.is_cuda and C_dev.dtype == out_dev.dtype
        n_mo = C_dev.shape[1]
        _check(load().cd_mo_vectors(self._h, ctypes.c_void_p(C_dev.data_ptr()), int(n_mo), int(P0),
                                    int(out_dev.shape[0]), int(slices), ctypes.c_void_p(out_dev.data_ptr()),
                                    CD_JK_DEVICE, _stream(stream)))

    def jk_device(self, C_dev, J_dev, K_dev, mode: int = CD_JK_FP64, stream=None):
        """J, K into torch CUDA tensors (no host copies)."""
        flags = mode | CD_JK_DEVICE
        if J_dev is None:
            flags |= CD_JK_ONLY_K
        if K_dev is None:
            flags |= CD_JK_ONLY_J
        _check(load().cd_jk(self._h, ctypes.c_void_p(C_dev.data_ptr()), int(C_dev.shape[1]),
                            ctypes.c_void_p(J_dev.data_ptr()) if J_dev is not None else None,
                            ctypes.c_void_p(K_dev.data_ptr()) if K_dev is not None else None,
                            int(flags), _stream(stream)))

    def free(self):
        if getattr(self, "_h", None):
            load().cd_factor_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def cd_eri_factor(basis, tau: float, schwarz: float = 0.0, vec_precision: int = CD_FP64, block: int = 0,
                  max_vectors: int = 0, mem_budget_gb: float = 0.0, forced=None, stream=None,
                  update: int = CD_UPDATE_SLICE, algorithm: int = CD_ALG_FULL, span: float = 0.0,
                  candidates=None, diag_shift: float = 0.0) -> Factor:
    """Full pipeline from a host basis (C ABI cd_eri_factor).  ``candidates``: mask
    over the screened rows (``System.rows()`` order) of the rows that may be pivots.
    ``diag_shift``: test hook (lowers every starting diagonal; see cd_opts_t)."""
    args = _BasisArgs(basis)
    o, keep = make_opts(tau, schwarz, vec_precision, block, max_vectors, mem_budget_gb, forced, update,
                        algorithm, span, candidates, diag_shift)
    h = ctypes.c_void_p()
    _check(load().cd_eri_factor(ctypes.byref(args.s), ctypes.byref(o), _stream(stream), ctypes.byref(h)))
    del keep
    return Factor(h)


def cd_eri_factor_sys(system: System, tau: float, vec_precision: int = CD_FP64, block: int = 0,
                      max_vectors: int = 0, mem_budget_gb: float = 0.0, forced=None, stream=None,
                      update: int = CD_UPDATE_SLICE, algorithm: int = CD_ALG_FULL, span: float = 0.0,
                      candidates=None) -> Factor:
    if candidates is not None and len(candidates) != system.n_rows:
        raise ValueError("candidates must have one entry per screened row")
    o, keep = make_opts(tau, 0.0, vec_precision, block, max_vectors, mem_budget_gb, forced, update, algorithm,
                        span, candidates)
    h = ctypes.c_void_p()
    _check(load().cd_eri_factor_sys(system._h, ctypes.byref(o), _stream(stream), ctypes.byref(h)))
    del keep
    return Factor(h, system)


def slice_matmul(X, Y, slices: int = 7, stream=None):
    """out = X @ Y.T for float64 CUDA tensors via the exact-slice tensor-core GEMM."""
    import torch
    assert X.dtype == torch.float64 and Y.dtype == torch.float64 and X.is_cuda and Y.is_cuda
    X = X.contiguous()
    Y = Y.contiguous()
    m, k = X.shape
    n, k2 = Y.shape
    assert k == k2
    out = torch.empty((m, n), dtype=torch.float64, device=X.device)
    _check(load().cd_slice_matmul(ctypes.c_void_p(X.data_ptr()), k, m, ctypes.c_void_p(Y.data_ptr()), k, n, k,
                                  int(slices), ctypes.c_void_p(out.data_ptr()), n, _stream(stream)))
    return out


def batch_run(systems, jk_mode: int = CD_JK_FP64, workers: int = 0, blocks=None, update: int = CD_UPDATE_SLICE,
              vec_precision: Optional[int] = None, stream=None):
    """Decompose and contract many independent systems (C ABI cd_batch_run).

    systems: sequence of synth.System-like objects (basis, C_occ, tau, schwarz).
    blocks: per-system speculative block size (e.g. from the autotuner), or None.
    Returns lists J, K of numpy arrays.
    """
    n = len(systems)
    if vec_precision is None:
        vec_precision = CD_FP64
    bargs = [_BasisArgs(s.basis) for s in systems]
    BasisArr = cd_basis_t * n
    OptsArr = cd_opts_t * n
    bases = BasisArr(*[b.s for b in bargs])
    opts = OptsArr(*[make_opts(s.tau, s.schwarz, vec_precision, int(blocks[i]) if blocks is not None else 0,
                               update=update)[0] for i, s in enumerate(systems)])
    Cs = [np.ascontiguousarray(s.C_occ, dtype=np.float64) for s in systems]
    Js = [np.zeros((c.shape[0], c.shape[0])) for c in Cs]
    Ks = [np.zeros((c.shape[0], c.shape[0])) for c in Cs]
    PArr = ctypes.c_void_p * n
    occ = np.array([c.shape[1] for c in Cs], dtype=np.int32)
    _check(load().cd_batch_run(n, ctypes.byref(bases), ctypes.byref(opts),
                               PArr(*[c.ctypes.data for c in Cs]), _p(occ),
                               PArr(*[j.ctypes.data for j in Js]), PArr(*[k.ctypes.data for k in Ks]),
                               int(jk_mode), int(workers), _stream(stream)))
    return Js, Ks


def batch_persistent(systems, blocks=None, max_vectors=None, mem_budget_gb: float = 0.0,
                     update: int = CD_UPDATE_SLICE, stream=None):
    """Decompose and contract many independent systems in FP64 with one
    persistent kernel launch recorded in a CUDA graph (C ABI cd_batch_persistent).

    systems: sequence of synth.System-like objects (basis, C_occ, tau, schwarz).
    blocks: per-system block size b <= 64 (e.g. from the autotuner), or None (64).
    max_vectors: per-system vector capacity, or None (8 N).
    update: CD_UPDATE_SLICE (exact 7-slice products on the tensor cores) or CD_UPDATE_FP64 (DFMA).
    Returns lists J, K of numpy arrays, the vector counts M and a dict of timings.
    """
    n = len(systems)
    bargs = [_BasisArgs(s.basis) for s in systems]
    bases = (cd_basis_t * n)(*[b.s for b in bargs])
    opts = (cd_opts_t * n)(*[make_opts(s.tau, s.schwarz, CD_FP64, int(blocks[i]) if blocks is not None else 0,
                                       int(max_vectors[i]) if max_vectors is not None else 0,
                                       float(mem_budget_gb) if i == 0 else 0.0, update=update)[0]
                             for i, s in enumerate(systems)])
    Cs = [np.ascontiguousarray(s.C_occ, dtype=np.float64) for s in systems]
    Js = [np.zeros((c.shape[0], c.shape[0])) for c in Cs]
    Ks = [np.zeros((c.shape[0], c.shape[0])) for c in Cs]
    PArr = ctypes.c_void_p * n
    occ = np.array([c.shape[1] for c in Cs], dtype=np.int32)
    M = np.zeros(n, dtype=np.int64)
    stats = np.zeros(40)
    _check(load().cd_batch_persistent(n, ctypes.byref(bases), ctypes.byref(opts),
                                      PArr(*[c.ctypes.data for c in Cs]), _p(occ),
                                      PArr(*[j.ctypes.data for j in Js]), PArr(*[k.ctypes.data for k in Ks]),
                                      _p(M), _p(stats), _stream(stream)))
    info = {"setup_ms": float(stats[0]), "upload_ms": float(stats[1]), "launch_device_ms": float(stats[2]),
            "launch_host_ms": float(stats[3]), "ctas": int(stats[4]), "bytes": float(stats[5]),
            "cta_s": {name: float(stats[6 + k]) for k, name in
                      [(1, "select"), (2, "gather"), (3, "update"), (4, "step"), (5, "density"), (6, "v"),
                       (7, "jp"), (8, "j_unpack"), (9, "slice"), (10, "eri"), (13, "b"), (14, "k_tiles"),
                       (15, "k_sum")]},
            "idle_cta_s": float(stats[22]), "waves": int(stats[39]),
            "fp64_ops": {name: float(stats[23 + k]) for k, name in
                         [(3, "update"), (4, "step"), (6, "v"), (7, "jp"), (10, "eri"), (13, "b"),
                          (14, "k_tiles")]}}
    return Js, Ks, [int(m) for m in M], info


def set_wait_limit(seconds: float) -> float:
    """Wall-clock limit of the bounded device waits (C ABI cd_set_wait_limit);
    returns the previous limit in seconds."""
    prev = ctypes.c_double()
    _check(load().cd_set_wait_limit(float(seconds), ctypes.byref(prev)))
    return prev.value


def kernel_launches() -> int:
    """Kernel launches issued by libcderi in this process."""
    return int(load().cd_kernel_launches())


def cd_version() -> str:
    return load().cd_version().decode()
