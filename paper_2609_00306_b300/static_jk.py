"""Binding of cd_jk_coulomb_static (include/cderi_static.h): the Coulomb
matrix for callers that cannot allocate device memory.  Its scratch is a
static device array of the library; the caller passes device buffers."""
from __future__ import annotations

import ctypes

from .cderi import _check, _stream, load

EXPORTS = ["cd_jk_coulomb_static"]


def coulomb_static(factor, C_dev, J_dev, stream=None) -> None:
    """J = sum_P L^P tr(L^P D), D = 2 C C^T, into the torch CUDA tensor J_dev."""
    lib = load()
    fn = lib.cd_jk_coulomb_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    _check(fn(factor._h, ctypes.c_void_p(C_dev.data_ptr()), int(C_dev.shape[1]),
              ctypes.c_void_p(J_dev.data_ptr()), _stream(stream)))
