"""C ABI checks that need no GPU: the library loads, exports every symbol
declared in include/cderi.h, and rejects malformed input on the host before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2609_00306_b300 as cd
from paper_2609_00306_b300 import cderi
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2609_00306_b300 import build
    build.build()
    return cd.load()


def test_exports_every_declared_symbol(lib):
    import glob
    declared = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        declared |= set(re.findall(r"\b(cd_[a-z0-9_]+)\s*\(", open(h).read()))
    assert declared, "no declarations parsed"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    bound = set(cderi.EXPORTS)
    try:
        from paper_2609_00306_b300 import static_jk
        bound |= set(static_jk.EXPORTS)
    except ImportError:
        pass
    assert declared == bound


def test_version(lib):
    assert "sm_103a" in cd.cd_version()


def _basis_struct(b):
    a = cderi._BasisArgs(b)
    return a


@pytest.mark.parametrize("mutate", ["nan_center", "neg_exp", "l2", "nprim0", "nan_coef", "zero_shells"])
def test_malformed_basis_is_einval(lib, mutate):
    s = synth.make_workload("sp8")
    b = synth.Basis(s.basis.center.copy(), s.basis.l.copy(), s.basis.nprim.copy(), s.basis.exps.copy(),
                    s.basis.coefs.copy())
    if mutate == "nan_center":
        b.center[3, 1] = np.nan
    elif mutate == "neg_exp":
        b.exps[5] = -0.3
    elif mutate == "l2":
        b.l[2] = 2
    elif mutate == "nprim0":
        b.nprim[0] = 0
    elif mutate == "nan_coef":
        b.coefs[1] = np.nan
    args = cderi._BasisArgs(b)
    if mutate == "zero_shells":
        args.s.n_shells = 0
    h = ctypes.c_void_p(1)
    rc = lib.cd_system_create(ctypes.byref(args.s), 0.0, None, ctypes.byref(h))
    assert rc == cderi.CD_EINVAL
    assert h.value is None
    assert len(lib.cd_last_error()) > 0


def test_bad_schwarz_is_einval(lib):
    s = synth.make_workload("sp8")
    args = cderi._BasisArgs(s.basis)
    h = ctypes.c_void_p()
    assert lib.cd_system_create(ctypes.byref(args.s), float("nan"), None, ctypes.byref(h)) == cderi.CD_EINVAL
    assert lib.cd_system_create(ctypes.byref(args.s), -1.0, None, ctypes.byref(h)) == cderi.CD_EINVAL


def test_null_arguments(lib):
    assert lib.cd_system_create(None, 0.0, None, None) == cderi.CD_EINVAL
    assert lib.cd_factor_info(None, None, None, None, None) == cderi.CD_EINVAL
    assert lib.cd_jk(None, None, 0, None, None, 0, None) == cderi.CD_EINVAL
    lib.cd_factor_free(None)
    lib.cd_system_free(None)
