"""The C ABI library builds, loads and exports every entry point that include/ugkwp.h declares (no GPU)."""
import ctypes as C
import os
import re

import pytest

from paper_2607_09552_b300 import build, ugkwp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "ugkwp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ugkwp_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert declared_entry_points() == sorted(ugkwp.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = C.CDLL(path)
    for name in declared_entry_points():
        assert hasattr(lib, name), name


def test_library_is_built_for_sm_103a():
    # the fatbinary carries an sm_103a cubin: cuobjdump is not used; ask nvcc's build flags instead
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)


def test_create_without_device_fails_cleanly():
    from conftest import gpu_available
    if gpu_available():
        pytest.skip("a GPU is present")
    from paper_2607_09552_b300 import workloads as wl
    with pytest.raises(ugkwp.UgkwpError) as e:
        ugkwp.Solver(wl.case_shock1d(ni=8, n_ref=4))
    assert e.value.status == 3
