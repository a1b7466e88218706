"""The C-ABI library builds for sm_103a, loads, and exports every function
include/h2ulv.h declares (no compute call: these run without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "h2ulv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(h2_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2208_10907_gb300 import build
    return build.build()


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(h2_[a-z_]+)", out))
    decl = declared_functions()
    assert decl, "no declarations parsed"
    missing = [f for f in decl if f not in exported]
    assert not missing, missing


def test_binding_loads_and_names_match(libpath):
    from paper_2208_10907_gb300 import h2ulv
    L = h2ulv.lib()
    for f in declared_functions():
        assert hasattr(L, f)
        assert f in h2ulv.EXPORTED


def test_argument_errors_need_no_gpu(libpath):
    """Invalid options are rejected before any device work."""
    import numpy as np
    from paper_2208_10907_gb300 import h2ulv as H
    X = np.zeros((10, 3))
    with pytest.raises(H.H2Error) as e:
        H.h2_construct(X, 10, H.make_kernel(), H.make_options(leaf=0))
    assert e.value.status == H.H2_ERR_ARG
    with pytest.raises(H.H2Error) as e:
        H.h2_construct(X, 10, H.make_kernel(), H.make_options(max_rank=257))
    assert e.value.status == H.H2_ERR_ARG
    Xn = np.full((10, 3), np.nan)
    with pytest.raises(H.H2Error) as e:
        H.h2_construct(Xn, 10, H.make_kernel(), H.make_options())
    assert e.value.status == H.H2_ERR_NONFINITE
