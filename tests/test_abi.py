"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function declared in include/*.h (no compute call is made here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(relu_qp_[a-z0-9_]+)\s*\(",
                             text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2311_18056_gb300 import build
    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for core in ("relu_qp_setup", "relu_qp_update", "relu_qp_solve", "relu_qp_destroy",
                 "relu_qp_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    import paper_2311_18056_gb300 as rq
    assert set(rq.EXPORTED_SYMBOLS) == declared_functions()
    rq.lib()  # loads and sets argtypes without touching the GPU


def test_setup_error_reporting_without_gpu(libpath):
    """Argument validation happens before any CUDA call, so it works on a CPU machine."""
    import numpy as np
    import paper_2311_18056_gb300 as rq
    with pytest.raises(rq.ReluQPError) as e:
        rq.ReluQP(np.eye(2), np.eye(2), [1.0, 0.0], [0.0, 1.0])   # l > u in row 0
    assert e.value.kind == "INVALID"
    with pytest.raises(rq.ReluQPError) as e:
        rq.ReluQP(np.array([[np.nan]]), None, None, None)
    assert e.value.kind == "INVALID"
