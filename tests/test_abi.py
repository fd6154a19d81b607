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
        for m in re.finditer(r"^\s*(?:const\s+)?(?:long\s+long|[A-Za-z_][A-Za-z0-9_]*)\s*\*?\s*(relu_qp_[a-z0-9_]+)\s*\(",
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


def header_struct_fields(name):
    """Field names, in order, of `typedef struct name { ... } name;` in include/relu_qp.h."""
    text = open(os.path.join(ROOT, "include", "relu_qp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct " + name + r"\s*\{(.*?)\}\s*" + name + ";", text, flags=re.S).group(1)
    return [m.group(1) for m in re.finditer(r"([A-Za-z_][A-Za-z0-9_]*)\s*;", body)]


def test_binding_structs_mirror_the_header(libpath):
    import paper_2311_18056_gb300 as rq
    for cname, pyt in (("relu_qp_opts", rq.Opts), ("relu_qp_info", rq.Info)):
        assert header_struct_fields(cname) == [f for f, _ in pyt._fields_], cname


def test_default_opts_without_gpu(libpath):
    """relu_qp_default_opts makes no CUDA call: the defaults of every field, the new ones included."""
    import paper_2311_18056_gb300 as rq
    o = rq.Opts()
    rq.lib().relu_qp_default_opts(ctypes.byref(o))
    assert (o.check_interval, o.adaptive_rho, o.rho0, o.eq_scale) == (25, 1, 0.1, 1e3)
    assert (o.keep_fp64, o.max_batch, o.batch_precision) == (0, 0, rq.PREC_FP32)
    assert o.scaling_iters == 0 and o.single_precision == rq.PREC_FP32


def test_new_options_are_validated_without_gpu(libpath):
    import numpy as np
    import paper_2311_18056_gb300 as rq
    P, A, l, u = np.eye(2), np.eye(2), -np.ones(2), np.ones(2)
    for kw in ({"scaling_iters": -1}, {"scaling_iters": 101}, {"single_precision": 5}):
        with pytest.raises(rq.ReluQPError) as e:
            rq.ReluQP(P, A, l, u, **kw)
        assert e.value.kind == "INVALID", kw
    # condensing: limits and sizes are checked before any GPU work
    with pytest.raises(rq.ReluQPError) as e:
        rq.condense_mpc(np.eye(2), np.ones((2, 1)), np.eye(2), np.eye(1), 5, umin=[1.0], umax=[-1.0])
    assert e.value.kind == "INVALID"
    with pytest.raises(rq.ReluQPError) as e:
        rq.condense_mpc(np.eye(2), np.ones((2, 1)), np.eye(2), np.eye(1), 0)
    assert e.value.kind == "INVALID"
    with pytest.raises(rq.ReluQPError) as e:
        rq.condense_mpc(np.array([[np.inf, 0], [0, 1]]), np.ones((2, 1)), np.eye(2), np.eye(1), 3)
    assert e.value.kind == "INVALID"


def test_product_path_fails_loudly_without_the_library(monkeypatch, tmp_path):
    """No CPU fallback: without librelu_qp.so every entry point raises before any work."""
    import numpy as np
    import paper_2311_18056_gb300 as rq
    monkeypatch.setattr(rq, "library_path", str(tmp_path / "librelu_qp.so"))
    monkeypatch.setattr(rq, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        rq.ReluQP(np.eye(2), np.eye(2), -np.ones(2), np.ones(2))
    with pytest.raises(RuntimeError, match="missing"):
        rq.condense_mpc(np.eye(2), np.ones((2, 1)), np.eye(2), np.eye(1), 3)


def test_product_path_does_not_import_the_oracle():
    """The binding, the package and the workload generators load without `oracle`."""
    import subprocess
    import sys
    code = ("import sys, paper_2311_18056_gb300, paper_2311_18056_gb300.build, workloads.mpc, "
            "workloads.random_qp; assert not any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules)")
    subprocess.run([sys.executable, "-c", code], cwd=ROOT, check=True)


def test_device_budget_is_validated_without_gpu(libpath):
    import numpy as np
    import paper_2311_18056_gb300 as rq
    o = rq.Opts()
    rq.lib().relu_qp_default_opts(ctypes.byref(o))
    assert o.device_budget == 0
    with pytest.raises(rq.ReluQPError) as e:
        rq.ReluQP(np.eye(2), np.eye(2), -np.ones(2), np.ones(2), device_budget=-1)
    assert e.value.kind == "INVALID"


def test_grid_barrier_logic_on_host_threads(libpath):
    """The grid barrier's arrival/wait template, run by host threads: with the
    right arrival count every round passes; with one arrival missing every
    thread gives up at its deadline (about 2 ms) and reports it, instead of
    waiting forever."""
    import paper_2311_18056_gb300 as rq
    L = rq.lib()
    n_to, ms = ctypes.c_int(-1), ctypes.c_double(0.0)
    assert L.relu_qp_diag_host_barrier(8, 0, 2000, 2_000_000_000, ctypes.byref(n_to), ctypes.byref(ms)) == 0
    assert n_to.value == 0
    assert L.relu_qp_diag_host_barrier(6, 1, 5, 2_000_000, ctypes.byref(n_to), ctypes.byref(ms)) == 0
    assert n_to.value == 6
    assert 1.5 <= ms.value < 2000.0
    # arguments are checked
    assert L.relu_qp_diag_host_barrier(0, 0, 1, 2_000_000, ctypes.byref(n_to), None) == -1


def test_single_launch_shape_calls_check_their_handle(libpath):
    """relu_qp_single_config / relu_qp_single_set_config refuse a NULL handle
    with INVALID (no GPU needed), and the device-wait diagnostics refuse kinds
    outside 0..5 before touching the device."""
    import paper_2311_18056_gb300 as rq
    L = rq.lib()
    c, k, r = ctypes.c_int(-7), ctypes.c_int(-7), ctypes.c_int(-7)
    assert L.relu_qp_single_config(None, ctypes.byref(c), ctypes.byref(k), ctypes.byref(r)) == -1
    assert (c.value, k.value, r.value) == (-7, -7, -7)
    assert L.relu_qp_single_set_config(None, 8, 8) == -1
    st, ms = ctypes.c_int(0), ctypes.c_double(0.0)
    assert L.relu_qp_diag_device_wait(6, 1_000_000, ctypes.byref(st), ctypes.byref(ms)) == -1
    assert L.relu_qp_diag_device_wait(-1, 1_000_000, ctypes.byref(st), ctypes.byref(ms)) == -1
