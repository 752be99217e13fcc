"""C-ABI checks that need no GPU: the library builds, loads, exports every
symbol include/bldtt.h declares, and validates arguments before any device
work."""
import ctypes
import os
import re

import pytest

import __graft_entry__
from paper_2012_06925_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bldtt.h")


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return B.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bldtt_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("bldtt_setup", "bldtt_compute", "bldtt_set_charges", "bldtt_stats",
                     "bldtt_destroy", "bldtt_status_string"):
        assert required in names
    assert set(names) == set(B.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_stats_struct_size_matches_header(lib, tmp_path):
    """The binding's Stats layout has the size and field offsets that a C
    compiler gives bldtt_stats_t from include/bldtt.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [name for name, _ in B.Stats._fields_]
    src = tmp_path / "sz.c"
    src.write_text('#include <stddef.h>\n#include <stdio.h>\n#include "bldtt.h"\nint main(void){'
                   'printf("%zu", sizeof(bldtt_stats_t));'
                   + "".join(f'printf(" %zu", offsetof(bldtt_stats_t, {f}));' for f in fields)
                   + 'return 0;}\n')
    exe = tmp_path / "sz"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    subprocess.run([cc, f"-I{inc}", str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(B.Stats)
    assert got[1:] == [getattr(B.Stats, f).offset for f in fields]


def test_status_strings(lib):
    assert B.status_string(0) == "BLDTT_OK"
    assert B.status_string(1) == "BLDTT_EINVAL"
    assert B.status_string(4) == "BLDTT_ETIMEOUT"
    assert B.status_string(12345) == "BLDTT_UNKNOWN_STATUS"


def test_wait_probe_rejects_limits_out_of_range(lib):
    # validated before any CUDA call (null stream: no device needed)
    assert lib.bldtt_wait_probe(999, None) == 1
    assert lib.bldtt_wait_probe(1_000_000_001, None) == 1
    assert "limit_ns" in lib.bldtt_last_error().decode()


DUMMY = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
GOOD = dict(kernel=0, kappa=0.0, n=4, theta=0.7, N0=10, M0=10, precision=1)


@pytest.mark.parametrize("change", [
    dict(n=0), dict(n=17), dict(theta=-0.1), dict(theta=float("nan")), dict(N0=0), dict(M0=0),
    dict(kernel=5), dict(kernel=1, kappa=-1.0), dict(kernel=1, kappa=float("inf")),
    dict(precision=2), dict(M=0), dict(N=0), dict(M=2 ** 31),
])
def test_setup_rejects_invalid_arguments(lib, change):
    args = dict(GOOD, M=100, N=100)
    args.update(change)
    st = B.setup_status(DUMMY, args["M"], DUMMY, args["N"], DUMMY, args["kernel"], args["kappa"],
                        args["n"], args["theta"], args["N0"], args["M0"], args["precision"])
    assert st == 1
    assert lib.bldtt_last_error().decode() != ""


def test_setup_rejects_null_pointers(lib):
    st = B.setup_status(None, 10, DUMMY, 10, DUMMY, 0, 0.0, 4, 0.7, 5, 5, 1)
    assert st == 1
    h = ctypes.c_void_p()
    assert lib.bldtt_setup(None, DUMMY, 10, DUMMY, 10, DUMMY, 0, 0.0, 4, 0.7, 5, 5, 1, None) == 1
    assert lib.bldtt_compute(None, None, None) == 1
    assert lib.bldtt_stats(None, None) == 1
    lib.bldtt_destroy(None)
    assert not h


def test_direct_sum_rejects_bad_arguments(lib):
    assert lib.bldtt_direct_sum(None, 1, DUMMY, 1, DUMMY, 0, 0.0, DUMMY, None) == 1
    assert lib.bldtt_direct_sum(DUMMY, 1, DUMMY, 1, DUMMY, 7, 0.0, DUMMY, None) == 1


def test_setup_ex_rejects_bad_variant_and_params(lib):
    h = ctypes.c_void_p()
    prm = B.Params(0, 0.0, 4, 0.7, 10, 10, 1, 7)          # unknown variant
    assert lib.bldtt_setup_ex(ctypes.byref(h), DUMMY, 100, DUMMY, 100, DUMMY, ctypes.byref(prm),
                              None) == 1
    assert lib.bldtt_setup_ex(ctypes.byref(h), DUMMY, 100, DUMMY, 100, DUMMY, None, None) == 1
    for kernel in (2, 3):                                  # parameter of the Sec. 4.6 kernels
        prm = B.Params(kernel, -0.5, 4, 0.7, 10, 10, 1, 0)
        assert lib.bldtt_setup_ex(ctypes.byref(h), DUMMY, 100, DUMMY, 100, DUMMY,
                                  ctypes.byref(prm), None) == 1
    assert not h


def test_setup_batch_rejects_bad_batches(lib):
    h = ctypes.c_void_p()
    prm = B.Params(0, 0.0, 4, 0.7, 10, 10, 1, 0)
    I64 = ctypes.c_int64 * 3
    ks = (ctypes.c_int * 2)(0, 1)
    kp = (ctypes.c_double * 2)(0.0, 0.5)
    def call(nprob, to, so, kernels=ks, kappas=kp):
        return lib.bldtt_setup_batch(ctypes.byref(h), nprob, DUMMY, to, DUMMY, so, DUMMY,
                                     kernels, kappas, ctypes.byref(prm), None)
    assert call(0, I64(0, 5, 9), I64(0, 5, 9)) == 1                    # no problems
    assert call(2, I64(1, 5, 9), I64(0, 5, 9)) == 1                    # offsets not from 0
    assert call(2, I64(0, 5, 5), I64(0, 5, 9)) == 1                    # empty problem
    assert call(2, I64(0, 5, 9), I64(0, 5, 9), kernels=(ctypes.c_int * 2)(0, 7)) == 1
    assert call(2, I64(0, 5, 9), I64(0, 5, 9), kappas=(ctypes.c_double * 2)(0.0, -1.0)) == 1
    assert not h


def test_setup_learned_rejects_bad_selectors(lib):
    h = ctypes.c_void_p()
    prm = B.Params(0, 0.0, 5, 0.7, 10, 10, 1, 0)

    def call(degrees, lo=None, hi=None, budget=-6.0, weights=None, prm_=prm):
        st = B.SelectorStruct()
        st.num_degrees = len(degrees)
        for i, d in enumerate(degrees):
            st.degrees[i] = d
        for i in range(6):
            st.feature_lo[i] = 0.0 if lo is None else lo[i]
            st.feature_hi[i] = 1.0 if hi is None else hi[i]
        st.log10_budget = budget
        if weights is not None:
            st.weights = weights
        return lib.bldtt_setup_learned(ctypes.byref(h), DUMMY, 100, DUMMY, 100, DUMMY,
                                       ctypes.byref(prm_), ctypes.byref(st), None)
    assert call([]) == 1                                   # no degrees
    assert call([3, 4, 5, 5]) == 1                         # not strictly increasing
    assert call([3, 4]) == 1                               # highest degree != params n
    assert call([3, 17]) == 1                              # degree out of range
    assert call([3, 5], lo=[0, 0, 0, 0, 2, 0], hi=[1] * 6) == 1    # empty feature box
    assert call([3, 5], budget=float("nan")) == 1
    assert lib.bldtt_setup_learned(ctypes.byref(h), DUMMY, 100, DUMMY, 100, DUMMY,
                                   ctypes.byref(prm), None, None) == 1
    assert not h


def test_training_entry_points_reject_bad_arguments(lib):
    assert lib.bldtt_selector_param_count(0) == -1
    assert lib.bldtt_selector_param_count(6) == 64 * 6 + 64 + 2 * (64 * 64 + 64) + 18 * 64 + 18
    assert lib.bldtt_mlp_forward(None, 3, DUMMY, 10, DUMMY, None) == 1
    assert lib.bldtt_mlp_forward(DUMMY, 25, DUMMY, 10, DUMMY, None) == 1      # > 24 outputs
    assert lib.bldtt_mlp_gradients(DUMMY, 3, DUMMY, DUMMY, None, 10, DUMMY, None, None) == 1
    assert lib.bldtt_mlp_adam(DUMMY, DUMMY, DUMMY, DUMMY, 10, 0, 1e-3, None) == 1   # step counts from 1
    deg = (ctypes.c_int * 2)(3, 5)
    assert lib.bldtt_pair_errors(None, 1, DUMMY, 64, 2, deg, DUMMY, None) == 1
    assert lib.bldtt_pair_features(None, 1, DUMMY, DUMMY, None) == 1
    assert lib.bldtt_list_classes(None, None, None, None) == 1


def test_binding_refuses_host_tensors(lib):
    """No CPU fallback: the binding hands only device pointers to the library
    and refuses host, non-FP64 or wrongly shaped tensors before any CUDA call."""
    import torch
    pts = torch.zeros(3, 10, dtype=torch.float64)
    q = torch.zeros(10, dtype=torch.float64)
    with pytest.raises(TypeError):
        B.Plan(pts, pts, q)
    with pytest.raises(TypeError):
        B.Plan(pts.float(), pts.float(), q.float())
    with pytest.raises(ValueError):
        B.Plan(pts.t(), pts.t(), q)


def test_autotune_table_rejects_null_arguments(lib):
    rows = ctypes.c_int(0)
    assert lib.bldtt_autotune_table(None, 0, ctypes.byref(rows), None, None, None, None) == 1
