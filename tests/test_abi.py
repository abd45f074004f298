"""CPU-side checks of the boundary: the CUDA library builds for sm_103a, loads,
and exports every function include/ebic.h declares; every entry point that
takes a handle rejects a null one before any device work; the binding fails
loudly when the library is missing."""
import ctypes
import os
import subprocess
import sys

import pytest

from helpers import ROOT, header_functions


@pytest.fixture(scope="module")
def libpath():
    from paper_1801_03039_gb300 import _build
    return _build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for want in ("ebic_load_matrix", "ebic_eval_population", "ebic_run_generations",
                 "ebic_free", "ebic_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in header_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_build_targets_sm_103a_only():
    from paper_1801_03039_gb300 import _build
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_marshals_names_of_the_header():
    import paper_1801_03039_gb300 as e
    for n in header_functions():
        if n in ("ebic_last_error", "ebic_abi_version", "ebic_kernel_launches"):
            continue
        assert hasattr(e, n), n


def test_binding_fails_loudly_without_library(tmp_path):
    code = (
        "import paper_1801_03039_gb300 as e, paper_1801_03039_gb300._build as b\n"
        f"b.LIB = {str(tmp_path / 'missing.so')!r}\n"
        "try:\n    e.lib()\nexcept RuntimeError as x:\n    print('raised', x)\n")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=ROOT)
    assert "raised" in r.stdout and "no CPU fallback" in r.stdout


def test_abi_version(libpath):
    L = ctypes.CDLL(libpath)
    assert L.ebic_abi_version() == 2


def _null_handle_calls():
    """(name, argtypes) of every status-returning entry point whose first
    argument is one of the library's opaque handles."""
    import re
    import paper_1801_03039_gb300 as e
    text = open(os.path.join(ROOT, "include", "ebic.h")).read()
    names = [m.group(1) for m in re.finditer(
        r"ebic_status\s+(ebic_\w+)\s*\(\s*(ebic_handle|ebic_batch|ebic_surrogate)\s+\w+", text)]
    return [(n, e._SIGS[n][0]) for n in names]


def test_null_handles_are_rejected_before_any_device_work():
    """A null handle is an argument error with a message, whatever the
    rest of the arguments (zeros and null pointers here; no GPU needed)."""
    import paper_1801_03039_gb300 as e
    L = e.lib()
    calls = _null_handle_calls()
    assert len(calls) >= 30
    for name, argtypes in calls:
        args = [0.0 if t in (ctypes.c_double, ctypes.c_float) else 0 for t in argtypes]
        args[0] = None
        status = getattr(L, name)(*args)
        if name == "ebic_surrogate_free":                  # like free(NULL): nothing to do
            assert status == 0
            continue
        assert status == 1, (name, status)                # EBIC_ERR_ARG
        assert L.ebic_last_error(), name


def test_matrix_shape_and_pointers_are_checked_on_the_host():
    import numpy as np
    import paper_1801_03039_gb300 as e
    L = e.lib()
    h = ctypes.c_void_p()
    A = np.zeros((4, 3), np.float32)
    p = A.ctypes.data_as(ctypes.c_void_p)
    for args in [(None, 4, 3, ctypes.byref(h)), (p, 4, 3, None), (p, 0, 3, ctypes.byref(h)),
                 (p, 4, 0, ctypes.byref(h)), (p, 4, 65536, ctypes.byref(h)),
                 (p, (1 << 26) + 1, 3, ctypes.byref(h))]:
        assert L.ebic_load_matrix(*args) == 1, args            # EBIC_ERR_ARG
        assert L.ebic_last_error()
    assert h.value is None                                     # nothing was created


def test_rows_binding_sizes_then_fills():
    """The binding's two-call protocol of the rows entry points (first call
    sizes the buffer, second fills it), against a fake that follows the
    header's contract."""
    import numpy as np
    import paper_1801_03039_gb300 as e
    want = [[0, 3, 5], [], [1, 2]]
    calls = []

    def fake(po, pc, P, ro, rw, cap):
        need = sum(len(w) for w in want)
        calls.append(cap._obj.value)
        if rw is None or cap._obj.value < need:
            cap._obj.value = need
            return 1                                   # EBIC_ERR_ARG, size in *cap
        roff = np.ctypeslib.as_array(ctypes.cast(ro, ctypes.POINTER(ctypes.c_int64)), (P + 1,))
        rows = np.ctypeslib.as_array(ctypes.cast(rw, ctypes.POINTER(ctypes.c_int32)), (need,))
        k = 0
        for i, w in enumerate(want):
            roff[i] = k
            rows[k:k + len(w)] = w
            k += len(w)
        roff[P] = k
        cap._obj.value = k
        return 0

    off = np.array([0, 2, 3, 5], np.int32)
    cols = np.array([0, 1, 2, 0, 1], np.int32)
    got = e._extract(fake, off, cols)
    assert [g.tolist() for g in got] == want and calls == [0, 5]
