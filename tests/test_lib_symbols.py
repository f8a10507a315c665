"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/povar.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "povar.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(povar_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_05079_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("povar_create", "povar_destroy", "povar_step", "povar_solve", "povar_cost",
              "povar_set_cameras", "povar_init_random", "povar_get_cameras",
              "povar_get_points", "povar_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_version_string_without_gpu(libpath):
    from paper_2405_05079_gb300 import povar
    assert "sm_103a" in povar.version()


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2405_05079_gb300 import povar
    monkeypatch.setattr(povar, "_lib", None)
    monkeypatch.setattr(povar, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not found"):
        povar.lib()


def test_create_rejects_empty_and_oversized_inputs_before_touching_the_device():
    """n_obs = 0 and n_obs >= 2^31 (32-bit observation indices) are rejected by
    the argument checks, before any CUDA call: this runs without a GPU."""
    import ctypes as C
    import numpy as np
    from paper_2405_05079_gb300 import povar
    L = povar.lib()
    cam = np.zeros(4, np.int32)
    pt = np.zeros(4, np.int32)
    meas = np.zeros((4, 2))
    h = C.c_void_p()
    args = (cam.ctypes.data_as(C.POINTER(C.c_int32)), pt.ctypes.data_as(C.POINTER(C.c_int32)),
            meas.ctypes.data_as(C.POINTER(C.c_double)), None, C.byref(h))
    assert L.povar_create(1, 1, 0, *args) == 1          # empty observation set
    assert L.povar_create(1, 1, 1 << 31, *args) == 1    # beyond 32-bit observation indices
    assert L.povar_create(0, 1, 4, *args) == 1          # no camera
    assert L.povar_create(1, 0, 4, *args) == 1          # no landmark
    assert not h.value


def test_create_rejects_invalid_arguments_on_the_host(libpath):
    """povar_create / povar_batch_create check sizes and pointers before any
    CUDA call (POVAR_EINVAL = 1, *out left NULL); povar_destroy(NULL) is a no-op."""
    C = ctypes
    lib = C.CDLL(libpath)
    for f in (lib.povar_create, lib.povar_batch_create):
        f.restype = C.c_int
    lib.povar_create.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
    lib.povar_batch_create.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_void_p)]
    lib.povar_destroy.argtypes = [C.c_void_p]
    cam = (C.c_int32 * 2)(0, 0)
    pt = (C.c_int32 * 2)(0, 0)
    meas = (C.c_double * 4)(0.0, 0.0, 0.1, 0.1)
    p = lambda a: C.cast(a, C.c_void_p)
    out = C.c_void_p(12345)
    cases = [(0, 1, 2, p(cam), p(pt), p(meas)),          # no cameras
             (1, 0, 2, p(cam), p(pt), p(meas)),          # no landmarks
             (1, 1, 0, p(cam), p(pt), p(meas)),          # no observations
             (1, 1, 1 << 31, p(cam), p(pt), p(meas)),    # observation count beyond int32
             (1, 1, 2, None, p(pt), p(meas)),
             (1, 1, 2, p(cam), None, p(meas)),
             (1, 1, 2, p(cam), p(pt), None)]
    for n_c, n_p, n_o, a, b, m in cases:
        out.value = 12345
        assert lib.povar_create(n_c, n_p, n_o, a, b, m, None, C.byref(out)) == 1
        assert out.value is None
    assert lib.povar_create(1, 1, 2, p(cam), p(pt), p(meas), None, None) == 1
    nc, npt, nob = (C.c_int32 * 1)(1), (C.c_int32 * 1)(1), (C.c_int64 * 1)(2)
    out.value = 12345
    assert lib.povar_batch_create(0, p(nc), p(npt), p(nob), p(cam), p(pt), p(meas), None,
                                  C.byref(out)) == 1
    assert out.value is None
    assert lib.povar_batch_create(1, None, p(npt), p(nob), p(cam), p(pt), p(meas), None,
                                  C.byref(out)) == 1
    lib.povar_destroy(None)


def test_estimate_bytes_grows_with_each_size(libpath):
    lib = ctypes.CDLL(libpath)
    lib.povar_estimate_bytes.restype = ctypes.c_int64
    lib.povar_estimate_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64]
    base = lib.povar_estimate_bytes(100, 10_000, 50_000)
    assert base > 50_000 * 12 + 10_000 * 40
    assert lib.povar_estimate_bytes(200, 10_000, 50_000) > base
    assert lib.povar_estimate_bytes(100, 20_000, 50_000) > base
    assert lib.povar_estimate_bytes(100, 10_000, 100_000) > base


def test_binding_noalloc_limit_equals_the_header():
    """The binding's copy of POVAR_NOALLOC_MAX_POINTS is the header's value."""
    from paper_2405_05079_gb300 import povar
    text = open(os.path.join(ROOT, "include", "povar.h")).read()
    m = re.search(r"POVAR_NOALLOC_MAX_POINTS\s*=\s*(\d+)", text)
    assert m and int(m.group(1)) == povar.NOALLOC_MAX_POINTS


def test_noalloc_rejects_misaligned_pointers_before_any_cuda_call(libpath):
    """povar_cost_noalloc checks the alignment of every device pointer on the
    host (P and meas 16 bytes, off_pt and cam 4, cost_out and X_out 8) and
    returns POVAR_EINVAL (1) before any CUDA call, so a misaligned caller
    pointer never reaches the device. The addresses below are never
    dereferenced: this runs without a GPU."""
    C = ctypes
    lib = C.CDLL(libpath)
    f = lib.povar_cost_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]
    base = 1 << 20
    good = dict(P=base, off=base + 0x1000, cam=base + 0x2000, meas=base + 0x3000,
                X=base + 0x4000, F=base + 0x5000)

    def call(**kw):
        a = {**good, **kw}
        return f(2, 3, 6, a["P"], a["off"], a["cam"], a["meas"], 0.1, a["X"], a["F"], None)

    for bad in (dict(P=base + 8), dict(meas=base + 0x3008), dict(off=base + 0x1002),
                dict(cam=base + 0x2001), dict(F=base + 0x5004), dict(X=base + 0x4004)):
        assert call(**bad) == 1, bad


def test_ctypes_structs_match_the_header(tmp_path):
    """The binding's Params and StepReport have the header's size and field
    offsets (compiled with the host C compiler against include/povar.h)."""
    import shutil
    import subprocess
    from paper_2405_05079_gb300 import povar
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"povar_params": povar.Params, "povar_step_report": povar.StepReport}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "povar.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "abi.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "abi"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
