"""The C ABI library builds for sm_103a, loads, and exports exactly what include/vrcube.h declares.
No GPU needed (no compute call is made)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vrcube.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"\b(vr_[a-z_0-9]+)\s*\(", src))


@pytest.fixture(scope="module")
def libpath():
    from paper_1008_0135_gb300.build_ext import build
    return build()


def test_every_declared_symbol_is_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    declared = _declared()
    assert declared, "no declarations parsed"
    assert declared == exported, (declared ^ exported)


def test_binding_covers_the_header(libpath):
    from paper_1008_0135_gb300 import _abi
    assert set(_abi.SIGNATURES) == _declared()
    L = _abi.lib()
    for name in _abi.SIGNATURES:
        assert getattr(L, name) is not None


def test_error_strings_and_no_gpu_create(libpath):
    from paper_1008_0135_gb300 import _abi
    import torch
    L = _abi.lib()
    for st in range(0, -8, -1):
        assert L.vr_error_string(st)
    if torch.cuda.is_available():
        pytest.skip("GPU present: creation is covered by the GPU tests")
    h = C.c_void_p()
    rc = L.vr_create(C.byref(h), 0, 0)
    assert rc in (_abi.VR_ERR_CUDA, _abi.VR_ERR_ARG) and not h.value


def test_null_context_calls_fail_cleanly(libpath):
    from paper_1008_0135_gb300 import _abi
    L = _abi.lib()
    assert L.vr_set_render_params(None, 0, 0.5, 0.99) == _abi.VR_ERR_ARG
    assert L.vr_set_timing(None, 1) == _abi.VR_ERR_ARG
    assert L.vr_reset_stats(None) == _abi.VR_ERR_ARG
    L.vr_destroy(None)
