"""The C-ABI library builds, loads and exports every symbol corr.h declares.

No compute calls here: these run on machines without a GPU.
"""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1501_05992_gb300 import build as corr_build
from paper_1501_05992_gb300 import corr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_functions() -> set[str]:
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([A-Za-z_][A-Za-z0-9_]*)\s*\([^;{]*\)\s*;", text):
            name = m.group(1)
            if name.startswith("corr_"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def lib_path():
    return corr_build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["corr_create", "corr_accumulate", "corr_dump", "corr_destroy",
                     "corr_workspace_bytes", "corr_bind_workspace", "corr_set_path",
                     "corr_get_state", "corr_set_state", "corr_last_error", "corr_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"
    lib = ctypes.CDLL(lib_path)
    for name in declared_functions():
        assert hasattr(lib, name)


def test_library_targets_sm103a_only(lib_path):
    """Every translation unit and the link are built with exactly one
    -gencode, for sm_103a, and the build fingerprint covers those flags."""
    arch = corr_build.ARCH
    assert arch == ["-gencode", "arch=compute_103a,code=sm_103a"], arch
    flags = corr_build.NVCC_FLAGS
    assert not any(f.startswith(("-arch", "--gpu-architecture", "-gencode", "--generate-code"))
                   for f in flags), flags
    stamp = os.path.join(os.path.dirname(lib_path), "libcorr.stamp")
    assert open(stamp).read().strip() == corr_build._fingerprint()


def test_strerror_and_version(lib_path):
    lib = corr.load()
    assert lib.corr_version() >= 100
    for code in [0, -1, -2, -3, -4, -5, -6, -7, -8]:
        assert lib.corr_strerror(code)
    assert lib.corr_strerror(12345) == b"unknown status"


@pytest.mark.parametrize("args", [(0, 1, 1), (1, 0, 1), (1, 1, 0), (-3, 4, 4),
                                  (16, 32, 1 << 24), (9000, 1, 1)])
def test_create_rejects_bad_sizes_without_touching_a_device(lib_path, args):
    lib = corr.load()
    assert not lib.corr_create(*args)
    assert lib.corr_last_error() == corr.CORR_E_ARG


def test_null_context_is_an_argument_error(lib_path):
    lib = corr.load()
    assert lib.corr_accumulate(None, None, 1, None) == corr.CORR_E_ARG
    assert lib.corr_dump(None, None, None) == corr.CORR_E_ARG
    assert lib.corr_destroy(None) == corr.CORR_E_ARG
    assert lib.corr_workspace_bytes(None) == 0
    assert lib.corr_last_error() == corr.CORR_E_ARG
    assert lib.corr_unpack(None, 4, 0, 4, None, 0, None) == corr.CORR_E_ARG
    assert lib.corr_unpack(None, 4, 2, 4, None, 0, None) == corr.CORR_E_ARG
    assert lib.corr_unpack(None, 0, 2, 4, None, 0, None) == corr.CORR_OK


def test_fine_pfb_rejects_bad_arguments_without_touching_a_device(lib_path):
    lib = corr.load()
    fake = ctypes.c_void_p(1 << 20)           # aligned, never dereferenced: every call below fails its checks
    null = ctypes.c_void_p(0)
    cases = [
        ((null, 1, 8, 1536, fake, 12, 1.0, fake, null, null), corr.CORR_E_ARG),        # no input
        ((fake, 1, 8, 1536, fake, 12, 1.0, null, null, null), corr.CORR_E_ARG),        # no output
        ((fake, 1, 8, 1500, fake, 12, 1.0, fake, null, null), corr.CORR_E_ARG),        # not whole blocks
        ((fake, 1, 8, 1408, fake, 12, 1.0, fake, null, null), corr.CORR_E_ARG),        # fewer than 12 blocks
        ((fake, 0, 8, 1536, fake, 12, 1.0, fake, null, null), corr.CORR_E_ARG),
        ((fake, 1, 8, 1536, ctypes.c_void_p((1 << 20) + 4), 12, 1.0, fake, null, null), corr.CORR_E_ARG),
        ((fake, 1, 8, 1536, fake, 12, float("nan"), fake, null, null), corr.CORR_E_ARG),
        ((fake, 1, 8, 1536, fake, 5, 1.0, fake, null, null), corr.CORR_E_UNSUPPORTED),
    ]
    for args, want in cases:
        assert lib.corr_fine_pfb(*args) == want, args


def test_probe_rejects_bad_kind_without_touching_a_device(lib_path):
    import ctypes as ct
    lib = corr.load()
    rate = ct.c_double()
    assert lib.corr_probe_rate(7, ct.byref(rate), None, None) == corr.CORR_E_ARG
    assert lib.corr_probe_rate(-1, ct.byref(rate), None, None) == corr.CORR_E_ARG
    assert lib.corr_probe_rate(0, None, None, None) == corr.CORR_E_ARG
