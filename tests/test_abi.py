"""The C-ABI library loads and exports every entry point include/hps.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

from paper_2511_00735_gb300 import build as B
from paper_2511_00735_gb300 import hps as H

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def libpath():
    srcs = [os.path.join(B.CSRC, f) for f in os.listdir(B.CSRC)]
    if not os.path.exists(B.LIB) or max(os.path.getmtime(s) for s in srcs) > os.path.getmtime(B.LIB):
        B.build()
    return B.LIB


def declared():
    txt = open(os.path.join(ROOT, "include", "hps.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hps_[A-Za-z_]+)\s*\(", txt)) - {"hps_alloc_fn", "hps_free_fn"})


def test_header_declares_the_binding_surface():
    assert declared() == sorted(H.EXPORTS)


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_device(libpath):
    lib = ctypes.CDLL(libpath)
    lib.hps_strerror.restype = ctypes.c_char_p
    assert lib.hps_strerror(0) == b"ok"
    assert b"unsupported" in lib.hps_strerror(-8) or b"not supported" in lib.hps_strerror(-8)


def test_null_context_is_rejected(libpath):
    lib = ctypes.CDLL(libpath)
    assert lib.hps_mesh(None, 4, 4, 8) == -1
    assert lib.hps_destroy(None) == 0


def test_plain_c_consumer(libpath, tmp_path):
    # the header compiles as C99 and a C program linked with the library runs (no GPU needed:
    # without a device hps_create reports HPS_ENODEV)
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "abi_consumer")
    libdir = os.path.dirname(libpath)
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "abi_consumer.c"), "-o", exe, libpath, "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() in ("no device", "device")


def test_autotune_table_and_null_context_without_device(libpath):
    # the tuning table is process-wide host state: empty until a tensor-core GEMM is tuned, and
    # readable (count only, or into a buffer cut to its length) without a device; the per-context
    # calls reject a null context
    lib = ctypes.CDLL(libpath)
    lib.hps_autotune_clear.restype = None
    lib.hps_autotune_clear()
    assert lib.hps_autotune_table(None, 0) == 0
    buf = ctypes.create_string_buffer(b"x" * 16)
    assert lib.hps_autotune_table(buf, 16) == 0
    assert buf.value == b""
    assert lib.hps_set_autotune(None, 1) == -1
    assert lib.hps_profile_kernels(None, 1) == -1
    assert lib.hps_profile_kernels_read(None, None, None, None, None) == -1
