"""CPU checks of the C-ABI library: it builds, loads without a GPU, exports
every function include/nk.h declares, and its host-side geometry logic
(nk_q_size) matches the architecture definition."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def libnk():
    from paper_2303_05420_gb300 import _lib

    if not os.path.exists(_lib.LIB_PATH):
        from paper_2303_05420_gb300 import build

        build.build()
    return _lib.lib()


def declared_functions():
    """Every function any header under include/ declares."""
    names = set()
    for hdr in HEADERS:
        src = open(hdr).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(nk_[a-z0-9_]+)\s*\(", src,
                                flags=re.M))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["nk_self_diag", "nk_block", "nk_pcg_solve", "nk_create", "nk_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libnk):
    from paper_2303_05420_gb300 import _lib

    names = declared_functions()
    missing = [n for n in names if not hasattr(libnk, n)]
    assert not missing, missing
    assert sorted(names) == sorted(_lib.EXPORTS)


def test_status_strings(libnk):
    for s in range(8):
        assert libnk.nk_status_string(s)


def test_q_size_host_logic(libnk):
    from paper_2303_05420_gb300._lib import make_arch

    a = make_arch((2, 1, 0))
    # two 32x32 layers and one 16x16 layer
    assert libnk.nk_q_size(ctypes.byref(a), 32, 32) == 2 * 1024 + 256
    a = make_arch((3, 3, 3))
    assert libnk.nk_q_size(ctypes.byref(a), 32, 32) == 3 * (1024 + 256 + 64)
    # odd size cannot be pooled
    assert libnk.nk_q_size(ctypes.byref(a), 30, 30) == -1  # 30 -> 15 cannot be pooled again
    assert libnk.nk_q_size(ctypes.byref(make_arch((2, 1, 0))), 31, 31) == -1
    bad = make_arch((0, 1))
    assert libnk.nk_q_size(ctypes.byref(bad), 8, 8) == -1
    assert libnk.nk_q_size(ctypes.byref(make_arch((2,), filt=5)), 8, 8) == -1
    # Erf keeps the layout; a LayerNorm appends one divisor per layer
    assert libnk.nk_q_size(ctypes.byref(make_arch((2, 1, 0), act="erf")), 32, 32) == 2 * 1024 + 256
    assert libnk.nk_q_size(ctypes.byref(make_arch((2, 1, 0), norm="layer")), 32, 32) == 2 * 1024 + 256 + 3
    assert libnk.nk_q_size(ctypes.byref(make_arch((3, 3, 3), act="erf", norm="layer")), 16, 16) == \
        3 * (256 + 64 + 16) + 9
    # a LayerNorm needs an activation
    assert libnk.nk_q_size(ctypes.byref(make_arch((2, 1, 0), act="identity", norm="layer")), 8, 8) == -1


def test_header_compiles_and_links_as_c(libnk, tmp_path):
    """include/nk.h compiles as C99 and libnk links from a C program that
    calls the host-only entry points (tests/c_abi_check.c)."""
    import shutil
    import subprocess

    from paper_2303_05420_gb300 import _lib

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(_lib.LIB_PATH)
    exe = str(tmp_path / "c_abi_check")
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_abi_check.c"), "-o", exe, "-L", libdir, "-lnk",
                    "-Wl,-rpath," + libdir], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.strip() == "ok"
