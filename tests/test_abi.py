"""C-ABI checks that need no GPU: the library builds, loads and exports every
entry point declared in include/hsgen.h; the binding refuses to run without it."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1602_06589_gb300 import hsgen

    return hsgen.load()


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "hsgen.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hsgen_[a-z_A-Z0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_1602_06589_gb300 import hsgen

    for n in declared_entry_points():
        assert n in hsgen.EXPORTS
        assert callable(getattr(hsgen, n))


def test_default_options(lib):
    from paper_1602_06589_gb300 import hsgen

    o = hsgen.hsgen_default_options()
    assert o.precision == hsgen.FP64 and o.uplo == ord("U") and o.target_rel_err == 1e-12
    assert o.wait_timeout_ns > 0


def test_null_arguments_are_rejected(lib):
    import ctypes as C

    from paper_1602_06589_gb300 import hsgen

    assert lib.hsgen_create(None, 0, None) == hsgen.EINVAL
    assert lib.hsgen_build_HS(None, 1, None, None, None, 1, None) == hsgen.EINVAL
    assert lib.hsgen_set_atoms(None, None, 1.0, 0, None, 0, None, None, None) == hsgen.EINVAL
    assert lib.hsgen_get_stats(None, None) == hsgen.EINVAL
    lib.hsgen_destroy(None)  # NULL-safe
    assert lib.hsgen_last_error(None) == b"null context"


def test_no_gpu_means_ecuda_not_fallback(lib):
    import torch

    from paper_1602_06589_gb300 import hsgen

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hsgen.HsgenError) as ei:
        hsgen.hsgen_create(0)
    assert ei.value.status in (hsgen.ECUDA, hsgen.EINVAL)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1602_06589_gb300 import hsgen

    with pytest.raises(RuntimeError, match="no non-CUDA fallback"):
        hsgen.load(str(tmp_path / "libhsgen.so"))


def test_header_is_plain_c_and_links_from_c(lib, tmp_path):
    """include/hsgen.h compiles as C11 (-Wall -Werror -pedantic) and a C program
    links against libhsgen.so and calls the entry points that need no GPU."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1602_06589_gb300 import build as cbuild

    libdir = os.path.dirname(cbuild.LIB)
    exe = str(tmp_path / "abi_from_c")
    src = os.path.join(ROOT, "tests", "c", "abi_from_c.c")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                        src, "-o", exe, "-L", libdir, "-lhsgen", "-Wl,-rpath," + libdir],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.stdout, r.stderr)
