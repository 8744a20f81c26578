"""The C-ABI library builds, loads and exports every symbol include/*.h declares (no GPU)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(kdt_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("kdt_create", "kdt_build", "kdt_step", "kdt_export_triangles", "kdt_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2308_06484_gb300 import kdt
    L = kdt.load()
    for name in declared_functions():
        assert hasattr(L, name), name
    assert set(declared_functions()) <= set(kdt.SYMBOLS)
    assert L.kdt_version() == 7
    assert L.kdt_stats_size() == ctypes.sizeof(kdt.Stats)
    assert L.kdt_config_size() == ctypes.sizeof(kdt.Config)
    assert L.kdt_num_cells(None) == 0 and L.kdt_num_points(None) == 0
    assert L.kdt_error_string(-3) == b"duplicate point or repeated move id"


def test_library_has_no_torch_dependency():
    from paper_2308_06484_gb300 import kdt
    out = subprocess.run(["ldd", kdt.lib_path()], capture_output=True, text=True).stdout
    libs = [line.split()[0] for line in out.splitlines() if line.strip()]
    assert not any("torch" in x or x.startswith("libc10") for x in libs), libs


def test_config_defaults_and_argument_errors():
    from paper_2308_06484_gb300 import kdt
    L = kdt.load()
    c = kdt.default_config()
    assert c.domain_bits == 28 and c.fallback == 1 and c.filter == 1 and c.retry_cap == 4096
    assert L.kdt_default_config(None) == -1
    assert L.kdt_create(None, None, 0, None) == -1
    # calls on a NULL handle are argument errors, never a crash
    assert L.kdt_build(None, None, 10) == -1
    assert L.kdt_step(None, None, 1) == -1
    n = ctypes.c_int64(0)
    assert L.kdt_export_triangles(None, None, 0, ctypes.byref(n)) == -1
    assert L.kdt_destroy(None) == 0
    assert L.kdt_num_points(None) == 0
