"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/hub.h declares; the Python binding wires every one of them (no GPU needed)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hub.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\*?\s+\*?(hub_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_23612_gb300 import build as b
    b.build()
    from paper_2507_23612_gb300 import binding
    return binding.load_library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hub_create_grid", "hub_set_atoms_projectors", "hub_apply_H",
                     "hub_chefsi_filter", "hub_occupation", "hub_rayleigh_ritz"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2507_23612_gb300.binding import library_path
    out = subprocess.run(["nm", "-D", "--defined-only", library_path()], capture_output=True,
                         text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_binding_covers_every_declared_function():
    from paper_2507_23612_gb300.binding import _SIGS
    assert set(declared_functions()) <= set(_SIGS)


def test_library_is_built_for_sm_103a_only():
    from paper_2507_23612_gb300 import build as b
    assert b.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_version_string(lib):
    import ctypes
    buf = ctypes.create_string_buffer(128)
    assert lib.hub_version(buf, 128) == 0
    assert b"sm_103a" in buf.value


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2507_23612_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in src.replace("oracle-free", ""), f
