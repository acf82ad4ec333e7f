"""Host-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every function that include/olb.h declares, with a ctypes signature
for each.  No CUDA call is made here (these run without a GPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "olb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(olb_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2307_11752_gb300 import build
    return build.build()


def test_header_declares_the_core_calls():
    names = _declared()
    for required in ("olb_lattice_create", "olb_set_material", "olb_set_bgk", "olb_step",
                     "olb_moments", "olb_adjoint_run"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (olb_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_ctypes_binding_covers_the_header(libpath):
    from paper_2307_11752_gb300 import olb
    assert sorted(olb.SIGNATURES) == _declared()
    lib = olb.load(libpath)
    for name in _declared():
        assert getattr(lib, name) is not None


def test_build_targets_sm_103a_only():
    from paper_2307_11752_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
