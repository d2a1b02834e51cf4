"""The C-ABI library builds, loads and exports every symbol its header declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fastmps.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fastmps_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("fastmps_create", "fastmps_load_site", "fastmps_sample", "fastmps_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import paper_2512_20064_gb300 as F

    lib = F.load_library()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert F.fastmps_version().startswith("fastmps-gb300")


def test_no_device_fails_loudly():
    """Without a GPU the library refuses to create a handle (there is no CPU fallback)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2512_20064_gb300 as F

    with pytest.raises(F.FastMPSError) as e:
        F.Sampler()
    assert e.value.code in (-5, -7)


def test_library_does_not_reference_oracle():
    """The product sources never mention the oracle package or its symbols."""
    src = os.path.join(ROOT, "paper_2512_20064_gb300")
    for dirpath, _, files in os.walk(src):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "orc_" not in text, f


def test_every_exported_symbol_is_declared():
    """The library exports no fastmps_* entry point that the header does not declare."""
    import shutil
    import subprocess

    import paper_2512_20064_gb300 as F

    if shutil.which("nm") is None:
        pytest.skip("nm not available")
    F.load_library()
    out = subprocess.run(["nm", "-D", "--defined-only", F.native.LIB], capture_output=True, text=True).stdout
    exported = sorted({ln.split()[-1] for ln in out.splitlines() if ln.split() and ln.split()[-1].startswith("fastmps_")})
    undeclared = [n for n in exported if n not in declared_functions()]
    assert exported and not undeclared, undeclared


def test_binding_carries_the_c_names():
    """The Python binding offers every declared entry point under its C name (argument marshalling only)."""
    import paper_2512_20064_gb300 as F

    missing = [n for n in declared_functions() if not callable(getattr(F, n, None))]
    assert not missing, missing
