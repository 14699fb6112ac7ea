"""The C-ABI library builds, loads and exports every entry point include/vip.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import re
from pathlib import Path

ROOT = Path(__file__).resolve().parents[1]


def declared():
    text = (ROOT / "include" / "vip.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vip_[a-z_0-9]+)\s*\(", text)))


def test_header_and_binding_agree():
    from paper_1401_6513_gb300 import vip
    assert declared() == sorted(vip.EXPORTS)


def test_library_exports_every_declared_symbol():
    import paper_1401_6513_gb300 as pkg
    lib = pkg.build()
    so = ctypes.CDLL(str(lib))
    missing = [s for s in declared() if not hasattr(so, s)]
    assert not missing, missing


def test_binding_refuses_missing_library(tmp_path):
    import pytest
    from paper_1401_6513_gb300 import vip
    with pytest.raises(ImportError):
        vip.lib(tmp_path / "libvip.so")


def test_header_is_plain_c():
    """The boundary is a C ABI: the header compiles as C99 (no C++ or torch types)
    and as C++, with warnings as errors."""
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc")
    if cc is None:
        pytest.skip("gcc not found")
    hdr = str(ROOT / "include" / "vip.h")
    for lang, std in (("c", "-std=c99"), ("c++", "-std=c++17")):
        r = subprocess.run([cc, "-fsyntax-only", std, "-Wall", "-Wextra", "-Werror", "-x", lang, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, (lang, r.stderr)
