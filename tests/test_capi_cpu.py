"""C ABI checks that need no GPU: the library builds, loads and exports every
symbol include/mps.h declares; the oracle and the product path stay apart."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1111_3124_gb300 import build as B
    B.build()
    import paper_1111_3124_gb300.mps as M
    return M.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "mps.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(mps_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("mps_create", "mps_apply_gate", "mps_amplitude", "mps_expectation", "mps_reduced_density"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_1111_3124_gb300 import build as B
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(mps_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    import paper_1111_3124_gb300.mps as M
    assert sorted(M.EXPORTS) == declared_symbols()


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_1111_3124_gb300.mps as M
    saved = M._lib
    M._lib = None
    try:
        with pytest.raises(ImportError):
            M.load_library(str(tmp_path / "missing.so"))
    finally:
        M._lib = saved


def test_oracle_and_product_share_no_code():
    pkg = os.path.join(ROOT, "paper_1111_3124_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f), errors="replace").read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "mps_oracle" not in src, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".cpp")):
            src = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_1111_3124_gb300" not in src.replace("paper_1111_3124_gb300/", ""), f
            assert "csrc" not in src, f
