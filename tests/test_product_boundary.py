"""The product path's boundary, CPU only: the package and the C ABI reference nothing under
oracle/ (the oracle is test infrastructure), and the binding fails loudly, with no CPU fallback,
when the CUDA library is missing."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PRODUCT = [os.path.join(ROOT, "paper_2305_03945_gb300"), os.path.join(ROOT, "include")]
SOURCES = (".py", ".cu", ".cuh", ".h", ".cpp", ".c")
# an import of the oracle package, a path into it, or a load of its library
ORACLE_REF = re.compile(r"^\s*(from\s+oracle\b|import\s+oracle\b)|oracle/|rd_oracle|librd_oracle|cpp_oracle", re.M)


def _product_files():
    for top in PRODUCT:
        for d, _, files in os.walk(top):
            for f in files:
                if f.endswith(SOURCES):
                    yield os.path.join(d, f)


def test_product_sources_reference_no_oracle():
    files = list(_product_files())
    assert len(files) > 20
    hits = []
    for p in files:
        for m in ORACLE_REF.finditer(open(p, encoding="utf-8").read()):
            hits.append("%s: %s" % (os.path.relpath(p, ROOT), m.group(0).strip()))
    assert hits == []


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_2305_03945_gb300 import rd
    monkeypatch.setattr(rd, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        rd.load(str(tmp_path / "librd_pdhg.so"))


def test_oracle_sources_reference_no_product_code():
    """The oracle shares nothing with the CUDA path: no import of the package, no path into its
    sources, no use of the product library."""
    product_ref = re.compile(r"^\s*(from|import)\s+paper_2305_03945_gb300|^\s*#\s*include\s*[<\"][^>\"]*"
                             r"(csrc|rd_pdhg|rd_internal|rd_device|rd_sweep)|librd_pdhg", re.M)
    d = os.path.join(ROOT, "oracle")
    files = [os.path.join(d, f) for f in os.listdir(d) if f.endswith(SOURCES)]
    assert len(files) >= 6
    hits = ["%s: %s" % (os.path.basename(p), m.group(0)) for p in files
            for m in product_ref.finditer(open(p, encoding="utf-8").read())]
    assert hits == []
