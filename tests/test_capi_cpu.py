"""The C-ABI library loads and exports every entry point include/navixgb.h
declares (no compute calls: CPU only)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "navixgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nx_[a-z_]+)\s*\(", src)) - {"nx_status"})


@pytest.fixture(scope="module")
def built():
    from paper_2407_19396_gb300 import build

    return build.build()


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (nx_[a-z_]+)$", out, flags=re.M))
    declared = _declared()
    assert declared, "no declarations found"
    missing = [s for s in declared if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_declared_symbol(built):
    from paper_2407_19396_gb300 import navixgb as nx

    L = nx.lib()
    for s in _declared():
        assert s in nx.SIGNATURES, s
        assert hasattr(L, s)


def test_status_strings_and_creation_errors_without_gpu(built):
    from paper_2407_19396_gb300 import navixgb as nx

    L = nx.lib()
    assert L.nx_status_str(nx.NX_E_BUDGET).decode() == "request exceeds the HBM budget"
    # argument validation happens before any device call
    for fam, size, n in [(nx.NX_N_FAMILIES, 5, 4), (-1, 5, 4), (0, 4, 4), (0, 20, 4), (0, 5, 0), (nx.NX_KEYCORRIDOR, 8, 4),
                          (nx.NX_KEYCORRIDOR, 5, 4)]:
        with pytest.raises(nx.NavixError) as ei:
            nx.nx_create(fam, size, n, 0)
        assert ei.value.status == nx.NX_E_INVAL
    # mixed descriptors: the 16-bit step counter's limit, variants beyond the
    # family's range, sizes outside 5..19 (one bad descriptor among good ones)
    good = (nx.NX_DOORKEY, 8, 0, 0)
    for bad in [(nx.NX_EMPTY, 5, 65536, 0), (nx.NX_LAVA_CROSSING, 9, 0, 99), (nx.NX_DISTSHIFT, 7, 0, 2),
                (nx.NX_EMPTY, 21, 0, 0), (nx.NX_DOORKEY, 8, 0, -1)]:
        with pytest.raises(nx.NavixError) as ei:
            nx.nx_create_mixed([good, bad, good], 0)
        assert ei.value.status == nx.NX_E_INVAL, bad


def test_product_binding_does_not_import_the_oracle():
    for f in os.listdir(os.path.join(ROOT, "paper_2407_19396_gb300")):
        if f.endswith(".py"):
            txt = open(os.path.join(ROOT, "paper_2407_19396_gb300", f)).read()
            assert "import oracle" not in txt and "from oracle" not in txt, f
