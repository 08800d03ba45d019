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


def test_binding_refuses_output_buffers_the_library_would_overrun():
    """The binding checks every caller-supplied output buffer before it
    hands a pointer to the library: element type, contiguity, [slots, n, ...]
    shape with enough slots, and host versus device memory."""
    import numpy as np
    import torch

    from paper_2407_19396_gb300.navixgb import check_out_buffer

    n, side = 5, 8
    check_out_buffer("obs_sym", np.zeros((3, n, 7, 7, 3), np.uint8), n, side, 3, device=False)
    check_out_buffer("obs_sym", np.zeros((4, n, 7, 7, 3), np.uint8), n, side, 3, device=False)  # more slots: fine
    check_out_buffer("reward", np.zeros((n,), np.float32), n, side, None, device=False)
    check_out_buffer("obs_full", torch.zeros((2, n, side, side, 3), dtype=torch.uint8), n, side, 2, device=False)
    check_out_buffer("action", torch.zeros((2, n), dtype=torch.int8), n, side, 2, device=False)
    bad = [
        ("obs_sym", np.zeros((2, n, 7, 7, 3), np.uint8), 3, False),         # fewer slots than the ring
        ("obs_sym", np.zeros((3, n + 1, 7, 7, 3), np.uint8), 3, False),     # another env count
        ("reward", np.zeros((3, n), np.uint8), 3, False),                   # 1-byte elements for 4-byte rewards
        ("reward", np.zeros((3, n), np.float64), 3, False),
        ("terminated", np.zeros((n, 3), np.uint8).T, 3, False),             # not C-contiguous
        ("obs_cat", np.zeros((3, n, side - 1, side - 1), np.uint8), 3, False),  # views of a smaller side
        ("obs_sym", np.zeros((n, 7, 7, 3), np.uint8), 3, False),            # no slot dimension
        ("mission", np.zeros((3, n), np.uint8), 3, True),                   # host array for a device output
        ("action", torch.zeros((3, n), dtype=torch.uint8), 3, False),       # unsigned actions
        ("reward", torch.zeros((3, n), dtype=torch.float32), 3, True),      # host tensor for a device output
        ("obs_sym", torch.zeros((3, n, 7, 7, 3), dtype=torch.uint8)[:, :, :, :, :1].expand(3, n, 7, 7, 3), 3, False),
    ]
    for key, a, slots, dev in bad:
        with pytest.raises(ValueError):
            check_out_buffer(key, a, n, side, slots, device=dev)


def test_ctypes_structs_match_the_header_layout(tmp_path):
    """Every struct the binding mirrors has, compiled from include/navixgb.h
    by the host C compiler, the size and field offsets of its ctypes twin: a
    field added, dropped, retyped or moved on one side only would hand the
    library records it misreads."""
    import ctypes

    from paper_2407_19396_gb300 import navixgb as nx

    classes = [nx.nx_desc, nx.nx_options, nx.nx_out, nx.nx_policy, nx.nx_info, nx.nx_request, nx.nx_result,
               nx.nx_server_stats]
    lines = ["#include <stdio.h>", '#include "navixgb.h"', "int main(void) {"]
    for c in classes:
        name = c.__name__
        lines.append(f'printf("{name} - %zu\\n", sizeof({name}));')
        for field in c._fields_:
            lines.append(f'printf("{name} {field[0]} %zu\\n", offsetof({name}, {field[0]}));')
    lines.append("return 0; }")
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    seen = 0
    for line in out.splitlines():
        name, field, value = line.split()
        c = getattr(nx, name)
        got = ctypes.sizeof(c) if field == "-" else getattr(c, field).offset
        assert got == int(value), f"{name}.{field}: ctypes {got}, C {value}"
        seen += 1
    assert seen == sum(1 + len(c._fields_) for c in classes)


def test_binding_constants_match_the_header(tmp_path):
    """Every NX_ constant of the binding, and its byte sizes, have the value
    the header gives them (families, status codes, flags, modes, sizes)."""
    from paper_2407_19396_gb300 import navixgb as nx

    pairs = {k: k for k in dir(nx) if k.startswith("NX_") and isinstance(getattr(nx, k), int)}
    pairs.update(OBS_SYM_BYTES="NX_OBS_SYM_BYTES", OBS_RGB_BYTES="NX_OBS_RGB_BYTES", ATLAS_BYTES="NX_ATLAS_BYTES",
                 AGENT_BYTES="NX_AGENT_BYTES")
    lines = ["#include <stdio.h>", '#include "navixgb.h"', "int main(void) {"]
    lines += [f'printf("{py} %lld\\n", (long long)({c}));' for py, c in pairs.items()]
    lines.append("return 0; }")
    src, exe = tmp_path / "consts.c", tmp_path / "consts"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    values = dict(line.split() for line in out.splitlines())
    assert len(values) == len(pairs) >= 35
    for py, v in values.items():
        assert getattr(nx, py) == int(v), f"{py}: binding {getattr(nx, py)}, header {v}"
    assert sorted(nx.FAMILIES.values()) == list(range(nx.NX_N_FAMILIES))
