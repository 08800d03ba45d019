"""Host-side pieces of bench.py that its JSON line depends on: the machine-read
fields of the committed ncu summaries (valid only for the kernel sources
they were captured from)."""
import os

import bench


def _summary(tmp_path, workload, lines):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / f"step_kernel_{workload}.md").write_text("\n".join(lines) + "\n")
    return str(tmp_path)


def test_profile_fields_valid_only_for_the_captured_sources(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()  # of the committed kernel sources
    root = _summary(tmp_path, "w", [f"- kernel_source_hash: `{h}`", "- dram_bytes_per_full_launch: `23442944`",
                                    "- warp_instructions_per_env_step: `183.64` (a note after the value)"])
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", root)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: h)
    assert bench.ncu_traffic("w") == 23442944.0
    assert bench.profile_field("w", "warp_instructions_per_env_step") == 183.64
    assert bench.profile_field("w", "missing_field") is None
    assert bench.ncu_traffic("no_such_workload") is None
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 16)  # sources changed since the capture
    assert bench.ncu_traffic("w") is None
    assert bench.profile_field("w", "warp_instructions_per_env_step") is None
    monkeypatch.setattr(bench, "ROOT", real_root)
