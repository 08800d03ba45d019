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


def test_reference_arm_under_torchrun_prints_one_line_from_rank_zero():
    """bench.py --impl reference launched as two ranks the way the multi-GPU
    runs launch it (gloo here, no GPU): rank 0 alone times the oracle and
    prints the one JSON line; every rank exits 0."""
    import json
    import socket
    import subprocess
    import sys

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(bench.ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3", "--workload", "empty5"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0 and d["unit"] == "env-steps/s"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
