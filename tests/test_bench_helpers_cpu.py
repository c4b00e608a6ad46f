"""Host helpers of bench.py (no GPU): split bookkeeping of the roofline line
and the matching of committed ncu counters to a run."""
import json
import os

import bench


def test_split_lengths_ignore_the_z_order():
    assert bench.split_lengths((160, 1, 80, 1, 16)) == bench.split_lengths((80, 1, 16, 1, 160)) == [160, 80, 16]
    assert bench.split_lengths((86, 2, 0, 0, 84)) == [86, 86, 84]
    assert bench.split_lengths((4, 16, 0, 0, 0)) == [4] * 16


def test_partial_floats_per_column_count_node_planes():
    # a segment of len planes keeps len / 2 + 1 node planes of 3 x (ox/2 + 1) x (oy/2 + 1)
    # entries, for the library's ox x oy output tile (3 x 15 x 7 for 28 x 12)
    from paper_1812_06765_gb300 import build, _lib
    build.build()
    ox, oy, _ = _lib.reg_fused_tile_shape()
    entries = 3 * (ox // 2 + 1) * (oy // 2 + 1)
    assert bench.split_partial_floats_per_column((160, 1, 80, 1, 16)) == (81 + 41 + 9) * entries
    assert bench.split_partial_floats_per_column((4, 16, 0, 0, 0)) == 16 * 3 * entries
    assert bench.split_partial_floats_per_column((0, 0, 0, 0, 70)) == 36 * entries


def test_committed_profile_needs_source_workload_and_split(tmp_path, monkeypatch):
    (tmp_path / "profiles").mkdir()
    entry = {"source_digest": "abc", "workload": "c2_ct256_4level", "fused_split": [160, 1, 80, 1, 16],
             "dram_bytes_per_launch_full_size": 1, "warp_instructions_per_launch": 2}
    with open(os.path.join(tmp_path, "profiles", "traffic.json"), "w") as f:
        json.dump({"objective_pass_fused": entry}, f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    get = bench.committed_profile
    assert get("objective_pass_fused", "abc", "c2_ct256_4level", (80, 1, 16, 1, 160))["warp_instructions_per_launch"] == 2
    assert get("objective_pass_fused", "abd", "c2_ct256_4level", (160, 1, 80, 1, 16)) == {}   # source changed
    assert get("objective_pass_fused", "abc", "c3_lung256x256x112_4level", (160, 1, 80, 1, 16)) == {}
    assert get("objective_pass_fused", "abc", "c2_ct256_4level", (86, 2, 0, 0, 84)) == {}   # other tiling
    assert get("objective_pass_multipass", "abc", "c2_ct256_4level", (160, 1, 80, 1, 16)) == {}


def test_source_digest_follows_the_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "a.cu").write_text("x")
    d1 = bench.source_digest(["a.cu"])
    (tmp_path / "a.cu").write_text("y")
    assert bench.source_digest(["a.cu"]) != d1


def _run_bench(args, env_extra=None):
    import subprocess
    import sys
    env = dict(os.environ, **(env_extra or {}))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, capture_output=True, text=True,
                          timeout=600, env=env, cwd=root)


def test_reference_arm_line_on_the_64cube_workload():
    out = _run_bench(["--impl", "reference", "--config", "0", "--steps", "2", "--warmup", "1"])
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["steps"] == 2 and line["warmup"] == 1 and line["higher_is_better"] is True
    assert line["value"] > 0 and abs(line["ms_per_step"] - 1000.0 / line["value"]) < 1e-6 * line["ms_per_step"]
    assert line["config"]["workload"] == "c0_64cube_1level" and line["dtype"] == "f64"
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"] and cpu["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_runs_on_rank_0_only():
    out = _run_bench(["--impl", "reference", "--config", "0", "--steps", "1", "--warmup", "1"],
                     {"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_cpu_oracle_sample_runs_for_its_time_budget():
    from synth import CONFIGS, make_pair
    c = CONFIGS[0]
    p = make_pair(0, dims=(16, 16, 16))
    rate, n, el, cores = bench.cpu_oracle_rate(p, c, 0.5)
    assert el >= 0.5 and n >= 1 and abs(rate - n / el) < 1e-9 * rate and cores >= 1
