"""Host logic of bench.py that needs no GPU: the argument defaults the timing
rules ask for, the algorithmic byte and FLOP counts the rooflines divide by,
and the rule that a recorded DRAM traffic figure is reported only for the
kernel source it was measured on."""
import json
import os

import bench


def test_defaults_run_one_gpu_with_enough_warmup():
    a = bench.parse_args([])
    assert a.gpus == 1 and a.impl == "ours"
    assert a.warmup >= 3 and a.steps >= 1
    assert (a.width, a.height) == (800, 800)


def test_algorithmic_bytes_and_flop_per_unit():
    # (bytes per sample, bytes per ray): packed write + offsets; t0, t1, sigma, rgb
    # read + per-ray outputs; the same read + gradients written + upstream gradients
    assert bench.BYTES == {"march": (12, 32), "render_fwd": (24, 32), "render_bwd": (40, 28)}
    assert bench.count_pass_flop(1000, 8) == 1000 * (11 * 8 + 14)
    assert sum(bench.KERNELS_PER_STEP.values()) == 11  # seven march kernels with a field + four


def test_recorded_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2305_04966_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = csrc / "k.cu"
    src.write_text("__global__ void k() {}\n")
    rec = {"stage_x": {"source": "k.cu", "source_sha": bench.src_sha(str(src)), "dram_bytes_per_sample": 2.5,
                       "dram_bytes_per_ray": 100.0}}
    tf = tmp_path / "traffic.json"
    tf.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tf))
    assert bench.recorded_traffic("stage_x", 1000, 10) == 2.5 * 1000 + 100.0 * 10
    assert bench.recorded_traffic("stage_y", 1000, 10) is None
    src.write_text("__global__ void k() { /* changed */ }\n")
    assert bench.recorded_traffic("stage_x", 1000, 10) is None  # measured on another version


def test_committed_traffic_records_name_existing_sources():
    recs = json.load(open(bench.TRAFFIC_FILE))
    for stage, r in recs.items():
        path = os.path.join(bench.ROOT, "paper_2305_04966_gb300", "csrc", r["source"])
        assert os.path.exists(path), stage
        assert r["dram_bytes_per_sample"] >= 0 and r.get("dram_bytes_per_ray", 0.0) >= 0


def test_reference_arm_prints_one_json_line():
    """`bench.py --impl reference` times the CPU oracle on the host (no GPU) and
    prints one JSON line with the arm's metric, unit, e2e and CPU-baseline keys."""
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--width", "160", "--height", "160"], capture_output=True, text=True,
                       timeout=600, cwd=bench.ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["metric"] == bench.METRIC and rec["unit"] == "rays/s"
    assert rec["value"] > 0 and rec["higher_is_better"] is True and rec["n_gpus"] == 1
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["cpu_baseline"]["cores"] >= 1
    assert rec["e2e"]["h2d_bytes_per_step"] == 0 and rec["e2e"]["value"] == rec["value"]
