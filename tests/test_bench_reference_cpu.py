"""bench.py's reference arm on CPU: the oracle's JSON line keeps the
benchmark contract (one line, the agreed keys, the oracle as its baseline)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line_on_the_small_cube():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--workload", "cube16b_512x512_K3"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "cube16b_512x512_K3"


def test_a_failing_extra_measurement_is_reported_not_raised():
    sys.path.insert(0, ROOT)
    import bench

    def boom(x):
        raise RuntimeError(f"extra failed on {x}")

    r = bench._extra(boom, 3)
    assert r == {"error": "RuntimeError: extra failed on 3"}
    assert bench._extra(lambda a, b=2: a * b, 5, b=4) == 20


def test_cpu_baselines_give_one_core_and_all_cores():
    """The oracle baselines beside the GPU line: the whole-page fit plus a
    band of the per-pixel work, on every host core and on one."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from synth import batch_workloads, make_workload

    try:
        w = make_workload(2024, 12, 160, 136, 3, (500, 400, 300), 2, separation=(1.0, 4.0), both=False)
        d = bench._both_baselines(w, 0.5)
        assert d["kind"] == "oracle" and d["value"] > 0 and d["unit"] == "Mpixel/s"
        assert d["cores"] == bench._host_cores()
        assert d["one_core"]["cores"] == 1 and d["one_core"]["value"] > 0
        assert d["ms_per_page"] >= d["fit_ms"] > 0
        ws = batch_workloads(3, sizes=[128, 256])
        b = bench._batch_baselines(ws)
        assert b["value"] > 0 and b["cores"] == bench._host_cores() and b["one_core"]["cores"] == 1
    finally:
        oracle.use_threads(1)
