"""Benchmark: CVA fit + projection + 8-bit rescale on a synthetic manuscript cube.

One step = one pass of the whole path on one cube already resident in HBM:
class moments of the training pixels, FP64 scatter and eigensolve, training
ranges, and the fused projection + 8-bit rescale of every pixel onto the top
canonical variates.  ``value`` is Mpixel/s of whole steps (all ranks), timed
with CUDA events on the launching stream; ``e2e`` repeats the step through the
Python binding with the cube and labels copied from pinned host memory and the
8-bit images copied back inside the timed region.

``--impl reference`` times the FP64 CPU oracle instead, on a bounded sample
of each step, on the host cores.

Multi-GPU (torchrun): every rank processes its own page (pages are
independent problems), no data-path collective; the timing is the max over
ranks and the value counts all ranks' pixels.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "CVA Mpixel/s (fit+project) & % HBM roofline; mixed vs FP64 path at ≤1e-4 err"
UNIT = "Mpixel/s"
DEFAULT_WORKLOAD = "cube23b_4096x4096_K4"
L2_BYTES = 126 * 1024 * 1024

# DRAM traffic of one k_project_v8<3, u8> launch on the 23-band 4096 x 4096
# cube, from ncu (dram__bytes_read.sum + dram__bytes_write.sum), valid while
# the projection source hashes to PROJECT_SRC_SHA256; null otherwise.
PROJECT_TRAFFIC_BYTES = 771801600 + 43983616
PROJECT_SRC_SHA256 = "19942c0bd60a130e690ad176aeba4ba2f87cd1c49aeac2c29a6f5689203c0c1c"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP64-form comparison")
    ap.add_argument("--no-forms", action="store_true", help="batch workload: skip the per-page forms")
    ap.add_argument("--pages", type=int, default=64, help="batch workload: number of pages (64 = the benchmark)")
    ap.add_argument("--split", action="store_true",
                    help="under torchrun: one page split by rows over the ranks (one all-reduce of the class "
                         "moments and one of the ranges per step; strong scaling) instead of a page per rank")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other configurations (small page, large cube, 64-page batch) in the line")
    return ap.parse_args()


def _dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(dist, value, device):
    """The largest of every rank's value (the step time the job is charged)."""
    import torch

    if dist is None:
        return value
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(world, pixels_per_rank, ms):
    """Whole-job throughput (Mpixel/s): every rank's pixels over the slowest
    rank's step time (weak scaling: each rank fits and projects its own page)."""
    return world * pixels_per_rank / (ms * 1e-3) / 1e6


def _workload(name, rank):
    from synth import named_workload

    return named_workload(name)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _src_hash():
    with open(os.path.join(ROOT, "paper_1612_06457_gb300", "csrc", "project.cu"), "rb") as f:
        h = hashlib.sha256(f.read())
    with open(os.path.join(ROOT, "paper_1612_06457_gb300", "csrc", "cva_internal.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        loaded = [r for r in rows if (num(r[4]) or 0) > 0] or rows
        sm = [num(r[1]) for r in loaded if num(r[1]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": num(rows[0][2]),
                "reasons": reasons, "samples": len(loaded),
                "power_w_max": max((num(r[3]) or 0) for r in loaded)}


def _host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # noqa: BLE001 - platforms without affinity masks
        return os.cpu_count() or 1


class OracleTimer:
    """The FP64 oracle on one page with a given number of threads.  The fit
    (class statistics and scatter of the training pixels, eigensolve, and the
    training pixels' scores for the training-score range) is timed as one
    piece on the whole page; the per-pixel part (projection and 8-bit
    rescale) is timed on bands of image rows and scaled to the page."""

    def __init__(self, w, threads):
        import oracle

        self.oracle = oracle
        self.w = w
        self.threads = oracle.use_threads(threads)
        self.f = None
        self.rng = None

    def fit(self):
        import numpy as np

        o, w = self.oracle, self.w
        t0 = time.perf_counter()
        f = o.fit(w.cube, w.labels, w.K)
        tr = np.flatnonzero(w.labels.reshape(-1))
        sub = w.cube.reshape(w.B, -1)[:, tr].reshape(w.B, 1, -1)
        rng = o.range_global(o.project(sub, f["V"], f["mu"], w.k))
        t = time.perf_counter() - t0
        self.f, self.rng = f, rng
        return t

    def band(self, r0, rows, keep=None):
        o, w = self.oracle, self.w
        t0 = time.perf_counter()
        y = o.project(w.cube, self.f["V"], self.f["mu"], w.k, r0 * w.W, (r0 + rows) * w.W)
        u8 = o.to_u8(y, self.rng)
        t = time.perf_counter() - t0
        if keep is not None:
            keep.update(fit=self.f, y=y, u8=u8, rows=rows, r0=r0)
        return t

    def rows_for(self, seconds_per_band):
        """Band height whose projection takes about `seconds_per_band`."""
        rows = min(self.w.H, 16)
        t = self.band(0, rows)
        return int(max(1, min(self.w.H, rows * seconds_per_band / max(t, 1e-6))))


def _cpu_baseline(w, seconds, threads):
    """Mpixel/s of the oracle on the page with `threads` threads, from about
    `seconds` of CPU work: the median of three whole-page fits plus the median
    band time scaled to all rows."""
    T = OracleTimer(w, threads)
    fits = [T.fit() for _ in range(3 if seconds > 2.0 else 1)]
    tf = statistics.median(fits)
    rows = T.rows_for(max(0.05, (seconds - sum(fits)) / 8))
    bands = []
    for i in range(8):
        r0 = (i * 977) % max(1, w.H - rows + 1)
        bands.append(T.band(r0, rows) * w.H / rows)
    tp = statistics.median(bands)
    t = tf + tp
    return {"value": w.P / t / 1e6, "unit": UNIT, "cores": T.threads, "kind": "oracle",
            "ms_per_page": t * 1e3, "fit_ms": tf * 1e3, "per_pixel_ms": tp * 1e3,
            "sample": (f"the oracle's whole-page fit with the training-score range (median of {len(fits)}) plus its "
                       f"projection and 8-bit rescale timed on 8 bands of {rows} of {w.H} rows and scaled to the "
                       f"page, {T.threads} thread(s)")}


REFERENCE_BUDGET_S = 90.0  # wall time of the whole --impl reference run, all steps
CPU_BASELINE_S = 8.0  # CPU work of each oracle baseline beside the GPU line
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e nominal bandwidth, reported beside the measured peak


def run_reference(a):
    """The FP64 oracle on every host core.  Each step is one page: the
    whole-page fit (timed once, median of three) plus the projection and
    8-bit rescale of a band of rows scaled to the page, the band sized so that
    the whole run stays within REFERENCE_BUDGET_S."""
    world, rank, _ = _dist_env()
    if rank != 0:
        return
    w = _workload(a.workload, 0)
    T = OracleTimer(w, _host_cores())
    tf = statistics.median([T.fit() for _ in range(3)])
    n = max(1, a.steps) + a.warmup
    rows = T.rows_for(max(1e-3, (REFERENCE_BUDGET_S - 3 * tf) / n))
    times = []
    for i in range(n):
        r0 = (i * 977) % max(1, w.H - rows + 1)
        tb = T.band(r0, rows) * w.H / rows
        if i >= a.warmup:
            times.append(tf + tb)
    t = statistics.median(times)
    value = w.P / t / 1e6
    sample = (f"each step: the oracle's whole-page fit with the training-score range (timed once, median of 3) "
              f"plus its projection and 8-bit rescale on a band of {rows} of {w.H} rows scaled to the page, "
              f"{T.threads} thread(s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(w),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": T.threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(w):
    return {"workload": w.name, "bands": w.B, "H": w.H, "W": w.W, "classes": w.K,
            "train_pixels": list(w.n_train), "variates": w.k, "range": "training-score (second rescale)",
            "l2": _l2_note(w.cube.nbytes + w.labels.nbytes)}


def _l2_note(nbytes):
    rel = "larger" if nbytes > L2_BYTES else "not larger"
    return f"inputs {rel} than L2 ({nbytes / 1e6:.0f} MB vs {L2_BYTES / 2**20:.0f} MiB)"


def _time_graphs(torch, graphs, stream, steps):
    with torch.cuda.stream(stream):
        for g in graphs:
            g.replay()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(steps):
            for g in graphs:
                g.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _precision_forms(cva, torch, w, m, cube, labels, out, stream, steps=5):
    """The FP64 form of the same step (CVA_PRECISION_FP64: FP64 training range,
    FP64 projection and 8-bit codes) timed the same way, and the mixed form's
    projections and codes against it over every pixel."""
    P = w.P
    y = {}
    u = {}
    res = {"bound": 1e-4}
    for mode, name in ((cva.CVA_PRECISION_FP64, "fp64"), (cva.CVA_PRECISION_MIXED, "mixed")):
        cva.cva_set_precision(m, mode)
        g_fit = torch.cuda.CUDAGraph()
        g_proj = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_fit, stream=stream):
            cva.cva_fit(cube, labels, w.K, m, stream=stream)
        with torch.cuda.graph(g_proj, stream=stream):
            cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, out, stream=stream)
        t = _time_graphs(torch, (g_fit, g_proj), stream, steps)
        res[name] = {"ms_per_step": t, "value": P / (t * 1e-3) / 1e6, "unit": UNIT, "steps": steps}
        u[name] = out.clone()
        yy = torch.empty((w.k, w.H, w.W), dtype=torch.float32, device=cube.device)
        with torch.cuda.stream(stream):
            cva.cva_project(cube, m, w.k, out_f32=yy, stream=stream)
        torch.cuda.synchronize()
        y[name] = yy.reshape(w.k, -1)
    d = (y["mixed"] - y["fp64"]).abs().amax(dim=1) / y["fp64"].abs().amax(dim=1)
    du = (u["mixed"].to(torch.int16) - u["fp64"].to(torch.int16)).abs()
    res["mixed_vs_fp64"] = {"projection_rel_err_max": float(d.max().item()),
                            "projection_rel_err_per_variate": [float(v) for v in d.tolist()],
                            "u8_within_1": float((du <= 1).float().mean().item()),
                            "u8_identical": float((du == 0).float().mean().item()),
                            "pixels": P}
    res["speedup_mixed_over_fp64"] = res["fp64"]["ms_per_step"] / res["mixed"]["ms_per_step"]
    cva.cva_set_precision(m, cva.CVA_PRECISION_MIXED)
    with torch.cuda.stream(stream):
        cva.cva_fit(cube, labels, w.K, m, stream=stream)
        cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, out, stream=stream)
    torch.cuda.synchronize()
    return res


def _extra(fn, *args, **kw):
    """Run one of the line's extra measurements; a failure is reported in the
    line as ``{"error": ...}`` instead of ending the run, so the headline keys
    (value, roofline, e2e, clocks) are always printed."""
    try:
        return fn(*args, **kw)
    except Exception as exc:  # noqa: BLE001 - any failure of an extra is recorded
        return {"error": f"{type(exc).__name__}: {exc}"}


def _time_calls(torch, fn, stream, reps=20):
    """Mean device time of one call of `fn`, replayed as a captured CUDA
    graph (so that a busy host, e.g. while other configs' inputs are being
    drawn, cannot leave gaps between the call's launches); timed eagerly if
    the call cannot be captured."""
    with torch.cuda.stream(stream):
        for _ in range(3):
            fn()
    torch.cuda.synchronize()
    g = None
    try:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            fn()
        torch.cuda.synchronize()
    except Exception:  # noqa: BLE001 - not capturable: eager timing below
        g = None
        torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if g is not None:
        with torch.cuda.stream(stream):
            for _ in range(3):
                g.replay()
    torch.cuda.synchronize()
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            if g is not None:
                g.replay()
            else:
                fn()
    e1.record(stream)
    torch.cuda.synchronize()
    _time_calls.graphed = g is not None
    return e0.elapsed_time(e1) / reps


def _page_stream(cva, torch, w, cube, labels, out, stream, steps):
    """Pages back to back on two streams: page i's fit runs while page i - 1 is
    being projected (a second page of the same recipe, its own model and
    buffers, alternates with the benchmark page so that no two pages in
    flight share data).  Every page is a full fit + fused projection."""
    from synth import make_workload

    w2 = make_workload(1101, w.B, w.H, w.W, w.K, w.n_train, w.k, separation=(1.0, 4.0), both=True)
    cubes = [cube, torch.from_numpy(w2.cube).to(cube.device)]
    labs = [labels, torch.from_numpy(w2.labels).to(cube.device)]
    outs = [out, torch.empty_like(out)]
    models = []
    for _ in range(2):
        mm = cva.Model(w.B, w.K)
        cva.cva_set_variates(mm, w.k)
        models.append(mm)
    streams = [stream, torch.cuda.Stream(device=cube.device)]
    graphs = []
    for i in range(2):
        with torch.cuda.stream(streams[i]):
            cva.cva_fit(cubes[i], labs[i], w.K, models[i], stream=streams[i])
            cva.cva_project_u8(cubes[i], models[i], w.k, cva.CVA_RANGE_TRAINING, outs[i], stream=streams[i])
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=streams[i]):
            cva.cva_fit(cubes[i], labs[i], w.K, models[i], stream=streams[i])
            cva.cva_project_u8(cubes[i], models[i], w.k, cva.CVA_RANGE_TRAINING, outs[i], stream=streams[i])
        graphs.append(g)
    torch.cuda.synchronize()

    def run(n):
        for i in range(n):
            with torch.cuda.stream(streams[i % 2]):
                graphs[i % 2].replay()

    run(4)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(streams[0])
    streams[1].wait_event(e0)
    run(steps)
    done = torch.cuda.Event()
    done.record(streams[1])
    streams[0].wait_event(done)
    e1.record(streams[0])
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    st = [cva.cva_status(mm, stream=streams[i]) for i, mm in enumerate(models)]
    for mm in models:
        mm.close()
    if any(x != cva.CVA_OK for x in st):
        raise SystemExit(f"page stream failed: {st}")
    return {"ms_per_page": ms, "value": w.P / (ms * 1e-3) / 1e6, "unit": UNIT, "pages": steps,
            "how": "two pages of the benchmark recipe alternate on two streams, each page a full fit + fused "
                   "projection through the binding (replayed graphs); a page's fit overlaps the previous "
                   "page's projection"}


def _other_outputs(cva, torch, w, m, cube, stream, peak):
    """The other image paths on the same cube, each timed alone: the FP32
    projection, the third rescale's trimmed range (1 % out of each tail, three
    passes over the projections), and the 8- and 16-bit rescales from FP32."""
    P, k = w.P, w.k
    y = torch.empty((k, w.H, w.W), dtype=torch.float32, device=cube.device)
    r = torch.empty(2 * k, dtype=torch.float32, device=cube.device)
    u8 = torch.empty((k, w.H, w.W), dtype=torch.uint8, device=cube.device)
    u16 = torch.empty((k, w.H, w.W), dtype=torch.uint16, device=cube.device)
    res = {}

    def entry(name, ms, nbytes):
        gbs = nbytes / (ms * 1e-3) / 1e9
        res[name] = {"ms": ms, "alg_bytes": nbytes, "GB/s": gbs, "frac_of_hbm": gbs / peak,
                     "timed": "replayed graph" if getattr(_time_calls, "graphed", False) else "eager calls"}

    entry("project_f32", _time_calls(torch, lambda: cva.cva_project(cube, m, k, out_f32=y, stream=stream), stream),
          P * (2 * w.B + 4 * k))
    entry("percentile_range_1pct", _time_calls(torch, lambda: cva.cva_percentile_range(y, 1.0, m, r, stream=stream),
                                               stream), 3 * 4 * k * P)
    entry("to_u8_given", _time_calls(torch, lambda: cva.cva_to_u8(y, cva.CVA_RANGE_GIVEN, u8, range=r, stream=stream),
                                     stream), 5 * k * P)
    entry("to_u16_given", _time_calls(torch, lambda: cva.cva_to_u16(y, cva.CVA_RANGE_GIVEN, u16, range=r,
                                                                     stream=stream), stream), 6 * k * P)
    t = res["project_f32"]["ms"] + res["percentile_range_1pct"]["ms"] + res["to_u8_given"]["ms"]
    res["third_rescale_u8_image_mpixel_s"] = P / (t * 1e-3) / 1e6
    # principal components of the whole page (exact moments of every pixel
    # on the tensor cores, then the 23 x 23 eigensolve), on a model of its own
    mp = cva.Model(w.B, 2)
    cva.cva_set_variates(mp, k)
    entry("pca_fit_whole_page", _time_calls(torch, lambda: cva.cva_pca_fit(cube, mp, stream=stream), stream),
          P * 2 * w.B)
    F = (w.B + 1 + 7) // 8 * 8
    res["pca_fit_whole_page"]["mma_tflops"] = P * (2 * F) ** 2 * 2 / (res["pca_fit_whole_page"]["ms"] * 1e-3) / 1e12
    mp.close()
    return res


def _errors_vs_oracle(cva, torch, w, m, cube, out, keep, stream):
    """Eigenvalues, canonical vectors (S_w norm), projections and codes of the
    mixed form against the FP64 oracle (projection rows: the oracle's band)."""
    import numpy as np

    f = keep["fit"]
    lam, V, mu, _ = cva.cva_model_get(m, stream=stream)
    r = min(w.K - 1, w.B)
    lam_rel = np.abs(lam[:r] - f["lam"][:r]) / f["lam"][:r]
    Sw = f["Sw"]
    vs = [float(np.sqrt((V[:, j] - f["V"][:, j]) @ Sw @ (V[:, j] - f["V"][:, j]))) for j in range(min(r, w.k))]
    p0, p1 = keep["r0"] * w.W, (keep["r0"] + keep["rows"]) * w.W
    yy = torch.empty((w.k, w.H, w.W), dtype=torch.float32, device=cube.device)
    with torch.cuda.stream(stream):
        cva.cva_project(cube, m, w.k, out_f32=yy, stream=stream)
    torch.cuda.synchronize()
    yg = yy.reshape(w.k, -1)[:, p0:p1].cpu().numpy().astype(np.float64)
    del yy
    yr = keep["y"]
    rel = np.abs(yg - yr).max(axis=1) / np.abs(yr).max(axis=1)
    ug = out.reshape(w.k, -1)[:, p0:p1].cpu().numpy().astype(np.int32)
    du = np.abs(ug - keep["u8"].astype(np.int32))
    return {"eigvals_rel_err": [float(v) for v in lam_rel], "eigvecs_sw_err": vs,
            "projection_rel_err_max": float(rel.max()), "u8_within_1": float((du <= 1).mean()),
            "u8_identical": float((du == 0).mean()), "pixels_compared": int(p1 - p0)}


def _oracle_errors(cva, torch, w, m, cube, out, stream, rows=256):
    """The oracle's fit of the page and a band of its rows, then
    _errors_vs_oracle (not timed)."""
    T = OracleTimer(w, _host_cores())
    T.fit()
    keep = {}
    rows = min(w.H, max(1, rows * 4096 // max(w.W, 1)))
    T.band((w.H - rows) // 2, rows, keep)
    return _errors_vs_oracle(cva, torch, w, m, cube, out, keep, stream)


def _both_baselines(w, seconds):
    """The oracle's Mpixel/s on every host core, with the single-core figure
    beside it."""
    allc = _cpu_baseline(w, seconds / 2, _host_cores())
    allc["one_core"] = _cpu_baseline(w, seconds, 1)
    return allc


# ---------------------------------------------------------------------------
# extra workloads of the line, drawn in the background
# ---------------------------------------------------------------------------

LARGE_WORKLOAD = "cube23b_8192x6144_K6"
SMALL_WORKLOAD = "cube16b_512x512_K3"
BATCH_WORKLOAD = "batch64_uneven"


def _start_extra_workloads(pages):
    """Spawn processes drawing the large cube and the batch's pages (fresh
    interpreters, so starting them after CUDA is initialized is safe; every
    page has its own seed, so they are the same as drawn in order)."""
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor

    from synth import cubes

    pool = ProcessPoolExecutor(max_workers=max(1, min(16, _host_cores() - 1)),
                               mp_context=multiprocessing.get_context("spawn"))
    futs = {"large": pool.submit(cubes.named_workload, LARGE_WORKLOAD),
            "batch": [pool.submit(cubes._batch_page, i, 100300, None) for i in range(pages)]}
    return pool, futs


def _collect_extra_workloads(pool, futs):
    out = {}
    try:
        out["large"] = futs["large"].result()
    except Exception as exc:  # noqa: BLE001 - reported in the line
        out["large"] = exc
    try:
        out["batch"] = [f.result() for f in futs["batch"]]
    except Exception as exc:  # noqa: BLE001 - reported in the line
        out["batch"] = exc
    pool.shutdown()
    return out


def _page_config(cva, torch, w, dev, steps, peak):
    """One page of another configuration: fit + fused projection to 8 bits
    (training-score range) as two replayed graphs, timed like the headline
    step; the projection launch timed by events around its graph."""
    cube = torch.from_numpy(w.cube).to(dev)
    labels = torch.from_numpy(w.labels).to(dev)
    out = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=dev)
    m = cva.Model(w.B, w.K)
    cva.cva_model_reserve(m, int(sum(w.n_train)) + 1024)
    cva.cva_set_variates(m, w.k)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        cva.cva_fit(cube, labels, w.K, m, stream=stream)
        cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, out, stream=stream)
    torch.cuda.synchronize()
    st = cva.cva_status(m, stream=stream)
    if st != cva.CVA_OK:
        raise RuntimeError(f"fit failed: {cva.cva_strerror(st)}")
    g_fit = torch.cuda.CUDAGraph()
    g_proj = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_fit, stream=stream):
        cva.cva_fit(cube, labels, w.K, m, stream=stream)
    with torch.cuda.graph(g_proj, stream=stream):
        cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, out, stream=stream)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for _ in range(3):
            g_fit.replay()
            g_proj.replay()
    pa = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    pb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for i in range(steps):
            g_fit.replay()
            pa[i].record(stream)
            g_proj.replay()
            pb[i].record(stream)
        t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / steps
    proj_ms = statistics.mean(pa[i].elapsed_time(pb[i]) for i in range(steps))
    alg = w.P * (2 * w.B + w.k)
    achieved = alg / (proj_ms * 1e-3) / 1e9
    res = {"value": w.P / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "fit_ms": ms - proj_ms,
           "steps": steps, "dtype": "f32", "config": _config(w),
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "kernel": "k_project_v8 (fused projection + u8)",
                        "alg_bytes_per_launch": alg, "launch_ms": proj_ms}}
    res["err_vs_oracle"] = _extra(_oracle_errors, cva, torch, w, m, cube, out, stream)
    m.close()
    return res


def _ragged_page(cva, torch, w, dev, steps, peak):
    """The benchmark page cropped to odd sides (H - 3) x (W - 1), so that its
    pixel count is not a multiple of 8 and no band starts on 16 bytes: the
    same fit + fused projection timed like the headline step."""
    import dataclasses

    import numpy as np

    H, W = w.H - 3, w.W - 1
    lab = np.ascontiguousarray(w.labels[:H, :W])
    w2 = dataclasses.replace(w, name=f"{w.name}_cropped_{H}x{W}", cube=np.ascontiguousarray(w.cube[:, :H, :W]),
                             labels=lab, classmap=np.ascontiguousarray(w.classmap[:H, :W]),
                             n_train=tuple(int((lab == c + 1).sum()) for c in range(w.K)))
    res = _page_config(cva, torch, w2, dev, steps, peak)
    res["pixels_mod_8"] = w2.P % 8
    res["roofline"]["kernel"] = "k_project_r8 (ragged fused projection + u8)"
    return res


def run_ours(a):
    import numpy as np
    import torch

    import paper_1612_06457_gb300 as cva

    world, rank, local = _dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    cva.load()

    w = _workload(a.workload, rank)
    cube_h = torch.from_numpy(w.cube).pin_memory()
    lab_h = torch.from_numpy(w.labels).pin_memory()
    cube = cube_h.to(dev)
    labels = lab_h.to(dev)
    out = torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=dev)
    m = cva.Model(w.B, w.K)
    cva.cva_set_variates(m, w.k)
    stream = torch.cuda.Stream(device=dev)
    P = w.P

    def fit():
        cva.cva_fit(cube, labels, w.K, m, stream=stream)

    def project():
        cva.cva_project_u8(cube, m, w.k, cva.CVA_RANGE_TRAINING, out, stream=stream)

    with torch.cuda.stream(stream):
        fit()
        project()
    torch.cuda.synchronize()
    st = cva.cva_status(m, stream=stream)
    if st != cva.CVA_OK:
        raise SystemExit(f"fit failed: {cva.cva_strerror(st)}")

    # the step's launches are captured once into two CUDA graphs (fit, then
    # projection); events recorded on the stream between the replays time the
    # projection kernel inside the timed region
    g_fit = torch.cuda.CUDAGraph()
    g_proj = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_fit, stream=stream):
        fit()
    with torch.cuda.graph(g_proj, stream=stream):
        project()
    torch.cuda.synchronize()

    def step(ev_a=None, ev_b=None):
        g_fit.replay()
        if ev_a is not None:
            ev_a.record(stream)
        g_proj.replay()
        if ev_b is not None:
            ev_b.record(stream)

    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    if rank == 0:
        sampler.start()
    with torch.cuda.stream(stream):
        for _ in range(a.warmup):
            step()
    pa = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    pb = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for i in range(a.steps):
            step(pa[i], pb[i])
        t1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if rank == 0 else None
    ms = t0.elapsed_time(t1) / a.steps
    proj_ms = statistics.mean(pa[i].elapsed_time(pb[i]) for i in range(a.steps))
    ms = _max_over_ranks(dist, ms, dev)

    # end to end through the binding: every step copies its cube and labels
    # from pinned host memory, fits, projects and copies the 8-bit images back.
    # Two buffer sets and three streams let the host-to-device copy of step
    # i + 1 and the device-to-host copy of step i - 1 run under the compute of
    # step i (the copies are bound by the host link, ~0.2 TB/s here).
    e2e_steps = a.e2e_steps if a.e2e_steps is not None else max(3, min(a.steps, 20))
    out_h = [torch.empty((w.k, w.H, w.W), dtype=torch.uint8).pin_memory() for _ in range(2)]
    cube_e = [torch.empty_like(cube) for _ in range(2)]
    lab_e = [torch.empty_like(labels) for _ in range(2)]
    out_e = [torch.empty_like(out) for _ in range(2)]
    h2d = torch.cuda.Stream(device=dev)
    d2h = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    computed = [torch.cuda.Event() for _ in range(2)]
    drained = [torch.cuda.Event() for _ in range(2)]
    for b in range(2):
        computed[b].record(stream)
        drained[b].record(d2h)

    def e2e_step(i):
        b = i % 2
        h2d.wait_event(computed[b])  # step i - 2 has finished reading this buffer set
        with torch.cuda.stream(h2d):
            cube_e[b].copy_(cube_h, non_blocking=True)
            lab_e[b].copy_(lab_h, non_blocking=True)
        copied[b].record(h2d)
        stream.wait_event(copied[b])
        stream.wait_event(drained[b])  # the images of step i - 2 have left the device
        cva.cva_fit(cube_e[b], lab_e[b], w.K, m, stream=stream)
        cva.cva_project_u8(cube_e[b], m, w.k, cva.CVA_RANGE_TRAINING, out_e[b], stream=stream)
        computed[b].record(stream)
        d2h.wait_event(computed[b])
        with torch.cuda.stream(d2h):
            out_h[b].copy_(out_e[b], non_blocking=True)
        drained[b].record(d2h)

    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(h2d)
    for i in range(e2e_steps):
        e2e_step(i)
    for b in range(2):
        d2h.wait_event(drained[b])
    e1.record(d2h)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_ms = _max_over_ranks(dist, e2e_ms, dev)
    st = cva.cva_status(m, stream=stream)
    if st != cva.CVA_OK:
        raise SystemExit(f"fit failed during timing: {cva.cva_strerror(st)}")
    del cube_e, lab_e, out_e

    # the other configurations' pages are drawn by spawn processes from here
    # on (not during the timed regions above: their host load would show in
    # the graph launches and the host copies)
    extras = None
    if rank == 0 and world == 1 and not a.no_extras:
        extras = _start_extra_workloads(a.pages)

    precision = None
    if rank == 0 and not a.no_precision:
        precision = _extra(_precision_forms, cva, torch, w, m, cube, labels, out, stream)
        cva.cva_set_precision(m, cva.CVA_PRECISION_MIXED)
    others = None
    if rank == 0 and not a.no_precision:
        others = _extra(_other_outputs, cva, torch, w, m, cube, stream, _peaks()[0])
        others["page_stream"] = _extra(_page_stream, cva, torch, w, cube, labels, out, stream,
                                       max(20, min(a.steps, 200)))
        others["ragged_page"] = _extra(_ragged_page, cva, torch, w, dev, max(20, min(a.steps, 200)), _peaks()[0])

    if rank == 0:
        peak, peak_kind = _peaks()
        alg_bytes = P * (2 * w.B + w.k)
        achieved = alg_bytes / (proj_ms * 1e-3) / 1e9
        traffic = PROJECT_TRAFFIC_BYTES if (PROJECT_SRC_SHA256 == _src_hash() and w.name == DEFAULT_WORKLOAD) else None
        # reset, label scan, gather + moments, eigensolve, training range (one
        # per 8 variates), projection (one per 8 variates)
        chunks = (w.k + 7) // 8
        launches_per_step = 4 + 2 * chunks
        line = {
            "metric": METRIC, "value": _job_value(world, P, ms), "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(w),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "k_project_v8 (fused projection + u8)",
                         "peak_kind": peak_kind, "alg_bytes_per_launch": alg_bytes,
                         "launch_ms": proj_ms, "nominal_peak": HBM_NOMINAL_GBS,
                         "frac_of_nominal": achieved / HBM_NOMINAL_GBS},
            "e2e": {"value": _job_value(world, P, e2e_ms), "unit": UNIT,
                    "h2d_bytes_per_step": int(w.cube.nbytes + w.labels.nbytes),
                    "d2h_bytes_per_step": int(out_h[0].numel()), "ms_per_step": e2e_ms, "steps": e2e_steps,
                    "overlap": "copies of neighbouring steps run under the compute (two buffer sets)"},
            "gpu_launches": launches_per_step * a.steps,
            "clocks": clocks,
            "fit_ms": ms - proj_ms,
            "precision": precision,
            "other_outputs": others,
        }

        # the other configurations, each on its own page(s)
        configs = None
        if extras is not None:
            from synth import named_workload

            drawn = _collect_extra_workloads(*extras)
            cfg_steps = max(20, min(a.steps, 200))
            configs = {}
            configs[SMALL_WORKLOAD] = _extra(_page_config, cva, torch, named_workload(SMALL_WORKLOAD), dev,
                                             cfg_steps, peak)
            large = drawn["large"]
            configs[LARGE_WORKLOAD] = (_extra(_page_config, cva, torch, large, dev, max(10, cfg_steps // 4), peak)
                                       if not isinstance(large, Exception)
                                       else {"error": f"{type(large).__name__}: {large}"})
            batch = drawn["batch"]
            configs[BATCH_WORKLOAD] = (_extra(_batch_measure, cva, torch, batch, dev, max(10, cfg_steps // 4),
                                              forms=("mixed",))
                                       if not isinstance(batch, Exception)
                                       else {"error": f"{type(batch).__name__}: {batch}"})
            line["configs"] = configs
            torch.cuda.empty_cache()

        # the oracle last, with no other work on the host cores
        if not a.no_cpu_baseline and world == 1:
            errs = _extra(_oracle_errors, cva, torch, w, m, cube, out, stream)
            if precision is not None:
                precision["err_vs_oracle"] = errs
            else:
                line["err_vs_oracle"] = errs
            line["cpu_baseline"] = _extra(_both_baselines, w, CPU_BASELINE_S)
            if configs is not None:
                if "error" not in configs[SMALL_WORKLOAD]:
                    configs[SMALL_WORKLOAD]["cpu_baseline"] = _extra(_both_baselines, named_workload(SMALL_WORKLOAD),
                                                                     2.0)
                if "error" not in configs[LARGE_WORKLOAD]:
                    configs[LARGE_WORKLOAD]["cpu_baseline"] = _extra(_both_baselines, drawn["large"],
                                                                     CPU_BASELINE_S)
                if "error" not in configs[BATCH_WORKLOAD]:
                    configs[BATCH_WORKLOAD]["cpu_baseline"] = _extra(_batch_baselines, drawn["batch"])
        print(json.dumps(line), flush=True)
    m.close()
    if dist is not None:
        dist.destroy_process_group()


def _batch_config(ws):
    P = sum(w.P for w in ws)
    nb = sum(w.cube.nbytes + w.labels.nbytes for w in ws)
    return {"workload": BATCH_WORKLOAD, "pages": len(ws), "pixels": P,
            "bands": [min(w.B for w in ws), max(w.B for w in ws)],
            "sides": [min(min(w.H, w.W) for w in ws), max(max(w.H, w.W) for w in ws)],
            "classes": [min(w.K for w in ws), max(w.K for w in ws)],
            "train_pixels": sum(sum(w.n_train) for w in ws), "variates": "K-1 per page",
            "range": "training-score (second rescale)",
            "l2": _l2_note(nb)}


def _batch_cpu_time(ws, threads, rows=8):
    """Oracle seconds for the whole batch with `threads` threads: every
    page's fit, plus its projection and 8-bit rescale on a band of `rows`
    rows scaled to the page."""
    t = 0.0
    used = 1
    for w in ws:
        T = OracleTimer(w, threads)
        used = T.threads
        t += T.fit()
        r = min(rows, w.H)
        t += T.band((w.H - r) // 2, r) * w.H / r
    return t, used


def _batch_baselines(ws):
    P = sum(w.P for w in ws)
    res = {}
    for key, threads in (("all", _host_cores()), ("one", 1)):
        t, used = _batch_cpu_time(ws, threads)
        res[key] = {"value": P / t / 1e6, "unit": UNIT, "cores": used, "kind": "oracle",
                    "ms_per_batch": t * 1e3,
                    "sample": "every page's whole fit with the training-score range, plus its projection and 8-bit "
                              "rescale on a band of 8 rows scaled to the page, summed over the batch"}
    out = res["all"]
    out["one_core"] = res["one"]
    return out


def _batch_launches(ws):
    """Kernel launches of one batched call on these pages: the set-up (24
    pages a launch) and page-table fill, the six fit passes (label counts,
    pool scan, compaction, gather + moments, eigensolves, training ranges),
    one batched projection per distinct variate count, and the single-page
    projection of each page the batched kernel does not take (pixel count not
    a multiple of 8; the pages are allocated by torch, so 16-byte aligned)."""
    n = len(ws)
    per_k = len({w.k for w in ws if w.P % 8 == 0})
    ragged = sum(1 for w in ws if w.P % 8 != 0)
    return (n + 23) // 24 + 1 + 6 + per_k + ragged


def _batch_measure(cva, torch, ws, dev, steps, forms=("mixed", "fp64"), warmup=3, sampler=None):
    """The batched form on the pages `ws`: autotune, then the whole batch (one
    graph) and its projection pass timed by CUDA events; the same pages
    through the single-page entry points one after another (`forms`); end to
    end from pinned host memory."""
    P = sum(w.P for w in ws)
    host = [(torch.from_numpy(w.cube).pin_memory(), torch.from_numpy(w.labels).pin_memory()) for w in ws]
    pages = [(c.to(dev), l.to(dev), w.K, w.k, torch.empty((w.k, w.H, w.W), dtype=torch.uint8, device=dev))
             for (c, l), w in zip(host, ws)]
    ntrain = sum(sum(w.n_train) for w in ws)
    b = cva.Batch(len(ws), P, int(ntrain * 1.05) + 1024)
    stream = torch.cuda.Stream(device=dev)
    tuned = cva.cva_batch_tune(b, pages, stream=stream)
    with torch.cuda.stream(stream):
        cva.cva_fit_project_batched(b, pages, stream=stream)
    torch.cuda.synchronize()
    st = cva.cva_batch_status(b, len(ws), stream=stream)
    if (st != cva.CVA_OK).any():
        raise RuntimeError(f"batch failed: {st.tolist()}")
    g_step = torch.cuda.CUDAGraph()
    g_proj = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g_step, stream=stream):
        cva.cva_fit_project_batched(b, pages, stream=stream)
    with torch.cuda.graph(g_proj, stream=stream):
        cva.cva_project_batched(b, pages, stream=stream)
    torch.cuda.synchronize()

    if sampler is not None:
        sampler.start()
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            g_step.replay()
    ms = _time_graphs(torch, (g_step,), stream, steps)
    clocks = sampler.stop() if sampler is not None else None
    proj_ms = _time_graphs(torch, (g_proj,), stream, steps)

    # the same pages one after another through the single-page entry points
    # (mixed form, then the FP64 form), each captured as one graph
    res_forms = {}
    for name in forms:
        mode = cva.CVA_PRECISION_MIXED if name == "mixed" else cva.CVA_PRECISION_FP64
        fsteps = max(3, steps // 4) if name == "mixed" else 3
        models = []
        outs = []
        for w, p in zip(ws, pages):
            mm = cva.Model(w.B, w.K)
            cva.cva_set_variates(mm, w.k)
            cva.cva_set_precision(mm, mode)
            models.append(mm)
            outs.append(torch.empty_like(p[4]))
        with torch.cuda.stream(stream):
            for mm, w, p, o in zip(models, ws, pages, outs):
                cva.cva_fit(p[0], p[1], w.K, mm, stream=stream)
                cva.cva_project_u8(p[0], mm, w.k, cva.CVA_RANGE_TRAINING, o, stream=stream)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for mm, w, p, o in zip(models, ws, pages, outs):
                cva.cva_fit(p[0], p[1], w.K, mm, stream=stream)
                cva.cva_project_u8(p[0], mm, w.k, cva.CVA_RANGE_TRAINING, o, stream=stream)
        t = _time_graphs(torch, (g,), stream, fsteps)
        same = all(torch.equal(o, p[4]) for o, p in zip(outs, pages)) if name == "mixed" else None
        res_forms["per_page_" + name] = {"ms_per_step": t, "value": P / (t * 1e-3) / 1e6, "unit": UNIT,
                                         "steps": fsteps, "identical_images": same}
        del g
        for mm in models:
            mm.close()

    # end to end: pinned host -> device, batch, images -> host
    outs_h = [torch.empty(p[4].shape, dtype=torch.uint8).pin_memory() for p in pages]
    e2e_steps = max(2, min(steps, 5))

    def e2e_step():
        with torch.cuda.stream(stream):
            for (c_h, l_h), p in zip(host, pages):
                p[0].copy_(c_h, non_blocking=True)
                p[1].copy_(l_h, non_blocking=True)
            cva.cva_fit_project_batched(b, pages, stream=stream)
            for o_h, p in zip(outs_h, pages):
                o_h.copy_(p[4], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps

    peak, peak_kind = _peaks()
    alg = sum(w.P * (2 * w.B + w.k) for w in ws)
    achieved = alg / (proj_ms * 1e-3) / 1e9
    res = {
        "value": P / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms, "steps": steps, "warmup": warmup,
        "dtype": "f32", "config": _batch_config(ws),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "kernel": "kb_project_v8 (batched fused projection + u8)",
                     "peak_kind": peak_kind, "alg_bytes_per_launch": alg, "launch_ms": proj_ms,
                     "nominal_peak": HBM_NOMINAL_GBS, "frac_of_nominal": achieved / HBM_NOMINAL_GBS},
        "e2e": {"value": P / (e2e_ms * 1e-3) / 1e6, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(w.cube.nbytes + w.labels.nbytes for w in ws)),
                "d2h_bytes_per_step": int(sum(o.numel() for o in outs_h)), "ms_per_step": e2e_ms,
                "steps": e2e_steps},
        "gpu_launches": _batch_launches(ws) * steps,
        "clocks": clocks,
        "autotuned": {"groups_per_item": tuned[0], "ctas_per_sm": tuned[1]},
        "forms": res_forms,
    }
    for name in res_forms:
        res["speedup_over_" + name] = res_forms[name]["ms_per_step"] / ms
    b.close()
    del pages, host
    return res


def run_batch_bench(a):
    import torch

    import paper_1612_06457_gb300 as cva
    from synth import batch_workloads

    world, rank, local = _dist_env()
    if rank != 0:
        return
    ws = batch_workloads(a.pages, workers=_host_cores())
    if a.impl == "reference":
        ts = []
        used = 1
        for i in range(a.warmup + a.steps):
            t, used = _batch_cpu_time(ws, _host_cores())
            if i >= a.warmup:
                ts.append(t)
        t = statistics.median(ts)
        v = sum(w.P for w in ws) / t / 1e6
        sample = ("every page's whole fit with the training-score range, plus its projection and 8-bit rescale on "
                  "a band of 8 rows scaled to the page, summed over the batch")
        print(json.dumps({"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
                          "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
                          "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": _batch_config(ws),
                          "cpu_baseline": {"value": v, "unit": UNIT, "cores": used, "kind": "oracle",
                                           "sample": sample},
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
              flush=True)
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cva.load()
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    res = _batch_measure(cva, torch, ws, dev, a.steps,
                         forms=() if a.no_forms else ("mixed", "fp64"), warmup=a.warmup, sampler=sampler)
    line = {"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic"}
    line.update(res)
    if not a.no_cpu_baseline:
        line["cpu_baseline"] = _batch_baselines(ws)
    print(json.dumps(line), flush=True)


def run_split_bench(a):
    """One page split by rows over the ranks (paper_1612_06457_gb300/split.py):
    every step each rank finds its band's class moments, the ranks sum them
    (NCCL all-reduce of int64), finish the same fit, merge the training-score
    ranges and project their bands.  Wall time per step, bracketed by a
    barrier and a device synchronization, max over ranks; value = the page's
    pixels / that time (strong scaling: the work is fixed as N grows)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_1612_06457_gb300 as cva
    from paper_1612_06457_gb300 import split

    world, rank, local = _dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    cva.load()
    w = _workload(a.workload, 0)
    r0, r1 = split.row_band(w.H, world, rank)
    cube = torch.from_numpy(np.ascontiguousarray(w.cube[:, r0:r1])).to(dev)
    labels = torch.from_numpy(np.ascontiguousarray(w.labels[r0:r1])).to(dev)
    out = torch.empty((w.k, r1 - r0, w.W), dtype=torch.uint8, device=dev)
    part = split.PagePart(cube, labels, w.K, w.k)

    def step():
        if world > 1:
            split.run_split(part, out)
        else:
            mom, _ = part.moments()
            rng, _ = part.fit(mom)
            part.project(rng, out)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = (time.perf_counter() - t0) * 1e3 / a.steps
    ms = _max_over_ranks(dist if world > 1 else None, ms, dev)
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": w.P / (ms * 1e-3) / 1e6, "unit": UNIT, "n_gpus": world,
                          "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True,
                          "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                          "config": dict(_config(w), parallelism=f"rows split over {world} ranks"),
                          "timing": "wall clock per step (the protocol synchronizes on the host)"}), flush=True)
    part.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    a = _args()
    if a.split and a.impl != "reference":
        run_split_bench(a)
        return
    if a.workload == BATCH_WORKLOAD:
        run_batch_bench(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
