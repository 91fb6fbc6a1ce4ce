"""Benchmark of the coupled D2Q9 + D2Q5 lattice Boltzmann time step on GB300.

A "step" is one coupled time step of the whole chip: pull-stream of f and g,
bounce-back walls, valve-switched Zou-He ports, moments, collision of f and
of g with the same step's velocity, and the fused FP64 mass/flux
diagnostics; one launch of the fused kernel.  The workload is the
4096 x 2048 two-channel chip (3.35 M fluid nodes, 0.94 GB of FP32
populations per copy, larger than the 129 MB L2), the configuration the HBM
roofline is quoted on.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line.  Under torchrun (N > 1) every rank advances its own
replica of the chip (no data exchange: the chips are independent) and rank 0
reports the aggregate over ranks with the time of the slowest rank.
"""
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
sys.path.insert(0, ROOT)

METRIC = "coupled D2Q9+D2Q5 GLUPS and % HBM roofline; adjoint/forward time ratio"
UNIT = "GLUPS"
BYTES_PER_NODE = 112  # 14 FP32 populations read + written per fluid node and step
KERNEL_SRC = [os.path.join(ROOT, "paper_1307_4703_gb300", "csrc", f)
              for f in ("lbm_device.cuh", "lbm_internal.h", "lbm_step.cuh", "lbm_kernels.cu")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "coupled_step_chip-4096x2048.json")
L2_GB = 0.129  # GB300 L2 cache


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20000)
    p.add_argument("--warmup", type=int, default=200)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default="large", choices=["large", "full", "small"])
    p.add_argument("--skip-extras", action="store_true",
                   help="skip the end-to-end and CPU-baseline legs (profiling runs)")
    p.add_argument("--cpu-seconds", type=float, default=8.0,
                   help="host time of the single-thread oracle sample")
    p.add_argument("--variant", type=int, default=0, choices=[0, 1, 2, 3, 4, 5],
                   help="step kernel: 0 library default, 1 registers, 2 bulk-copy pipeline, "
                        "3 self-refilling pipeline, 4 registers with async-copy prefetch, "
                        "5 registers on 64-node tiles (FP32)")
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp16", "bf16"],
                   help="storage of the populations of the timed chip (profiling runs)")
    p.add_argument("--kernel", default="step", choices=["step", "scalar", "adjoint"],
                   help="profiling runs: time the scalar-only step or the adjoint instead of the coupled step "
                        "(prints a short JSON line)")
    return p.parse_args()


def _problem(name):
    from paper_1307_4703_gb300 import workloads as W
    if name == "large":
        return W.config_large_chip()
    if name == "full":
        return W.config_full_chip()
    return W.config_small()


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_hash():
    h = hashlib.sha256()
    for path in KERNEL_SRC:
        with open(path, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _traffic(nodes_now, precision):
    """DRAM bytes (read + written) per launch of the step kernel from the
    committed ncu figures, if they were taken on the current kernel source
    and storage type (else None).  They come from one launch that ncu runs
    with cold caches: reads include the first touch of every row, and writes
    leave out what is still dirty in L2 when the kernel ends."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256_16") != _kernel_hash():
        return None
    per = rec.get("per_precision", {}).get(precision)
    if not per:
        return None
    return float(per["dram_bytes_per_launch"]) * nodes_now / float(rec["fluid_nodes"])


class _Clocks:
    """nvidia-smi sampler running during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.before = ""
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def _once(self):
        """One read-only query (no setting is changed)."""
        try:
            out = subprocess.run(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                  "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
            return out.stdout
        except (OSError, subprocess.SubprocessError):
            return ""

    def start(self):
        self.before = self._once()
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        after = self._once()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        # a sample right before and right after the timed region, beside the
        # 50 ms poll (a short timed region may fall between two polls)
        text = self.before + self.out.read() + after
        rows = [r.split(",") for r in text.strip().splitlines() if r.strip()]
        self.out.close()
        os.unlink(self.out.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                s = float(r[1])
                smax = float(r[2])
            except (ValueError, IndexError):
                continue
            sm.append(s)
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "samples": len(sm), "reasons": sorted(reasons),
                "sampling": "nvidia-smi read-only queries: one right before and one right after the timed "
                            "region, and every 50 ms during it"}


def _cpu_baseline(seconds):
    """The FP64 oracle as it stands, timed on the host cores on the 512 x 256
    downscaled copy of the chip: the serial build for about `seconds` of one
    core, then the all-cores build of the same source (OpenMP over rows, the
    same bits) over the first 1000 steps from rest.  Returns the
    cpu_baseline record and the all-cores run's fields after those 1000
    steps, the reference of the storage-precision accuracy figures."""
    import oracle
    from paper_1307_4703_gb300 import workloads as W
    prob = W.config_large_chip(512, 256)
    fluid = W.fluid_count(prob)
    sched = lambda t: W.valve_word(prob, t)  # noqa: E731
    ref = oracle.from_problem(prob)
    ref.step(1, 5)
    t0 = time.perf_counter()
    n = 0
    while True:
        ref.step(W.valve_word(prob, n), 10)
        n += 10
        dt1 = time.perf_counter() - t0
        if dt1 >= seconds:
            break
    ref.close()
    single = fluid * n / dt1 / 1e9
    par = oracle.from_problem(prob, parallel=True)
    threads = oracle.num_threads(True)
    t0 = time.perf_counter()
    par.run(1000, sched)
    dtp = time.perf_counter() - t0
    fields = par.fields()
    par.close()
    record = {"value": fluid * 1000 / dtp / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
              "nproc": os.cpu_count(),
              "sample": "FP64 C oracle, all-cores build (OpenMP over rows, %d threads), the first 1000 steps "
                        "of the 512x256 downscaled copy (%d fluid nodes) from rest, %.1f s" % (threads, fluid, dtp),
              "single_thread": {"value": single, "unit": UNIT, "cores": 1,
                                "sample": "serial build, %d steps of the same copy, %.1f s" % (n, dt1)}}
    return record, (prob, fields)


def _workload_config(prob, precision):
    """The `config` keys that name the workload (both arms)."""
    from paper_1307_4703_gb300 import workloads as W
    return {"workload": "%s two-channel gradient chip, %s populations" % (prob["name"], precision.upper()),
            "nx": prob["nx"], "ny": prob["ny"], "fluid_nodes": W.fluid_count(prob),
            "tau": prob["tau"], "tau_c": prob["tau_c"], "valve_period": prob["period"]}


def _reference(args):
    """The reference arm: the oracle, as it stands, on the host cores (its
    all-cores build).  Each step is one time step of the 4096 x 2048 chip
    itself when the run holds at most 200 steps (warm-up included), else of
    its 512 x 256 downscaled copy, so that the run ends within minutes."""
    import oracle
    from paper_1307_4703_gb300 import workloads as W
    ws, rank, _ = _dist()
    if rank != 0:
        return
    full = args.steps + args.warmup <= 200
    prob = W.config_large_chip() if full else W.config_large_chip(512, 256)
    fluid = W.fluid_count(prob)
    ref = oracle.from_problem(prob, parallel=True)
    threads = oracle.num_threads(True)
    for t in range(args.warmup):
        ref.step(W.valve_word(prob, t))
    t0 = time.perf_counter()
    for t in range(args.steps):
        ref.step(W.valve_word(prob, args.warmup + t))
    dt = time.perf_counter() - t0
    ref.close()
    value = fluid * args.steps / dt / 1e9
    sample = ("FP64 C oracle, all-cores build (OpenMP over rows, %d threads, %s host cores); each step one time "
              "step of the %s (%d fluid nodes)"
              % (threads, os.cpu_count(), "4096x2048 chip" if full else "512x256 downscaled copy of the chip",
                 fluid))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _workload_config(W.config_large_chip(), "fp32"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _adjoint_ratio(device):
    """Cost of the gradient on the gradient workload (the 1024 x 512 chip,
    4000 steps, two valve toggles) relative to a forward run of the same
    4000 steps with the same options: the whole lbm_adjoint call (its own
    forward sweep, the recomputation of every checkpoint segment but the
    last, and the reverse sweep) over the forward run, and (call - forward
    run) / forward run, the reverse sweep and recomputation alone.  Wall
    clock with the stream synchronised, best of two calls (device memory from
    PyTorch's caching allocator, so the second call allocates nothing).
    Checkpoints every 250 steps (the workload's setting) and every state
    kept (ckpt_every = 1, 117 GB, nothing recomputed); one launch per step,
    and multi_step runs of up to 1000 steps (forward run and adjoint
    alike)."""
    import numpy as np
    from paper_1307_4703_gb300 import lbm, workloads as W
    prob = W.config_adjoint_chip()
    cx0, cx1, cy0, cy1 = prob["chamber"]
    oy = np.arange(cy0, cy1)
    ox = np.full_like(oy, (cx0 + cx1) // 2)
    target = (oy - cy0) / max(1, cy1 - 1 - cy0)
    n = prob["steps"]
    out = {}
    for ms in (0, 1000):
        for K in (250, 1):
            best = None
            for _ in range(2):
                chip = lbm.Chip.from_problem(prob, device=device, torch_alloc=True, multi_step=ms)
                chip.set_valve_schedule(prob["period"], prob["states"])
                chip.step(10)
                chip.synchronize()
                t0 = time.perf_counter()
                chip.step(n)
                chip.synchronize()
                tf = time.perf_counter() - t0
                t0 = time.perf_counter()
                chip.adjoint(n, ox, oy, target, ckpt_every=K)
                ta = time.perf_counter() - t0
                chip.close()
                r = {"whole_call": ta / tf, "beyond_forward": (ta - tf) / tf,
                     "forward_us_per_step": tf / n * 1e6, "adjoint_call_us_per_step": ta / n * 1e6}
                best = r if best is None or r["whole_call"] < best["whole_call"] else best
            out[(ms, K)] = best
    import torch
    torch.cuda.empty_cache()
    return {"value": out[(0, 250)]["whole_call"], "workload": "chip-1024x512, 4000 steps, checkpoints every 250",
            "definition": "whole lbm_adjoint call (forward sweep + recomputation + reverse sweep) / forward run "
                          "of the same steps; one launch per step",
            "ckpt_every_250": out[(0, 250)], "ckpt_every_1": out[(0, 1)],
            "multi_step_1000": {"ckpt_every_250": out[(1000, 250)], "ckpt_every_1": out[(1000, 1)]}}


def _frozen_scalar(chip, prob, steps, stream, peak):
    """The scalar-only step on stored velocity fields (the paper's own
    workflow): 48 bytes per fluid node and step (5 populations read and
    written, 2 velocity components read).  Device time over `steps` steps."""
    import torch
    from paper_1307_4703_gb300 import workloads as W
    fluid = W.fluid_count(prob)
    for w in sorted(set(prob["states"])):
        chip.store_velocity(w)  # the current flow field stands in for each valve state
    chip.scalar_step(10, 2.0)
    chip.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        chip.scalar_step(1, 2.0)
    e1.record(stream)
    stream.synchronize()
    s = e0.elapsed_time(e1) / 1e3
    achieved = fluid * 48 * steps / s / 1e9
    return {"value": fluid * steps / s / 1e9, "unit": UNIT, "steps": steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "bytes_per_launch": fluid * 48}}


def _reduced_precision(prob, steps, stream, device, peak, reference=None):
    """The same coupled step with 16-bit population storage (FP16 and BF16
    deviations, FP32 arithmetic): 56 bytes per fluid node and step.  Device
    time over `steps` single-step calls after 50 warm-up steps.  Accuracy:
    the fields of each storage type after the first 1000 steps of the
    512 x 256 copy against `reference` = (problem, FP64 oracle fields) of the
    CPU-baseline leg, or, without it (ranks of a multi-GPU run), against
    FP32 storage."""
    import numpy as np
    import torch
    from paper_1307_4703_gb300 import lbm, workloads as W
    fluid = W.fluid_count(prob)
    out = {}
    for prec in ("fp16", "bf16"):
        chip = lbm.Chip.from_problem(prob, stream=stream, torch_alloc=True, device=device, precision=prec)
        chip.set_valve_schedule(prob["period"], prob["states"])
        chip.step(50)
        chip.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            chip.step(1)
        e1.record(stream)
        stream.synchronize()
        s = e0.elapsed_time(e1) / 1e3
        chip.diagnostics()  # raises on a numeric error flag
        info = chip.info()
        chip.close()
        achieved = info["algorithmic_bytes_per_step"] * steps / s / 1e9
        out[prec] = {"value": fluid * steps / s / 1e9, "unit": UNIT, "steps": steps,
                     "us_per_step": s / steps * 1e6,
                     "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak,
                                  "bytes_per_launch": info["algorithmic_bytes_per_step"]}}
    small = W.config_large_chip(512, 256) if reference is None else reference[0]
    fields = {}
    for prec in ("fp32", "fp16", "bf16"):
        chip = lbm.Chip.from_problem(small, stream=stream, torch_alloc=True, device=device, precision=prec)
        chip.set_valve_schedule(small["period"], small["states"])
        chip.step(1000)
        fields[prec] = chip.fields()
        chip.close()
    fl = ~np.asarray(small["solid"], bool)
    ref = fields["fp32"] if reference is None else reference[1]
    against = ("FP32 storage" if reference is None else "the FP64 oracle") + ", chip-512x256 copy, 1000 steps from rest"
    out["fp32"] = {}
    for prec in ("fp32", "fp16", "bf16") if reference is not None else ("fp16", "bf16"):
        f = fields[prec]
        drho = np.abs(f[0] - ref[0])[fl].max()
        du = max(np.abs(f[k] - ref[k])[fl].max() for k in (1, 2)) / small["u_max"]
        dC = np.abs(f[3] - ref[3])[fl].max()
        dm = abs(f[0][fl].astype(np.float64).sum() - ref[0][fl].sum()) / ref[0][fl].sum()
        out[prec]["accuracy"] = {"max_drho": float(drho), "max_du_over_u_max": float(du), "max_dC": float(dC),
                                 "mass_rel": float(dm), "against": against}
    if not out["fp32"]:
        del out["fp32"]
    return out


def _batch(steps, stream, device, peak, n_chips=64):
    """64 independent chips of 256 x 128 ... 1024 x 512 (seeded sizes,
    relaxation times and valve periods): all in one handle, one launch per
    step; the same handle autotuned with CUDA graphs of 100 steps, and with
    runs of up to 1000 steps in one persistent cooperative launch
    (multi_step); against the same chips stepped one handle after another."""
    import torch
    from paper_1307_4703_gb300 import lbm, workloads as W
    chips = W.config_batch(n_chips)
    fluid = sum(W.fluid_count(p) for p in chips)

    def timed(fn, n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        stream.synchronize()
        return e0.elapsed_time(e1) / 1e3

    batch = lbm.Chip.batch(chips, stream=stream, torch_alloc=True, device=device)
    for k, p in enumerate(chips):
        batch.set_instance_schedule(k, p["period"], p["states"])
    batch.step(20)
    batch.synchronize()
    s_batch = timed(lambda: batch.step(1), steps)
    info = batch.info()
    batch.diagnostics()
    batch.close()
    modes = {}
    for key, kw in (("graphs_100_autotuned", {"graph_steps": 100}), ("multi_step_1000", {"multi_step": 1000})):
        b = lbm.Chip.batch(chips, stream=stream, torch_alloc=True, device=device, **kw)
        for k, p in enumerate(chips):
            b.set_instance_schedule(k, p["period"], p["states"])
        if "graph_steps" in kw:
            b.autotune()
        b.step(200)
        b.synchronize()
        s_mode = timed(lambda: b.step(steps), 1)
        b.diagnostics()
        b.close()
        modes[key] = {"value": fluid * steps / s_mode / 1e9, "unit": UNIT, "steps": steps,
                      "roofline_frac": info["algorithmic_bytes_per_step"] * steps / s_mode / 1e9 / peak}
    singles = [lbm.Chip.from_problem(p, stream=stream, torch_alloc=True, device=device) for p in chips]
    for c, p in zip(singles, chips):
        c.set_valve_schedule(p["period"], p["states"])
        c.step(5)
    n_single = max(1, steps // 10)

    def one_by_one():
        for c in singles:
            c.step(1)

    s_single = timed(one_by_one, n_single)
    for c in singles:
        c.close()
    achieved = info["algorithmic_bytes_per_step"] * steps / s_batch / 1e9
    return {"value": fluid * steps / s_batch / 1e9, "unit": UNIT, "chips": n_chips, "fluid_nodes": fluid,
            "steps": steps, "one_by_one": fluid * n_single / s_single / 1e9, "one_by_one_steps": n_single,
            **modes,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "bytes_per_launch": info["algorithmic_bytes_per_step"]}}


def _small_chips(steps, stream, device, peak):
    """Chips of a few microseconds per step, where launch costs show: the
    1024 x 768 chip (the paper's 1 um lattice, 313,600 fluid nodes) with
    single-step launches, replayed CUDA graphs of 100 steps (both after
    lbm_autotune) and runs of up to 1000 steps in one cooperative launch
    (multi_step); the 1024 x 512 chip (two buffers in L2) with single-step
    launches and multi_step runs."""
    import torch
    from paper_1307_4703_gb300 import lbm, workloads as W
    out = {}
    for prob, modes in ((W.config_full_chip(), (("launches", {}), ("graphs_100", {"graph_steps": 100}),
                                                ("multi_step_1000", {"multi_step": 1000}))),
                        (W.config_adjoint_chip(), (("launches", {}), ("multi_step_1000", {"multi_step": 1000})))):
        fluid = W.fluid_count(prob)
        res = {"workload": "chip-%dx%d, %d fluid nodes" % (prob["nx"], prob["ny"], fluid)}
        for key, kw in modes:
            chip = lbm.Chip.from_problem(prob, stream=stream, torch_alloc=True, device=device, **kw)
            chip.set_valve_schedule(prob["period"], prob["states"])
            info = chip.autotune() if "multi_step" not in kw else chip.info()
            chip.step(200)
            chip.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            chip.step(steps)
            e1.record(stream)
            stream.synchronize()
            s = e0.elapsed_time(e1) / 1e3
            chip.diagnostics()
            chip.close()
            achieved = info["algorithmic_bytes_per_step"] * steps / s / 1e9
            res[key] = {"value": fluid * steps / s / 1e9, "unit": UNIT, "steps": steps,
                        "us_per_step": s / steps * 1e6, "roofline_frac": achieved / peak}
            if "multi_step" not in kw:
                res[key]["launch"] = {k: info[k] for k in ("variant", "grid", "block", "stages")}
        out["chip-%dx%d" % (prob["nx"], prob["ny"])] = res
    return out


def _e2e(prob, steps, device):
    """The same metric through the public C ABI with host buffers: create the
    chip from host arrays, then every step upload the step's valve word and
    run the step with its diagnostics written by the step kernel into
    page-locked host memory (lbm_step_diagnostics, one row per step, read
    after the final synchronisation), and finally read the fields back into
    the caller's page-locked arrays; all inside the timed region."""
    import numpy as np
    import torch
    from paper_1307_4703_gb300 import lbm, workloads as W
    fluid = W.fluid_count(prob)
    nx, ny = prob["nx"], prob["ny"]
    warm = lbm.Chip.from_problem(prob, device=device)
    warm.step(2)
    warm.diagnostics()
    warm.close()
    rows = torch.zeros((steps, 4), dtype=torch.float64, pin_memory=True)
    # the caller's page-locked buffers for the fields read at the end
    out = [torch.empty((ny, nx), dtype=torch.float32, pin_memory=True).numpy() for _ in range(4)]
    t0 = time.perf_counter()
    chip = lbm.Chip.from_problem(prob, device=device)
    chip.synchronize()
    t1 = time.perf_counter()
    for t in range(steps):
        chip.set_valves(W.valve_word(prob, t))
        chip.step_diagnostics(1, rows[t].data_ptr())
    chip.synchronize()
    t2 = time.perf_counter()
    fields = chip.fields(out=out)
    t3 = time.perf_counter()
    chip.close()
    dt = time.perf_counter() - t0
    assert np.isfinite(rows.numpy()).all()
    h2d_once = nx * ny + 2 * 2 * ny * 4 + len(prob["ports"]) * 32
    d2h_once = sum(a.nbytes for a in fields)
    return {"value": fluid * steps / dt / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": 4 + h2d_once / steps,
            "d2h_bytes_per_step": 32 + d2h_once / steps,
            "steps": steps, "seconds": dt,
            "breakdown_s": {"create": t1 - t0, "steps": t2 - t1, "read_fields": t3 - t2, "destroy": dt - (t3 - t0)}}


def reduce_max(value, world_size):
    """Largest value over the ranks (the slowest rank's time); the value
    itself on a single process.  Works on the NCCL and on the gloo backend."""
    if world_size <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_glups(per_rank_units, seconds, world_size):
    """Whole-job throughput: the units every rank processed over the time
    of the slowest rank (weak scaling: each rank advances its own chip)."""
    return world_size * per_rank_units / reduce_max(seconds, world_size) / 1e9


def _profile_target(args, device):
    """The scalar-only step (after `warmup` coupled steps, on the velocity
    field of the chip at that point) or the adjoint of `steps` steps of the
    gradient chip with every state kept, for kernel profiles."""
    import numpy as np
    import torch
    from paper_1307_4703_gb300 import lbm, workloads as W
    stream = torch.cuda.Stream()
    if args.kernel == "scalar":
        prob = _problem(args.workload)
        chip = lbm.Chip.from_problem(prob, stream=stream, torch_alloc=True, device=device)
        chip.set_valve_schedule(prob["period"], prob["states"])
        chip.step(max(args.warmup, 1))
        for w in sorted(set(prob["states"])):
            chip.store_velocity(w)
        chip.scalar_step(max(args.warmup, 1), 2.0)
        chip.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            chip.scalar_step(1, 2.0)
        e1.record(stream)
        stream.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / max(args.steps, 1)
        out = {"kernel": "lbm_scalar_step (default kernel: scalar_frozen_regs)", "workload": prob["name"],
               "us_per_step": us,
               "glups": W.fluid_count(prob) / us / 1e3}
    else:
        prob = W.config_adjoint_chip()
        cx0, cx1, cy0, cy1 = prob["chamber"]
        oy = np.arange(cy0, cy1)
        ox = np.full_like(oy, (cx0 + cx1) // 2)
        chip = lbm.Chip.from_problem(prob, stream=stream, torch_alloc=True, device=device)
        chip.set_valve_schedule(prob["period"], prob["states"])
        chip.step(max(args.warmup, 1))
        chip.synchronize()
        t0 = time.perf_counter()
        chip.step(args.steps)
        chip.synchronize()
        tf = time.perf_counter() - t0
        t0 = time.perf_counter()
        chip.adjoint(args.steps, ox, oy, (oy - cy0) / max(1, cy1 - 1 - cy0), ckpt_every=1)
        ta = time.perf_counter() - t0
        out = {"kernel": "adjoint", "workload": prob["name"], "steps": args.steps,
               "forward_us_per_step": tf / args.steps * 1e6, "adjoint_call_seconds": ta,
               "reverse_us_per_step": (ta - tf) / args.steps * 1e6}
    chip.close()
    print(json.dumps(out), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        _reference(args)
        return
    import torch
    from paper_1307_4703_gb300 import build, lbm, workloads as W

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    build.build()
    torch.cuda.set_device(local)
    if args.kernel != "step":
        _profile_target(args, local)
        return
    prob = _problem(args.workload)
    fluid = W.fluid_count(prob)
    stream = torch.cuda.Stream()
    chip = lbm.Chip.from_problem(prob, stream=stream, torch_alloc=True, device=local, variant=args.variant,
                                 precision=args.precision)
    chip.set_valve_schedule(prob["period"], prob["states"])
    info = chip.info()

    for _ in range(max(args.warmup, 0)):
        chip.step(1)
    chip.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    clocks = _Clocks(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        chip.step(1)  # one launch of the fused step kernel (with diagnostics)
    ev1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    d = chip.diagnostics()  # raises on a numeric error flag
    value = aggregate_glups(fluid * args.steps, ms / 1e3, ws)
    ms = reduce_max(ms, ws)
    ms_per_step = ms / max(args.steps, 1)
    peak, peak_src = _peak()
    achieved = info["algorithmic_bytes_per_step"] / (ms_per_step / 1e3) / 1e9
    extras = {}
    if not args.skip_extras:
        reference = None
        if ws == 1 and rank == 0:
            extras["cpu_baseline"], reference = _cpu_baseline(args.cpu_seconds)
        extras["frozen_scalar_step"] = _frozen_scalar(chip, prob, min(args.steps, 2000), stream, peak)
        extras["reduced_precision_storage"] = _reduced_precision(prob, min(args.steps, 5000), stream, local, peak,
                                                                 reference)
        extras["batch_64_chips"] = _batch(min(args.steps, 10000), stream, local, peak)
        extras["small_chips"] = _small_chips(min(args.steps, 20000), stream, local, peak)
        e2e_steps = args.steps  # the device-timed region's step count
        e = _e2e(prob, e2e_steps, local)
        e["value"] = aggregate_glups(fluid * e2e_steps, e["seconds"], ws)
        extras["e2e"] = {k: e[k] for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step", "steps",
                                           "breakdown_s")}
        extras["adjoint_forward_ratio"] = _adjoint_ratio(local)
    chip.close()
    if rank == 0:
        # two copies of the populations alternate: 2 x this many bytes per step
        copy_gb = info["pitch"] * prob["ny"] * 14 * (4 if args.precision == "fp32" else 2) / 1e9
        l2_note = ("inputs larger than L2 (%.2f GB of populations per copy)" % copy_gb
                   if 2 * copy_gb > L2_GB else
                   "inputs fit in L2 (%.3f GB of populations per copy, not flushed: a small chip steps in L2)"
                   % copy_gb)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_workload_config(prob, args.precision), **{
                       "l2": l2_note,
                       "parallelism": "replicas" if ws > 1 else "single GPU",
                       "launch": {"variant": {1: "registers", 2: "bulk-copy pipeline", 3: "self-refilling pipeline",
                                              4: "registers + async-copy prefetch",
                                              5: "registers on 64-node tiles"}[
                                      info["variant"]],
                                  "grid": info["grid"], "block": info["block"],
                                  "stages": info["stages"], "tiles": info["n_tiles"]}}),
            "all_node_glups": ws * prob["nx"] * prob["ny"] * args.steps / (ms / 1e3) / 1e9,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": _traffic(fluid, args.precision),
                         "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch with "
                                         "cold caches (committed figures, null when the kernel source changed); "
                                         "writes still dirty in L2 at the kernel's end are not counted",
                         "peak_source": "%s (hbm_gbs)" % peak_src,
                         "bytes_per_launch": info["algorithmic_bytes_per_step"]},
            "gpu_launches": args.steps,
            "clocks": clk,
            "diagnostics": {"mass": d[0], "scalar": d[1]},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
