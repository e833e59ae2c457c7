#!/usr/bin/env python
"""Benchmark of the e-ph collision-integral hot path on one GB300 (or N replicas).

One step = one classic RK4 step of the rt-BTE (four collision-integral sweeps,
Eq. 2) plus one three-direction transport iteration (one weighted sweep), on
the 40^3 workload: 4 bands, 6 modes, per-band 0.3 eV window, 1.36e8 channels.
The metric is channel evaluations per second (5 sweeps x channels per step).

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded row sample of the same workload instead.
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

SWEEPS_PER_STEP = 5  # 4 RK4 collision sweeps + 1 transport sweep
LAUNCHES_PER_STEP = 13  # rk4: 1 conversion + 8 graph kernels; transport: 1 conversion + 3 kernels
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=5,
                    help="timed blocks of --steps steps each; value and ms_per_step are their median")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="window40")
    ap.add_argument("--variant", default="ff")
    ap.add_argument("--tile-sweep", type=int, default=0, help="pb_dev_opts.tile_sweep of the bench device")
    ap.add_argument("--ctas-per-sm", type=int, default=0, help="pb_dev_opts.ctas_per_sm of the bench device")
    ap.add_argument("--transport-gather", type=int, default=0,
                    help="pb_dev_opts.transport_gather of the bench device (the transport sweep shape)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--mixed-steps", type=int, default=1000)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--only-adjoint", action="store_true",
                    help="print only the adjoint workload's report (for profiling its kernels)")
    ap.add_argument("--adjoint-steps", type=int, default=200)
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--batched-instances", type=int, default=64)
    ap.add_argument("--batched-steps", type=int, default=500)
    return ap.parse_args()


def workload_config(name: str) -> dict:
    if name == "window40":
        return {"workload": "rt-BTE RK4 step + 3-direction transport iteration, 40^3 k/q grids, 4 bands, "
                            "6 modes, per-band 0.3 eV window, sigma 8 meV, T 300 K",
                "grid": [40, 40, 40], "bands": 4, "modes": 6, "dt_fs": 1.0}
    if name == "tiny":
        return {"workload": "rt-BTE RK4 step + 3-direction transport iteration, 8^3 full BZ, 2 bands, 3 modes, "
                            "sigma 5 meV, T 300 K", "grid": [8, 8, 8], "bands": 2, "modes": 3, "dt_fs": 1.0}
    return {"workload": name}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while the GPU is busy."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,clocks.mem")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def has_sample(self) -> bool:
        try:
            return self.proc is not None and os.path.getsize(self.path) > 0
        except OSError:
            return False

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                mem = float(parts[9]) if len(parts) > 9 else float("nan")
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], mem))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        mx = max(r[1] for r in rows)
        loaded = [r for r in rows if r[0] > 0.5 * mx] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower() == "active"})
        mems = [r[3] for r in loaded if r[3] == r[3]]
        return {"sm_mhz": statistics.median(r[0] for r in loaded), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "mem_mhz": statistics.median(mems) if mems else None}


def measured_hbm():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM, "fallback (6.8 TB/s)"


def function_source(text: str, name: str) -> str:
    """Source of the device function or kernel `name` in kernels.cuh: from its template/
    qualifier line to the brace that closes its body (every overload, concatenated)."""
    out = []
    lines = text.split("\n")
    for i, line in enumerate(lines):
        if (f" {name}(" not in line and f" {name}<" not in line) or line.strip().startswith("//") \
                or line.rstrip().endswith(";"):
            continue
        if "__device__" not in line and "__global__" not in line and "__launch_bounds__" not in line:
            continue
        start = i
        while start > 0 and lines[start - 1].startswith("template"):
            start -= 1
        depth, j, seen = 0, i, False
        while j < len(lines):
            depth += lines[j].count("{") - lines[j].count("}")
            seen = seen or "{" in lines[j]
            if seen and depth == 0:
                break
            j += 1
        out.append("\n".join(lines[start:j + 1]))
    return "\n".join(out)


HOT_FUNCTIONS = ("ff_split", "ff_to_double", "ff_mac", "ff_mac_lazy", "ff_add", "warp_sum", "partners4", "group_f",
                 "k_stream_ff", "k_stream_sym", "ff_prod", "ff_reduce_scatter",
                 "sym_columns_out", "mbar_init", "mbar_expect_tx", "mbar_try_wait", "mbar_wait", "bulk_g2s",
                 "fence_proxy_async", "k_stream_sym_bulk", "half_smem", "k_stream_sym_half")


# the FP32 coefficient-tile sweep (tiles32.cuh) and the helpers of kernels.cuh it inlines
HOT_FUNCTIONS_C32 = ("c32_smem", "c32_term", "f32_reduce_scatter", "c32_columns_out", "k_stream_c32", "ff_split",
                     "mbar_init", "mbar_expect_tx", "mbar_try_wait", "mbar_wait", "bulk_g2s", "fence_proxy_async")


def kernel_source_hash(variant: str = "ff") -> str:
    """Hash of the collision sweep's own source (the kernel and the helpers it inlines)."""
    csrc = os.path.join(ROOT, "paper_2511_03683_gb300", "csrc")
    text = open(os.path.join(csrc, "kernels.cuh")).read()
    names = HOT_FUNCTIONS
    if variant == "c32":
        text += "\n" + open(os.path.join(csrc, "tiles32.cuh")).read()
        names = HOT_FUNCTIONS_C32
    h = hashlib.sha256()
    for n in names:
        h.update(function_source(text, n).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload: str, variant: str, bytes_per_launch: float):
    """DRAM bytes per launch of the collision sweep from the committed ncu summary, if it
    was captured on the current kernel source and the same streamed layout (the same
    algorithmic bytes per launch); else None."""
    try:
        d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        e = d[f"{workload}:{variant}"]
        if e.get("source_hash") != kernel_source_hash(variant):
            return None
        if abs(float(e["algorithmic_bytes_per_launch"]) - bytes_per_launch) > 1e-6 * bytes_per_launch:
            return None
        return float(e["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The largest value of x over all ranks (the timed region's max-over-ranks)."""
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as tdist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(units_per_rank: float, ws: int, seconds_max: float) -> float:
    """Throughput of the whole job: units processed by all replicas / slowest rank's time."""
    return ws * units_per_rank / seconds_max


def dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def emit(obj):
    print(json.dumps(obj), flush=True)


# ---------------------------------------------------------------- CPU oracle


def oracle_step_sample(o, f, f0, v, rows):
    """One bounded oracle 'step' on a row sample: four collision row-passes and one
    transport-map row-pass (the GPU step's sweep mix)."""
    import numpy as np

    for _ in range(4):
        o.collision(f, rows=rows)
    o.transport_map(f0, v, np.zeros_like(v), rows=rows)


def cpu_baseline(m, sample_every=4, reps=1):
    import numpy as np

    import oracle

    o = oracle.Oracle(m)
    f = o.window_values(m.f_hot())
    f0 = o.window_values(m.f_fermi(m.emin() - 0.2))
    v = o.window_values(m.vel)
    rows = np.arange(0, o.nstate, sample_every, dtype=np.int32)
    ch_rows = o_rows_channels(m, o, rows)
    t = time.perf_counter()
    for _ in range(reps):
        oracle_step_sample(o, f, f0, v, rows)
    dt = time.perf_counter() - t
    value = SWEEPS_PER_STEP * ch_rows * reps / dt
    return {"value": value, "unit": "channels/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{reps} oracle step(s) (4 collision + 1 transport-map row passes) over every "
                      f"{sample_every}th window state ({len(rows)} rows, {ch_rows} channels per pass), "
                      f"{dt:.1f} s"}, (o, f, f0, v, rows, ch_rows)


def o_rows_channels(m, o, rows):
    """Channels in the listed rows, counted from the model by the oracle's own rule."""
    import numpy as np

    nb = m.nbands
    nk = m.nk
    ids = o.ids
    ik = ids // nb
    j = np.stack([ik // (nk[1] * nk[2]), (ik // nk[2]) % nk[1], ik % nk[2]], axis=1)
    npos = (m.omega > 0).sum(axis=1)
    total = 0
    for r in rows:
        q = (j - j[r]) % np.array(nk)
        iq = (q[:, 0] * nk[1] + q[:, 1]) * nk[2] + q[:, 2]
        total += int(npos[iq].sum())
    return total


def run_reference(args):
    ws, rank, _ = dist()
    if rank != 0:
        return 0
    import synth

    m = synth.make_config(args.workload)
    every = 16 if args.workload == "window40" else 4
    base, (o, f, f0, v, rows, ch_rows) = cpu_baseline(m, sample_every=every, reps=1)
    for _ in range(args.warmup):
        oracle_step_sample(o, f, f0, v, rows)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle_step_sample(o, f, f0, v, rows)
    dt = time.perf_counter() - t
    value = SWEEPS_PER_STEP * ch_rows * args.steps / dt
    cfg = workload_config(args.workload)
    cfg["sample"] = f"every {every}th window state ({len(rows)} rows)"
    emit({"impl": "reference", "metric": "e-ph channels/s", "value": value, "unit": "channels/s", "n_gpus": ws,
          "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
          "config": cfg,
          "cpu_baseline": {"value": value, "unit": "channels/s", "cores": base["cores"], "kind": "oracle",
                           "sample": f"{args.steps} oracle steps (4 collision + 1 transport-map row passes) over "
                                     f"every {every}th window state ({len(rows)} rows)"},
          "e2e": {"value": value, "unit": "channels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    return 0


# ---------------------------------------------------------------- GPU


def time_calls(fn, n, stream):
    import torch

    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    fn()
    for a, b in evs:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in evs)


_flush_buf = None


def sweep_ms_flushed(dev, f, n, stream):
    """Median device time of one collision sweep launch, with L2 flushed before each (a 256 MB
    buffer written, twice the 129 MB L2), for sweeps whose streamed bytes fit in L2."""
    global _flush_buf
    import torch

    if _flush_buf is None:
        _flush_buf = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ts = []
    dev.time_sweep(f, 1, stream=stream)
    for _ in range(n):
        _flush_buf.zero_()
        ts.append(dev.time_sweep(f, 1, stream=stream))
    return statistics.median(ts)


def adjoint_report(pb, stream, nsteps=200):
    """The adjoint workload: 24^3, 4 bands, 6 modes; loss = carrier energy after 200 RK4
    steps of 1 fs; gradient with respect to f0 and every stored |g|^2 through checkpoints
    every 20 steps (forward + backward), FP64-accurate (FF) and FP32 (G32) devices."""
    every = min(20, nsteps)
    import numpy as np
    import torch

    import synth
    from paper_2511_03683_gb300 import autograd as pa

    m = synth.make_config("window24")
    ch = pb.Channels.from_model(m)
    ids = ch.state_ids()
    eps = torch.tensor(m.eps.reshape(-1)[ids], device="cuda")
    out = {"workload": f"24^3, 4 bands, 6 modes, {nsteps} RK4 steps of 1 fs, checkpoints every {every}",
           "channels": ch.nchannels}
    grads = {}
    for v in ("ff", "g32"):
        # the |g|^2 gradient is deferred to per-pair accumulators and flushed once
        dev = pb.Device(ch, variant=v, adjoint=True)
        g2 = pa.g2_tensor(ch)
        times = []
        for rep in range(3):
            f0 = torch.tensor(m.f_hot().reshape(-1)[ids], device="cuda", requires_grad=True)
            g2r = g2.clone().requires_grad_(True)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            (eps * pa.trajectory(dev, f0, g2r, 1.0, nsteps, every)).sum().backward()
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        grads[v] = (f0.grad.cpu().numpy(), g2r.grad.cpu().numpy())
        out[v] = {"forward_backward_ms": min(times), "forward_steps": nsteps, "recomputed_steps": nsteps,
                  "adjoint_steps": nsteps, "g2_gradient": "deferred" if dev.deferred else "per step"}
        dev.close()
    out["g32_grad_err_vs_ff"] = {
        "f0": float(np.abs(grads["g32"][0] - grads["ff"][0]).max() / np.abs(grads["ff"][0]).max()),
        "g2": float(np.abs(grads["g32"][1] - grads["ff"][1]).max() / np.abs(grads["ff"][1]).max())}
    ch.close()
    return out


def batched_report(pb, ninst, nsteps, stream):
    """The batched workload: ninst instances (grids 16^3..36^3, 2-4 bands, 3-6 modes,
    T 100-500 K, excitation 0.1-0.5 eV) in one launch per RK4 stage with FP32 |g|^2, against
    the same instances advanced one after the other on the unbatched FP32 path (the same
    arithmetic) and on the FP64-accurate paths (branch-merged and one entry per channel)."""
    import numpy as np
    import torch

    import synth

    inst = [synth.make_batch_instance(i) for i in range(ninst)]
    t0 = time.perf_counter()
    chs = [pb.Channels.from_model(m) for m, _ in inst]
    build_s = time.perf_counter() - t0
    fs = [m.f_hot(e_exc=e).reshape(-1)[c.state_ids()] for (m, e), c in zip(inst, chs)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = pb.Batch(chs)
    create_b = time.perf_counter() - t0
    f = torch.tensor(np.concatenate(fs), device="cuda")
    item, ctas, tune_ms = b.autotune(f)
    nch = b.nchannels
    g = f.clone()
    b.rk4(g, 1.0, 3)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    b.rk4(g, 1.0, nsteps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    Ib = b.collision(f).cpu().numpy()

    def sequential(variant, **kw):
        devs = [pb.Device(c, variant=variant, **kw) for c in chs]
        fl = [torch.tensor(x, device="cuda") for x in fs]
        for d, x in zip(devs, fl):
            d.rk4(x, 1.0, 2)
        torch.cuda.synchronize()
        e0.record(stream)
        for d, x in zip(devs, fl):
            d.rk4(x, 1.0, nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        err = 0.0
        if variant == "ff":
            for i, (d, x) in enumerate(zip(devs, fs)):
                ref = d.collision(torch.tensor(x, device="cuda")).cpu().numpy()
                a, e = b.offsets[i], b.offsets[i + 1]
                err = max(err, float(np.abs(Ib[a:e] - ref).max() / max(np.abs(ref).max(), 1e-300)))
        for d in devs:
            d.close()
        return ms, err

    ms_ff, err = sequential("ff")
    ms_ffc, _ = sequential("ff", merge_branches=2)
    ms_g, _ = sequential("g32")
    ms_64, _ = sequential("f64")  # the plain FP64 GPU path (native FP64 FMAs, branch-merged)
    b.close()

    def accurate(precision, layout):
        """One FP64-accurate or FP32-pair batch: autotuned, nsteps RK4 steps timed, and df/dt
        against each instance on its own FF device (max over instances, normwise)."""
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        bx = pb.Batch(chs, precision=precision, layout=layout)
        create_s = time.perf_counter() - t1
        tuned = bx.autotune(f)
        g = f.clone()
        bx.rk4(g, 1.0, 3)
        torch.cuda.synchronize()
        e0.record(stream)
        bx.rk4(g, 1.0, nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        bx.check()
        Ix = bx.collision(f).cpu().numpy()
        errx = 0.0
        for i, (c, x) in enumerate(zip(chs, fs)):
            d = pb.Device(c)
            ref = d.collision(torch.tensor(x, device="cuda")).cpu().numpy()
            d.close()
            a, e = bx.offsets[i], bx.offsets[i + 1]
            errx = max(errx, float(np.abs(Ix[a:e] - ref).max() / max(np.abs(ref).max(), 1e-300)))
        tiled = bx.tiled
        bx.close()
        return ms, tuned, errx, tiled, create_s

    # the same batch on the FP64-accurate branch-merged coefficients (symmetric tiles by
    # default, rows beside them) and as FP32 pairs (net terms per entry)
    ms_bf, (item_f, ctas_f, tune_f), err_f, tiled_f, create_f = accurate("ff", 0)
    ms_bfr, (item_fr, ctas_fr, tune_fr), _, _, _ = accurate("ff", 1)
    ms_bc, (item_c, ctas_c, tune_c), err_c, tiled_c, create_c = accurate("c32", 0)
    ms_bcr, (item_cr, ctas_cr, tune_cr), _, _, _ = accurate("c32", 1)

    def rows_leg(ms, item_, ctas_, tune_):
        return {"autotuned": {"item_entries": item_, "ctas_per_sm": ctas_, "sweep_ms": tune_}, "batched_ms": ms,
                "batched_rk4_steps_per_s": nsteps / (ms * 1e-3)}

    return {"instances": ninst, "states": b.nstate, "channels": nch, "build_channels_s": build_s,
            "create_s": create_b,
            "autotuned": {"item_channels": item, "ctas_per_sm": ctas, "sweep_ms": tune_ms},
            "rk4_steps": nsteps, "batched_ms": ms_b,
            "batched_channels_per_s": 4 * nch * nsteps / (ms_b * 1e-3),
            "batched_rk4_steps_per_s": nsteps / (ms_b * 1e-3),
            "sequential_ff_ms": ms_ff, "sequential_ff_per_channel_ms": ms_ffc, "sequential_g32_ms": ms_g,
            "sequential_f64_ms": ms_64, "speedup_vs_sequential_f64": ms_64 / ms_b,
            "speedup_vs_sequential_fp32": ms_g / ms_b, "speedup_vs_sequential_ff": ms_ff / ms_b,
            "speedup_vs_sequential_ff_per_channel": ms_ffc / ms_b,
            "ff_batch": {"layout": "tiles" if tiled_f else "rows", "create_s": create_f,
                         "autotuned": {"item_entries": item_f, "ctas_per_sm": ctas_f, "sweep_ms": tune_f},
                         "batched_ms": ms_bf, "batched_rk4_steps_per_s": nsteps / (ms_bf * 1e-3),
                         "batched_channels_per_s": 4 * nch * nsteps / (ms_bf * 1e-3),
                         "speedup_vs_sequential_ff": ms_ff / ms_bf, "speedup_vs_sequential_f64": ms_64 / ms_bf,
                         "speedup_vs_sequential_ff_per_channel": ms_ffc / ms_bf,
                         "dfdt_err_vs_unbatched_ff_max_over_instances": err_f,
                         "rows": rows_leg(ms_bfr, item_fr, ctas_fr, tune_fr)},
            "c32_batch": {"layout": "tiles" if tiled_c else "rows", "create_s": create_c,
                          "autotuned": {"item_entries": item_c, "ctas_per_sm": ctas_c, "sweep_ms": tune_c},
                          "batched_ms": ms_bc, "batched_rk4_steps_per_s": nsteps / (ms_bc * 1e-3),
                          "batched_channels_per_s": 4 * nch * nsteps / (ms_bc * 1e-3),
                          "speedup_vs_sequential_ff": ms_ff / ms_bc, "speedup_vs_ff_batch": ms_bf / ms_bc,
                          "speedup_vs_sequential_f64": ms_64 / ms_bc,
                          "speedup_vs_sequential_fp32": ms_g / ms_bc,
                          "dfdt_err_vs_fp64_max_over_instances": err_c,
                          "rows": rows_leg(ms_bcr, item_cr, ctas_cr, tune_cr)},
            "dfdt_err_vs_fp64_max_over_instances": err}


def ablation_report(pb, m, ch_full, stream):
    """The paper's own layout (each channel once, sc_col written then gathered with signs)
    against the full-list fused sweep, one entry per channel (the layout comparison proper)
    and branch-merged (the default), on the whole list and with the paper's cutoffs on
    (delta at 6 sigma, |g|^2 >= 1e-5 eV^2)."""
    import torch

    out = {}
    for label, kw in (("no_cutoffs", None), ("cutoffs_delta6sigma_g2min1e-5", {"g2_min": 1e-5, "delta_nsigma": 6.0})):
        ch = ch_full if kw is None else pb.Channels.from_model(m, **kw)
        ids = ch.state_ids()
        f = torch.tensor(m.f_hot().reshape(-1)[ids], device="cuda")
        res = {"channels": ch.nchannels}
        for v, dkw in (("ff", {}), ("ff_per_channel", {"merge_branches": 2}), ("paper", {})):
            d = pb.Device(ch, variant="ff" if v.startswith("ff") else v, **dkw)
            o = torch.empty(d.nstate, dtype=torch.float64, device="cuda")
            ms = time_calls(lambda: d.collision(f, out=o), 20, stream)
            res[v] = {"collision_ms": ms, "channels_per_s": ch.nchannels / (ms * 1e-3),
                      "bytes_per_channel": d.bytes_per_channel,
                      "algorithmic_gb_s": d.bytes_per_channel * ch.nchannels / (ms * 1e-3) / 1e9}
            d.close()
        res["paper_time_over_ff"] = res["paper"]["collision_ms"] / res["ff"]["collision_ms"]
        res["paper_time_over_ff_per_channel"] = res["paper"]["collision_ms"] / res["ff_per_channel"]["collision_ms"]
        out[label] = res
        if kw is not None:
            ch.close()
    return out


def compare_variants(pb, ch, dev_ff, fh, ff_ms, mixed_steps, stream):
    """Collision sweep of every variant on the same channel list: time, channels/s, df/dt
    error against the default (which the tests hold to the FP64 oracle at 1e-12), and
    speed-ups over three FP64 GPU paths: the branch-merged native-FP64 coefficient sweep
    (f64), the same with one entry per channel (f64_per_channel), and the literal per-channel
    FP64 form that evaluates the Gaussians and occupations of every channel (literal)."""
    import numpy as np
    import torch

    f = torch.tensor(fh, device="cuda")
    ref = dev_ff.collision(f).cpu().numpy()
    out = {}
    ms = {"ff": ff_ms}
    devs = {}
    peak, _ = measured_hbm()
    for v in ("ff_per_channel", "f64", "f64_per_channel", "literal", "g32", "g16", "h16", "c32"):
        kw = {"merge_branches": 2} if v.endswith("_per_channel") else {}
        d = pb.Device(ch, variant=v.replace("_per_channel", ""), **kw)
        o = torch.empty(d.nstate, dtype=torch.float64, device="cuda")
        ms[v] = time_calls(lambda: d.collision(f, out=o), 5 if v == "literal" else 20, stream)
        err = float(np.abs(o.cpu().numpy() - ref).max() / np.abs(ref).max())
        out[v] = {"collision_ms": ms[v], "channels_per_s": dev_ff.nchannels / (ms[v] * 1e-3),
                  "hbm_gb_s": d.bytes_per_channel * d.nchannels / (ms[v] * 1e-3) / 1e9,
                  "bytes_per_channel": d.bytes_per_channel, "speedup_vs_ff": ff_ms / ms[v],
                  "dfdt_err_vs_fp64": err}
        if v in ("c32", "g32", "g16", "h16", "f64"):
            # the sweep kernel alone, one launch at a time with L2 flushed before each (the C32
            # tiles, 93 MB, fit in the 129 MB L2); beside it the average over back-to-back launches
            k_ms = sweep_ms_flushed(d, f, 30, stream)
            gbs = d.bytes_per_channel * d.nchannels / (k_ms * 1e-3) / 1e9
            out[v]["sweep_kernel"] = {"ms": k_ms, "algorithmic_gb_s": gbs, "frac_of_hbm": gbs / peak,
                                      "timing": "one launch per pair of events, L2 flushed before each",
                                      "ms_back_to_back": d.time_sweep(f, 50, stream=stream)}
            rv = torch.empty_like(o)
            out[v]["rates_ms"] = time_calls(lambda: d.rates(f, out=rv), 10, stream)
        if v in ("g32", "g16", "h16", "c32"):
            devs[v] = d
        else:
            d.close()
    out["ff"] = {"collision_ms": ff_ms, "channels_per_s": dev_ff.nchannels / (ff_ms * 1e-3),
                 "bytes_per_channel": dev_ff.bytes_per_channel}
    for v in out:
        for base in ("f64", "f64_per_channel", "literal"):
            out[v][f"speedup_vs_{base}"] = ms[base] / ms[v]
    # mixed precision along an FP64-accurate RK4 trajectory: per-step df/dt error
    if mixed_steps > 0:
        traj = torch.tensor(fh, device="cuda")
        a = torch.empty_like(traj)
        errs = {v: [] for v in devs}
        bufs = {v: torch.empty_like(traj) for v in devs}
        for _ in range(mixed_steps):
            dev_ff.collision(traj, out=a)
            for v, d in devs.items():
                d.collision(traj, out=bufs[v])
            an = a.abs().max()
            for v in devs:
                errs[v].append(((bufs[v] - a).abs().max() / an))
            dev_ff.rk4(traj, 1.0, 1)
        for v in devs:
            e = torch.stack(errs[v]).cpu().numpy()
            out[v]["dfdt_err_over_steps"] = {"steps": mixed_steps, "max": float(e.max()), "median": float(np.median(e)),
                                             "final": float(e[-1])}
            rk_ms = time_calls(lambda: devs[v].rk4(traj.clone(), 1.0, 20), 3, stream)
            out[v]["rk4_steps_per_s"] = 20 / (rk_ms * 1e-3)
    for d in devs.values():
        d.close()
    return out


def run_ours(args):
    import numpy as np
    import torch

    import synth
    import paper_2511_03683_gb300 as pb

    ws, rank, local = dist()
    torch.cuda.set_device(local)
    if args.only_adjoint:
        if rank == 0:
            print(json.dumps({"adjoint": adjoint_report(pb, torch.cuda.current_stream(), args.adjoint_steps)}))
        return 0
    if ws > 1:
        import torch.distributed as tdist

        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if ws > 1:
            import torch.distributed as tdist

            tdist.barrier()
        torch.cuda.synchronize()

    def rank_max(x: float) -> float:
        return max_over_ranks(x, ws, device="cuda")

    m = synth.make_config(args.workload)
    t0 = time.perf_counter()
    ch = pb.Channels.from_model(m)
    build_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    dev = pb.Device(ch, variant=args.variant, transport=True, tile_sweep=args.tile_sweep, ctas_per_sm=args.ctas_per_sm,
                    transport_gather=args.transport_gather)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    ids = ch.state_ids()
    ns, nch = dev.nstate, dev.nchannels
    fh = m.f_hot().reshape(-1)[ids]
    f0h = m.f_fermi(m.emin() - 0.2).reshape(-1)[ids]
    vh = m.vel.reshape(-1, 3)[ids]
    f = torch.tensor(fh, device="cuda")
    f0 = torch.tensor(f0h, device="cuda")
    v = torch.tensor(vh, device="cuda")
    Fa = torch.zeros((ns, 3), dtype=torch.float64, device="cuda")
    Fb = torch.zeros_like(Fa)
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    dev.transport_setup(f0)
    dt = 1.0
    stream = torch.cuda.current_stream()

    def step(F_in, F_out):
        dev.rk4(f, dt, 1)
        dev.transport_iterate(v, F_in, out=F_out, resid=res)

    clocks = Clocks(local)
    for i in range(args.warmup):
        step(Fa, Fb) if i % 2 == 0 else step(Fb, Fa)
    clocks.start()
    # keep the GPU busy with further untimed steps until the sampler has taken its first
    # sample (at most 3 s), so that its samples cover the timed region
    t_wait = time.time()
    i = 0
    while clocks.proc is not None and not clocks.has_sample() and time.time() - t_wait < 3.0:
        step(Fa, Fb) if i % 2 == 0 else step(Fb, Fa)
        i += 1
        torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    block_ms = []
    for _ in range(max(1, args.repeats)):
        # each block: exactly --steps steps, a barrier and a device synchronisation on both sides
        barrier()
        e0.record(stream)
        for i in range(args.steps):
            step(Fa, Fb) if i % 2 == 0 else step(Fb, Fa)
        e1.record(stream)
        barrier()
        block_ms.append(rank_max(e0.elapsed_time(e1)))
    ms_max = statistics.median(block_ms)
    value = whole_job_value(SWEEPS_PER_STEP * nch * args.steps, ws, ms_max * 1e-3)

    # rt-BTE RK4 steps per second (one call, graph replay)
    nrk = 200
    g = torch.tensor(fh, device="cuda")
    dev.rk4(g, dt, 5)
    torch.cuda.synchronize()
    e0.record(stream)
    dev.rk4(g, dt, nrk)
    e1.record(stream)
    torch.cuda.synchronize()
    rk_ms = e0.elapsed_time(e1)
    # transport iterations per second (device only)
    ntr = 100
    e0.record(stream)
    for i in range(ntr):
        dev.transport_iterate(v, Fa, out=Fb, resid=res) if i % 2 == 0 else dev.transport_iterate(v, Fb, out=Fa, resid=res)
    e1.record(stream)
    torch.cuda.synchronize()
    tr_ms = e0.elapsed_time(e1)

    # dominant kernel: the collision sweep, timed per call on the launching stream
    ncall = 40
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ncall)]
    out = torch.empty(ns, dtype=torch.float64, device="cuda")
    for a, b in evs:
        a.record(stream)
        dev.collision(f, out=out)
        b.record(stream)
    torch.cuda.synchronize()
    coll_ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    rates_ms = None
    if args.variant != "paper":  # the paper layout computes the collision integral only
        for a, b in evs[:10]:
            a.record(stream)
            dev.rates(f, out=out)
            b.record(stream)
        torch.cuda.synchronize()
        rates_ms = statistics.mean(a.elapsed_time(b) for a, b in evs[:10])
    # the sweep kernel alone: CUDA events on this stream around back-to-back launches of it
    # (its 0.19 GB exceed the L2), and one launch at a time with L2 flushed before each
    sweep_ms = dev.time_sweep(f, 50, stream=stream)
    sweep_ms_fl = sweep_ms_flushed(dev, f, 30, stream)
    # back-to-back launches alternating the tile order, as the RK4 stages run them (each sweep
    # starts on the tiles the one before it left in L2)
    sweep_ms_alt = dev.time_sweep(f, 50, order=1, stream=stream)
    clk = clocks.stop()

    bytes_launch = dev.bytes_per_channel * nch
    achieved = bytes_launch / (sweep_ms * 1e-3) / 1e9
    peak, peak_src = measured_hbm()
    traffic = ncu_traffic(args.workload, args.variant, bytes_launch)

    # full transport solve for x, y, z to 1e-10 (the workload's second half)
    solve = None
    if not args.no_solve:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Fs, iters, resid, ok = dev.transport(f0, v, tol=1e-10, maxit=1000)
        solve = {"iterations": iters, "residual": resid, "converged": ok, "seconds": time.perf_counter() - t0}

    # end to end through the C ABI's host-buffer calls from pinned host memory: every step is
    # pb_rtbte_rk4_host (f host -> device, one RK4 step, f device -> host, synchronise) and
    # pb_transport_iterate_host (F host -> device, one transport pass, F device -> host,
    # synchronise), so the host holds both results after every step
    e2e = None
    if not args.no_e2e:
        f_host = torch.tensor(fh).pin_memory()
        F_host = torch.zeros((ns, 3), dtype=torch.float64).pin_memory()
        fnp, Fnp = f_host.numpy(), F_host.numpy()

        def e2e_step():
            dev.rk4_host(f_host, dt, 1, out=f_host, stream=stream)
            dev.transport_iterate_host(v, F_host, out=F_host, stream=stream)

        for _ in range(max(3, min(args.warmup, 5))):
            e2e_step()
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = rank_max(time.perf_counter() - t0)
        assert np.isfinite(fnp).all() and np.isfinite(Fnp).all()
        e2e = {"value": ws * SWEEPS_PER_STEP * nch * args.steps / e2e_s, "unit": "channels/s",
               "h2d_bytes_per_step": 8 * ns + 24 * ns, "d2h_bytes_per_step": 8 * ns + 24 * ns,
               "calls": "pb_rtbte_rk4_host + pb_transport_iterate_host per step (pinned host buffers)"}

    variants = None
    if not args.no_variants and ws == 1:
        variants = compare_variants(pb, ch, dev, fh, coll_ms, args.mixed_steps, stream)

    ablation = None
    if not args.no_ablation and ws == 1:
        ablation = ablation_report(pb, m, ch, stream)

    adjoint = None
    if not args.no_adjoint and ws == 1 and args.workload == "window40":
        adjoint = adjoint_report(pb, stream)

    batched = None
    if not args.no_batched and ws == 1:
        dev.close()
        batched = batched_report(pb, args.batched_instances, args.batched_steps, stream)

    base = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        base, _ = cpu_baseline(m, sample_every=1 if args.workload != "window40" else 4)

    if rank == 0:
        cfg = workload_config(args.workload)
        cfg.update({"nstate": ns, "channels": nch, "variant": args.variant, "tile_sweep": args.tile_sweep,
                    "ctas_per_sm": args.ctas_per_sm, "transport_gather": args.transport_gather,
                    "l2": "inputs larger than L2 "
                    f"({dev.bytes_per_channel * nch / 1e9:.2f} GB streamed per sweep vs 0.13 GB L2)"
                    if args.workload == "window40" else "inputs fit in L2 (latency/parity workload)",
                    "parallelism": f"{ws} independent replica(s)"})
        emit({
            "metric": "e-ph channels/s", "value": value, "unit": "channels/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"ff": "f32x2", "paper": "f32x2", "f64": "f64", "literal": "f64", "g32": "f32",
                      "g16": "f32 (bf16 |g|^2)", "h16": "f32 (fp16 |g|^2 x 2^k)",
                      "c32": "f32 (fp32 coefficient tiles)"}.get(args.variant, args.variant),
            "data": "synthetic", "config": cfg,
            "rk4_steps_per_s": nrk / (rk_ms * 1e-3), "transport_iters_per_s": ntr / (tr_ms * 1e-3),
            "collision_ms": coll_ms, "rates_ms": rates_ms,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "kernel": f"collision sweep ({args.variant} variant), its own launches",
                         "kernel_ms": sweep_ms, "kernel_ms_l2_flushed": sweep_ms_fl,
                         "kernel_ms_alternating_order": sweep_ms_alt,
                         "frac_l2_flushed": bytes_launch / (sweep_ms_fl * 1e-3) / 1e9 / peak, "call_ms": coll_ms,
                         "call_gb_s": bytes_launch / (coll_ms * 1e-3) / 1e9,
                         "bytes_per_channel": dev.bytes_per_channel, "bytes_per_launch": bytes_launch,
                         "layout": "one entry per state pair (branches merged)" if dev.merged else "one entry per channel",
                         "peak_source": peak_src},
            "cpu_baseline": base, "e2e": e2e, "gpu_launches": LAUNCHES_PER_STEP * args.steps,
            "repeats": {"blocks": len(block_ms), "steps_per_block": args.steps, "ms_per_step": [b / args.steps for b in block_ms],
                        "median": ms_max / args.steps, "min": min(block_ms) / args.steps,
                        "max": max(block_ms) / args.steps},
            "state_pairs": {"per_sweep": ns * ns, "per_s": whole_job_value(SWEEPS_PER_STEP * ns * ns * args.steps, ws, ms_max * 1e-3),
                            "channels_per_pair": nch / (ns * ns),
                            "note": "the sweeps stream coefficients summed once per state pair (branches merged at "
                                    "setup); value counts the physical channels those pairs carry"},
            "setup_ms": create_s * 1e3, "setup_in_steps": create_s * 1e3 / (ms_max / args.steps),
            "clocks": clk, "setup": {"build_channels_s": build_s, "device_create_s": create_s},
            "transport_solve": solve, "variants": variants, "batched": batched, "paper_layout": ablation,
            "adjoint": adjoint,
        })
    if ws > 1:
        import torch.distributed as tdist

        tdist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
