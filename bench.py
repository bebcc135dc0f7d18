"""Benchmark: particle-steps/s of the RNA / ARNA filter step on GB300.

Workload (the tracking scenario): one 512x512 spot-tracking sequence, G = 64
groups x 16384 particles (1,048,576), particles initialised at the truth,
ARNA (adaptive exchange share, random ring each step); the RNA 10% fixed-ring
run on the same Philox streams is reported beside it.  Synthetic frames
(see paper_1310_4624_gb300/synth.py).

One timed step = one pf_step over all particles: frame preparation,
exchange + propagation + likelihood, per-group resampling and the global
reduction / next-step ring and ratio.  L2 is flushed (a 256 MB write)
between timed steps, outside the timed interval; each step is timed with
CUDA events on the launch stream.

Beside the headline line's own figures it reports the other forms of the
step on their workloads: the batched form (512 independent tracks of mixed
sizes, one graph-captured launch sequence per frame, against the same tracks
stepped one by one), the adjoint form (forward with ancestry recording plus
pf_backward, against the plain forward), the information-sharing start
(steps until every group mean is within 2 px, PE_eff / G per step) and the
tracking accuracy over 10 sequences (RMSE, ARNA against RNA 10 %).
--no-extras skips them.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]
Under torchrun each rank runs an independent replica (its own seed and
sequence): the path does not shard across GPUs, so N > 1 is weak scaling.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (propagate+weight+ARNA)"
UNIT = "particle-steps/s"

# Algorithmic work per particle-step, fixed for the roofline: FP32 / INT32
# lane operations (likelihood 121 pixels x 3 + 44 Gaussian arguments + 11
# hoisted products, propagation 10, Box-Muller ~15, uniform maps 6, Philox 2
# calls x 10 rounds x ~8), MUFU operations (22 ex2, 3 lg2, 3 sqrt, 6
# sin/cos), and HBM bytes (parent state 20 + new state 20 + ancestor written
# 4 + ancestor read 4).  These are counts of the method, not of the kernels:
# arithmetic the kernels save (fused multiply-adds, recurrences) raises the
# reported fraction and does not lower the work credited.
ALG_LANE_OPS = 610
ALG_SFU_OPS = 34
ALG_BYTES = 48
# The same lane count with two fused multiply-adds per pixel, a tighter
# reading of the likelihood (reported beside the fixed one, labelled).
ALG_LANE_OPS_FMA = 540


def kernel_source_hash() -> str:
    """sha256 of the kernel sources' code (comments and blank lines left
    out, so that editing a comment keeps a profile valid); ncu figures in
    profiles/ are tied to it."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("pf_kernels.cu", "pf_device.cuh", "pf_math.cuh", "pf_launch.h"):
        with open(os.path.join(ROOT, "paper_1310_4624_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        code = "\n".join(line.rstrip() for line in text.splitlines() if line.strip())
        h.update(code.encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from profiles/*.md, if captured on
    the current kernel sources (else None)."""
    import glob
    import re
    src = kernel_source_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        text = open(path).read()
        m = re.search(r"kernel sources sha256\[:16\]: ([0-9a-f]{16})", text)
        if not m or m.group(1) != src:
            continue
        t = re.search(r"traffic_bytes_per_launch %s: ([0-9]+)" % re.escape(kernel), text)
        if t:
            return int(t.group(1)), os.path.basename(path)
    return None, None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=sorted(reasons), samples=len(rows))
        return out


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int, dev) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def time_filter(pf, fr, first: int, K: int, flush, profile: bool):
    """Device time (ms) of K steps, L2 flushed before each."""
    import torch
    stream = pf.stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    if profile:
        pf.profile(True)
    for i in range(K):
        flush.zero_()
        evs[i][0].record(stream)
        pf.step(fr[first + i])
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    if profile:
        pf.profile(False)
    return sum(a.elapsed_time(b) for a, b in evs)


def _oracle_rate(wl, frames, truth, steps: int, threads: int, first: int = 1):
    """particle-steps/s of the FP64 oracle (as it stands) over steps
    first .. first+steps-1 of `wl` after untimed steps 0 .. first-1, on
    `threads` host threads; returns (rate, seconds, threads used)."""
    import oracle as ora
    from paper_1310_4624_gb300 import synth
    ocfg = ora.cfg_from_workload(wl)
    kind, x0, lo, hi, rad = synth.init_arrays(wl, np.float32(truth[0]).astype(np.float64))
    f = lambda a: np.float32(a).astype(np.float64)  # noqa: E731
    pop = ora.init_population(ocfg, kind, f(x0), f(lo), f(hi), float(np.float32(rad)))
    used = ora.set_threads(threads)
    try:
        lam = None
        for k in range(first):
            r = ora.step(ocfg, k, frames[k], pop, lam)
            pop, lam = r.pop_out, r.Lambda
        t0 = time.perf_counter()
        for k in range(first, first + steps):
            r = ora.step(ocfg, k, frames[k], pop, lam)
            pop, lam = r.pop_out, r.Lambda
        dt = time.perf_counter() - t0
    finally:
        ora.set_threads(1)
    return wl.N * steps / dt, dt, used


def cpu_baseline(wl, frames, truth, steps: int = 8, steps_single: int = 4):
    """The FP64 oracle as it stands on the full workload population: `steps`
    steps with its loops on every host core (OpenMP over particles and
    groups), and `steps_single` steps on one thread, each after an untimed
    step 0."""
    cores = os.cpu_count() or 1
    v, dt, used = _oracle_rate(wl, frames, truth, steps, cores)
    v1, dt1, _ = _oracle_rate(wl, frames, truth, steps_single, 1)
    return {"value": v, "unit": UNIT, "cores": used, "kind": "oracle", "host_cpu_count": cores,
            "sample": "%d oracle steps (k=1..%d) of the full %d-particle workload, FP64, %d threads, %.1f s"
                      % (steps, steps, wl.N, used, dt),
            "single_thread": {"value": v1, "cores": 1,
                              "sample": "%d steps (k=1..%d), 1 thread, %.1f s" % (steps_single, steps_single, dt1)}}


def bench_oracle_configs():
    """The oracle timed on the host cores (all of them, OpenMP; and one
    thread) per workload: the small RNA run and the information-sharing run
    in full, the tracking and differentiable runs on their first 5 frames,
    and 8 tracks drawn from the batched workload."""
    from paper_1310_4624_gb300 import synth
    cores = os.cpu_count() or 1
    out = {"host_cpu_count": cores}
    jobs = [("small_rna", synth.small_rna(), None, 0),
            ("sharing_arna", synth.sharing(mode=synth.ARNA), None, 0),
            ("tracking_arna", synth.tracking(mode=synth.ARNA), 5, 0),
            ("differentiable", synth.differentiable(), 5, 0)]
    for name, wl, T, _ in jobs:
        T = wl.T if T is None else T
        frames, truth = synth.make_sequence(wl, T=T)
        v, dt, used = _oracle_rate(wl, frames, truth, T, cores, first=0)
        row = {"value": v, "unit": UNIT, "threads": used, "steps": T, "particles": wl.N, "seconds": dt}
        if name == "small_rna":
            v1, dt1, _ = _oracle_rate(wl, frames, truth, T, 1, first=0)
            row["single_thread"] = {"value": v1, "seconds": dt1}
        out[name] = row
    # batched: 8 of the 512 tracks (every 64th), 50 frames each
    wls = synth.batched_tracks(512)[::64]
    n, secs = 0, 0.0
    for wl in wls:
        frames, truth = synth.make_sequence(wl)
        v, dt, used = _oracle_rate(wl, frames, truth, wl.T, cores, first=0)
        n += wl.N * wl.T
        secs += dt
    out["batched_8_tracks"] = {"value": n / secs, "unit": UNIT, "threads": used, "tracks": len(wls),
                               "particle_steps": n, "seconds": secs}
    return out


def run_reference(args, ws, rank):
    """The reference arm: the FP64 CPU oracle, timed as it stands, on the
    same workload (all 64 x 16384 particles of the tracking run, ARNA), its
    per-particle and per-group loops on every host core; W untimed steps,
    then K timed steps."""
    if rank != 0:
        return
    from paper_1310_4624_gb300 import synth
    K, W = args.steps, args.warmup
    wl = synth.tracking(mode=synth.ARNA, T=K + W + 1)
    frames, truth = synth.make_sequence(wl)
    cores = os.cpu_count() or 1
    value, dt, used = _oracle_rate(wl, frames, truth, K, cores, first=W)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
            "warmup": W, "ms_per_step": dt / K * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "particles": wl.N, "G": wl.G, "Np": wl.Np,
                       "frame": "%dx%d" % (wl.H, wl.W), "mode": "ARNA", "init": "all particles at the truth"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": used, "kind": "oracle",
                             "sample": "steps %d..%d of the full %d-particle workload, FP64 oracle, %d threads, %.1f s"
                                       % (W, W + K - 1, wl.N, used, dt)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _lane_peak(dev):
    """SMs x 128 lanes x the maximum SM clock (per second)."""
    import torch
    peaks, _ = _peaks()
    return torch.cuda.get_device_properties(dev).multi_processor_count * 128 * float(
        peaks.get("sm_max_mhz", 2070.0)) * 1e6


def _events(stream, fn):
    """Device time (ms) of fn() on `stream`, synchronised on both sides."""
    import torch
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def bench_configs(dev, reps: int = 3):
    """GPU particle-steps/s of the other single-track workloads, whole
    sequences timed with CUDA events (best of `reps`; L2 not flushed inside a
    sequence): the small RNA run (20 frames 64 x 64, G = 4 x 1024, RNA 10 %)
    through pf_step and through the CUDA-graph step (pf_graph_step, frames
    from a device table), and the information-sharing run (100 frames 512 x
    512, G = 256 x 4096, sharing start) for ARNA and RNA 10 %."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    out = {}
    wl = synth.small_rna()
    frames, truth = synth.make_sequence(wl)
    fr = torch.from_numpy(frames).to(dev)
    pf = ParticleFilter([config_from_workload(wl, truth[0])], history=wl.T + 1, device=dev)
    table = pf.frame_table([fr])
    best_step, best_graph = 1e30, 1e30
    for _ in range(reps):
        pf.reset()
        best_step = min(best_step, _events(pf.stream, lambda: [pf.step(fr[k]) for k in range(wl.T)]))
        pf.reset()
        best_graph = min(best_graph, _events(pf.stream, lambda: [pf.step_table(table, graph=True)
                                                                  for _ in range(wl.T)]))
    pf.close()
    n = wl.N * wl.T
    out["small_rna"] = {"workload": wl.name, "particles": wl.N, "steps": wl.T, "unit": UNIT,
                        "pf_step": {"value": n / (best_step / 1e3), "ms_per_step": best_step / wl.T},
                        "graph": {"value": n / (best_graph / 1e3), "ms_per_step": best_graph / wl.T}}
    frames = fr = None
    for mode, name in ((synth.ARNA, "sharing_arna"), (synth.RNA, "sharing_rna10")):
        wl = synth.sharing(mode=mode)
        if frames is None:
            frames, truth = synth.make_sequence(wl)
            fr = torch.from_numpy(frames).to(dev)
        pf = ParticleFilter([config_from_workload(wl, truth[0])], history=wl.T + 1, device=dev)
        best = 1e30
        for _ in range(reps):
            pf.reset()
            best = min(best, _events(pf.stream, lambda: [pf.step(fr[k]) for k in range(wl.T)]))
        pf.close()
        out[name] = {"workload": wl.name, "particles": wl.N, "steps": wl.T, "unit": UNIT,
                     "value": wl.N * wl.T / (best / 1e3), "ms_per_step": best / wl.T}
    return out


def bench_batched(dev, K: int, W: int, flush, n_tracks: int = 512, k_alone: int = 8):
    """512 independent tracks (256 x 256 frames, 50-frame sequences; particle
    counts log-uniform in [4096, 262144], groups log-uniform in [4, 128],
    spot amplitude U[5, 20], PSF width U[1.2, 2.0]) in one handle: autotuned
    launch shapes, frames through a device table, each step one CUDA graph
    launch.  Against it, the same tracks in 512 handles stepped one by one
    with pf_step (the first `k_alone` timed steps)."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    T = max(50, W + K + 6)  # autotuned step, warm-up, timed steps, three profiled steps
    wls = synth.batched_tracks(n_tracks, T=T)
    frames, truths = synth.render_batched_torch(wls, dev, seed=0)
    cfgs = [config_from_workload(wl, truths[t][0], track_id=t) for t, wl in enumerate(wls)]
    n_total = sum(wl.N for wl in wls)
    pf = ParticleFilter(cfgs, history=4, device=dev)
    table = pf.frame_table([frames[t] for t in range(n_tracks)])
    grid, cluster = pf.autotune([frames[t, 0] for t in range(n_tracks)])
    for _ in range(W):
        pf.step_table(table, graph=True)
    ms = 0.0
    for _ in range(K):
        flush.zero_()
        ms += _events(pf.stream, lambda: pf.step_table(table, graph=True))
    # the kernels of a step (per-kernel events serialise them; not the timed steps)
    pf.profile(True)
    for _ in range(3):
        flush.zero_()
        pf.step_table(table, graph=False)
    prof = pf.profile_read()
    pf.profile(False)
    _, logz, st = pf.estimate()
    pf.close()
    pixels = sum(wl.H * wl.W for wl in wls)
    # the same tracks one by one through the plain entry point
    alone = [ParticleFilter([c], history=4, device=dev) for c in cfgs]
    for k in range(W):
        for t, a in enumerate(alone):
            a.step(frames[t, k])
    Ka = min(K, k_alone)

    def one_by_one(k):
        for t, a in enumerate(alone):
            a.step(frames[t, k])
    ms_alone = 0.0
    for k in range(W, W + Ka):
        flush.zero_()
        ms_alone += _events(alone[0].stream, lambda: one_by_one(k))
    for a in alone:
        a.close()
    del frames, table
    return {"workload": "batched_%dtracks_256x256" % n_tracks, "tracks": n_tracks, "particles": n_total,
            "G_range": [min(w.G for w in wls), max(w.G for w in wls)],
            "particles_range": [min(w.N for w in wls), max(w.N for w in wls)],
            "value": n_total * K / (ms / 1e3), "ms_per_step": ms / K, "unit": UNIT,
            "form": "one handle, autotuned (propagate grid %d, resample cluster %d), CUDA graph per step"
                    % (grid, cluster),
            "one_by_one": {"value": n_total * Ka / (ms_alone / 1e3), "ms_per_step": ms_alone / Ka,
                           "steps": Ka, "form": "512 handles, pf_step each, same stream"},
            "speedup": (ms_alone / Ka) / (ms / K), "degenerate_status": int(st),
            "roofline_frac": ALG_LANE_OPS * n_total / (ms / K / 1e3) / _lane_peak(dev),
            "kernels": {n: {"launches": c, "ms_per_launch": t / max(1, c)} for n, (c, t) in prof.items() if c > 0},
            "frame_prep_hbm_bound_ms": 8.0 * pixels / (float(_peaks()[0]["hbm_gbs"]) * 1e9) * 1e3}


def bench_adjoint(dev, flush, reps: int = 3):
    """Differentiable workload: 50 frames 512 x 512, G = 16 x 65536, ARNA.
    Forward without recording, forward recording the ancestry, and
    pf_backward (replay + adjoint of log Z over the 50 steps); each timed
    `reps` times after a warm-up pass, L2 flushed before each pass."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wl = synth.differentiable()
    frames, truth = synth.make_sequence(wl)
    fr = torch.from_numpy(frames).to(dev)
    flist = [fr[k] for k in range(wl.T)]

    def forward(pf):
        pf.reset()
        for k in range(wl.T):
            pf.step(fr[k])

    out = {}
    for rec in (False, True):
        pf = ParticleFilter([config_from_workload(wl, truth[0], record_ancestors=rec)], history=wl.T + 1,
                            device=dev)
        forward(pf)
        if rec:
            pf.backward(flist)
        f_ms, b_ms = [], []
        for _ in range(reps):
            flush.zero_()
            f_ms.append(_events(pf.stream, lambda: forward(pf)))
            if rec:
                flush.zero_()
                grad = []
                b_ms.append(_events(pf.stream, lambda: grad.append(pf.backward(flist))))
        out["fwd_rec" if rec else "fwd"] = min(f_ms)
        if rec:
            out["bwd"] = min(b_ms)
            g, lz = grad[-1]
            out["grad"] = [float(v) for v in g[0].cpu()]
            out["log_Z"] = float(lz[0])
        if rec:
            out["fit"] = adam_fit(pf, wl, fr, truth)
            out["fit_observation"] = adam_fit(pf, wl, fr, truth, fit=(0, 1, 2))
        pf.close()
    n = wl.N * wl.T
    lane = _lane_peak(dev)
    return {"fit": out["fit"], "fit_observation_only": out["fit_observation"], "workload": wl.name,
            "fwd_roofline_frac": ALG_LANE_OPS * n / (out["fwd"] / 1e3) / lane,
            "fwd_bwd_rate_over_fwd_roofline": ALG_LANE_OPS * n / ((out["fwd_rec"] + out["bwd"]) / 1e3) / lane, "particles": wl.N, "steps": wl.T, "unit": UNIT,
            "fwd": {"value": n / (out["fwd"] / 1e3), "ms": out["fwd"]},
            "fwd_recording": {"value": n / (out["fwd_rec"] / 1e3), "ms": out["fwd_rec"]},
            "fwd_bwd": {"value": n / ((out["fwd_rec"] + out["bwd"]) / 1e3), "ms": out["fwd_rec"] + out["bwd"]},
            "bwd_ms": out["bwd"], "fwd_bwd_over_fwd": (out["fwd_rec"] + out["bwd"]) / out["fwd"],
            "grad_theta": dict(zip(("sigma_psf", "A", "b", "sigma_pos", "sigma_v"), out["grad"])),
            "log_Z": out["log_Z"], "timing": "best of %d passes, CUDA events" % reps}


def adam_fit(pf, wl, fr, truth, iters: int = 200, lr: float = 0.02, fit=(0, 1, 2, 3, 4)):
    """Maximum-likelihood fit of theta = (sigma_psf, A, b, sigma_pos, sigma_v)
    by Adam on log theta, from theta_true x 1.3 on the components in `fit`
    (the others held at the truth), each iteration one forward run
    (ancestry recorded) and one pf_backward (common random numbers: the
    filter's seed is fixed).  The gradient holds the resampling ancestry
    fixed, so it is biased for sigma_pos and sigma_v, which move particles
    across the resampling decisions; sigma_psf, A and b do not."""
    import torch
    from paper_1310_4624_gb300.filter import LogLikelihood
    names = ("sigma_psf", "A", "b", "sigma_pos", "sigma_v")
    true = np.array([wl.sigma_psf, float(np.float32(truth[0][4])), wl.background, wl.sigma_pos, wl.sigma_v])
    mask = torch.tensor([1.0 if q in fit else 0.0 for q in range(5)], dtype=torch.float64)
    start = np.where(mask.numpy() > 0, true * 1.3, true)
    logt = torch.tensor(np.log(start), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([logt], lr=lr)
    first = last = None
    t0 = time.perf_counter()
    for it in range(iters):
        opt.zero_grad()
        lz = LogLikelihood.apply(torch.exp(logt), pf, fr)
        (-lz).backward()
        logt.grad.mul_(mask)
        opt.step()
        v = float(lz.detach())
        first = v if first is None else first
        last = v
    dt = time.perf_counter() - t0
    pf.set_theta(true)
    lz_true = float(LogLikelihood.apply(torch.tensor(true), pf, fr))
    end = np.exp(logt.detach().numpy())
    return {"iters": iters, "lr_log_theta": lr, "theta_true": dict(zip(names, true.round(4).tolist())),
            "fitted": [names[q] for q in fit],
            "theta_start": dict(zip(names, start.round(4).tolist())),
            "theta_end": dict(zip(names, end.round(4).tolist())),
            "log_Z_start": first, "log_Z_end": last, "log_Z_at_true": lz_true, "seconds": dt}


def bench_sharing(dev):
    """Information-sharing start: 100 frames 512 x 512, G = 256 x 4096, group
    0 in a 2 px disc around the truth, the other groups uniform over the
    image.  For ARNA, RNA 10 %, ARNA with keyed random send sets, and the
    topologies of Sec. VI (ARNA on a ring that keeps nodes of 16 groups
    together; ARNA and RNA 10 % on the hypercube), under the patch-residual
    likelihood and the frame likelihood ratio: the first step at which every group mean is
    within 2 px of the truth, the first steps at which PE_eff / G reaches 0.5
    and 0.9 (Sec. V-B's recovery of PE_eff), the final estimate's error, and
    PE_eff / G per step."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    out = {}
    frames = truth = fr = None
    for obs_name, obs in (("patch", 0), ("frame", 1)):
        res = {}
        runs = (("arna", dict(mode=synth.ARNA)), ("rna10", dict(mode=synth.RNA)),
                ("arna_keyed", dict(mode=synth.ARNA, send_rule=1)),
                ("arna_node_ring16", dict(mode=synth.ARNA, topology=1, node_groups=16)),
                ("arna_hypercube", dict(mode=synth.ARNA, topology=2)),
                ("rna10_hypercube", dict(mode=synth.RNA, topology=2)))
        for name, kw in runs:
            wl = synth.sharing(obs_model=obs, **kw)
            if frames is None:
                frames, truth = synth.make_sequence(wl)
                fr = torch.from_numpy(frames).to(dev)
            pf = ParticleFilter([config_from_workload(wl, truth[0])], history=wl.T + 1, device=dev)
            for k in range(wl.T):
                pf.step(fr[k])
            pe, nex, first = [], [], None
            for k in range(wl.T):
                st = pf.stats(k)
                gx = st["group_xhat"]
                d = np.hypot(gx[0] - truth[k, 0], gx[1] - truth[k, 1])
                if first is None and np.all(d <= 2.0):
                    first = k
                pe.append(round(st["pe_eff"] / wl.G, 4))
                nex.append(st["n_ex"])
            xhat, _, _ = pf.estimate()
            pf.close()

            def first_at(level):
                return next((k for k, v in enumerate(pe) if k >= 1 and v >= level), None)
            res[name] = {
                "steps_to_all_groups_within_2px": first, "steps_to_pe_eff_0.5": first_at(0.5),
                "steps_to_pe_eff_0.9": first_at(0.9), "pe_eff_over_G_last": pe[-1],
                "final_error_px": float(np.hypot(*(xhat[0, :2] - truth[-1, :2]))),
                "pe_eff_over_G": pe[:40], "n_ex": nex[:40]}
        out[obs_name] = res
    out["workload"] = synth.sharing().name.rsplit("_", 1)[0]
    return out


def bench_pe_eff_recovery(dev, G_list=(24, 96, 192, 384), Np: int = 4096, T: int = 30):
    """PE_eff / G per iteration from the information-sharing start (group 0
    at the truth, the others spread over the image), for 24, 96, 192 and 384
    groups of 4096 particles, ARNA against RNA with 10 % and 50 % exchange,
    under the frame likelihood ratio (with which spread-out groups can find
    the spot).  The quantity of Sec. V-B's recovery figure; the paper quotes
    it after 10 and 20 iterations."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    out = {}
    base = synth.sharing(T=T, obs_model=1)
    frames, truth = synth.make_sequence(base)
    fr = torch.from_numpy(frames).to(dev)
    modes = {"arna": dict(mode=synth.ARNA), "rna10": dict(mode=synth.RNA, ex_ratio=0.10),
             "rna50": dict(mode=synth.RNA, ex_ratio=0.50)}
    for G in G_list:
        row = {}
        for name, kw in modes.items():
            wl = base.replace(G=G, Np=Np, **kw)
            pf = ParticleFilter([config_from_workload(wl, truth[0])], history=T + 1, device=dev)
            for k in range(T):
                pf.step(fr[k])
            pe = [h["pe_eff"] / G for h in pf.history_stats(0, T)]
            pf.close()
            row[name] = {"at_10": round(pe[10], 4), "at_20": round(pe[min(20, T - 1)], 4),
                         "curve": [round(v, 4) for v in pe]}
        out["G%d" % G] = row
    out["particles_per_group"] = Np
    return out


def bench_rmse_vs_groups(dev, G_list=(24, 96, 192, 384), Np: int = 40, n_seq: int = 5):
    """Tracking accuracy with a constant 40 particles per group, initialised
    at the target (Sec. V-A's accuracy figure): position RMSE over `n_seq`
    tracking sequences for 24 ... 384 groups, ARNA against RNA with 10 % and
    50 % exchange."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wls = [synth.tracking(data_seed=s) for s in range(n_seq)]
    frames, truths = synth.render_batched_torch(wls, dev, seed=2)
    modes = {"arna": dict(mode=synth.ARNA), "rna10": dict(mode=synth.RNA, ex_ratio=0.10),
             "rna50": dict(mode=synth.RNA, ex_ratio=0.50)}
    out = {}
    for G in G_list:
        row = {}
        for name, kw in modes.items():
            se, n = 0.0, 0
            for s, wl0 in enumerate(wls):
                wl = wl0.replace(G=G, Np=Np, **kw)
                pf = ParticleFilter([config_from_workload(wl, truths[s][0])], history=wl.T + 1, device=dev)
                for k in range(wl.T):
                    pf.step(frames[s, k])
                for h in pf.history_stats(0, wl.T):
                    se += float(np.sum((h["xhat"][:2] - truths[s][h["step"], :2]) ** 2))
                    n += 1
                pf.close()
            row[name] = round(math.sqrt(se / n), 4)
        out["G%d" % G] = row
    out["particles_per_group"] = Np
    out["sequences"] = n_seq
    return out


def bench_multi_object(dev, n_obj: int = 64, G: int = 16, Np: int = 1024, T: int = 50):
    """Multi-object tracking as one filter per object: 64 spots on 512 x 512
    frames (one per 64 x 64 cell, drifting), one ARNA track of 16 groups x
    1024 particles per spot (1 048 576 particles), every track reading the
    same frame.  Device time of the whole sequence (CUDA events, L2 not
    flushed), particle-steps/s and the per-object position RMSE."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wls = synth.multi_object(n_obj=n_obj, G=G, Np=Np, H=512, W=512, T=T, cell=64)
    frames, truths = synth.make_multi_sequence(wls)
    fr = torch.from_numpy(frames).to(dev)
    pf = ParticleFilter([config_from_workload(wl, truths[t][0], track_id=t) for t, wl in enumerate(wls)],
                        history=T + 1, device=dev)
    pf.step([fr[0]] * n_obj)
    ms = _events(pf.stream, lambda: [pf.step([fr[k]] * n_obj) for k in range(1, T)])
    rmse = []
    for t in range(n_obj):
        hs = pf.history_stats(0, T, track=t)
        e = np.array([np.sum((h["xhat"][:2] - truths[t][h["step"], :2]) ** 2) for h in hs])
        rmse.append(float(math.sqrt(e.mean())))
    pf.close()
    N = n_obj * G * Np
    return {"workload": wls[0].name, "objects": n_obj, "particles": N, "unit": "particle-steps/s",
            "value": N * (T - 1) / (ms / 1e3), "ms_per_step": ms / (T - 1),
            "rmse_px_mean": float(np.mean(rmse)), "rmse_px_max": float(np.max(rmse))}


def bench_accuracy(dev, n_seq: int = 10):
    """Tracking accuracy and per-mode step time on the tracking workload over
    `n_seq` sequences (data seeds 0..n_seq-1, rendered on the device):
    position RMSE of the global estimate against the truth, for ARNA and RNA
    with 0 %, 10 % and 50 % exchange on identical Philox streams (the paper's
    comparison, Sec. V-A), ARNA and RNA 10 % that resample a group only when
    its N_eff falls below Np / 2 (Alg. 1's test), and the mean device time
    per step of each (CUDA events around whole 100-step runs; L2 not flushed
    between steps) with the mean number of groups that resampled per step."""
    import torch
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload
    wls = [synth.tracking(mode=synth.ARNA, data_seed=s) for s in range(n_seq)]
    frames, truths = synth.render_batched_torch(wls, dev, seed=1)
    modes = {"arna": dict(mode=synth.ARNA), "rna0": dict(mode=synth.RNA, ex_ratio=0.0),
             "rna10": dict(mode=synth.RNA, ex_ratio=0.10), "rna50": dict(mode=synth.RNA, ex_ratio=0.50),
             "arna_ess50": dict(mode=synth.ARNA, resample_rule=1, ess_fraction=0.5),
             "arna_keyed": dict(mode=synth.ARNA, send_rule=1),
             "rna10_ess50": dict(mode=synth.RNA, ex_ratio=0.10, resample_rule=1, ess_fraction=0.5)}
    out = {}
    for name, kw in modes.items():
        se, per, ms, nres = 0.0, [], 0.0, 0
        for s, wl in enumerate(wls):
            wl = wl.replace(**kw)
            pf = ParticleFilter([config_from_workload(wl, truths[s][0])], history=wl.T + 1, device=dev)
            ms += _events(pf.stream, lambda: [pf.step(frames[s, k]) for k in range(wl.T)])
            hs = pf.history_stats(0, wl.T)
            e = np.array([np.sum((h["xhat"][:2] - truths[s][h["step"], :2]) ** 2) for h in hs])
            per.append(float(math.sqrt(e.mean())))
            se += float(e.sum())
            nres += sum(h["resampled"] for h in hs)
            pf.close()
        out[name] = {"rmse_px": math.sqrt(se / (n_seq * wls[0].T)), "per_sequence": [round(v, 4) for v in per],
                     "ms_per_step": ms / (n_seq * wls[0].T),
                     "resampled_groups_per_step": nres / (n_seq * wls[0].T)}
    out["sequences"] = n_seq
    out["workload"] = wls[0].name.rsplit("_", 1)[0]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched / adjoint / sharing / accuracy forms")
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    K, W = args.steps, max(3, args.warmup)

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as ge
    ge.build()
    from paper_1310_4624_gb300 import synth
    from paper_1310_4624_gb300.filter import ParticleFilter, config_from_workload

    KP = min(K, 20)          # profiled steps (per-kernel events), after the timed ones
    T = W + K + KP + 1
    res = {}
    for mode in (synth.ARNA, synth.RNA):
        wl = synth.tracking(mode=mode, T=T, seed=rank, data_seed=rank)
        frames, truth = synth.make_sequence(wl)
        fr = torch.from_numpy(frames).to(dev)
        pf = ParticleFilter([config_from_workload(wl, truth[0], track_id=0)], history=T + 1, device=dev)
        for k in range(W):
            pf.step(fr[k])
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        torch.cuda.synchronize()
        sampler = ClockSampler(local) if mode == synth.ARNA else None
        barrier(ws)
        if sampler:
            sampler.start()
        ms = time_filter(pf, fr, W, K, flush, profile=False)
        clocks = sampler.stop() if sampler else None
        barrier(ws)
        # per-kernel CUDA events on further steps (events between the kernels
        # serialise them, so these steps are not the timed ones)
        time_filter(pf, fr, W + K, KP, flush, profile=True)
        prof = pf.profile_read()
        hs = pf.history_stats(0, W + K + KP)
        rmse = math.sqrt(np.mean([np.sum((h["xhat"][:2] - truth[h["step"], :2]) ** 2) for h in hs]))
        res[mode] = dict(wl=wl, ms=reduce_max(ms, ws, dev), prof=prof, clocks=clocks, rmse=rmse,
                         n_ex=[h["n_ex"] for h in hs], frames=frames, truth=truth)
        pf.close()
        del flush

    # end to end through the public API, every step: pf_step_host on the
    # frame in page-locked host memory (the library uploads it on its own
    # stream into a device staging slot, so frame k+1 uploads while step k
    # runs), and the estimate read back to page-locked host memory
    # (pf_estimate_async: the finishing kernel stores it there); the host
    # consumes step k's estimate after enqueueing step k+1, and the clock
    # stops once the last estimate is on the host
    wl = res[synth.ARNA]["wl"]
    frames = res[synth.ARNA]["frames"]
    truth = res[synth.ARNA]["truth"]
    host = torch.from_numpy(frames).pin_memory()
    host_k = [host[k] for k in range(host.shape[0])]
    pf = ParticleFilter([config_from_workload(wl, truth[0])], history=T + 1, device=dev)
    ev_done = [torch.cuda.Event() for _ in range(2)]
    x_out = [torch.zeros((1, 5), dtype=torch.float32).pin_memory() for _ in range(2)]
    z_out = [torch.zeros(1, dtype=torch.float64).pin_memory() for _ in range(2)]
    est = []

    def enqueue(k):
        b = k & 1
        pf.step_host(host_k[k])
        pf.estimate_async(x_out[b], z_out[b])
        ev_done[b].record(pf.stream)

    def run(first, count):
        for k in range(first, first + count):
            enqueue(k)
            if k > first:
                ev_done[(k - 1) & 1].synchronize()
                est.append(x_out[(k - 1) & 1][0, :2].tolist())
        ev_done[(first + count - 1) & 1].synchronize()
        est.append(x_out[(first + count - 1) & 1][0, :2].tolist())

    run(0, W)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    run(W, K)
    t1 = time.perf_counter()
    e2e_s = reduce_max(t1 - t0, ws, dev)
    pf.estimate()  # reports any device error of the run
    pf.close()

    a = res[synth.ARNA]
    n_all = wl.N * ws
    value = n_all * K / (a["ms"] / 1e3)
    peaks, src = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    lane_peak = sms * 128 * f_max
    prof_launches = sum(c for c, _ in a["prof"].values())
    # the dominant kernel: the fused step (one launch per step), or the
    # propagate kernel of the two-launch step
    fused = a["prof"].get("fused_step", (0, 0.0))[0] > 0
    k1_name = "fused_step" if fused else "propagate_weight"
    k1_launches, k1_ms = a["prof"][k1_name]
    k1_avg_s = k1_ms / 1e3 / max(1, k1_launches)
    achieved = ALG_LANE_OPS * wl.N / k1_avg_s
    traffic, traffic_src = profiled_traffic("k_propagate_weight")
    step_s = a["ms"] / K / 1e3
    hbm = float(peaks["hbm_gbs"]) * 1e9
    sfu_peak = sms * 16 * f_max
    sm_mhz = a["clocks"]["sm_mhz"] if a["clocks"] and a["clocks"].get("sm_mhz") else None
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": lane_peak / 1e12, "unit": "Tops/s",
                "frac": achieved / lane_peak, "traffic": traffic, "traffic_source": traffic_src,
                "kernel": "k_propagate_weight (fused step)" if fused else "k_propagate_weight", "peak_source": "%d SMs x 128 lanes x %.0f MHz (%s sm_max_mhz)"
                % (sms, f_max / 1e6, src),
                "work_per_particle": {"lane_ops": ALG_LANE_OPS, "mufu": ALG_SFU_OPS, "hbm_bytes": ALG_BYTES},
                "kernel_ms": k1_avg_s * 1e3,
                "frac_at_sampled_clock": achieved / (sms * 128 * sm_mhz * 1e6) if sm_mhz else None,
                "frac_fma_count": ALG_LANE_OPS_FMA * wl.N / k1_avg_s / lane_peak,
                "hbm_frac": ALG_BYTES * wl.N / k1_avg_s / hbm,
                "sfu_frac": ALG_SFU_OPS * wl.N / k1_avg_s / sfu_peak,
                # the whole step (every kernel of pf_step, device-timed), against
                # the step's bound: the slowest of lane ops, MUFU and HBM bytes
                "step": {"ms": step_s * 1e3, "achieved": ALG_LANE_OPS * wl.N / step_s / 1e12,
                         "frac": ALG_LANE_OPS * wl.N / step_s / lane_peak,
                         "frac_at_sampled_clock": (ALG_LANE_OPS * wl.N / step_s / (sms * 128 * sm_mhz * 1e6)
                                                   if sm_mhz else None),
                         "bound_ms": 1e3 * wl.N * max(ALG_LANE_OPS / lane_peak, ALG_SFU_OPS / sfu_peak,
                                                       ALG_BYTES / hbm),
                         "hbm_frac": ALG_BYTES * wl.N / step_s / hbm}}
    kernels = {n: {"launches": c, "ms_per_launch": ms / max(1, c), "share": ms / max(1e-12, sum(
        v[1] for v in a["prof"].values()))} for n, (c, ms) in a["prof"].items() if c > 0}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": W,
            "ms_per_step": a["ms"] / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": a["wl"].name, "particles": wl.N, "G": wl.G, "Np": wl.Np,
                       "frame": "%dx%d" % (wl.H, wl.W), "mode": "ARNA", "init": "all particles at the truth",
                       "parallelism": "replicas" if ws > 1 else "single",
                       "l2": "flushed (256 MB write) before every timed step, outside the timed interval"},
            "e2e": {"value": n_all * K / e2e_s, "unit": UNIT, "h2d_bytes_per_step": wl.H * wl.W * 4,
                    "d2h_bytes_per_step": 5 * 4 + 8,
                    "form": "wall clock; per step pf_step_host on a page-locked host frame (uploaded by the "
                            "library on its own stream, overlapping the previous step), pf_estimate_async into "
                            "page-locked memory (stored by the finishing kernel), the estimate consumed on the "
                            "host one step later"},
            "gpu_launches": int(round(prof_launches / KP * K)),
            "roofline": roofline,
            "kernels": kernels,
            "clocks": a["clocks"],
            "rmse_px": a["rmse"],
            "rna10": {"value": n_all * K / (res[synth.RNA]["ms"] / 1e3), "ms_per_step": res[synth.RNA]["ms"] / K,
                      "rmse_px": res[synth.RNA]["rmse"]},
            "arna_n_ex": a["n_ex"][:12]}
    if not args.no_extras:
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
        line["configs"] = bench_configs(dev)
        line["batched"] = bench_batched(dev, K, W, flush)
        line["adjoint"] = bench_adjoint(dev, flush)
        line["sharing"] = bench_sharing(dev)
        line["accuracy"] = bench_accuracy(dev)
        line["multi_object"] = bench_multi_object(dev)
        line["pe_eff_recovery"] = bench_pe_eff_recovery(dev)
        line["rmse_vs_groups"] = bench_rmse_vs_groups(dev)
        del flush
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl, frames, truth)
        if not args.no_extras:
            line["oracle_by_config"] = bench_oracle_configs()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
