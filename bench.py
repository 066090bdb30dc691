#!/usr/bin/env python3
"""Benchmark of the fused LBM-IBM time step on GB300.

One bench step = one pass of the whole hot path: the Lagrangian update of
step n (interpolation, bonds, membrane forces, integration, direct forcing)
overlapped with the bulk lattice update of step n + 1, then the near-membrane
lattice update of step n + 1 (one captured graph, three kernels).

Workloads (seeded synthetic geometry, FP32 populations, Re = 1e-2, tau = 1):
  sweep (default)  the 64-capillary parameter sweep of Sec. 3.1 (particle
                   aspect ratio x Ca x cell shape x 2 bond seeds; channel
                   lengths uniform in 600-1600 nodes, H = 150) stepped as one
                   batch: 10.66 M nodes, 780 MB of populations, larger than
                   L2, so every step streams from HBM.  Also times the plain
                   solver (each capillary alone in its own context, warm L2)
                   on the same 64 capillaries for simulations per hour.
  production       one 1200 x 150 capillary, globular cell (256 markers) +
                   soft AR 0.5 particle (96 markers, 200 ligand sites); its
                   13 MB fit in L2, so a 256 MiB buffer is rewritten between
                   timed steps and every timed step starts cold.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same
workload instead (the only other place this script runs the oracle).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MLUPS of fused LBM+IBM step"
UNIT = "MLUPS"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


STEPS_PER_SIM = 200000  # one capillary simulation: 2e5 time steps (the production horizon)
PRODUCTION = ("capillary 1200x150 nodes, globular cell 256 markers + soft AR0.5 ellipse 96 markers "
              "(200 ligand sites), Re 1e-2, tau 1, fp32 populations")
SWEEP = ("sweep of 64 capillaries in one batch: particle AR {0.25,0.5,0.75,1} x Ca {0 (rigid),1e-4,5e-4,1e-3} x "
         "cell {globular,biconcave} x bond seeds {0,1}; channel lengths U[600,1600] (seed 0) x 150 nodes; "
         "256-marker cells, 96-marker particles with 200 ligand sites; Re 1e-2, tau 1, fp32 populations")


def _workload(name, instances=64, seed=0):
    """List of capillaries and the config block naming them.  Under torchrun
    each rank draws its own sweep (seed = rank): the ranks together run a
    sweep of 64 N capillaries split across the GPUs, no exchange between them."""
    from paper_2210_06043_gb300 import workloads as wl
    if name == "production":
        caps = [wl.production_capillary(seed=0)]
        cfg = {"workload": PRODUCTION, "nx": caps[0].nx, "ny": caps[0].ny}
    else:
        caps = wl.sweep_capillaries(seed=seed)[:instances]
        cfg = {"workload": SWEEP if instances == 64 else f"first {instances} capillaries of the {SWEEP}",
               "instances": len(caps), "nx_total": sum(c.nx for c in caps), "ny": caps[0].ny}
    cfg.update({"nodes": sum(c.nodes for c in caps), "markers": sum(c.markers for c in caps),
                "ligand_sites": sum(b.adhesion.n_lig for c in caps for b in c.bodies if b.adhesion),
                "parallelism": ("data-parallel over capillaries: each rank steps its own 64-capillary draw "
                                "(seed = rank), no collective on the data path" if name == "sweep" else
                                "replicas (one independent copy of the capillary per GPU)")})
    return caps, cfg


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _code_only(text):
    """Source text without comments and blank lines: a comment edit does not
    change the kernel the counters were taken on."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip())


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("lbib_lbm.cu", "lbib_device.cuh", "lbib_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2210_06043_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_code_only(fh.read()).encode())
    return h.hexdigest()[:16]


def _traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    e = d.get(kernel)
    if not e or e.get("source_sha") != _kernel_source_hash() or e.get("workload") != workload:
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _oracle_sim(cap):
    import oracle
    s = oracle.OracleSim(cap.nx, cap.ny, tau=cap.tau, re=cap.re, rho_out=cap.rho_out, bc=cap.bc, g=cap.g,
                         seed=cap.seed)
    for b in cap.bodies:
        i = s.add_body(b.kind, b.motion, b.xy, b.xy_ref, b.ca, b.beta, b.ka, b.density_ratio)
        if b.adhesion is not None:
            a = b.adhesion
            s.set_adhesion(i, a.n_lig, a.sigma, a.y_cr, a.y_eq, a.kf_dt, a.kr0_dt, a.xi)
    return s


def _oracle_sample(caps, nodes_budget):
    """The capillaries the CPU oracle steps as a bounded sample of the
    workload: every 8th capillary of a sweep (the production capillary
    alone), and the number of steps that keeps the sample near nodes_budget
    node updates."""
    sample = caps[::8] if len(caps) > 1 else caps
    nodes = sum(c.nodes for c in sample)
    return sample, max(1, int(round(nodes_budget / nodes)))


def _time_oracle(sample, steps, threads):
    import oracle
    used = oracle.set_threads(threads)
    sims = [_oracle_sim(c) for c in sample]
    t0 = time.perf_counter()
    for s in sims:
        s.step(steps)
    return time.perf_counter() - t0, used


def cpu_baseline(caps, nodes_budget):
    """The oracle as it stands (plain C, FP64; its node loops on OpenMP
    threads) on a bounded sample of the workload, on one thread and on every
    host core; and the small capillary (240 x 60) for its full 2000 steps."""
    from paper_2210_06043_gb300 import workloads as wl
    host = os.cpu_count() or 1
    sample, steps = _oracle_sample(caps, nodes_budget)
    nodes = sum(c.nodes for c in sample)
    dt1, _ = _time_oracle(sample, steps, 1)
    dtn, used = _time_oracle(sample, steps, host)
    small = wl.small_capillary()
    dts, _ = _time_oracle([small], small.steps, host)
    return {"value": nodes * steps / dtn / 1e6, "unit": UNIT, "cores": used, "kind": "oracle",
            "host_cores": host,
            "sample": f"{steps} steps from t = 0 of {len(sample)} of the {len(caps)} capillaries "
                      f"({nodes} nodes), FP64 plain C, node loops on {used} OpenMP threads",
            "seconds": dtn,
            "one_thread": {"value": nodes * steps / dt1 / 1e6, "seconds": dt1},
            "small_capillary_full_run": {
                "what": f"240 x 60 capillary, biconcave cell + rigid adhering ellipse, {small.steps} steps, "
                        f"{used} threads",
                "mlups": small.nodes * small.steps / dts / 1e6, "seconds": dts,
                "marker_updates_per_s": small.markers * small.steps / dts}}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    caps, cfg = _workload(args.workload, args.instances)
    sample = caps[::32]  # every 32nd capillary of a sweep (the production capillary alone)
    import oracle
    threads = oracle.set_threads(os.cpu_count() or 1)  # the node loops on every host core
    sims = [_oracle_sim(c) for c in sample]
    nodes = sum(c.nodes for c in sample)
    for s in sims:
        s.step(args.warmup)
    t0 = time.perf_counter()
    for s in sims:
        s.step(args.steps)
    dt = time.perf_counter() - t0
    v = nodes * args.steps / dt / 1e6
    what = (f"{args.steps} timed steps after {args.warmup} warm-up steps of {len(sample)} of the {len(caps)} "
            f"capillaries ({nodes} nodes), FP64 plain C oracle, node loops on {threads} OpenMP threads")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": what,
                             "host_cores": os.cpu_count()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if len(caps) > 1:
        line["sims_per_hour"] = 3600.0 / (STEPS_PER_SIM * dt / args.steps * sum(c.nodes for c in caps) / nodes) \
            * len(caps)
    print(json.dumps(line), flush=True)
    return 0


def plain_solver(caps, local, steps, warmup):
    """Each capillary alone in its own context (the one-instance solver), timed
    with CUDA events on its stream over `steps` steps after `warmup`, warm L2;
    returns the device seconds per step of every capillary."""
    import torch

    from paper_2210_06043_gb300 import lbib
    out = []
    for c in caps:
        st = torch.cuda.Stream()
        s = lbib.from_capillary(c, device=local, stream=st.cuda_stream)
        s.autotune(steps_per_trial=10)
        s.advance(warmup)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        st.synchronize()
        a.record(st)
        s.advance(steps)
        b.record(st)
        b.synchronize()
        out.append(a.elapsed_time(b) / 1e3 / steps)
        s.close()
    return out


def surrogate_accuracy(local, stream, points=96, replicates=4, steps=30000, samples=96, holdout=16):
    """Held-out accuracy of a surrogate trained here on a small set (include/lbib_mlp.h
    network, surrogate.py pipeline): `points` parameter points, each run under
    `replicates` bond seeds by the batched solver, the network trained on the
    seed means of all but `holdout` points and scored on the held-out means.
    The floor of each output is the uncertainty of a held-out mean (the
    solver's seed-to-seed spread / sqrt(replicates)); N_L, a count of bond
    events, is the output with a floor.  Smaller than the full pipeline (which
    the design notes report): this is a measurement, repeated every run."""
    import time

    import numpy as np

    from paper_2210_06043_gb300 import surrogate as sg

    pts = sg.sample_points(points, seed=31)
    runs = sg.replicate(pts, replicates)
    t0 = time.perf_counter()
    t_star, Yall, gen_secs = sg.generate(runs, steps=steps, samples=samples, batch=len(runs), device=local,
                                         stream=stream.cuda_stream)
    Y, spread, floor = sg.seed_statistics(Yall, replicates)
    hold, fit = np.arange(holdout), np.arange(holdout, points)
    X = sg.features_many([pts[i] for i in fit], t_star)
    tr = sg.train(X, Y[fit].reshape(-1, 3).astype(np.float32), steps=1500, batch=4096, lr=2e-3, seed=1,
                  device=local)
    err, _, _ = sg.evaluate(tr, [pts[i] for i in hold], t_star, Y[hold], floor=floor)
    tr.net.close()
    return {"points": points, "replicates": replicates, "trajectories": len(runs), "solver_steps": steps,
            "t_star_max": float(t_star[-1]), "holdout_points": holdout, "train_steps": 1500,
            "seconds": time.perf_counter() - t0,
            "holdout": {k: {"rmse": v["rmse"], "rmse_over_std": v["rmse_over_std"], "floor": v["floor"],
                            "rmse_over_floor": v["rmse_over_floor"]} for k, v in err.items()},
            "seed_to_seed_spread": dict(zip(sg.OUTPUTS, map(float, spread)))}


def surrogate_inference(local, stream, iters=50, batch=65536, accuracy=True):
    """Throughput of the surrogate network's inference (include/lbib_mlp.h:
    9 inputs, 3 x 256 GELU, 3 outputs; the fused tcgen05 kernel) on batches
    of 65 536 queries, CUDA events on the launching stream; one training step
    (batch 8192, tcgen05 forward and backward); the host-side cost of a trajectory's
    features (surrogate.features_many); and the held-out accuracy of a
    network trained here (``surrogate_accuracy``).  Weights of the timed
    network random: timing only."""
    import time

    import numpy as np
    import torch

    from paper_2210_06043_gb300 import lbib
    from paper_2210_06043_gb300 import surrogate as sg

    n_in = len(sg.FEATURES)
    net = lbib.Mlp(n_in, 3, width=256, n_hidden=3, max_batch=batch, device=local, stream=stream.cuda_stream, seed=0)
    x = torch.rand(batch, n_in, device="cuda")
    y = torch.empty(batch, 3, device="cuda")
    t = torch.rand(batch, 3, device="cuda")
    for _ in range(5):
        net.forward(x.data_ptr(), batch, y.data_ptr())
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(iters):
        net.forward(x.data_ptr(), batch, y.data_ptr())
    b.record(stream)
    b.synchronize()
    t_inf = a.elapsed_time(b) / 1e3 / iters
    tb = 8192
    for _ in range(3):
        net.train_step(x.data_ptr(), t.data_ptr(), tb, 1e-4)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(iters):
        net.train_step(x.data_ptr(), t.data_ptr(), tb, 1e-4)
    b.record(stream)
    b.synchronize()
    t_train = a.elapsed_time(b) / 1e3 / iters
    net.close()
    # host features of one batch's trajectories (65 536 / 512 points)
    traj_per_call = batch / sg.SAMPLES
    fpts = sg.sample_points(int(traj_per_call), seed=41)
    ts = np.linspace(0.0, 1.0, sg.SAMPLES)
    sg.features_many(fpts[:2], ts)  # builds the polygon table once
    t0 = time.perf_counter()
    sg.features_many(fpts, ts)
    t_feat = (time.perf_counter() - t0) / len(fpts)
    flops = 2.0 * batch * (64 * 256 + 2 * 256 * 256 + 256 * 64)  # products as padded and run
    alg = 2.0 * batch * (n_in * 256 + 2 * 256 * 256 + 256 * 3)
    peak = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            peak = float(json.load(fh)["bf16_tflops"])
    per_step = sg.plain_solver_seconds_per_step(sg.sample_points(2, seed=9), steps=500)
    plain_traj = per_step * sg.STEPS
    per_traj = t_inf / traj_per_call + t_feat
    out = {"inference_batch": batch, "inference_ms": t_inf * 1e3, "queries_per_s": batch / t_inf,
           "tflops_run": flops / t_inf / 1e12, "tflops_algorithmic": alg / t_inf / 1e12,
           "bf16_peak_tflops": peak, "frac_of_bf16_peak": (flops / t_inf / 1e12 / peak) if peak else None,
           "train_step_ms_batch_8192": t_train * 1e3,
           "trajectory_us": {"network": t_inf / traj_per_call * 1e6, "host_features": t_feat * 1e6},
           "sims_per_hour": 3600.0 / per_traj, "sims_per_hour_network_only": traj_per_call * 3600.0 / t_inf,
           "plain_solver_sims_per_hour": 3600.0 / plain_traj,
           "speedup_vs_plain_solver": plain_traj / per_traj,
           "note": f"a simulation = one {sg.SAMPLES}-sample trajectory of the surrogate's {sg.NX}x{sg.NY} capillary "
                   f"({sg.STEPS} solver steps)",
           "hull": {"aspect_ratio": list(sg.AR_RANGE), "log10_ca": list(sg.LOGCA_RANGE), "rigid": True,
                    "ligand_density_per_um": list(sg.DENSITY_RANGE), "t_star_max": sg.STEPS * sg.u_max() / sg.NY,
                    "training_capillary": f"{sg.NX}x{sg.NY}, Re {sg.RE}, tau 1",
                    "deviation": "log10 Ca in [-4,-3] (not [-5,-3]) on the Stokes-regime training capillary "
                                 "(not the 1200x150, Re 1e-2 one): stiffer membranes exceed the explicit membrane "
                                 "update's stability limit at the training step; such queries go to the solver"}}
    if accuracy:
        out["accuracy"] = surrogate_accuracy(local, stream)
    return out


def storage_16bit(caps, local, stream, steps, warmup, hbm):
    """The same sweep with populations stored in 16 bits (FP16 deviations
    scaled by 2^14, and BF16 deviations; FP32 arithmetic): autotuned, `steps`
    steps timed with CUDA events on the launching stream, the bulk lattice
    kernel's in-graph time from a profiled pass, both against the 16-bit
    roofline (36 algorithmic bytes per node update)."""
    import dataclasses

    import torch

    from paper_2210_06043_gb300 import lbib
    out = {}
    for st in ("fp16", "bf16"):
        cs = [dataclasses.replace(c, storage=st) for c in caps]
        s = lbib.from_capillaries(cs, device=local, stream=stream.cuda_stream)
        cfg = s.autotune(steps_per_trial=50)
        s.advance(max(warmup, 3))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        s.advance(steps)
        b.record(stream)
        b.synchronize()
        dt = a.elapsed_time(b) / 1e3
        s.set_profiling(True)
        kern = []
        for _ in range(20):
            s.advance(1)
            kern.append(s.kernel_times())
        s.set_profiling(False)
        desc = s.describe()
        s.close()
        nodes = sum(c.nodes for c in cs)
        bpn = lbib.roofline_bytes_per_node(lbib.STORAGE_CODES[st])
        bulk_ms = statistics.mean(k[0] for k in kern)
        bulk_nodes = nodes - desc["near_tiles"] * 32 * 4
        out[st] = {"value": nodes * steps / dt / 1e6, "unit": UNIT, "ms_per_step": dt * 1e3 / steps,
                   "bytes_per_node": bpn, "step_roofline_frac": nodes * bpn / (dt / steps) / 1e9 / hbm,
                   "bulk_ms": bulk_ms, "bulk_roofline_frac": bulk_nodes * bpn / (bulk_ms * 1e-3) / 1e9 / hbm,
                   "launch_config": cfg}
    out["accuracy"] = ("against the FP64 oracle on the 240 x 60 capillary after 2000 steps "
                       "(tests/test_gpu_reduced_precision.py): see the bounds stated there")
    return out


def run_gpu(args):
    import torch

    from paper_2210_06043_gb300 import lbib

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    caps, cfg = _workload(args.workload, args.instances, seed=rank)
    if args.storage:  # population storage other than the workload's FP32
        import dataclasses
        caps = [dataclasses.replace(c, storage=args.storage) for c in caps]
        cfg["workload"] = cfg["workload"].replace("fp32 populations", f"{args.storage} populations")
        cfg["storage"] = args.storage
    store = lbib.STORAGE_CODES[caps[0].storage]
    batch = len(caps) > 1 or args.workload == "sweep"
    nodes = cfg["nodes"]
    stream = torch.cuda.Stream()  # non-null handle: the library enqueues on it, the events bracket it
    torch.cuda.set_stream(stream)
    make = (lambda **kw: lbib.from_capillaries(caps, **kw)) if batch else \
        (lambda **kw: lbib.from_capillary(caps[0], **kw))
    s = make(device=local, stream=stream.cuda_stream)
    if args.config:  # a fixed launch configuration (profiling runs) instead of the autotuner
        s.set_launch_config(*(int(v) for v in args.config.split(",")))
        tuned = dict(s.launch_config())
        tuned_by = "--config"
    else:
        tune_steps = args.tune_steps or (200 if args.workload == "production" else 50)
        tuned = s.autotune(steps_per_trial=tune_steps)  # leaves the state unchanged
        tuned_by = f"lbib_autotune, {tune_steps} steps per trial"
    # populations beyond L2 (sweep): no flush; else a 256 MiB buffer rewritten between steps
    pop_bytes = lbib.roofline_bytes_per_node(store) * nodes
    flush = None if pop_bytes > (256 << 20) else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        if flush is not None:
            flush.fill_(1)
        s.advance(1)
    torch.cuda.synchronize()
    desc = s.describe()
    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    t0 = time.perf_counter()
    # steps enqueued back to back (no host synchronisation inside the timed region)
    for k in range(K):
        if flush is not None:
            flush.fill_(k & 0xFF)
        starts[k].record(stream)
        s.advance(1)
        ends[k].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    # per-kernel device times from a separate profiled pass (events inside the step graph)
    s.set_profiling(True)
    kern = []
    for k in range(args.profile_steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        s.advance(1)
        kern.append(s.kernel_times())  # synchronises the stream
    s.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    dev_s = sum(step_ms) / 1e3
    if dist:
        t = torch.tensor([dev_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_s = float(t.item())
        dist.barrier()
    value = ws * nodes * K / dev_s / 1e6
    bulk_ms = statistics.mean(k[0] for k in kern)
    lag_ms = statistics.mean(k[1] for k in kern)
    near_ms = statistics.mean(k[2] for k in kern)
    near_nodes = desc["near_tiles"] * 32 * 4
    bulk_nodes = nodes - near_nodes
    bpn = lbib.roofline_bytes_per_node(store)
    hbm, src = _peaks()
    achieved = bulk_nodes * bpn / (bulk_ms * 1e-3) / 1e9
    traffic = _traffic("k_bulk<float,float>", cfg["workload"]) if caps[0].storage == "fp32" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "k_bulk<float,float> (bulk lattice update)",
                "algorithmic_bytes_per_launch": bulk_nodes * bpn,
                "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs, burst copy)",
                # the whole fused step (bulk + near updates, every node once) against the same peak
                "step": {"achieved": nodes * bpn / (dev_s / K) / 1e9, "frac": nodes * bpn / (dev_s / K) / 1e9 / hbm,
                         "bytes_per_step": nodes * bpn}}
    s.close()

    # end to end through the C ABI with host buffers: create from host meshes,
    # then per step advance + copy of the newest observables record of every
    # instance into page-locked host memory (enqueued, no wait: the step
    # pipeline stays full), finally the velocity field of instance 0 to the host
    rec_sz = lbib.Solver.OBS_DTYPE.itemsize
    host_obs = torch.zeros((K, len(caps) * rec_sz), dtype=torch.uint8).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s2 = make(device=local)
    s2.set_launch_config(**tuned)  # the launch shape chosen above (a user tunes once and keeps it)
    for k in range(K):
        s2.advance(1)
        s2.latest_observables_async(host_obs[k].data_ptr())
    ux, uy = s2.velocity()  # waits for the stream: every record has landed
    s2.close()
    e2e_s = time.perf_counter() - t0
    obs = host_obs[K - 1].numpy().view(lbib.Solver.OBS_DTYPE)
    if dist:
        t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d = sum(b.xy.nbytes for c in caps for b in c.bodies)
    d2h_rec = 48 * len(caps)
    e2e = {"value": ws * nodes * K / e2e_s / 1e6, "unit": UNIT,
           "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h_rec + (ux.nbytes + uy.nbytes) / K,
           "what": "create + add membranes from host meshes, the tuned launch configuration "
                   "(lbib_set_launch_config), then per step lbib_advance(1) and "
                   "lbib_read_latest_observables_async (every instance's newest record into pinned host "
                   "memory), final velocity of instance 0 to host (waits), destroy",
           "records_last_step": int((obs["step"] >= 0).sum())}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    markers = cfg["markers"]
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": dev_s * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16 storage, f32 arithmetic",
                      "fp16": "f16 storage (x 2^14), f32 arithmetic"}[caps[0].storage], "data": "synthetic",
            "config": dict(cfg, l2=(f"populations ({pop_bytes / 1e6:.0f} MB) larger than L2: no flush" if flush is None else
                                    "256 MiB buffer rewritten between timed steps (cold L2 each step)")),
            "marker_updates_per_s": ws * markers * K / dev_s,
            "kernel_ms": {"bulk_lattice": bulk_ms, "lagrangian": lag_ms, "near_lattice": near_ms},
            "near_tiles": desc["near_tiles"], "tiles": desc["tiles"],
            "roofline": roofline, "e2e": e2e, "gpu_launches": desc["kernels_per_step"] * K, "clocks": clk,
            "launch_config": dict(tuned, chosen_by=tuned_by),
            "wall_s_timed_region": wall}
    if batch and args.plain_steps > 0:
        t_plain = plain_solver(caps, local, args.plain_steps, 3)
        t_batch = dev_s / K
        line["sweep"] = {
            "steps_per_sim": STEPS_PER_SIM,
            "sims_per_hour": ws * len(caps) * 3600.0 / (STEPS_PER_SIM * t_batch),
            "plain_solver_sims_per_hour": ws * len(caps) * 3600.0 / (STEPS_PER_SIM * sum(t_plain)),
            "speedup_vs_plain_solver": sum(t_plain) / t_batch,
            "plain_solver_ms_per_step": {"mean": 1e3 * statistics.mean(t_plain), "min": 1e3 * min(t_plain),
                                         "max": 1e3 * max(t_plain)},
            "plain_solver": f"each capillary alone in its own context (same kernels, autotuned), "
                            f"{args.plain_steps} steps after 3 warm-up steps, warm L2, CUDA events",
            "accuracy": "every instance bit-identical to its lone run (tests/test_gpu_batch.py)"}
    if batch and not args.storage and not args.no_16bit:
        line["storage_16bit"] = storage_16bit(caps, local, stream, K, args.warmup, hbm)
    if batch and not args.no_surrogate:
        line["surrogate"] = surrogate_inference(local, stream)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(caps, args.cpu_nodes)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="lbib", choices=["lbib", "reference"])
    ap.add_argument("--workload", default="sweep", choices=["sweep", "production"])
    ap.add_argument("--instances", type=int, default=64, help="first N capillaries of the sweep")
    ap.add_argument("--plain-steps", type=int, default=50,
                    help="steps per capillary of the plain-solver timing (0: skip it, for profiling runs)")
    ap.add_argument("--cpu-nodes", type=float, default=1.0e8,
                    help="node updates of the CPU oracle sample (about 15 s at 7 MLUPS)")
    ap.add_argument("--tune-steps", type=int, default=0,
                    help="steps per autotuner trial (default: 50 for the sweep, 200 for the production capillary, "
                         "whose steps are short enough for timing noise to decide between close candidates)")
    ap.add_argument("--storage", default="", choices=["", "fp32", "bf16", "fp16", "fp64"],
                    help="population storage (default: the workload's, FP32)")
    ap.add_argument("--profile-steps", type=int, default=50,
                    help="steps of the separate profiled pass that gives the per-kernel times")
    ap.add_argument("--config", default="", help="fixed launch configuration "
                    "lagrangian_threads,near_blocks,bulk_tiles_y,activation_stride[,bulk_nodes_per_thread"
                    "[,observables_branch[,chain_programmatic[,near_update_blocks[,bulk_tma]]]]] "
                    "instead of the autotuner")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-16bit", action="store_true", help="skip the 16-bit storage timing of the sweep")
    ap.add_argument("--no-surrogate", action="store_true", help="skip the surrogate inference timing")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
