#!/usr/bin/env python3
"""Benchmark of the fused LBM-IBM time step on GB300.

One bench step = one pass of the whole hot path: the Lagrangian update of
step n (interpolation, bonds, membrane forces, integration, direct forcing)
overlapped with the bulk lattice update of step n + 1, then the near-membrane
lattice update of step n + 1 (one captured graph, three kernels).

Workload (N = 1): the production capillary, 1200 x 150 nodes, globular cell
(256 markers) + soft AR 0.5 particle (96 markers, 200 ligand sites), FP32
populations, Re = 1e-2, seeded synthetic geometry.  Its 13 MB of populations
fit in L2, so the 256 MiB flush buffer is rewritten between timed steps and
every timed step starts cold.

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the same
workload instead (the only other place this script runs the oracle).
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
sys.path.insert(0, ROOT)

METRIC = "MLUPS of fused LBM+IBM step"
UNIT = "MLUPS"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _workload():
    from paper_2210_06043_gb300 import workloads as wl
    cap = wl.production_capillary(seed=0)
    cfg = {"workload": "capillary 1200x150 nodes, globular cell 256 markers + soft AR0.5 ellipse 96 markers "
                       "(200 ligand sites), Re 1e-2, tau 1, fp32 populations",
           "nx": cap.nx, "ny": cap.ny, "markers": cap.markers,
           "ligand_sites": sum(b.adhesion.n_lig for b in cap.bodies if b.adhesion),
           "parallelism": "replicas (one independent instance per GPU)"}
    return cap, cfg


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _kernel_source_hash():
    h = hashlib.sha256()
    for f in ("lbib_lbm.cu", "lbib_device.cuh", "lbib_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2210_06043_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
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


def cpu_baseline(cap, steps):
    """The oracle as it stands (single-threaded plain C, FP64) on a bounded
    sample of the workload."""
    s = _oracle_sim(cap)
    t0 = time.perf_counter()
    s.step(steps)
    dt = time.perf_counter() - t0
    return {"value": cap.nodes * steps / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{steps} steps of the same capillary from t = 0 (of {cap.steps}), FP64 plain C, one thread",
            "seconds": dt}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    cap, cfg = _workload()
    s = _oracle_sim(cap)
    s.step(args.warmup)
    t0 = time.perf_counter()
    s.step(args.steps)
    dt = time.perf_counter() - t0
    v = cap.nodes * args.steps / dt / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed steps after {args.warmup} warm-up steps, FP64 "
                                       f"plain C oracle, one thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch

    from paper_2210_06043_gb300 import lbib

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cap, cfg = _workload()
    nodes = cap.nodes
    stream = torch.cuda.Stream()  # non-null handle: the library enqueues on it, the events bracket it
    torch.cuda.set_stream(stream)
    s = lbib.from_capillary(cap, device=local, stream=stream.cuda_stream)
    s.set_profiling(True)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        s.advance(1)
    torch.cuda.synchronize()
    desc = s.describe()
    K = args.steps
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    kern = []
    clocks = Clocks(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)
    t0 = time.perf_counter()
    for k in range(K):
        flush.fill_(k & 0xFF)
        starts[k].record(stream)
        s.advance(1)
        ends[k].record(stream)
        kern.append(s.kernel_times())  # synchronises the stream
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
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
    bpn = lbib.roofline_bytes_per_node(lbib.LBIB_STORE_FP32)
    hbm, src = _peaks()
    achieved = bulk_nodes * bpn / (bulk_ms * 1e-3) / 1e9
    traffic = _traffic("k_bulk<float,float>", cfg["workload"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "k_bulk<float,float> (bulk lattice update)",
                "algorithmic_bytes_per_launch": bulk_nodes * bpn, "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs)"}
    s.close()

    # end to end through the C ABI with host buffers: create from host meshes,
    # then per step advance + read that step's observables record to the host,
    # finally the velocity field to the host
    if True:
        K2 = K
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = lbib.from_capillary(cap, device=local)
        for _ in range(K2):
            s2.advance(1)
            obs = s2.observables(cap=4)
        ux, uy = s2.velocity()
        s2.close()
        e2e_s = time.perf_counter() - t0
        if dist:
            t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_s = float(t.item())
        h2d = sum(b.xy.nbytes for b in cap.bodies)
        d2h_rec = 48
        e2e = {"value": ws * nodes * K2 / e2e_s / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d / K2, "d2h_bytes_per_step": d2h_rec + (ux.nbytes + uy.nbytes) / K2,
               "what": "lbib_create + add_membrane (host meshes) + per step lbib_advance(1) and "
                       "lbib_read_observables to host + final lbib_read_velocity to host + destroy",
               "records_read_last_step": len(obs)}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
            "ms_per_step": dev_s * 1e3 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": dict(cfg, l2="256 MiB buffer rewritten between timed steps (cold L2 each step)"),
            "marker_updates_per_s": ws * cap.markers * K / dev_s,
            "kernel_ms": {"bulk_lattice": bulk_ms, "lagrangian": lag_ms, "near_lattice": near_ms},
            "near_tiles": desc["near_tiles"], "tiles": desc["tiles"],
            "roofline": roofline, "e2e": e2e, "gpu_launches": 3 * K, "clocks": clk,
            "wall_s_timed_region": wall}
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cap, args.cpu_steps)
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
    ap.add_argument("--cpu-steps", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
