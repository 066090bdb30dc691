"""A sweep split across ranks (paper_2210_06043_gb300/sweep.py): balanced
assignment, and a world-size-2 gloo run on CPU whose gathered trajectories
equal a serial run.  The per-capillary work is the CPU oracle on tiny
capillaries (the ranks' GPU solver is replaced, the sharding and gathering
logic is the one the GPU path uses)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2210_06043_gb300 import sweep
from paper_2210_06043_gb300 import workloads as wl


def test_assign_balances_and_covers():
    rng = np.random.default_rng(0)
    sizes = rng.integers(600, 1601, 64) * 150
    for world in (1, 2, 3, 8):
        parts = sweep.assign(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(64))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
        assert parts == sweep.assign(sizes, world)  # deterministic
    assert sweep.assign([5], 3) == [[0], [], []]


def _caps():
    out = []
    for k, nx in enumerate((40, 52, 44, 60, 48)):
        cell = wl.circle(24, 12.0, 8.0, 3.5)
        part = wl.ellipse(16, 28.0, 1.6, 4.0, 1.5)
        out.append(wl.Capillary(f"tiny {k}", nx, 16, 1.0, 0.05, 40, "fp64", k, [
            wl.Body(wl.CELL, wl.DEFORMABLE, cell, ca=1e-2, beta=0.0),
            wl.Body(wl.PARTICLE, wl.RIGID, part, ca=0.0, beta=0.0, density_ratio=1.1,
                    adhesion=wl.Adhesion(12, 1.0, 0.3, 0.15, 0.1, 0.01, 10.0))]))
    return out


def _runner(share):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from helpers import oracle_from
    res = []
    for cap in share:
        o = oracle_from(cap)
        rows = []
        for _ in range(4):
            o.step(10)
            ob = o.obs()
            rows.append([ob["n_l"], ob["delta_p"], ob["r"]])
        res.append(rows)
    return np.asarray(res)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    full = sweep.run_sharded(_caps(), _runner, rank, world)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), full)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gather_the_serial_result(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    serial = _runner(_caps())
    for r in range(2):
        assert np.array_equal(np.load(tmp_path / f"rank{r}.npy"), serial)
