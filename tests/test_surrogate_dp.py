"""Data-parallel training of the surrogate network
(paper_2210_06043_gb300/surrogate.py ``data_parallel_step``): a world-size-2
gloo run on CPU ends with the same parameters on both ranks, equal to a serial
run on the whole batches.  The network's backward pass and Adam update are
the CPU oracle's here (the library's kernels need a GPU); the sharding,
all-reduce and scaling are the code the GPU path runs."""
import ctypes
import os
import socket
import sys

import numpy as np
import torch
import torch.multiprocessing as mp

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from oracle import mlp  # noqa: E402
from paper_2210_06043_gb300 import surrogate  # noqa: E402

N_IN, WIDTH, HIDDEN, N_OUT = 5, 8, 2, 3
GLOBAL_BATCH, STEPS, LR = 16, 4, 1e-2


def _f32(ptr, n):
    return np.ctypeslib.as_array((ctypes.c_float * n).from_address(ptr))


class OracleNet:
    """Stand-in with lbib.Mlp's backward / apply_gradient signatures, on host
    float32 buffers, computed by the FP64 oracle."""

    def __init__(self, seed=0):
        rng = np.random.default_rng(seed)
        dims = [N_IN] + [WIDTH] * HIDDEN + [N_OUT]
        self.p = mlp.flat([(rng.normal(0, 0.5, (o, i)), rng.normal(0, 0.1, o)) for i, o in zip(dims[:-1], dims[1:])])
        self.m = np.zeros_like(self.p)
        self.v = np.zeros_like(self.p)
        self.t = 0
        self.applied = []
        self.norm = dict(c_in=np.zeros(N_IN), s_in=np.ones(N_IN), c_out=np.full(N_OUT, 0.1), s_out=np.full(N_OUT, 2.0))

    def backward(self, x_ptr, t_ptr, batch, grad_ptr, n, loss_ptr):
        x = _f32(x_ptr, batch * N_IN).reshape(batch, N_IN).astype(np.float64)
        t = _f32(t_ptr, batch * N_OUT).reshape(batch, N_OUT).astype(np.float64)
        layers = mlp.split_params(self.p, N_IN, WIDTH, HIDDEN, N_OUT)
        loss, grads = mlp.gradients(layers, x, t, **self.norm)
        _f32(grad_ptr, n)[:] = mlp.flat(grads)
        _f32(loss_ptr, 1)[0] = loss

    def apply_gradient(self, grad_ptr, n, scale, lr):
        g = scale * _f32(grad_ptr, n).astype(np.float64)
        self.applied.append(g)
        self.t += 1
        self.p, self.m, self.v = mlp.adam_step(self.p, g, self.m, self.v, self.t, lr)


def _batches():
    rng = np.random.default_rng(7)
    return [(torch.tensor(rng.uniform(-1, 1, (GLOBAL_BATCH, N_IN)), dtype=torch.float32),
             torch.tensor(rng.normal(0, 1, (GLOBAL_BATCH, N_OUT)), dtype=torch.float32)) for _ in range(STEPS)]


def _train(rank, world):
    net = OracleNet()
    grad = torch.zeros(net.p.size, dtype=torch.float32)
    loss = torch.zeros(1, dtype=torch.float32)
    for xb, yb in _batches():
        surrogate.data_parallel_step(net, xb, yb, grad, loss, LR, rank, world)
    return np.concatenate([net.p] + net.applied)


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), _train(rank, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_train_like_one(tmp_path):
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
    p0, p1 = (np.load(tmp_path / f"rank{r}.npy") for r in range(2))
    assert np.array_equal(p0, p1)  # the copies stay identical
    serial = _train(0, 1)
    n = OracleNet().p.size
    start = OracleNet().p
    # the applied gradient (1/2 the all-reduced sum) is the whole batch's: the
    # loss is a batch mean; they differ by the float32 rounding of the shards
    for k in range(STEPS):
        gd, gs = p0[n * (k + 1):n * (k + 2)], serial[n * (k + 1):n * (k + 2)]
        assert np.abs(gd - gs).max() <= 1e-6 * np.abs(gs).max(), k
    assert np.abs(p0[:n] - serial[:n]).max() < 1e-6 * LR * STEPS
    assert np.abs(serial[:n] - start).max() > 0.5 * LR  # the steps moved the parameters


def test_uneven_global_batch_is_refused():
    net = OracleNet()
    x, y = _batches()[0]
    grad = torch.zeros(net.p.size)
    loss = torch.zeros(1)
    try:
        surrogate.data_parallel_step(net, x[:15], y[:15], grad, loss, LR, 0, 2)
    except ValueError:
        return
    raise AssertionError("an uneven split must be refused")
