"""GPU parity of the surrogate network's kernels (include/lbib_mlp.h) against
the CPU oracle (oracle/mlp.py, quantize=True: the same bfloat16 roundings).

Tolerances: the GPU accumulates products in FP32 and evaluates GELU in FP32
with the hardware tanh approximation (relative error about 2^-11), so an
activation sitting on a bfloat16 rounding boundary can round the other
way (one unit, 2^-8 relative); such flips are rare and propagate as small
noise, so outputs and gradients are compared in relative L2 (5e-3 and 2e-2),
not element by element."""
import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2210_06043_gb300 import lbib

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N_IN, N_OUT, WIDTH, HIDDEN = 7, 3, 256, 3


@pytest.fixture(autouse=True)
def one_stream():
    """The network and torch's copies share one stream (ordering by the stream)."""
    st = torch.cuda.Stream()
    prev = torch.cuda.current_stream()
    torch.cuda.set_stream(st)
    yield st
    torch.cuda.synchronize()
    torch.cuda.set_stream(prev)


def _norm(rng):
    return dict(c_in=rng.uniform(-0.3, 0.3, N_IN).astype(np.float32), s_in=rng.uniform(0.5, 2, N_IN).astype(np.float32),
                c_out=rng.uniform(-1, 1, N_OUT).astype(np.float32), s_out=rng.uniform(0.5, 2, N_OUT).astype(np.float32))


def _net(norm, max_batch=4096, seed=1):
    return lbib.Mlp(N_IN, N_OUT, width=WIDTH, n_hidden=HIDDEN, max_batch=max_batch, seed=seed,
                    stream=torch.cuda.current_stream().cuda_stream,
                    in_shift=norm["c_in"], in_scale=norm["s_in"], out_shift=norm["c_out"], out_scale=norm["s_out"])


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def test_forward_matches_quantized_oracle():
    rng = np.random.default_rng(0)
    norm = _norm(rng)
    net = _net(norm)
    x = rng.uniform(-1, 1, (1000, N_IN)).astype(np.float32)  # ragged: not a multiple of the 64-row tile
    xd, yd = _dev(x), torch.zeros(1000, N_OUT, device="cuda")
    net.forward(xd.data_ptr(), 1000, yd.data_ptr())
    torch.cuda.synchronize()
    layers = omlp.split_params(net.get_params(), N_IN, WIDTH, HIDDEN, N_OUT)
    y, _, _ = omlp.forward(layers, x, quantize=True, **norm)
    assert _rel(yd.cpu().numpy(), y) < 5e-3
    net.close()


# a ragged batch, one of whole tiles, and one of 313 tiles (ragged): up to three 128-row tiles per
# CTA of the fused training kernels, so both tile slots and the staging of a slot's next tile run
@pytest.mark.parametrize("B", [500, 1024, 40000])
def test_gradients_match_quantized_oracle_and_repeat_exactly(B):
    rng = np.random.default_rng(1)
    norm = _norm(rng)
    net = _net(norm, max_batch=max(4096, B), seed=7)
    x = rng.uniform(-1, 1, (B, N_IN)).astype(np.float32)
    t = (rng.normal(0, 1, (B, N_OUT)) * norm["s_out"] + norm["c_out"]).astype(np.float32)
    xd, td = _dev(x), _dev(t)
    g1, l1 = net.gradients(xd.data_ptr(), td.data_ptr(), B)
    g2, l2 = net.gradients(xd.data_ptr(), td.data_ptr(), B)
    assert np.array_equal(g1, g2) and l1 == l2  # fixed-order reductions
    layers = omlp.split_params(net.get_params(), N_IN, WIDTH, HIDDEN, N_OUT)
    lo, go = omlp.gradients(layers, x, t, quantize=True, **norm)
    assert abs(l1 - lo) <= 1e-3 * lo
    k = 0
    for (dW, db) in go:
        gw = g1[k:k + dW.size].reshape(dW.shape)
        k += dW.size
        gb = g1[k:k + db.size]
        k += db.size
        assert _rel(gw, dW) < 2e-2 and _rel(gb, db) < 2e-2
    net.close()


# other shapes through the same tensor-core training path: width 64 (one output
# tile per layer), 192 (a 64-row second tile and three column tiles), eight
# hidden layers; a batch of one row, and ragged ones
@pytest.mark.parametrize("width,hidden,B", [(64, 1, 1), (192, 2, 333), (128, 8, 2500)])
def test_gradients_of_other_shapes(width, hidden, B):
    rng = np.random.default_rng(width + hidden)
    norm = _norm(rng)
    net = lbib.Mlp(N_IN, N_OUT, width=width, n_hidden=hidden, max_batch=4096, seed=3,
                   stream=torch.cuda.current_stream().cuda_stream,
                   in_shift=norm["c_in"], in_scale=norm["s_in"], out_shift=norm["c_out"], out_scale=norm["s_out"])
    x = rng.uniform(-1, 1, (B, N_IN)).astype(np.float32)
    t = (rng.normal(0, 1, (B, N_OUT)) * norm["s_out"] + norm["c_out"]).astype(np.float32)
    xd, td = _dev(x), _dev(t)
    g1, l1 = net.gradients(xd.data_ptr(), td.data_ptr(), B)
    g2, l2 = net.gradients(xd.data_ptr(), td.data_ptr(), B)
    assert np.array_equal(g1, g2) and l1 == l2
    layers = omlp.split_params(net.get_params(), N_IN, width, hidden, N_OUT)
    lo, go = omlp.gradients(layers, x, t, quantize=True, **norm)
    assert abs(l1 - lo) <= 1e-3 * lo
    k = 0
    for (dW, db) in go:
        gw = g1[k:k + dW.size].reshape(dW.shape)
        k += dW.size
        gb = g1[k:k + db.size]
        k += db.size
        # one row: a flipped bf16 rounding is not averaged out over the batch
        tol = 6e-2 if B == 1 else 2e-2
        assert _rel(gw, dW) < tol and _rel(gb, db) < tol
    assert k == g1.size
    net.close()


def test_wide_network_on_the_general_path():
    """Width 320 (above the fused kernels' 256): every product on the general
    tensor-core GEMM path.  Outputs and gradients against the quantized
    oracle, gradients repeat exactly, and backward + apply(1) equals
    train_step bit for bit over two steps."""
    rng = np.random.default_rng(9)
    norm = _norm(rng)
    width, hidden, B = 320, 2, 700

    def make(seed):
        return lbib.Mlp(N_IN, N_OUT, width=width, n_hidden=hidden, max_batch=1024, seed=seed,
                        stream=torch.cuda.current_stream().cuda_stream,
                        in_shift=norm["c_in"], in_scale=norm["s_in"], out_shift=norm["c_out"],
                        out_scale=norm["s_out"])

    a, b = make(5), make(5)
    x = rng.uniform(-1, 1, (B, N_IN)).astype(np.float32)
    t = (rng.normal(0, 1, (B, N_OUT)) * norm["s_out"] + norm["c_out"]).astype(np.float32)
    xd, td, yd = _dev(x), _dev(t), torch.zeros(B, N_OUT, device="cuda")
    a.forward(xd.data_ptr(), B, yd.data_ptr())
    torch.cuda.synchronize()
    layers = omlp.split_params(a.get_params(), N_IN, width, hidden, N_OUT)
    y, _, _ = omlp.forward(layers, x, quantize=True, **norm)
    assert _rel(yd.cpu().numpy(), y) < 5e-3
    g1, l1 = a.gradients(xd.data_ptr(), td.data_ptr(), B)
    g2, l2 = a.gradients(xd.data_ptr(), td.data_ptr(), B)
    assert np.array_equal(g1, g2) and l1 == l2
    lo, go = omlp.gradients(layers, x, t, quantize=True, **norm)
    assert abs(l1 - lo) <= 1e-3 * lo
    k = 0
    for (dW, db) in go:
        gw = g1[k:k + dW.size].reshape(dW.shape)
        k += dW.size
        gb = g1[k:k + db.size]
        k += db.size
        assert _rel(gw, dW) < 2e-2 and _rel(gb, db) < 2e-2
    n = a.param_count()
    grad = torch.zeros(n, device="cuda")
    for lr in (1e-3, 5e-4):
        a.backward(xd.data_ptr(), td.data_ptr(), B, grad.data_ptr(), n, None)
        a.apply_gradient(grad.data_ptr(), n, 1.0, lr)
        b.train_step(xd.data_ptr(), td.data_ptr(), B, lr)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    a.close()
    b.close()


def test_training_fits_a_smooth_function():
    rng = np.random.default_rng(2)
    norm = dict(c_in=np.zeros(N_IN, np.float32), s_in=np.ones(N_IN, np.float32),
                c_out=np.zeros(N_OUT, np.float32), s_out=np.ones(N_OUT, np.float32))
    net = _net(norm, max_batch=4096, seed=3)

    def target(x):
        return np.stack([np.sin(np.pi * x[:, 0]) * x[:, 1], x[:, 2] ** 2 - x[:, 3], np.cos(2 * x[:, 4]) + x[:, 5] * x[:, 6]],
                        1).astype(np.float32)

    xtr = rng.uniform(-1, 1, (4096, N_IN)).astype(np.float32)
    xte = rng.uniform(-1, 1, (2048, N_IN)).astype(np.float32)
    xd, td = _dev(xtr), _dev(target(xtr))
    loss = torch.zeros(1, device="cuda")
    losses = []
    for k in range(600):
        net.train_step(xd.data_ptr(), td.data_ptr(), 4096, 2e-3 if k < 400 else 5e-4, loss.data_ptr())
        if k % 100 == 0 or k == 599:
            losses.append(float(loss.item()))
    assert losses[-1] < losses[0] / 30, losses
    yd = torch.zeros(2048, N_OUT, device="cuda")
    net.forward(_dev(xte).data_ptr(), 2048, yd.data_ptr())
    err = np.mean((yd.cpu().numpy() - target(xte)) ** 2)
    assert err < 3 * losses[-1] + 1e-3, (err, losses[-1])
    net.close()


def test_params_roundtrip_and_invalid_arguments():
    rng = np.random.default_rng(3)
    norm = _norm(rng)
    net = _net(norm, max_batch=128)
    p = net.get_params()
    assert p.size == net.param_count() == (N_IN * WIDTH + WIDTH) + 2 * (WIDTH * WIDTH + WIDTH) + (WIDTH * N_OUT + N_OUT)
    q = rng.normal(0, 0.05, p.size).astype(np.float32)
    net.set_params(q)
    assert np.array_equal(net.get_params(), q)
    x = _dev(np.zeros((256, N_IN)))
    y = torch.zeros(256, N_OUT, device="cuda")
    with pytest.raises(lbib.LbibError):
        net.forward(x.data_ptr(), 256, y.data_ptr())  # beyond max_batch
    with pytest.raises(lbib.LbibError):
        net.train_step(x.data_ptr(), y.data_ptr(), 64, -1.0)
    with pytest.raises(lbib.LbibError):
        lbib.Mlp(40, 3)  # n_in > 32
    with pytest.raises(lbib.LbibError):
        lbib.Mlp(7, 3, width=100)
    net.close()


def test_data_parallel_calls():
    """lbib_mlp_backward equals lbib_mlp_gradients bit for bit; backward + apply
    (scale 1) equals train_step bit for bit; apply_gradient is the oracle's
    Adam update on the FP32 masters; the mean of two shards' gradients is the
    whole batch's (what the ranks of a data-parallel step exchange)."""
    rng = np.random.default_rng(5)
    norm = _norm(rng)
    B = 2048
    x = rng.uniform(-1, 1, (B, N_IN)).astype(np.float32)
    t = rng.normal(0, 1, (B, N_OUT)).astype(np.float32)
    xd, td = _dev(x), _dev(t)
    a, b = _net(norm, seed=3), _net(norm, seed=3)
    n = a.param_count()
    grad = torch.zeros(n, device="cuda")
    loss = torch.zeros(1, device="cuda")
    a.backward(xd.data_ptr(), td.data_ptr(), B, grad.data_ptr(), n, loss.data_ptr())
    g_host, l_host = a.gradients(xd.data_ptr(), td.data_ptr(), B)
    torch.cuda.synchronize()
    assert np.array_equal(grad.cpu().numpy(), g_host) and float(loss.item()) == l_host
    # backward + apply(1) == train_step, two steps
    for lr in (1e-3, 5e-4):
        a.backward(xd.data_ptr(), td.data_ptr(), B, grad.data_ptr(), n, None)
        a.apply_gradient(grad.data_ptr(), n, 1.0, lr)
        b.train_step(xd.data_ptr(), td.data_ptr(), B, lr)
    torch.cuda.synchronize()
    assert np.array_equal(a.get_params(), b.get_params())
    # apply_gradient against the oracle's Adam on a fresh network (first step)
    c = _net(norm, seed=4)
    p0 = c.get_params().astype(np.float64)
    gg = rng.normal(0, 1e-2, n).astype(np.float32)
    gd = _dev(gg)
    c.apply_gradient(gd.data_ptr(), n, 0.5, 1e-3)
    p1, m1, v1 = omlp.adam_step(p0, 0.5 * gg.astype(np.float64), np.zeros(n), np.zeros(n), 1, 1e-3)
    assert np.abs(c.get_params() - p1).max() < 1e-6
    # shard gradients: mean of two halves == whole batch (bf16 roundings differ slightly)
    d = _net(norm, seed=6)
    g1, g2 = torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    d.backward(xd[: B // 2].data_ptr(), td[: B // 2].data_ptr(), B // 2, g1.data_ptr(), n, None)
    d.backward(xd[B // 2:].data_ptr(), td[B // 2:].data_ptr(), B // 2, g2.data_ptr(), n, None)
    d.backward(xd.data_ptr(), td.data_ptr(), B, grad.data_ptr(), n, None)
    torch.cuda.synchronize()
    assert _rel(0.5 * (g1 + g2).cpu().numpy(), grad.cpu().numpy().astype(np.float64)) < 1e-2
    for bad in (lambda: a.backward(xd.data_ptr(), td.data_ptr(), B, grad.data_ptr(), n - 1, None),
                lambda: a.apply_gradient(grad.data_ptr(), n, float("nan"), 1e-3),
                lambda: a.apply_gradient(grad.data_ptr(), n, 1.0, 0.0)):
        with pytest.raises(lbib.LbibError):
            bad()


def test_fused_forward_many_tiles_ragged_and_after_new_weights():
    """The fused inference kernel on 305 tiles of 128 rows (the last one
    ragged; each persistent CTA runs 2 or 3 tiles, so both tensor-memory
    slots and an odd tile count per CTA occur), against the oracle on sampled
    rows; then again after new weights (the packed copy is refreshed)."""
    rng = np.random.default_rng(11)
    norm = _norm(rng)
    B = 304 * 128 + 77
    net = _net(norm, max_batch=B, seed=2)
    x = rng.uniform(-1, 1, (B, N_IN)).astype(np.float32)
    xd, yd = _dev(x), torch.zeros(B, N_OUT, device="cuda")
    rows = np.concatenate([np.arange(0, 300), rng.choice(B, 1200, replace=False), np.arange(B - 200, B)])
    for attempt in range(2):
        if attempt == 1:
            p = net.get_params()
            net.set_params(p + rng.normal(0, 0.02, p.size).astype(np.float32))
        net.forward(xd.data_ptr(), B, yd.data_ptr())
        torch.cuda.synchronize()
        layers = omlp.split_params(net.get_params(), N_IN, WIDTH, HIDDEN, N_OUT)
        y, _, _ = omlp.forward(layers, x[rows], quantize=True, **norm)
        assert _rel(yd.cpu().numpy()[rows], y) < 5e-3, attempt
        assert np.isfinite(yd.cpu().numpy()).all()
