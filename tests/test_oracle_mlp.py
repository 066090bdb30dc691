"""Pins of the surrogate network's CPU oracle (oracle/mlp.py) against facts
other than itself: finite differences of the FP64 loss, closed forms of the
Gaussian error linear unit, and the bfloat16 rounding rule."""
import math

import numpy as np

from oracle import mlp


def _tiny(seed=0, n_in=3, width=5, n_hidden=2, n_out=2):
    rng = np.random.default_rng(seed)
    dims = [n_in] + [width] * n_hidden + [n_out]
    layers = [(rng.normal(0, 0.7, (o, i)), rng.normal(0, 0.2, o)) for i, o in zip(dims[:-1], dims[1:])]
    x = rng.uniform(-1, 1, (7, n_in))
    t = rng.normal(0, 1, (7, n_out))
    norm = dict(c_in=rng.uniform(-0.2, 0.2, n_in), s_in=rng.uniform(0.5, 2, n_in),
                c_out=rng.uniform(-1, 1, n_out), s_out=rng.uniform(0.5, 2, n_out))
    return layers, x, t, norm


def test_gradients_match_central_differences():
    layers, x, t, norm = _tiny()
    loss, grads = mlp.gradients(layers, x, t, **norm)
    h = 1e-6
    for l, (W, b) in enumerate(layers):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            it = np.nditer(arr, flags=["multi_index"])
            for _ in it:
                idx = it.multi_index
                old = arr[idx]
                arr[idx] = old + h
                lp, _ = mlp.gradients(layers, x, t, **norm)
                arr[idx] = old - h
                lm, _ = mlp.gradients(layers, x, t, **norm)
                arr[idx] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(fd)), (l, idx, fd, g[idx])
    # the loss is the mean squared standardised error
    _, yraw, _ = mlp.forward(layers, x, **norm)
    ts = (t - norm["c_out"]) / norm["s_out"]
    assert abs(loss - np.mean((yraw - ts) ** 2)) < 1e-15


def test_gelu_closed_forms():
    z = np.linspace(-6, 6, 241)
    assert mlp.gelu(0.0) == 0.0 and abs(mlp.gelu_d(0.0) - 0.5) < 1e-16
    # GELU(z) - GELU(-z) = z (tanh is odd)
    assert np.abs(mlp.gelu(z) - mlp.gelu(-z) - z).max() < 1e-14
    # derivative by central differences
    h = 1e-6
    fd = (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_d(z)).max() < 1e-8
    # limits: the identity for large z, zero for large -z
    assert mlp.gelu(10.0) == 10.0 and abs(float(mlp.gelu(-10.0))) == 0.0
    assert mlp.gelu_d(10.0) == 1.0 and abs(float(mlp.gelu_d(-10.0))) == 0.0


def test_gelu_tanh_form_is_close_to_z_phi_z():
    """The tanh form approximates the exact unit z Phi(z), Phi the standard
    normal distribution function (here from the error function of the C
    library): within 4.8e-4 in value and 9e-4 in slope on [-8, 8] (largest
    near z = -2.7); a dropped term or a wrong constant breaks the bound."""
    z = np.linspace(-8, 8, 16001)
    phi = 0.5 * (1.0 + np.array([math.erf(v / math.sqrt(2.0)) for v in z]))
    dens = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    assert np.abs(mlp.gelu(z) - z * phi).max() < 4.8e-4
    assert np.abs(mlp.gelu_d(z) - (phi + z * dens)).max() < 9e-4
    # Phi(1) = 0.841344746068543 (standard normal table): the exact unit above
    assert abs(0.5 * (1.0 + math.erf(1.0 / math.sqrt(2.0))) - 0.8413447460685429) < 1e-15


def test_bf16_rounding_rule():
    # 8 significant bits: 1 + 2^-7 is representable, 1 + 2^-8 is a tie -> even (1), 1 + 3 * 2^-8 -> 1 + 2^-6
    v = np.array([1.0, 1 + 2.0**-7, 1 + 2.0**-8, 1 + 3 * 2.0**-8, -2.5, 3.0e-30], np.float64)
    r = mlp.bf16(v)
    assert r[0] == 1.0 and r[1] == 1 + 2.0**-7 and r[2] == 1.0 and r[3] == 1 + 2.0**-6 and r[4] == -2.5
    assert abs(r[5] - 3.0e-30) <= 2.0**-8 * 3.0e-30
    rng = np.random.default_rng(1)
    x = rng.normal(0, 10, 10000)
    q = mlp.bf16(x)
    assert (np.abs(q - x) <= 2.0**-8 * np.abs(x) + 1e-45).all()
    assert np.array_equal(mlp.bf16(q), q)  # idempotent


def test_quantized_oracle_stays_near_the_exact_one():
    layers, x, t, norm = _tiny(seed=3, width=16)
    l64, g64 = mlp.gradients(layers, x, t, **norm)
    lq, gq = mlp.gradients(layers, x, t, quantize=True, **norm)
    assert abs(lq - l64) <= 0.05 * l64
    f64, fq = mlp.flat(g64), mlp.flat(gq)
    assert np.linalg.norm(fq - f64) <= 0.05 * np.linalg.norm(f64)


def test_adam_closed_forms():
    """Adam's bias correction makes the first step, and every step under a
    constant gradient, move each parameter by lr g / (|g| + eps): lr against
    the gradient's sign (Kingma & Ba 2015, Sec. 2.1: the effective step is
    bounded by the step size and equals it in these cases)."""
    rng = np.random.default_rng(3)
    p0 = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    g[0] = 0.0
    lr = 1e-3
    m = v = np.zeros(50)
    p1, m, v = mlp.adam_step(p0, g, m, v, 1, lr)
    want = lr * g / (np.abs(g) + 1e-8)
    assert np.abs((p0 - p1) - want).max() < 1e-15
    assert p1[0] == p0[0]  # zero gradient, zero moments: no move
    # a constant gradient keeps m_hat = g and v_hat = g^2 at every step
    p = p1
    for t in range(2, 40):
        pn, m, v = mlp.adam_step(p, g, m, v, t, lr)
        assert np.abs((p - pn) - want).max() < 1e-12, t
        p = pn
    # steps scale with lr and not with the gradient's magnitude
    q1, _, _ = mlp.adam_step(p0, 1e3 * g, np.zeros(50), np.zeros(50), 1, 2 * lr)
    assert np.abs((p0 - q1) - 2 * lr * g / (np.abs(g) + 1e-11)).max() < 1e-14
