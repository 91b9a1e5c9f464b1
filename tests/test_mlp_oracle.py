"""Pins of the warm-start network's FP64 oracle (CPU): the analytic gradient against central finite
differences, the closed form of a network with zero hidden weights, the invariances of the centred
loss, Adam's first step, SiLU and its derivative, and bfloat16 rounding."""
import numpy as np

from oracle import mlp_oracle as mo

SHIFT = np.array([-1.5, 0.2, 1.0, 0.4, 0.0, 0.0])
SCALE = np.array([1.0, 20.0, 1.0, 5.0, 10.0, 10.0])


def _params(rng, s=1.0):
    d = {}
    for name, shp in mo.SHAPES:
        fan = shp[0] if len(shp) == 2 else mo.H
        d[name] = rng.uniform(-1, 1, shp) * s / np.sqrt(fan) if shp else rng.uniform(-0.5, 0.5)
    for b in ("b1", "b2", "b3"):
        d[b] = rng.uniform(-0.3, 0.3, mo.H)
    return mo.pack(d)


def _inputs(rng, M):
    x = np.zeros((M, 6))
    x[:, 0] = rng.uniform(-3.5, 0, M)
    x[:, 1] = rng.choice([1 / 4, 1 / 5, 1 / 6, 1 / 8], M)
    x[:, 2] = 1.0
    x[:, 3] = rng.uniform(0.2, 0.6, M)
    x[:, 4] = rng.uniform(-0.1, 0.1, M)
    return x


def test_param_count_matches_library_constant():
    assert mo.N_PARAMS == 34049


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    x = _inputs(rng, 14)
    t = rng.normal(0, 0.3, 14)
    seg = [0, 5, 6, 14]           # runs of 5, 1 and 8 samples
    L, g = mo.loss_and_grad(p, x, t, seg, SHIFT, SCALE)
    # probe parameters in every block (first, last and random entries)
    idx, o = [], 0
    for _, shp in mo.SHAPES:
        n = int(np.prod(shp))
        idx += [o, o + n - 1] + list(rng.integers(o, o + n, 4))
        o += n
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mo.loss_and_grad(pp, x, t, seg, SHIFT, SCALE)[0] - mo.loss_and_grad(pm, x, t, seg, SHIFT, SCALE)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(g[i]), (i, fd, g[i])


def test_zero_hidden_weights_closed_form():
    rng = np.random.default_rng(2)
    d = mo.unpack(_params(rng))
    d = {k: np.array(v, copy=True) for k, v in d.items()}
    for k in ("WT1", "WT2", "WT3"):
        d[k][:] = 0.0
    p = mo.pack(d)
    x = _inputs(rng, 7)
    y, _ = mo.forward(p, x, SHIFT, SCALE)
    b3 = d["b3"]
    want = float(d["b4"]) + float(np.dot(d["WT4"], b3 / (1 + np.exp(-b3))))
    assert np.allclose(y, want, rtol=0, atol=1e-14)


def test_centred_loss_ignores_a_constant_per_run():
    rng = np.random.default_rng(3)
    p = _params(rng)
    x = _inputs(rng, 12)
    seg = [0, 4, 12]
    y, _ = mo.forward(p, x, SHIFT, SCALE)
    # targets equal to the output up to a constant per run: zero loss and zero gradient
    t = y.copy()
    t[:4] += 3.0
    t[4:] -= 7.5
    L, g = mo.loss_and_grad(p, x, t, seg, SHIFT, SCALE)
    assert L < 1e-25 and np.max(np.abs(g)) < 1e-12
    t2 = rng.normal(0, 1, 12)
    L1, g1 = mo.loss_and_grad(p, x, t2, seg, SHIFT, SCALE)
    t3 = t2.copy()
    t3[4:] += 11.0
    L2, g2 = mo.loss_and_grad(p, x, t3, seg, SHIFT, SCALE)
    assert abs(L1 - L2) < 1e-12 * max(1.0, L1) and np.allclose(g1, g2, rtol=1e-10, atol=1e-14)
    # a one-sample run contributes nothing
    L3, _ = mo.centred_loss(np.array([1.0, 2.0, 5.0]), np.array([0.0, 0.0, -4.0]), [0, 2, 3])
    assert abs(L3 - 0.5 / 3) < 1e-15


def test_adam_first_step_is_a_signed_step():
    rng = np.random.default_rng(4)
    p = rng.normal(0, 1, 50)
    g = rng.normal(0, 1, 50)
    p1, m, v = mo.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=1e-3, eps=0.0)
    assert np.allclose(p1, p - 1e-3 * np.sign(g), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_silu_and_derivative():
    assert mo.silu(0.0) == 0.0 and mo.silu_prime(0.0) == 0.5
    z = np.linspace(-8, 8, 33)
    fd = (mo.silu(z + 1e-6) - mo.silu(z - 1e-6)) / 2e-6
    assert np.allclose(mo.silu_prime(z), fd, rtol=1e-7, atol=1e-9)
    assert abs(mo.silu(40.0) - 40.0) < 1e-15


def test_bf16_rounding():
    one = 1.0
    cases = {one: one, one + 2 ** -8: one, one + 3 * 2 ** -8: one + 2 ** -6, one + 2 ** -8 + 2 ** -20: one + 2 ** -7,
             -2.5: -2.5, 3.0e-3: None}
    for v, want in cases.items():
        r = mo.bf16_round(np.float32(v))
        if want is None:
            assert abs(r - v) <= abs(v) * 2 ** -8   # half a unit of the 8-bit significand
        else:
            assert r == want, (v, r, want)
