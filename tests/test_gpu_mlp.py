"""The warm-start network's CUDA kernels (forward, centred loss, backward, reduction, Adam) against
the FP64 oracle, evaluated with the same BF16-rounded weights the kernels use.  Sizes span one
partial tile up to many tiles per persistent CTA, with runs of one sample and ragged tails."""
import numpy as np
import pytest

import paper_1411_4212_gb300 as rw
from oracle import mlp_oracle as mo

pytestmark = pytest.mark.gpu

SHIFT = np.array([-1.5, 0.2, 1.0, 0.4, 0.0, 0.0], dtype=np.float32)
SCALE = np.array([1.0, 20.0, 1.0, 5.0, 10.0, 10.0], dtype=np.float32)


def _params(rng):
    d = {}
    for name, shp in mo.SHAPES:
        fan = shp[0] if len(shp) == 2 else mo.H
        d[name] = rng.uniform(-1, 1, shp) / np.sqrt(fan) if shp else 0.1
    for b in ("b1", "b2", "b3"):
        d[b] = rng.uniform(-0.3, 0.3, mo.H)
    return mo.pack(d).astype(np.float32)


def _inputs(rng, M):
    x = np.zeros((M, 6), dtype=np.float32)
    x[:, 0] = rng.uniform(-3.5, 0, M)
    x[:, 1] = rng.choice([1 / 4, 1 / 5, 1 / 6, 1 / 8], M)
    x[:, 2] = 1.0
    x[:, 3] = rng.uniform(0.2, 0.6, M)
    x[:, 4] = rng.uniform(-0.1, 0.1, M)
    return x


def _runs(rng, M):
    cuts = np.sort(rng.choice(np.arange(1, M), size=max(1, M // 40), replace=False))
    seg = np.concatenate([[0], cuts, [M]]).astype(np.int32)
    return seg


@pytest.mark.parametrize("M", [1, 15, 16, 17, 333, 5000])
def test_forward_loss_and_gradient_match_oracle(M):
    rng = np.random.default_rng(M)
    net = rw.Mlp(SHIFT, SCALE, seed=3)
    p = _params(rng)
    net.set_params(p)
    pb = net.params(bf16=True).astype(np.float64)
    assert np.array_equal(pb, mo.bf16_round(p))
    x = _inputs(rng, M)
    y = net.forward(x)
    yo, _ = mo.forward(pb, x.astype(np.float64), SHIFT.astype(np.float64), SCALE.astype(np.float64))
    assert np.max(np.abs(y - yo)) <= 2e-5 * (1 + np.max(np.abs(yo)))
    t = (yo + rng.normal(0, 0.2, M)).astype(np.float32)
    seg = _runs(rng, M) if M > 1 else np.array([0, 1], dtype=np.int32)
    L, g = net.gradient(x, t, seg)
    Lo, go = mo.loss_and_grad(pb, x.astype(np.float64), t.astype(np.float64), seg, SHIFT.astype(np.float64),
                              SCALE.astype(np.float64))
    assert abs(L - Lo) <= 1e-4 * Lo + 1e-9
    scale = np.max(np.abs(go)) + 1e-12
    assert np.max(np.abs(g - go)) <= 2e-4 * scale, np.max(np.abs(g - go)) / scale
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go) + 1e-12
    net.close()


def test_gradient_is_deterministic():
    rng = np.random.default_rng(7)
    net = rw.Mlp(SHIFT, SCALE, seed=1)
    x = _inputs(rng, 3001)
    t = rng.normal(0, 1, 3001).astype(np.float32)
    seg = _runs(rng, 3001)
    L1, g1 = net.gradient(x, t, seg)
    L2, g2 = net.gradient(x, t, seg)
    assert L1 == L2 and np.array_equal(g1.view(np.int32), g2.view(np.int32))
    net.close()


def test_adam_steps_match_oracle():
    rng = np.random.default_rng(11)
    net = rw.Mlp(SHIFT, SCALE, seed=5)
    p0 = _params(rng)
    net.set_params(p0)
    x = _inputs(rng, 400)
    t = rng.normal(0, 1, 400).astype(np.float32)
    seg = _runs(rng, 400)
    # the oracle's Adam, fed the kernels' gradient at each step, against three device steps
    p, m, v = p0.astype(np.float64), np.zeros(p0.size), np.zeros(p0.size)
    for step in range(1, 4):
        net_state = net.params()
        _, g = net.gradient(x, t, seg)
        p, m, v = mo.adam_step(net_state.astype(np.float64), g.astype(np.float64), m, v, step, lr=1e-3)
        net.train(x, t, seg, steps=1, lr=1e-3)
        got = net.params().astype(np.float64)
        assert np.max(np.abs(got - p)) <= 1e-6, step
        assert np.array_equal(net.params(bf16=True).astype(np.float64), mo.bf16_round(net.params()))
    net.close()


def test_training_fits_a_smooth_family():
    """A family of smooth curves (different per 'run'), known up to a constant: training lowers the
    centred loss by orders of magnitude."""
    rng = np.random.default_rng(5)
    runs, xs, ts = 24, [], []
    for r in range(runs):
        n = int(rng.integers(40, 90))
        x = np.zeros((n, 6), dtype=np.float32)
        j2, j3 = rng.uniform(0.2, 0.6), rng.uniform(-0.1, 0.1)
        L = rng.choice([4, 5, 6])
        e = np.linspace(-3.0, 0.0, n)
        x[:, 0], x[:, 1], x[:, 2], x[:, 3], x[:, 4] = e, 1.0 / L, 1.0, j2, j3
        ts.append((np.sqrt(e + 3.2) * (1 + j2) + 0.5 * j3 * e + 7.0 * r).astype(np.float32))
        xs.append(x)
    x = np.concatenate(xs)
    t = np.concatenate(ts)
    seg = np.cumsum([0] + [len(a) for a in ts]).astype(np.int32)
    net = rw.Mlp(SHIFT, SCALE, seed=2)
    hist = net.train(x, t, seg, steps=600, lr=2e-3)
    assert hist[-1] < hist[0] / 100, (hist[0], hist[-1])
    net.close()
