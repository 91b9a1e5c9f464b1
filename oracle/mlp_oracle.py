"""Oracle of the learned warm start's network, in plain numpy FP64.  TEST INFRASTRUCTURE ONLY: used by
tests/, __graft_entry__.smoke() and bench.py's CPU legs, never by the library.

The network (the paper has no learned part; it is this project's warm start): inputs
x = (E/N, 1/L, J1, J2, J3, J4), normalised x' = (x - shift) * scale; three hidden layers of 128 units
with SiLU(z) = z / (1 + exp(-z)); a linear output y ~ ln g / N.  Parameters are one flat vector:
WT1 [6][128] | b1 [128] | WT2 [128][128] | b2 | WT3 [128][128] | b3 | WT4 [128] | b4, with WT[k][j]
the weight from input k to unit j (so a layer is z = a_prev @ WT + b).

Loss over runs g (ln g of a run is defined up to a constant, so each run's residual is centred):
    L = (1/M) sum_g sum_{s in g} (r_s - mean_g r)^2,   r = y - target,   M = number of samples.
Gradient by the chain rule written out layer by layer (back-propagation); Adam as published
(Kingma & Ba, 2015) with bias correction.
"""
import numpy as np

N_IN, H = 6, 128
SHAPES = [("WT1", (N_IN, H)), ("b1", (H,)), ("WT2", (H, H)), ("b2", (H,)), ("WT3", (H, H)), ("b3", (H,)),
          ("WT4", (H,)), ("b4", ())]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = p[o:o + n].reshape(shp) if shp else p[o]
        o += n
    assert o == p.size
    return out


def pack(d):
    return np.concatenate([np.ravel(np.asarray(d[name], dtype=np.float64)) for name, _ in SHAPES])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_prime(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, x, shift, scale):
    """Returns y [M] and the activations needed by backward."""
    w = unpack(p)
    a0 = (np.asarray(x, dtype=np.float64) - np.asarray(shift, dtype=np.float64)) * np.asarray(scale, dtype=np.float64)
    z1 = a0 @ w["WT1"] + w["b1"]
    a1 = silu(z1)
    z2 = a1 @ w["WT2"] + w["b2"]
    a2 = silu(z2)
    z3 = a2 @ w["WT3"] + w["b3"]
    a3 = silu(z3)
    y = a3 @ w["WT4"] + w["b4"]
    return y, (a0, z1, a1, z2, a2, z3, a3)


def centred_loss(y, target, run_offsets):
    """L and dL/dy."""
    y = np.asarray(y, dtype=np.float64)
    r = y - np.asarray(target, dtype=np.float64)
    M = y.size
    L = 0.0
    dy = np.zeros(M)
    for g in range(len(run_offsets) - 1):
        a, b = run_offsets[g], run_offsets[g + 1]
        c = r[a:b] - r[a:b].mean()
        L += float(np.sum(c * c))
        dy[a:b] = 2.0 * c / M
    return L / M, dy


def backward(p, cache, dy):
    """Gradient of sum_s dy_s y_s with respect to p (flat)."""
    w = unpack(p)
    a0, z1, a1, z2, a2, z3, a3 = cache
    g = {}
    g["WT4"] = a3.T @ dy
    g["b4"] = dy.sum()
    da3 = np.outer(dy, w["WT4"])
    dz3 = da3 * silu_prime(z3)
    g["WT3"] = a2.T @ dz3
    g["b3"] = dz3.sum(0)
    da2 = dz3 @ w["WT3"].T
    dz2 = da2 * silu_prime(z2)
    g["WT2"] = a1.T @ dz2
    g["b2"] = dz2.sum(0)
    da1 = dz2 @ w["WT2"].T
    dz1 = da1 * silu_prime(z1)
    g["WT1"] = a0.T @ dz1
    g["b1"] = dz1.sum(0)
    return pack(g)


def loss_and_grad(p, x, target, run_offsets, shift, scale):
    y, cache = forward(p, x, shift, scale)
    L, dy = centred_loss(y, target, run_offsets)
    return L, backward(p, cache, dy)


def adam_step(p, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (p, m, v)."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a):
    """Round FP32 values to bfloat16 (nearest, ties to even), returned as FP64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
