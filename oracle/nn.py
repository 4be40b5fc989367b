"""Oracle (test infrastructure only): the displacement-correction network in FP64.

The paper has no learned component; this network is the learned correction of the build's
scope: a coarse, few-step COLA run's final displacement field Psi (3 channels on the
Lagrangian grid) is mapped to a correction dPsi (3 channels) by four periodic 3x3x3
convolutions, C_in -> 16 -> 16 -> 16 -> 3, with ReLU between layers, trained with the mean
squared error against Psi_fine - Psi_coarse.

Layout: fields are channels-last arrays [z][y][x][c]; a layer's weights are W[tap][c_out][c_in]
with tap = (dz + 1) 9 + (dy + 1) 3 + (dx + 1), and

    out[v][o] = b[o] + sum_tap sum_i W[tap][o][i] in[v + d_tap][i]      (periodic in v)

(a cross-correlation, the usual convolution layer). The backward pass is written out by hand:

    dW[tap][o][i] = sum_v dz[v][o] a[v + d_tap][i]
    db[o]         = sum_v dz[v][o]
    da[u][i]      = sum_tap sum_o W[tap][o][i] dz[u - d_tap][o]
    dz_prev       = da * (a > 0)                         (ReLU)
"""
import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(a, d):
    """b[v] = a[v + d] with periodic wrap over the three spatial axes."""
    dz, dy, dx = d
    return np.roll(a, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def conv(a, w, b):
    """Periodic 3x3x3 cross-correlation of a [.., C_in] with w [27, C_out, C_in] plus bias b."""
    out = np.zeros(a.shape[:3] + (w.shape[1],))
    for t, d in enumerate(TAPS):
        out += shift(a, d) @ w[t].T
    return out + b


def forward(x, params, store=None):
    """params: list of (W, b). Returns the output and the list of layer inputs/outputs.

    store (optional) maps each hidden activation to the values kept between layers, e.g.
    bf16_round to model activations stored in BF16; arithmetic stays FP64."""
    acts = [x]
    h = x
    for l, (w, b) in enumerate(params):
        z = conv(h, w, b)
        if l < len(params) - 1:
            h = np.maximum(z, 0.0)
            if store is not None:
                h = store(h)
        else:
            h = z
        acts.append(h)
    return h, acts


def loss_and_grads(x, target, params, store=None):
    """Mean squared error over all voxels and channels, and its gradients [(dW, db)] per layer."""
    pred, acts = forward(x, params, store)
    diff = pred - target
    loss = float(np.mean(diff * diff))
    dz = 2.0 * diff / diff.size
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        w, _ = params[l]
        a_in = acts[l]
        dw = np.zeros_like(w)
        flat_dz = dz.reshape(-1, dz.shape[-1])
        for t, d in enumerate(TAPS):
            dw[t] = flat_dz.T @ shift(a_in, d).reshape(-1, a_in.shape[-1])
        db = flat_dz.sum(axis=0)
        grads[l] = (dw, db)
        if l > 0:
            da = np.zeros(a_in.shape)
            for t, d in enumerate(TAPS):
                da += shift(dz, (-d[0], -d[1], -d[2])) @ w[t]
            dz = da * (acts[l] > 0)
    return loss, grads


def adam_step(params, grads, m1, m2, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of flat arrays; t counts from 1.
    Returns the new (params, m1, m2)."""
    m1 = beta1 * m1 + (1.0 - beta1) * grads
    m2 = beta2 * m2 + (1.0 - beta2) * grads * grads
    mh = m1 / (1.0 - beta1 ** t)
    vh = m2 / (1.0 - beta2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m1, m2


def flatten(params):
    """Flat parameter vector: per layer W[27][c_out][c_in] then b[c_out]."""
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def unflatten(flat, sizes=(3, 16, 16, 16, 3)):
    out, k = [], 0
    for i in range(len(sizes) - 1):
        nw = 27 * sizes[i + 1] * sizes[i]
        w = np.asarray(flat[k:k + nw], dtype=np.float64).reshape(27, sizes[i + 1], sizes[i])
        k += nw
        b = np.asarray(flat[k:k + sizes[i + 1]], dtype=np.float64)
        k += sizes[i + 1]
        out.append((w, b))
    assert k == len(flat)
    return out


def init_params(channels, seed=0, c_in=3, c_out=3, hidden=16):
    """He-style random weights (FP64) for c_in -> hidden x3 -> c_out."""
    rng = np.random.default_rng(seed)
    sizes = [c_in, hidden, hidden, hidden, c_out] if channels is None else channels
    params = []
    for i in range(len(sizes) - 1):
        fan_in = 27 * sizes[i]
        params.append((rng.standard_normal((27, sizes[i + 1], sizes[i])) * np.sqrt(2.0 / fan_in),
                       rng.standard_normal(sizes[i + 1]) * 0.01))
    return params


def bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1))
    r = ((bits + bias) & np.uint64(0xFFFF0000)).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)
