"""Pins of the oracle's correction network: finite differences, definitions, BF16 rounding."""
import numpy as np

from oracle import nn


def small_problem(seed=0, n=5, sizes=(3, 4, 4, 4, 3)):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, n, n, sizes[0]))
    t = rng.standard_normal((n, n, n, sizes[-1]))
    params = nn.init_params(list(sizes), seed=seed + 1)
    return x, t, params


def test_conv_matches_direct_definition():
    # Brute force over voxels and taps on a tiny grid (periodic indices written out).
    rng = np.random.default_rng(2)
    n, ci, co = 4, 2, 3
    a = rng.standard_normal((n, n, n, ci))
    w = rng.standard_normal((27, co, ci))
    b = rng.standard_normal(co)
    out = nn.conv(a, w, b)
    ref = np.zeros((n, n, n, co))
    for z in range(n):
        for y in range(n):
            for x in range(n):
                acc = b.copy()
                for dz in (-1, 0, 1):
                    for dy in (-1, 0, 1):
                        for dx in (-1, 0, 1):
                            t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)
                            acc += w[t] @ a[(z + dz) % n, (y + dy) % n, (x + dx) % n]
                ref[z, y, x] = acc
    assert np.abs(out - ref).max() < 1e-12


def test_gradients_match_central_finite_differences():
    x, t, params = small_problem()
    loss, grads = nn.loss_and_grads(x, t, params)
    rng = np.random.default_rng(3)
    h = 1e-6
    for l in range(len(params)):
        w, b = params[l]
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in w.shape)
            wp = [(ww.copy(), bb.copy()) for ww, bb in params]
            wm = [(ww.copy(), bb.copy()) for ww, bb in params]
            wp[l][0][idx] += h
            wm[l][0][idx] -= h
            fd = (nn.loss_and_grads(x, t, wp)[0] - nn.loss_and_grads(x, t, wm)[0]) / (2 * h)
            assert abs(fd - grads[l][0][idx]) < 1e-7 + 1e-5 * abs(fd)
        j = int(rng.integers(0, b.shape[0]))
        bp = [(ww.copy(), bb.copy()) for ww, bb in params]
        bm = [(ww.copy(), bb.copy()) for ww, bb in params]
        bp[l][1][j] += h
        bm[l][1][j] -= h
        fd = (nn.loss_and_grads(x, t, bp)[0] - nn.loss_and_grads(x, t, bm)[0]) / (2 * h)
        assert abs(fd - grads[l][1][j]) < 1e-7 + 1e-5 * abs(fd)


def test_identity_network_and_relu_gate():
    # One layer with the centre tap = identity reproduces its input; ReLU zeroes the negative half.
    n = 3
    x = np.random.default_rng(4).standard_normal((n, n, n, 2))
    w = np.zeros((27, 2, 2))
    w[13] = np.eye(2)
    out, _ = nn.forward(x, [(w, np.zeros(2))])
    assert np.array_equal(out, x)
    out2, _ = nn.forward(x, [(w, np.zeros(2)), (w, np.zeros(2))])
    assert np.array_equal(out2, np.maximum(x, 0))


def test_bf16_round_half_to_even():
    one = 1.0
    ulp = 2.0 ** -7                                      # BF16 spacing in [1, 2)
    vals = np.array([one, one + ulp / 2, one + 1.5 * ulp, one + ulp / 4, -3.0], dtype=np.float32)
    out = nn.bf16_round(vals)
    assert list(out) == [1.0, 1.0, one + 2 * ulp, 1.0, -3.0]


def test_flatten_roundtrip_and_size():
    params = nn.init_params(None, seed=5)
    flat = nn.flatten(params)
    assert flat.size == 16467                      # 27*(3*16 + 16*16*2 + 16*3) + 16*3 + 3
    back = nn.unflatten(flat)
    for (w, b), (w2, b2) in zip(params, back):
        assert np.array_equal(w, w2) and np.array_equal(b, b2)


def test_adam_closed_forms():
    # Step 1: m_hat = g and v_hat = g^2, so each weight moves by -lr g/(|g| + eps), i.e. -lr sign(g).
    g = np.array([3.0, -2e-3, 5e-1, 0.0])
    p0 = np.zeros(4)
    p1, m1, m2 = nn.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    assert np.allclose(p1[:3], -0.01 * np.sign(g[:3]), rtol=1e-5) and p1[3] == 0.0
    # A constant gradient keeps m_hat = g and v_hat = g^2 at every step: the same move each time.
    p, a, b = p1, m1, m2
    for t in range(2, 6):
        p, a, b = nn.adam_step(p, g, a, b, t, lr=0.01)
    assert np.allclose(p[:3], -0.05 * np.sign(g[:3]), rtol=1e-5)


def test_stored_activation_rounding_changes_only_storage():
    x, t, params = small_problem(seed=7)
    out, acts = nn.forward(x, params, store=nn.bf16_round)
    for a in acts[1:-1]:
        assert np.array_equal(a, nn.bf16_round(a))
    ref, _ = nn.forward(x, params)
    assert np.sqrt(np.mean((out - ref) ** 2)) < 1e-2 * np.sqrt(np.mean(ref ** 2))
