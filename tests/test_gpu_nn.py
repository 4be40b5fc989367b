"""The learned correction's kernels through the C ABI against the FP64 oracle network.

Scales s_in and s_out are powers of two so that the input scaling is exact on both sides; the
oracle then sees exactly the GPU's BF16 inputs and weights and (with store=bf16_round) keeps its
hidden activations at the precision the GPU stores them in. What remains is FP32 against FP64
accumulation, BF16 storage of the backward gradients, and the odd activation rounded the other way.
"""
import numpy as np
import pytest

from oracle import ics as oics
from oracle import nn as onn

pytestmark = pytest.mark.gpu

S_IN, S_OUT = 4.0, 0.5


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1506_03737_gb300 import colapm
    return colapm, torch


def smooth_field(n, seed, scale):
    """[n^3][3] random field with a few-cell correlation length (particle-id order)."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((3, n, n, n))
    k = np.fft.fftfreq(n) * n
    kk = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    f = np.real(np.fft.ifftn(np.fft.fftn(f, axes=(1, 2, 3)) * np.exp(-kk / 20.0), axes=(1, 2, 3)))
    f *= scale / f.std()
    return np.ascontiguousarray(np.stack([f[j].ravel() for j in range(3)], axis=1), dtype=np.float32)


def emulated(params_flat):
    """Oracle parameters as the GPU uses them: BF16 weights, FP32 biases."""
    out = []
    for w, b in onn.unflatten(params_flat.astype(np.float64)):
        out.append((onn.bf16_round(w), b.astype(np.float32).astype(np.float64)))
    return out


def grid(a, n):
    return a.reshape(n, n, n, 3).astype(np.float64)


def make_net(C, n, seed=1, lr=1e-3, engine=0):
    return C.colapm_nn_create(n, C.nn_default_config(s_in=S_IN, s_out=S_OUT, seed=seed, lr=lr, engine=engine))


@pytest.mark.parametrize("n", [16, 48])
def test_forward_matches_oracle(env, n):
    C, torch = env
    net = make_net(C, n)
    try:
        psi = smooth_field(n, 3, 3.0)
        d_psi = torch.from_numpy(psi).cuda()
        out = torch.empty_like(d_psi)
        C.colapm_nn_forward(net, d_psi, out)
        got = grid(out.cpu().numpy(), n)
        params = C.colapm_nn_get_params(net)
        x = onn.bf16_round(grid(psi, n) / S_IN)
        ref, _ = onn.forward(x, emulated(params), store=onn.bf16_round)
        ref *= S_OUT
        rms = np.sqrt(np.mean(ref ** 2))
        assert np.sqrt(np.mean((got - ref) ** 2)) < 2e-3 * rms
        assert np.max(np.abs(got - ref)) < 2e-2 * rms
        # Against the plain FP64 network on unrounded inputs: BF16 storage error only.
        plain, _ = onn.forward(grid(psi, n) / S_IN, onn.unflatten(params.astype(np.float64)))
        assert np.sqrt(np.mean((got - S_OUT * plain) ** 2)) < 2e-2 * rms
        # add = 1 returns psi + correction
        out2 = torch.empty_like(d_psi)
        C.colapm_nn_forward(net, d_psi, out2, add=True)
        assert np.allclose(out2.cpu().numpy(), psi + out.cpu().numpy(), atol=1e-5)
    finally:
        C.colapm_nn_destroy(net)


def test_gradients_match_oracle_and_are_deterministic(env):
    C, torch = env
    n = 32
    net = make_net(C, n, seed=2)
    try:
        psi = smooth_field(n, 4, 3.0)
        tgt = smooth_field(n, 5, 0.4)
        d_psi, d_tgt = torch.from_numpy(psi).cuda(), torch.from_numpy(tgt).cuda()
        g, loss = C.colapm_nn_grads(net, d_psi, d_tgt)
        g2, loss2 = C.colapm_nn_grads(net, d_psi, d_tgt)
        assert np.array_equal(g, g2)
        params = C.colapm_nn_get_params(net)
        x = onn.bf16_round(grid(psi, n) / S_IN)
        lref, gref = onn.loss_and_grads(x, grid(tgt, n) / S_OUT, emulated(params), store=onn.bf16_round)
        assert abs(loss / lref - 1) < 1e-4
        gl = onn.unflatten(g.astype(np.float64))
        for l, ((gw, gb), (rw, rb)) in enumerate(zip(gl, gref)):
            assert np.linalg.norm(gw - rw) < 1e-2 * np.linalg.norm(rw), l
            assert np.linalg.norm(gb - rb) < 1e-2 * np.linalg.norm(rb) + 1e-12, l
    finally:
        C.colapm_nn_destroy(net)


def test_adam_step_moves_by_lr_sign_on_first_step(env):
    C, torch = env
    n = 16
    lr = 1e-3
    net = make_net(C, n, seed=3, lr=lr)
    try:
        psi = smooth_field(n, 6, 3.0)
        tgt = smooth_field(n, 7, 0.4)
        d_psi, d_tgt = torch.from_numpy(psi).cuda(), torch.from_numpy(tgt).cuda()
        g, _ = C.colapm_nn_grads(net, d_psi, d_tgt)
        p0 = C.colapm_nn_get_params(net)
        C.colapm_nn_train_step(net, d_psi, d_tgt)
        p1 = C.colapm_nn_get_params(net)
        assert C.colapm_nn_steps(net) == 1
        want, _, _ = onn.adam_step(p0.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, lr=lr)
        assert np.max(np.abs(p1 - want)) < 1e-7
        moved = np.abs(g) > 1e-3                   # eps / |g| < 1e-5
        assert np.allclose(p1[moved] - p0[moved], -lr * np.sign(g[moved]), atol=2e-7)
    finally:
        C.colapm_nn_destroy(net)


def test_overfits_one_pair(env):
    C, torch = env
    n = 32
    net = make_net(C, n, seed=4, lr=3e-3)
    teacher = make_net(C, n, seed=11)
    try:
        psi = torch.from_numpy(smooth_field(n, 8, 3.0)).cuda()
        tgt = torch.empty_like(psi)
        C.colapm_nn_forward(teacher, psi, tgt)      # a target the architecture can represent
        first = C.colapm_nn_train_step(net, psi, tgt)
        for _ in range(400):
            last = C.colapm_nn_train_step(net, psi, tgt)
        assert last < 0.05 * first
    finally:
        C.colapm_nn_destroy(net)
        C.colapm_nn_destroy(teacher)


def test_displacement_accessors(env):
    C, torch = env
    p = C.default_params(np=32, nm=64, box=256.0, seed=21, n_steps=4)
    ctx = C.colapm_create(p)
    try:
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, -1)
        n = 32 ** 3
        psi = C.colapm_get_displacement(ctx, np.empty((n, 3), np.float32))
        pos, _ = C.colapm_get_particles(ctx, np.empty((n, 3), np.float32))
        q = oics.lagrangian_grid(32, 256.0, 64)
        d = pos.astype(np.float64) - q
        d -= 256.0 * np.rint(d / 256.0)
        assert np.max(np.abs(psi - d)) < 1e-3
        k0, p0, n0 = C.colapm_power(ctx, 20)
        # Round trip through x = q + Psi, from a device array.
        C.colapm_set_displacement(ctx, torch.from_numpy(psi).cuda())
        psi2 = C.colapm_get_displacement(ctx, np.empty((n, 3), np.float32))
        assert np.max(np.abs(psi2 - psi)) < 1e-4
        k1, p1, n1 = C.colapm_power(ctx, 20)
        assert np.array_equal(n0, n1)
        ok = n0 > 0
        assert np.max(np.abs(p1[ok] / p0[ok] - 1)) < 1e-4
        with pytest.raises(C.ColapmError):
            C.colapm_set_displacement(ctx, np.full((n, 3), 1e4, np.float32))
    finally:
        C.colapm_destroy(ctx)


def test_rejects_bad_arguments(env):
    C, torch = env
    with pytest.raises(C.ColapmError):
        C.colapm_nn_create(24, C.nn_default_config())
    with pytest.raises(C.ColapmError):
        C.colapm_nn_create(32, C.nn_default_config(s_in=0.0))
    net = make_net(C, 16)
    try:
        host = np.zeros((16 ** 3, 3), np.float32)
        with pytest.raises(C.ColapmError):
            C.colapm_nn_forward(net, host, np.zeros_like(host))
    finally:
        C.colapm_nn_destroy(net)


def test_tcgen05_forward_matches_oracle_on_sampled_blocks(env):
    # engine 1 at n = 128 runs the convolutions on the tcgen05 tensor cores. The oracle computes the network on
    # 24^3 neighbourhoods: with a receptive field of 4 voxels the central 16^3 of each block is
    # exact although the block wraps periodically at its own edges.
    C, torch = env
    n = 128
    net = make_net(C, n, seed=5, engine=1)
    try:
        psi = smooth_field(n, 9, 3.0)
        d_psi = torch.from_numpy(psi).cuda()
        out = torch.empty_like(d_psi)
        C.colapm_nn_forward(net, d_psi, out)
        got = grid(out.cpu().numpy(), n)
        params = emulated(C.colapm_nn_get_params(net))
        x = onn.bf16_round(grid(psi, n) / S_IN)
        for cz, cy, cx in [(0, 0, 0), (70, 33, 101), (127, 64, 5)]:
            iz, iy, ix = [(c + np.arange(-12, 12)) % n for c in (cz, cy, cx)]
            ref, _ = onn.forward(x[np.ix_(iz, iy, ix)], params, store=onn.bf16_round)
            ref = S_OUT * ref[4:20, 4:20, 4:20]
            g = got[np.ix_(iz[4:20], iy[4:20], ix[4:20])]
            rms = np.sqrt(np.mean(ref ** 2))
            assert np.sqrt(np.mean((g - ref) ** 2)) < 2e-3 * rms
            assert np.max(np.abs(g - ref)) < 2e-2 * rms
    finally:
        C.colapm_nn_destroy(net)


def test_tcgen05_and_mma_sync_engines_agree(env):
    C, torch = env
    n = 128
    tc = C.colapm_nn_create(n, C.nn_default_config(s_in=S_IN, s_out=S_OUT, seed=6, engine=1))
    ms = C.colapm_nn_create(n, C.nn_default_config(s_in=S_IN, s_out=S_OUT, seed=6, engine=0))
    try:
        psi = torch.from_numpy(smooth_field(n, 10, 3.0)).cuda()
        tgt = torch.from_numpy(smooth_field(n, 11, 0.4)).cuda()
        oa, ob = torch.empty_like(psi), torch.empty_like(psi)
        C.colapm_nn_forward(tc, psi, oa)
        C.colapm_nn_forward(ms, psi, ob)
        C.colapm_nn_sync(tc)
        C.colapm_nn_sync(ms)
        a, b = oa.double(), ob.double()
        assert torch.sqrt(torch.mean((a - b) ** 2)).item() < 1e-3 * torch.sqrt(torch.mean(b ** 2)).item()
        ga, la = C.colapm_nn_grads(tc, psi, tgt)
        gb, lb = C.colapm_nn_grads(ms, psi, tgt)
        assert abs(la / lb - 1) < 1e-4
        for l, ((wa, ba), (wb, bb)) in enumerate(zip(onn.unflatten(ga.astype(np.float64)),
                                                       onn.unflatten(gb.astype(np.float64)))):
            assert np.linalg.norm(wa - wb) < 5e-3 * np.linalg.norm(wb), l
            assert np.linalg.norm(ba - bb) < 5e-3 * np.linalg.norm(bb) + 1e-12, l
    finally:
        C.colapm_nn_destroy(tc)
        C.colapm_nn_destroy(ms)
