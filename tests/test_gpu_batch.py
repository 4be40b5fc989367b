"""Batched mocks of uneven sizes (one CUDA graph) and the autotuner, through the C ABI.

The batch must give each mock exactly what a single context gives for the same parameters and
seed, and (for the sizes the oracle finishes in seconds) the oracle's P(k) within 1e-3 per bin.
"""
import numpy as np
import pytest

from oracle import cola as ocola, cosmology as ocosmo, power as opower

pytestmark = pytest.mark.gpu

# (np, nm, box): power-of-two and mixed-radix meshes (96 = 2^5 3, 160 = 2^5 5)
MOCKS = [(16, 32, 64.0), (32, 64, 128.0), (32, 96, 160.0), (32, 160, 200.0), (16, 16, 100.0), (32, 64, 96.0)]


@pytest.fixture(scope="module")
def C():
    from paper_1506_03737_gb300 import colapm
    return colapm


def single_power(C, p, nbins):
    ctx = C.colapm_create(p)
    try:
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, -1)
        return C.colapm_power(ctx, nbins)
    finally:
        C.colapm_destroy(ctx)


def test_batch_matches_single_contexts_and_oracle(C):
    params = [C.default_params(np=a, nm=b, box=L, seed=500 + i, n_steps=6) for i, (a, b, L) in enumerate(MOCKS)]
    b = C.colapm_batch_create(params, nstreams=0)
    try:
        nbins = 24
        k, p, cnt = C.colapm_batch_run(b, len(params), nbins)
        assert C.colapm_batch_streams(b) in (1, 2, 4, 8)
        for i, prm in enumerate(params):
            ks, ps, ns = single_power(C, prm, nbins)
            assert np.array_equal(cnt[i], ns)
            ok = ns > 0
            assert np.max(np.abs(p[i][ok] / ps[ok] - 1)) < 1e-9
            assert np.max(np.abs(k[i][ok] / ks[ok] - 1)) < 1e-9
        pk = ocosmo.linear_pk(0.3, 0.7, 0.96, 0.8)
        for i in (0, 1):                        # sizes the oracle runs in seconds
            a, bm, L = MOCKS[i]
            r = ocola.Run(L, a, bm, 0.3, 9.0, 0.0, 6)
            r.make_ics(500 + i, pk)
            r.run()
            kr, pr, nr = opower.power_from_positions(r.x, L, a, bm, nbins)
            assert np.array_equal(cnt[i], nr)
            ok = nr > 0
            assert np.max(np.abs(p[i][ok] / pr[ok] - 1)) < 1e-3
        # New seeds through the pinned buffer give new mocks; the old seeds reproduce the old ones.
        k2, p2, _ = C.colapm_batch_run(b, len(params), nbins, seeds=[900 + i for i in range(len(params))])
        assert not np.allclose(p2[1], p[1])
        k3, p3, cnt3 = C.colapm_batch_run(b, len(params), nbins, seeds=[500 + i for i in range(len(params))])
        assert np.array_equal(cnt3, cnt)
        assert np.allclose(p3, p, rtol=1e-9, equal_nan=True)
    finally:
        C.colapm_batch_destroy(b)


def test_autotune_preserves_state_and_results(C):
    p = C.default_params(np=64, nm=128, box=200.0, seed=31)
    a, b = C.colapm_create(p), C.colapm_create(p)
    try:
        for ctx in (a, b):
            C.colapm_make_ics(ctx)
            C.colapm_step(ctx, 2)
        n = 64 ** 3
        before = [np.empty((n, 3), np.int32), np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)]
        C.colapm_get_state(a, *before)
        choice = C.colapm_autotune(a)
        assert choice["block"] in (128, 256, 512)
        after = [np.empty_like(x) for x in before]
        C.colapm_get_state(a, *after)
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        assert C.colapm_steps_done(a) == 2
        C.colapm_step(a, -1)
        C.colapm_step(b, -1)
        sa = [np.empty_like(x) for x in before]
        sb = [np.empty_like(x) for x in before]
        C.colapm_get_state(a, *sa)
        C.colapm_get_state(b, *sb)
        ua = sa[0] + sa[1].astype(np.float64)
        ub = sb[0] + sb[1].astype(np.float64)
        d = ua - ub
        d -= 128 * np.rint(d / 128)
        assert np.sqrt(np.mean(d ** 2)) < 1e-4                  # cells; engines differ only in FP32 rounding
    finally:
        C.colapm_destroy(a)
        C.colapm_destroy(b)


def test_lockstep_and_per_mock_schedules_agree(C):
    """The lockstep schedule (multi-mock persistent deposit and gather over work items of every
    mock, uneven sizes and step counts) against each mock run on its own, in one batch: the same
    mode counts and the same P(k) up to the order of the FP64 bin sums (atomic, so not fixed from
    run to run), replay after replay (the ticket counters reset themselves)."""
    params = [C.default_params(np=a, nm=b, box=L, seed=700 + i, n_steps=4 + (i % 3)) for i, (a, b, L) in enumerate(MOCKS)]
    b = C.colapm_batch_create(params, nstreams=2)
    try:
        nbins = 16
        seeds = [40 + i for i in range(len(params))]
        C.colapm_batch_set_lockstep(b, True)
        k1, p1, n1 = C.colapm_batch_run(b, len(params), nbins, seeds=seeds)
        k1b, p1b, _ = C.colapm_batch_run(b, len(params), nbins, seeds=seeds)
        C.colapm_batch_set_lockstep(b, False)
        k2, p2, n2 = C.colapm_batch_run(b, len(params), nbins, seeds=seeds)
        assert np.array_equal(n1, n2)
        for a, b_ in ((p1, p2), (k1, k2), (p1, p1b), (k1, k1b)):
            assert np.allclose(a, b_, rtol=1e-12, atol=0.0, equal_nan=True)
        assert C.LIB.colapm_batch_set_lockstep(b, 2) == C.LIB.colapm_batch_set_lockstep(None, 1) != 0
    finally:
        C.colapm_batch_destroy(b)


@pytest.mark.parametrize("np_,nm", [(96, 192), (160, 320), (256, 512)])
def test_every_plan_mask_gives_the_same_force(C, np_, nm):
    """Each pass on either radix plan (16 masks; at 512^3 only the all-two-stage mask keeps the
    blocked layout): the force meshes agree to FP32 rounding, and the autotuner's choice is one of
    them and is reported whole by colapm_get_config."""
    import torch
    ctx = C.colapm_create(C.default_params(np=np_, nm=nm, box=300.0, seed=3))
    try:
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, 4)
        out = {}
        for plan in range(16):
            C.colapm_set_plan(ctx, plan)
            f = torch.empty(3 * nm ** 3, dtype=torch.float32, device="cuda")
            C.colapm_get_force(ctx, f)
            out[plan] = f
        ref = out[C.PLAN_ALL].double()
        scale = torch.sqrt(torch.mean(ref ** 2)).item()
        for plan, f in out.items():
            diff = f.double() - ref
            assert torch.sqrt(torch.mean(diff ** 2)).item() < 1e-5 * scale, plan
        if nm >= 512:   # default reordering: once, before step 2 n_steps / 5
            cfg = C.colapm_get_config(ctx)
            assert cfg["sort_every"] == 10 and cfg["sort_first"] == 4 and cfg["sort_tiles"] == 2
        if nm < 512:   # (tuning is remembered per size for the rest of the process)
            C.colapm_autotune(ctx)
            cfg = C.colapm_get_config(ctx)
            assert 0 <= cfg["plan"] <= C.PLAN_ALL and cfg["block"] in (128, 256, 512)
            assert C.colapm_steps_done(ctx) == 4
    finally:
        C.colapm_destroy(ctx)


def test_plan_arguments_are_checked(C):
    ctx = C.colapm_create(C.default_params(np=16, nm=32, box=100.0))
    try:
        for bad in (-1, 16):
            with pytest.raises(C.ColapmError):
                C.colapm_set_plan(ctx, bad)
        C.colapm_set_plan(ctx, C.PLAN_Y | C.PLAN_Z)
        assert C.colapm_get_config(ctx)["plan"] == C.PLAN_Y | C.PLAN_Z
    finally:
        C.colapm_destroy(ctx)


def test_uneven_batch_mocks_match_oracle_at_full_size(C):
    """Mocks r = 0..7 of the 64-mock uneven batch (N_p = 64 + 32 (r mod 5), N_m = 2 N_p,
    L = 128 + 96 (r mod 5) Mpc/h, seed 1000 + r, 10 steps): every mock equals a single context,
    and the two the FP64 oracle runs in under a minute (r = 0, 1) match it within 0.1% per bin."""
    params = []
    for r in range(8):
        k = r % 5
        npp = 64 + 32 * k
        params.append(C.default_params(np=npp, nm=2 * npp, box=128.0 + 96.0 * k, seed=1000 + r))
    b = C.colapm_batch_create(params, nstreams=0)
    try:
        nbins = 100
        kb, pb, nb = C.colapm_batch_run(b, len(params), nbins)
    finally:
        C.colapm_batch_destroy(b)
    for i, prm in enumerate(params[:5]):          # the five distinct sizes
        ks, ps, ns = single_power(C, prm, nbins)
        assert np.array_equal(nb[i], ns)
        ok = ns > 0
        assert np.max(np.abs(pb[i][ok] / ps[ok] - 1)) < 1e-9
    pk = ocosmo.linear_pk(0.3, 0.7, 0.96, 0.8)
    for i in (0, 1):
        prm = params[i]
        r = ocola.Run(prm.box, prm.np, prm.nm, 0.3, 9.0, 0.0, 10, fft="numpy")
        r.make_ics(prm.seed, pk)
        r.run()
        kr, pr, nr = opower.power_from_positions(r.x, prm.box, prm.np, prm.nm, nbins, fft="numpy")
        assert np.array_equal(nb[i], nr)
        ok = nr > 0
        assert np.max(np.abs(pb[i][ok] / pr[ok] - 1)) < 1e-3
        assert np.max(np.abs(kb[i][ok] / kr[ok] - 1)) < 1e-6
