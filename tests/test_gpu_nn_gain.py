"""What the trained network gains over plain COLA, on held-out seeds.

A scaled-down copy of the 128^3 workload with the same particle spacing (2 Mpc/h): 64^3 particles
in 128 Mpc/h; coarse = 64^3 mesh, 5 steps; fine = 192^3 mesh, 50 steps; 32 training and 8 test
seeds. The network, trained on the GPU by the library's own kernels, must bring the coarse run
closer to the fine one in displacement, P(k) below the particle Nyquist frequency, and the
cross-correlation of the densities at high k; without it nothing changes (plain COLA).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_network_beats_plain_cola_on_test_seeds():
    import torch  # noqa: F401
    from paper_1506_03737_gb300 import colapm as C, learned
    pc, pf = learned.pair_params(64, 128.0, 64, 5, 192, 50)
    pairs = learned.Pairs(pc, pf, range(2000, 2040), nbins=16)
    try:
        train_idx, test_idx = list(range(32)), list(range(32, 40))
        s_in, s_out = pairs.scales(train_idx)
        net = C.colapm_nn_create(64, C.nn_default_config(s_in=s_in, s_out=s_out, lr=1e-3, seed=1))
        try:
            before = learned.evaluate(net, pairs, test_idx)
            learned.train(net, pairs, train_idx, 1500, seed=0)
            res = learned.evaluate(net, pairs, test_idx, cross_seeds=2)
        finally:
            C.colapm_nn_destroy(net)
        assert before["mse_net"] > res["mse_net"]                          # training helped
        assert res["mse_net"] < 0.9 * res["mse_plain"]
        assert res["pk_err_net"] < 0.5 * res["pk_err_plain"]
        hi = slice(8, 16)
        r_plain, r_net = np.array(res["r_plain"])[hi], np.array(res["r_net"])[hi]
        assert np.nanmean(1 - r_net) < np.nanmean(1 - r_plain)
    finally:
        pairs.close()
