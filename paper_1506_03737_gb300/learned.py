"""Training and evaluation driver for the learned displacement correction.

Every step runs in the library through its C calls (colapm_* and colapm_nn_*); this module only
orders the calls and keeps device buffers (torch tensors) alive.

A pair comes from two COLA runs of the same seed and cosmology: a coarse run (few steps, a mesh
as fine as the particle grid) and a fine run (many steps on a finer mesh). The network learns
dPsi = Psi_fine - Psi_coarse from Psi_coarse; the corrected run is Psi_coarse + dPsi_net, placed
back into the coarse context with colapm_set_displacement so that colapm_power measures it.
"""
import time

import numpy as np

from . import colapm as C


def pair_params(np_, box, coarse_nm, coarse_steps, fine_nm, fine_steps, cosmo=None):
    kw = dict(cosmo or {})
    return (C.default_params(np=np_, nm=coarse_nm, box=box, n_steps=coarse_steps, **kw),
            C.default_params(np=np_, nm=fine_nm, box=box, n_steps=fine_steps, **kw))


class Pairs:
    """Coarse displacements, targets and P(k) of both runs for a list of seeds (device-resident)."""

    def __init__(self, coarse_params, fine_params, seeds, nbins=24, stream=0):
        import torch
        self.np = coarse_params.np
        self.box = coarse_params.box
        self.seeds = list(seeds)
        self.nbins = nbins
        self.kmax = np.pi * self.np / self.box            # particle Nyquist frequency
        n3 = self.np ** 3
        self.cc = C.colapm_create(coarse_params, stream)
        self.cf = C.colapm_create(fine_params, stream)
        self.cx = C.colapm_create(coarse_params, stream)   # partner context of the cross-correlations
        C.colapm_make_ics(self.cx)                          # (its particles are placed by displacement)
        self.coarse, self.target, self.pk_coarse, self.pk_fine = [], [], [], []
        self.nm = coarse_params.nm
        self.secs = {"coarse": 0.0, "fine": 0.0}
        for s in self.seeds:
            disp = {}
            for name, ctx in (("fine", self.cf), ("coarse", self.cc)):
                t0 = time.perf_counter()
                C.colapm_reseed(ctx, s)
                C.colapm_make_ics(ctx)
                C.colapm_step(ctx, -1)
                d = torch.empty((n3, 3), dtype=torch.float32, device="cuda")
                C.colapm_get_displacement(ctx, d)
                torch.cuda.synchronize()
                self.secs[name] += time.perf_counter() - t0
                disp[name] = d
            # Both spectra on the coarse context's mesh, so that only the particles differ.
            self.k, pc, self.nmodes = C.colapm_power(self.cc, nbins, 0.0, self.kmax)
            C.colapm_set_displacement(self.cc, disp["fine"])
            _, pf, _ = C.colapm_power(self.cc, nbins, 0.0, self.kmax)
            self.coarse.append(disp["coarse"])
            self.target.append(disp["fine"] - disp["coarse"])
            self.pk_coarse.append(pc)
            self.pk_fine.append(pf)

    def scales(self, idx):
        """Power-of-two input and output scales near the rms of Psi_coarse and of the targets."""
        s_in = float(np.mean([float(self.coarse[i].std()) for i in idx]))
        s_out = float(np.mean([float(self.target[i].std()) for i in idx]))
        return 2.0 ** np.round(np.log2(s_in)), 2.0 ** np.round(np.log2(s_out))

    def close(self):
        C.colapm_destroy(self.cc)
        C.colapm_destroy(self.cf)
        C.colapm_destroy(self.cx)


def train(net, pairs, idx, steps, seed=0, log_every=0):
    """Adam steps on pairs drawn uniformly from idx; returns the losses that were read back.
    The pairs' tensors must be complete before the network's stream reads them (Pairs ensures it)."""
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(steps):
        i = idx[int(rng.integers(len(idx)))]
        want = log_every and it % log_every == 0
        loss = C.colapm_nn_train_step(net, pairs.coarse[i], pairs.target[i], want_loss=bool(want))
        if want:
            losses.append((it, loss))
    C.colapm_nn_sync(net)
    return losses


def evaluate(net, pairs, idx, cross_seeds=0):
    """Errors of plain COLA and of COLA + network against the fine runs on the pairs idx.

    mse: mean squared displacement error (Mpc/h)^2; pk_err: mean over k-bins below the particle
    Nyquist frequency of |<P>/<P_fine> - 1| with <> the mean over the pairs; for the first
    cross_seeds pairs also the cross-correlation coefficient r(k) with the fine run's density.
    """
    import torch
    out = torch.empty_like(pairs.coarse[idx[0]])
    mse_plain = mse_net = 0.0
    pk_net = []
    r_plain, r_net = [], []
    for j, i in enumerate(idx):
        C.colapm_nn_forward(net, pairs.coarse[i], out, add=False)
        C.colapm_nn_sync(net)                     # torch reads `out` on its own stream
        mse_plain += float((pairs.target[i] ** 2).mean()) * 3
        mse_net += float(((pairs.target[i] - out) ** 2).mean()) * 3
        C.colapm_nn_forward(net, pairs.coarse[i], out, add=True)
        C.colapm_nn_sync(net)
        C.colapm_set_displacement(pairs.cc, out)
        _, p, _ = C.colapm_power(pairs.cc, pairs.nbins, 0.0, pairs.kmax)
        pk_net.append(p)
        if j < cross_seeds:   # the coarse context holds the corrected particles here
            C.colapm_set_displacement(pairs.cx, pairs.coarse[i] + pairs.target[i])
            r_net.append(C.colapm_cross_correlation(pairs.cc, pairs.cx, pairs.nbins, 0.0, pairs.kmax)[1])
            C.colapm_set_displacement(pairs.cc, pairs.coarse[i])
            r_plain.append(C.colapm_cross_correlation(pairs.cc, pairs.cx, pairs.nbins, 0.0, pairs.kmax)[1])
    ok = pairs.nmodes > 0
    pf = np.mean([pairs.pk_fine[i] for i in idx], axis=0)[ok]
    pc = np.mean([pairs.pk_coarse[i] for i in idx], axis=0)[ok]
    pn = np.mean(pk_net, axis=0)[ok]
    res = {"mse_plain": mse_plain / len(idx), "mse_net": mse_net / len(idx),
           "pk_err_plain": float(np.mean(np.abs(pc / pf - 1))), "pk_err_net": float(np.mean(np.abs(pn / pf - 1))),
           "pk_ratio_plain": (pc / pf).tolist(), "pk_ratio_net": (pn / pf).tolist(), "k": pairs.k[ok].tolist()}
    if cross_seeds:
        res["r_plain"] = np.mean(r_plain, axis=0).tolist()
        res["r_net"] = np.mean(r_net, axis=0).tolist()
    return res
