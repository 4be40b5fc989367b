"""Self-referenced accuracy studies of the method's free parameters (§7.3).

The paper measures how the force mesh (N_m = N_p, N_p/2, N_p/4), the spacing of the steps (linear
or logarithmic in a), the stepping (modified with nLPT, or Quinn et al.), the value of nLPT and
COLA against plain PM change the power spectrum and the cross-correlation with a full N-body run.
No N-body run is available here; the reference is instead a converged COLA run of the same seed:
many steps (50) on the finest mesh of the study (N_m = 2 N_p). Every run and every spectrum goes
through the library's C calls; this module only orders them.

All spectra are measured on one mesh (N_m = 2 N_p) by moving each run's particles into a
measurement context (colapm_set_displacement), so that only the particles differ; the
cross-correlation is colapm_cross_correlation against the reference run's particles.
"""
import time

import numpy as np

from . import colapm as C


def variants(np_):
    """(name, params overrides) of the runs compared with the reference (10 steps each)."""
    return [
        ("COLA modified lin-a, N_m = N_p", dict(nm=np_)),
        ("COLA modified lin-a, N_m = N_p/2", dict(nm=np_ // 2)),
        ("COLA modified lin-a, N_m = N_p/4", dict(nm=np_ // 4)),
        ("COLA modified lin-a, N_m = 2 N_p", dict(nm=2 * np_)),
        ("COLA modified log-a, N_m = N_p", dict(nm=np_, spacing=1)),
        ("COLA Quinn lin-a, N_m = N_p", dict(nm=np_, stepping=1)),
        ("COLA Quinn log-a, N_m = N_p", dict(nm=np_, stepping=1, spacing=1)),
        ("PM lin-a, N_m = N_p", dict(nm=np_, cola=0, stepping=1)),
        ("PM log-a, N_m = N_p", dict(nm=np_, cola=0, stepping=1, spacing=1)),
        ("COLA modified nLPT = -1.5, N_m = N_p", dict(nm=np_, nlpt=-1.5)),
        ("COLA modified nLPT = -0.5, N_m = N_p", dict(nm=np_, nlpt=-0.5)),
        ("COLA modified nLPT = +0.5, N_m = N_p", dict(nm=np_, nlpt=0.5)),
    ]


def _displacement(params, seed, stream):
    """Run one realisation; return its displacement field (device tensor) and the run's wall ms."""
    import torch
    ctx = C.colapm_create(params, stream)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        C.colapm_reseed(ctx, seed)
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, -1)
        C.colapm_sync(ctx)
        ms = 1e3 * (time.perf_counter() - t0)
        d = torch.empty((params.np ** 3, 3), dtype=torch.float32, device="cuda")
        C.colapm_get_displacement(ctx, d)
        C.colapm_sync(ctx)
        return d, ms
    finally:
        C.colapm_destroy(ctx)


def run(np_=256, box=512.0, seeds=(1, 2), nbins=24, steps=10, ref_steps=50, cosmo=None, stream=0):
    """The study on N_p^3 particles in a box of side `box` (Mpc/h), z = 9 to 0.

    Returns {"k": bin centres, "variants": {name: {"pk_ratio", "r", "ms"}}, "reference": ...}: the
    mean over the seeds of P_variant / P_reference and of r(k) per bin (log bins from 2 pi / L to the
    particle Nyquist frequency pi N_p / L), and the mean wall time of one run."""
    import torch
    kw = dict(cosmo or {})
    kmax = np.pi * np_ / box
    base = dict(np=np_, box=box, n_steps=steps, **kw)
    meas_p = C.default_params(np=np_, nm=2 * np_, box=box, **kw)
    ma = C.colapm_create(meas_p, stream)
    mb = C.colapm_create(meas_p, stream)
    C.colapm_make_ics(ma)
    C.colapm_make_ics(mb)
    out = {"variants": {}, "reference": {"steps": ref_steps, "nm": 2 * np_, "stepping": "modified, nLPT = -2.5",
                                         "spacing": "linear in a"}}
    try:
        refs, ref_pk, ref_ms = [], [], []
        for s in seeds:
            d, ms = _displacement(C.default_params(nm=2 * np_, **dict(base, n_steps=ref_steps)), s, stream)
            C.colapm_set_displacement(ma, d)
            k, p, cnt = C.colapm_power(ma, nbins, 0.0, kmax)
            refs.append(d)
            ref_pk.append(p)
            ref_ms.append(ms)
        out["k"] = k.tolist()
        out["nmodes"] = cnt.tolist()
        out["reference"]["ms"] = float(np.mean(ref_ms))
        for name, over in variants(np_):
            ratios, rs, mss = [], [], []
            for s, dref, pref in zip(seeds, refs, ref_pk):
                d, ms = _displacement(C.default_params(**dict(base, **over)), s, stream)
                C.colapm_set_displacement(ma, d)
                _, p, _ = C.colapm_power(ma, nbins, 0.0, kmax)
                C.colapm_set_displacement(mb, dref)
                _, r, _ = C.colapm_cross_correlation(ma, mb, nbins, 0.0, kmax)
                ratios.append(p / pref)
                rs.append(r)
                mss.append(ms)
                del d
            out["variants"][name] = {"pk_ratio": np.mean(ratios, axis=0).tolist(), "r": np.mean(rs, axis=0).tolist(),
                                     "ms": float(np.mean(mss))}
        torch.cuda.synchronize()
    finally:
        C.colapm_destroy(ma)
        C.colapm_destroy(mb)
    return out


def summary(res, k_cut=(0.1, 0.3)):
    """Per variant: the largest |P/P_ref - 1| over bins with k below each cut, and r in the highest bin."""
    k = np.asarray(res["k"])
    rows = {}
    for name, v in res["variants"].items():
        pr = np.asarray(v["pk_ratio"])
        r = np.asarray(v["r"])
        row = {f"max_pk_err_k<{c}": float(np.nanmax(np.abs(pr[k < c] - 1))) for c in k_cut}
        row["r_highest_bin"] = float(r[np.isfinite(r)][-1])
        row["ms"] = v["ms"]
        rows[name] = row
    return rows
