"""Error of each GPU result against the FP64 oracle at the benchmark sizes (a report, not a test).

    python tests/report_errors.py [--full-run]

Prints one markdown table: for the 2LPT fields, forces, positions and momenta the max and rms
absolute error relative to the rms of the oracle's value (forces: per component, the worst one);
for P(k) the largest per-bin relative error; for the density the number of cells that differ.
Sizes: the 256^3 / 512^3 and 512^3 / 1024^3 workloads wherever the oracle fits the host (ICs, one
COLA step from a shared state, P(k) on shared positions, density), the clustered force at 512^3;
--full-run adds the oracle's own 10-step run of 256^3 / 512^3 from the same seed (several minutes).
The oracle uses numpy's FFT as its transform primitive (pinned against its own FFT).
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from oracle import cola as ocola, cosmology as ocosmo, ics as oics, pm as opm, power as opower  # noqa: E402
from paper_1506_03737_gb300 import colapm as C, workloads  # noqa: E402

ROWS = []


def row(result, size, err_max, err_rms, note=""):
    ROWS.append((result, size, err_max, err_rms, note))
    print(f"  {result} {size}: max {err_max:.2e} rms {err_rms:.2e} {note}", flush=True)


def rel(a, b):
    """(max |a - b|, rms |a - b|) over rms(b)."""
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    s = np.sqrt(np.mean(b * b))
    d = np.abs(a - b)
    return float(d.max() / s), float(np.sqrt(np.mean(d * d)) / s)


def state(ctx, n):
    cell, off, mom = np.empty((n, 3), np.int32), np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)
    C.colapm_get_state(ctx, cell, off, mom)
    return cell, off, mom


def lpt(ctx, np_):
    a, b = np.empty(3 * np_ ** 3, np.float32), np.empty(3 * np_ ** 3, np.float32)
    C.colapm_get_lpt(ctx, a, b)
    return a.reshape(3, np_, np_, np_), b.reshape(3, np_, np_, np_)


def oracle_run(kw):
    return ocola.Run(kw["box"], kw["np"], kw["nm"], kw["omega_m"], kw["z_init"], kw["z_final"], kw["n_steps"],
                     fft="numpy")


def min_image(d, period):
    return d - period * np.rint(d / period)


def workload(name, full_run):
    kw = workloads.run_params(name)
    np_, nm, box, seed = kw["np"], kw["nm"], kw["box"], kw["seed"]
    n = np_ ** 3
    size = f"{np_}^3 / {nm}^3"
    pk = ocosmo.linear_pk(kw["omega_m"], kw["h"], kw["n_s"], kw["sigma8"])
    ctx = C.colapm_create(C.default_params(**kw))
    try:
        C.colapm_make_ics(ctx)
        g1, g2 = lpt(ctx, np_)
        dk = oics.gaussian_field(np_, box, seed, pk)
        p1, p2 = oics.lpt_displacements(dk, box, fft="numpy")
        del dk
        row("Psi1 (2LPT ICs)", size, *rel(g1, p1))
        row("Psi2 (2LPT ICs)", size, *rel(g2, p2))
        del p1, p2
        # one step from the GPU's state after 5 steps (the oracle's whole-mesh force needs ~170 GB of host
        # memory at 1024^3: there only the density of that state is compared)
        C.colapm_step(ctx, 5)
        if nm > 512:
            cell, off, _ = state(ctx, n)
            rho_ref = opm.cic_deposit(cell + off.astype(np.float64), nm)
            rho = np.empty(nm ** 3, np.int64)
            C.colapm_get_density(ctx, rho)
            row("density (int64)", size, float(np.count_nonzero(rho != rho_ref.ravel())), 0.0, "cells that differ")
            del rho, rho_ref, cell, off
            C.colapm_step(ctx, -1)
            k, p, cnt = C.colapm_power(ctx, 100)
            cell, off, _ = state(ctx, n)
            kr, pr, nr = opower.power_from_positions((cell + off.astype(np.float64)) * (box / nm), box, np_, nm, 100,
                                                     fft="numpy")
            ok = nr > 0
            row("P(k) (shared positions)", size, float(np.max(np.abs(p[ok] / pr[ok] - 1))), 0.0,
                f"max per-bin relative; mode counts {'equal' if np.array_equal(cnt, nr) else 'DIFFER'}")
            return
        cell, off, mom = state(ctx, n)
        r = oracle_run(kw)
        r.set_displacements(g1.astype(np.float64), g2.astype(np.float64))
        r.x = (cell + off.astype(np.float64)) * (box / nm)
        r.p = mom.astype(np.float64) * (box / nm)
        r.step_index = 5
        rho_ref = opm.cic_deposit(r.x * (nm / box), nm)
        rho = np.empty(nm ** 3, np.int64)
        C.colapm_get_density(ctx, rho)
        row("density (int64)", size, float(np.count_nonzero(rho != rho_ref.ravel())), 0.0, "cells that differ")
        del rho, rho_ref
        x0 = r.x.copy()
        r.step()
        C.colapm_step(ctx, 1)
        cell2, off2, mom2 = state(ctx, n)
        d = min_image((cell2 + off2.astype(np.float64)) * (box / nm) - r.x, box)
        move = min_image(r.x - x0, box)
        s = np.sqrt(np.mean(move ** 2))
        row("positions (1 step)", size, float(np.abs(d).max() / s), float(np.sqrt(np.mean(d ** 2)) / s),
            "relative to the rms move of the step")
        row("momenta (1 step)", size, *rel(mom2 * (box / nm), r.p))
        del r, x0, d, move
        # P(k) on the GPU's positions after the last step
        C.colapm_step(ctx, -1)
        k, p, cnt = C.colapm_power(ctx, 100)
        cell, off, _ = state(ctx, n)
        kr, pr, nr = opower.power_from_positions((cell + off.astype(np.float64)) * (box / nm), box, np_, nm, 100,
                                                 fft="numpy")
        ok = nr > 0
        row("P(k) (shared positions)", size, float(np.max(np.abs(p[ok] / pr[ok] - 1))), 0.0,
            f"max per-bin relative; mode counts {'equal' if np.array_equal(cnt, nr) else 'DIFFER'}")
        if full_run:
            gp, gm = np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)
            C.colapm_get_particles(ctx, gp, gm)
            t0 = time.time()
            r = oracle_run(kw)
            r.make_ics(seed, pk)
            r.run()
            d = min_image(gp.astype(np.float64) - r.x, box)
            s = np.sqrt(np.mean(r.displacement() ** 2))
            row("positions (10-step run)", size, float(np.abs(d).max() / s), float(np.sqrt(np.mean(d ** 2)) / s),
                f"relative to the rms displacement; oracle run {time.time() - t0:.0f} s")
            row("momenta (10-step run)", size, *rel(gm, r.p))
            kr, pr, nr = opower.power_from_positions(r.x, box, np_, nm, 100, fft="numpy")
            ok = nr > 0
            row("P(k) (10-step run)", size, float(np.max(np.abs(p[ok] / pr[ok] - 1))), 0.0,
                "max per-bin relative, independent runs")
    finally:
        C.colapm_destroy(ctx)


def force_512():
    np_, nm, box = 256, 512, 512.0
    ctx = C.colapm_create(C.default_params(np=np_, nm=nm, box=box))
    try:
        C.colapm_make_ics(ctx)
        cell, off, _ = workloads.clustered_state(np_, nm, 29)
        C.colapm_set_state(ctx, cell, off, None)
        f = np.empty(3 * nm ** 3, np.float32)
        C.colapm_get_force(ctx, f)
    finally:
        C.colapm_destroy(ctx)
    f = f.reshape(3, nm, nm, nm)
    rho = opm.cic_deposit(cell.astype(np.float64) + off, nm)
    ref = opm.force_mesh(opm.density_contrast(rho, np_, nm), box, 1, fft="numpy") * (nm / box)
    errs = [rel(f[j], ref[j]) for j in range(3)]
    row("force mesh (clustered state)", f"{nm}^3", max(e[0] for e in errs), max(e[1] for e in errs),
        "worst component")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--full-run", action="store_true")
    args = ap.parse_args()
    force_512()
    workload("cola_256p_512m_512mpc", args.full_run)
    workload("cola_512p_1024m_1024mpc", False)
    print("\n| result | particles / mesh | max error | rms error | note |\n|---|---|---|---|---|")
    for r, s, a, b, note in ROWS:
        print(f"| {r} | {s} | {a:.2e} | {b:.2e} | {note} |")


if __name__ == "__main__":
    main()
