"""Oracle (test infrastructure only): periodic-box power spectrum and cross-correlation (§7.1).

For a periodic cube the FKP estimator the paper uses reduces to the binned mode
power. With delta from the fixed-point CIC deposit of ``pm`` and delta_k its
unnormalised DFT:

    P(k_mode) = L^3 |delta_k|^2 / (N_m^6 W(k)^2),  W = prod_i sinc^2(pi n_i / N_m)

binned in ``nbins`` logarithmic bins with edges e_b = kmin (kmax/kmin)^(b/nbins);
a mode belongs to bin b when e_b <= |k| < e_{b+1}. Modes are counted over the full
complex grid; k = 0 and modes with any index at N_m/2 are excluded. Per bin: the
mean |k|, the mean P and the mode count. Shot noise is not subtracted (§7.1).

Cross-correlation (§7.1): r(k) = <Re delta_a delta_b^*> / sqrt(<|delta_a|^2> <|delta_b|^2>)
per bin. The printed formula lacks the square root; without it r is not
dimensionless, so the square root is read as intended.

Redshift space (§7.1): each particle is moved along the line of sight by
s_los = v_los / (H(a) a). With the momentum p = a^3 E dx/da of the method (H0 = 1, lengths
in Mpc/h) the peculiar velocity is v = a dx/dt = p / a and H = E(a). The line of sight is
radial from an observer at the centre of the box (the paper's choice) or, as an option, one
of the axes (plane-parallel). Redshift-space positions wrap periodically.
"""
import math

import numpy as np

from .fft import fftn
from .ics import wavevectors
from . import cosmology, pm


def bin_edges(nbins, kmin, kmax):
    b = np.arange(nbins + 1, dtype=np.float64)
    return kmin * (kmax / kmin) ** (b / nbins)


def mode_bins(nm, box, nbins, kmin, kmax):
    """(|k|, bin index or -1) for every mode of the full [z][y][x] grid."""
    kx, ky, kz, nyq = wavevectors(nm, box)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    edges = bin_edges(nbins, kmin, kmax)
    b = np.searchsorted(edges, kmag, side="right") - 1
    b[(b < 0) | (b >= nbins) | nyq] = -1
    return kmag, b


def binned_power(delta_k, box, nbins, kmin, kmax, window=True):
    nm = delta_k.shape[0]
    kmag, b = mode_bins(nm, box, nbins, kmin, kmax)
    p = box ** 3 * np.abs(delta_k) ** 2 / float(nm) ** 6
    if window:
        p = p / pm.cic_window(nm) ** 2
    sel = b >= 0
    cnt = np.bincount(b[sel], minlength=nbins).astype(np.int64)
    ksum = np.bincount(b[sel], weights=kmag[sel], minlength=nbins)
    psum = np.bincount(b[sel], weights=p[sel], minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, psum / cnt, cnt


def power_from_positions(x, box, np_, nm, nbins=100, kmin=None, kmax=None, fft=None):
    """Deposit, transform and bin (defaults: kmin = 2 pi / L, kmax = pi N_m / L); fft="numpy" takes
    numpy's FFT as the transform primitive."""
    kmin = 2.0 * math.pi / box if kmin is None else kmin
    kmax = math.pi * nm / box if kmax is None else kmax
    u = np.mod(np.asarray(x, dtype=np.float64) * (nm / box), nm)
    rho = pm.cic_deposit(u, nm)
    delta = pm.density_contrast(rho, np_, nm)
    dk = np.fft.fftn(delta) if fft == "numpy" else fftn(delta)
    return binned_power(dk, box, nbins, kmin, kmax)


def cross_correlation(dka, dkb, box, nbins, kmin, kmax):
    nm = dka.shape[0]
    _, b = mode_bins(nm, box, nbins, kmin, kmax)
    sel = b >= 0
    cab = np.bincount(b[sel], weights=(dka * np.conj(dkb)).real[sel], minlength=nbins)
    caa = np.bincount(b[sel], weights=(np.abs(dka) ** 2)[sel], minlength=nbins)
    cbb = np.bincount(b[sel], weights=(np.abs(dkb) ** 2)[sel], minlength=nbins)
    with np.errstate(invalid="ignore", divide="ignore"):
        return cab / np.sqrt(caa * cbb)


def redshift_space(x, p, a, om, box, los=-1):
    """Redshift-space positions (P,3) of particles at x (Mpc/h) with momenta p (Mpc/h) at scale
    factor a (§7.1): los = -1 radial from the box centre, 0/1/2 along that axis."""
    x = np.asarray(x, dtype=np.float64)
    v = np.asarray(p, dtype=np.float64) / a
    scale = 1.0 / (cosmology.hubble_e(a, om) * a)
    if los < 0:
        r = x - 0.5 * box
        d = np.sqrt(np.sum(r * r, axis=1))
        rhat = np.zeros_like(r)
        ok = d > 0
        rhat[ok] = r[ok] / d[ok, None]
        s = x + (np.sum(v * rhat, axis=1) * scale)[:, None] * rhat
    else:
        s = x.copy()
        s[:, los] += v[:, los] * scale
    return np.mod(s, box)
