"""Oracle (test infrastructure only): FP64 background cosmology.

Units: H0 = 1, lengths in Mpc/h, k in h/Mpc. Flat LCDM, Omega_L = 1 - Omega_m.

* Growth factors. D1 solves the linear growth equation and D2 the second-order
  one whose source is (D2 - D1^2); these are the exact 2LPT growth factors that
  the Bouchet approximation of §2.1 (Eq. eq:2LPTgrowth) and the Matsubara
  expression quoted at the end of §2.3 approximate. In terms of a:
      d/da (a^3 E D1') = 1.5 Om D1 / (a^2 E)
      d/da (a^3 E D2') = 1.5 Om (D2 - D1^2) / (a^2 E)
  started on the growing mode at a = 1e-5 (D1 = a, D2 = -3/7 a^2) and
  normalised to D1(1) = 1.
* Kick-Drift-Kick coefficients (§2.3). The momentum variable is p = a^3 E dx/da
  (= a^2 dx/dt), the one for which the drift integral of §2.3 holds. Its
  equation of motion is dp/da = 1.5 Om F / (a^2 E) with F = -grad(psi),
  lap(psi) = delta (the comoving Poisson equation of §2.4 step 2 with its 1/a
  factor written out), so:
      Quinn kick   K_i = int_{a_{i-1/2}}^{a_{i+1/2}} da / (a^2 E)
      Quinn drift  S_i = int_{a_i}^{a_{i+1}} da / (a^3 E)
      modified kick  K_i = (a_{i+1/2}^n - a_{i-1/2}^n) / (n a_i^(n-1)) / (a_i^2 E_i)
      modified drift S_i = a_{i+1/2}^(-n) int_{a_i}^{a_{i+1}} a^(n-3) / E da
  (Eq. eq:modifiedt, n = nLPT). The modified kick is the integral of the
  acceleration per unit a, 1.5 Om F_i /(a_i^2 E_i), under the assumption that it
  scales as a^(n-1) across the step; its small-step limit equals the Quinn one.
  The kick coefficients returned below include the factor 1.5 Om.
* BBKS transfer function (Bardeen et al. 1986) with Gamma = Om h, P(k) = A k^ns T^2,
  A fixed by sigma_8 (top-hat of radius 8 Mpc/h).
"""
import math

import numpy as np
from scipy import integrate

A_START = 1e-5
RK4_STEPS = 4000


def hubble_e(a, om):
    """E(a) = H(a)/H0 for flat LCDM."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(om * a ** -3 + (1.0 - om))


def _growth_raw(a_targets, om, nsteps=RK4_STEPS):
    """RK4 in ln a of y = (D1, P1, D2, P2), P = a^3 E dD/da, from A_START to each target.

    d D / d ln a = P / (a^2 E);   d P1 / d ln a = 1.5 Om D1 / (a E);
    d P2 / d ln a = 1.5 Om (D2 - D1^2) / (a E).
    """
    at = np.atleast_1d(np.asarray(a_targets, dtype=np.float64))
    l0 = math.log(A_START)
    h = (np.log(at) - l0) / nsteps

    def rhs(lna, y):
        a = np.exp(lna)
        e = hubble_e(a, om)
        d1, p1, d2, p2 = y
        return np.array([p1 / (a * a * e), 1.5 * om * d1 / (a * e),
                         p2 / (a * a * e), 1.5 * om * (d2 - d1 * d1) / (a * e)])

    a0 = A_START
    e0 = hubble_e(a0, om)
    y = np.empty((4, at.size))
    y[0] = a0
    y[1] = a0 ** 3 * e0 * 1.0
    y[2] = -3.0 / 7.0 * a0 * a0
    y[3] = a0 ** 3 * e0 * (-6.0 / 7.0 * a0)
    lna = np.full(at.size, l0)
    for _ in range(nsteps):
        k1 = rhs(lna, y)
        k2 = rhs(lna + 0.5 * h, y + 0.5 * h * k1)
        k3 = rhs(lna + 0.5 * h, y + 0.5 * h * k2)
        k4 = rhs(lna + h, y + h * k3)
        y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        lna = lna + h
    return y


def growth(a, om):
    """Return (D1, D2, P1, P2) at scale factors ``a``; D1(1) = 1, D2 scaled by the same factor squared.

    P1 = a^3 E dD1/da and P2 = a^3 E dD2/da are the LPT momenta per unit displacement
    (the reference-frame velocity that §2.3 removes at the start and adds back at the end).
    """
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    y = _growth_raw(a, om)
    norm = _growth_raw(np.array([1.0]), om)[0, 0]
    return y[0] / norm, y[2] / norm ** 2, y[1] / norm, y[3] / norm ** 2


def growth_matter_era(om):
    """D1(a = 1) normalised to D1 = a deep in matter domination (the growth of a density mode since the
    matter era: the factor by which Lambda suppresses it, g(Om) in the literature)."""
    return float(_growth_raw(np.array([1.0]), om)[0, 0])


def _quad(f, lo, hi):
    if hi == lo:
        return 0.0
    val, _ = integrate.quad(f, lo, hi, epsabs=0.0, epsrel=1e-13, limit=200)
    return val


def scale_factors(z_init, z_final, n_steps, spacing="lin"):
    """a_0 .. a_N, linearly (default) or logarithmically spaced in a (§7.3)."""
    a0 = 1.0 / (1.0 + z_init)
    an = 1.0 / (1.0 + z_final)
    i = np.arange(n_steps + 1, dtype=np.float64)
    if spacing == "lin":
        return a0 + (an - a0) * i / n_steps
    if spacing == "log":
        return a0 * (an / a0) ** (i / n_steps)
    raise ValueError(spacing)


def kick_coeff(a_lo, a_hi, a_f, om, stepping="modified", nlpt=-2.5):
    """1.5 Om times the kick integral over [a_lo, a_hi] for a force evaluated at a_f (§2.3)."""
    if stepping == "quinn":
        k = _quad(lambda x: 1.0 / (x * x * hubble_e(x, om)), a_lo, a_hi)
    elif stepping == "modified":
        n = nlpt
        k = (a_hi ** n - a_lo ** n) / (n * a_f ** (n - 1.0)) / (a_f * a_f * hubble_e(a_f, om))
    else:
        raise ValueError(stepping)
    return 1.5 * om * k


def drift_coeff(a_i, a_next, a_mid, om, stepping="modified", nlpt=-2.5):
    """Drift integral from a_i to a_next with the momentum taken at a_mid (§2.3)."""
    if stepping == "quinn":
        return _quad(lambda x: 1.0 / (x ** 3 * hubble_e(x, om)), a_i, a_next)
    if stepping == "modified":
        n = nlpt
        return a_mid ** (-n) * _quad(lambda x: x ** (n - 3.0) / hubble_e(x, om), a_i, a_next)
    raise ValueError(stepping)


def timestep_table(om, z_init, z_final, n_steps, spacing="lin", stepping="modified", nlpt=-2.5):
    """Per-step FP64 coefficients of the COLA / PM Kick-Drift-Kick loop (§2.3).

    Step i (0 <= i < N): force at a_i, kick p over [a_{i-1/2}, a_{i+1/2}] (a_{-1/2} = a_0),
    drift x over [a_i, a_{i+1}] with p_{i+1/2}. ``kick_final`` closes the last half step
    (force at a_N, kick over [a_{N-1/2}, a_N]).
    """
    a = scale_factors(z_init, z_final, n_steps, spacing)
    ah = 0.5 * (a[:-1] + a[1:])
    alo = np.concatenate([[a[0]], ah[:-1]])
    d1, d2, p1, p2 = growth(a, om)
    kick = np.array([kick_coeff(alo[i], ah[i], a[i], om, stepping, nlpt) for i in range(n_steps)])
    drift = np.array([drift_coeff(a[i], a[i + 1], ah[i], om, stepping, nlpt) for i in range(n_steps)])
    kick_final = kick_coeff(ah[-1], a[-1], a[-1], om, stepping, nlpt)
    return {
        "a": a, "a_half": ah, "D1": d1, "D2": d2, "P1": p1, "P2": p2,
        "kick": kick, "drift": drift, "kick_final": kick_final,
        "dD1": d1[1:] - d1[:-1], "dD2": d2[1:] - d2[:-1],
    }


# --- linear power spectrum -------------------------------------------------------------

def t_bbks(k, om, h):
    """BBKS (1986) CDM transfer function, q = k / (Om h) with k in h/Mpc."""
    k = np.asarray(k, dtype=np.float64)
    q = k / (om * h)
    x = 2.34 * q
    with np.errstate(divide="ignore", invalid="ignore"):
        lead = np.where(x > 0, np.log1p(x) / np.where(x > 0, x, 1.0), 1.0)
    poly = 1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
    return lead * poly ** -0.25


def tophat_window(x):
    """Fourier transform of the unit-volume spherical top-hat, 3 (sin x - x cos x) / x^3."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 1e-3
    xs = np.where(small, 1.0, x)
    w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    return np.where(small, 1.0 - x * x / 10.0, w)


def sigma_r2(pk, r, lnk_min=math.log(1e-5), lnk_max=math.log(1e2), n=1 << 16):
    """sigma^2(R) = (1 / 2 pi^2) int k^3 P(k) W^2(kR) dln k, composite Simpson in ln k."""
    lnk = np.linspace(lnk_min, lnk_max, n + 1)
    k = np.exp(lnk)
    f = k ** 3 * pk(k) * tophat_window(k * r) ** 2 / (2.0 * math.pi ** 2)
    hstep = (lnk_max - lnk_min) / n
    return hstep / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())


def linear_pk(om, h, ns, sigma8):
    """Return P(k) [(Mpc/h)^3], BBKS shape, normalised so that sigma(8 Mpc/h) = sigma8 at z = 0."""
    def shape(k):
        return k ** ns * t_bbks(k, om, h) ** 2
    amp = sigma8 ** 2 / sigma_r2(shape, 8.0)

    def pk(k):
        return amp * shape(np.asarray(k, dtype=np.float64))
    return pk
