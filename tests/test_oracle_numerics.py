"""Pins of the oracle's numerical building blocks against definitions and closed forms.

Each test checks the oracle against something other than itself: the DFT definition,
closed-form growth factors and integrals, published known-answer vectors.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology, fft, philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- FFT: the oracle's own transform vs the O(N^2) definition -------------------------

def test_fft_matches_bruteforce_dft_8cubed():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((8, 8, 8)) + 1j * rng.standard_normal((8, 8, 8))
    ref = a
    for ax in range(3):
        ref = fft.dft_bruteforce(ref, ax)
    assert np.abs(fft.fftn(a) - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("n", [2, 3, 5, 6, 10, 12, 15, 24, 30, 40])
def test_fft_mixed_radix_lengths(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((3, n)) + 1j * rng.standard_normal((3, n))
    for sign in (-1, 1):
        ref = fft.dft_bruteforce(a, -1, sign)
        assert np.abs(fft.fft_axis(a, -1, sign) - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_fft_roundtrip_and_library_special_case():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((12, 10, 8))
    assert np.abs(fft.ifftn(fft.fftn(a)) - a).max() < 1e-13
    # A library routine computes the same transform (numpy.fft is used only here, as a check).
    assert np.abs(fft.fftn(a) - np.fft.fftn(a)).max() < 1e-11


def test_dft_definition_single_mode():
    # A pure exponential exp(2 pi i m n / N) transforms to N at bin m and zero elsewhere.
    n, m = 16, 3
    x = np.exp(2j * np.pi * m * np.arange(n) / n)
    out = fft.fft_axis(x)
    expect = np.zeros(n, complex)
    expect[m] = n
    assert np.abs(out - expect).max() < 1e-12


# --- Philox4x32-10 known-answer vectors ------------------------------------------------

def test_philox_known_answers():
    rows = [line.split() for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_uniform_open_interval():
    u = philox.uniform_open(np.array([0, 0xFFFFFFFF, 1 << 31], dtype=np.uint64))
    assert u[0] == 2.0 ** -24 and u[1] == 1.0 - 2.0 ** -24 and u[2] == 0.5 + 2.0 ** -24
    assert np.all(u.astype(np.float32).astype(np.float64) == u)   # exact in FP32


# --- Growth factors: Einstein-de Sitter closed forms, Heath integral, Bouchet --------

def test_growth_eds_closed_form():
    a = np.array([0.05, 0.1, 0.37, 0.8, 1.0])
    d1, d2, p1, p2 = cosmology.growth(a, 1.0)
    assert np.abs(d1 / a - 1).max() < 1e-10
    assert np.abs(d2 / (-3.0 / 7.0 * a * a) - 1).max() < 1e-10
    # P = a^3 E dD/da with E = a^-3/2: P1 = a^(3/2), P2 = -6/7 a^(5/2).
    assert np.abs(p1 / a ** 1.5 - 1).max() < 1e-10
    assert np.abs(p2 / (-6.0 / 7.0 * a ** 2.5) - 1).max() < 1e-10


@pytest.mark.parametrize("om", [0.25, 0.3, 0.5])
def test_growth_lcdm_matches_heath_integral(om):
    # Linear growing mode of flat LCDM: D1 proportional to E(a) * int_0^a da' / (a' E(a'))^3.
    def heath(a):
        val, _ = integrate.quad(lambda x: 1.0 / (x * cosmology.hubble_e(x, om)) ** 3, 0.0, a,
                                epsabs=0, epsrel=1e-13)
        return cosmology.hubble_e(a, om) * val
    a = np.array([0.1, 0.3, 0.6, 0.9])
    d1, _, _, _ = cosmology.growth(a, om)
    ref = np.array([heath(x) for x in a]) / heath(1.0)
    assert np.abs(d1 / ref - 1).max() < 1e-8


def test_d2_close_to_bouchet_approximation():
    # Eq. eq:2LPTgrowth: D2 ~ -3/7 D1^2 Om(a)^(-1/143) -- an approximation good to ~1%.
    om = 0.3
    a = np.array([0.1, 0.5, 1.0])
    d1, d2, _, _ = cosmology.growth(a, om)
    om_a = om * a ** -3 / cosmology.hubble_e(a, om) ** 2
    approx = -3.0 / 7.0 * d1 ** 2 * om_a ** (-1.0 / 143.0)
    assert np.abs(d2 / approx - 1).max() < 1e-2


# --- Kick / drift coefficients: EdS closed forms -------------------------------------

def test_quinn_coefficients_eds():
    t = cosmology.timestep_table(1.0, 9.0, 0.0, 10, stepping="quinn")
    a, ah = t["a"], t["a_half"]
    alo = np.concatenate([[a[0]], ah[:-1]])
    # int da/(a^2 E) = 2 (sqrt(hi) - sqrt(lo)); int da/(a^3 E) = 2 (lo^-1/2 - hi^-1/2) in EdS.
    kick = 1.5 * 2.0 * (np.sqrt(ah) - np.sqrt(alo))
    drift = 2.0 * (a[:-1] ** -0.5 - a[1:] ** -0.5)
    assert np.abs(t["kick"] / kick - 1).max() < 1e-11
    assert np.abs(t["drift"] / drift - 1).max() < 1e-11
    # the closing half kick of finalize covers [a_{N-1/2}, a_N]
    assert abs(t["kick_final"] / (1.5 * 2.0 * (math.sqrt(a[-1]) - math.sqrt(ah[-1]))) - 1) < 1e-11


def test_modified_coefficients_eds():
    n = -2.5
    t = cosmology.timestep_table(1.0, 9.0, 0.0, 10, stepping="modified", nlpt=n)
    a, ah = t["a"], t["a_half"]
    alo = np.concatenate([[a[0]], ah[:-1]])
    kick = 1.5 * (ah ** n - alo ** n) / (n * a[:-1] ** (n - 1)) / (a[:-1] ** 2 * a[:-1] ** -1.5)
    # int a^(n-3) / E da = int a^(n - 3/2) da in EdS.
    drift = ah ** -n * (a[1:] ** (n - 0.5) - a[:-1] ** (n - 0.5)) / (n - 0.5)
    assert np.abs(t["kick"] / kick - 1).max() < 1e-11
    assert np.abs(t["drift"] / drift - 1).max() < 1e-11


def test_log_spacing_is_geometric_in_a():
    # §7.3: steps logarithmic in a. From z = 9 to 0 in 10 steps a_i = 10^((i - 10) / 10).
    a = cosmology.scale_factors(9.0, 0.0, 10, "log")
    assert np.abs(a / 10.0 ** ((np.arange(11) - 10) / 10.0) - 1).max() < 1e-14
    lin = cosmology.scale_factors(9.0, 0.0, 10, "lin")
    assert np.abs(lin - (0.1 + 0.09 * np.arange(11))).max() < 1e-15
    # the table follows the spacing it is given: EdS Quinn drift over each geometric step
    t = cosmology.timestep_table(1.0, 9.0, 0.0, 10, spacing="log", stepping="quinn")
    drift = 2.0 * (a[:-1] ** -0.5 - a[1:] ** -0.5)
    assert np.abs(t["drift"] / drift - 1).max() < 1e-11


def test_modified_and_quinn_kick_agree_for_small_steps():
    tq = cosmology.timestep_table(0.3, 9.0, 0.0, 2000, stepping="quinn")
    tm = cosmology.timestep_table(0.3, 9.0, 0.0, 2000, stepping="modified")
    assert np.abs(tm["kick"][1:] / tq["kick"][1:] - 1).max() < 1e-4
    assert np.abs(tm["drift"] / tq["drift"] - 1).max() < 1e-4


# --- Linear power spectrum ---------------------------------------------------------------

def test_sigma_integral_closed_form_power_law():
    # For P(k) = k^-2 the correlation function is 1/(4 pi r), so sigma^2(R) is the mean of 1/(4 pi r12)
    # over pairs in a uniform ball: (1/4pi) (6/5) / R = 3 / (10 pi R) (uniform-sphere self energy).
    for r in (4.0, 8.0, 16.0):
        s2 = cosmology.sigma_r2(lambda k: k ** -2.0, r, lnk_min=math.log(1e-7), lnk_max=math.log(1e4),
                                n=1 << 18)
        assert abs(s2 / (3.0 / (10.0 * math.pi * r)) - 1) < 1e-6


def test_bbks_limits_and_normalisation():
    om, h = 0.3, 0.7
    # Small q: ln(1+x)/x ~ 1 - x/2 and poly^-1/4 ~ 1 - 3.89 q / 4, so T ~ 1 - (2.34/2 + 3.89/4) q.
    q = 1e-6
    assert abs(cosmology.t_bbks(q * om * h, om, h) - (1.0 - (2.34 / 2 + 3.89 / 4) * q)) < 1e-10
    # Large q: T -> ln(2.34 q) / (2.34 q) * (6.71 q)^-1.
    q = 1e4
    k = q * om * h
    asym = math.log(2.34 * q) / (2.34 * q) / (6.71 * q)
    assert abs(cosmology.t_bbks(k, om, h) / asym - 1) < 1e-3
    pk = cosmology.linear_pk(om, h, 0.96, 0.8)
    assert abs(math.sqrt(cosmology.sigma_r2(pk, 8.0)) - 0.8) < 1e-12
