"""Pins of the oracle's method steps: closed forms, invariants and brute force on tiny inputs.

Each test would fail on a plausible slip in the oracle (a dropped term, a wrong sign or
index, a transposed operand, a missing normalisation).
"""
import itertools
import math

import numpy as np
import pytest

from scipy import integrate

from oracle import cola, cosmology, fft, ics, pm, power

BOX = 256.0


def plane_wave_field(n, amps):
    """delta_k for delta(q) = sum A cos(2 pi m.q / N) with integer index vectors m."""
    dk = np.zeros((n, n, n), complex)
    for (mx, my, mz), a in amps:
        dk[mz % n, my % n, mx % n] += a * n ** 3 / 2
        dk[-mz % n, -my % n, -mx % n] += a * n ** 3 / 2
    return dk


# --- Gaussian field (§5) -----------------------------------------------------------------

def test_gaussian_field_hermitian_and_masked():
    n = 16
    pk = cosmology.linear_pk(0.3, 0.7, 0.96, 0.8)
    dk = ics.gaussian_field(n, BOX, 7, pk)
    real = fft.ifftn(dk)
    assert np.abs(real.imag).max() < 1e-14 * np.abs(real.real).max()
    assert dk[0, 0, 0] == 0
    h = n // 2
    assert np.all(dk[h] == 0) and np.all(dk[:, h] == 0) and np.all(dk[:, :, h] == 0)


def test_gaussian_field_power_statistics():
    # <|delta_k|^2> = N^6 P(k) / L^3: the mean ratio over ~N^3/2 independent modes is 1 +- a few sqrt(1/modes).
    n = 32
    pk = cosmology.linear_pk(0.3, 0.7, 0.96, 0.8)
    dk = ics.gaussian_field(n, BOX, 3, pk)
    kx, ky, kz, nyq = ics.wavevectors(n, BOX)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    sel = (k > 0) & ~nyq
    ratio = np.abs(dk[sel]) ** 2 / (n ** 6 * pk(k[sel]) / BOX ** 3)
    nind = sel.sum() / 2
    assert abs(ratio.mean() - 1) < 5 / math.sqrt(nind)
    # |g|^2 = -ln(u1) is exponential with unit mean: its variance is 1 as well.
    assert abs(ratio.var() - 1) < 10 / math.sqrt(nind)


def test_gaussian_field_seed_determinism():
    pk = cosmology.linear_pk(0.3, 0.7, 0.96, 0.8)
    a = ics.gaussian_field(8, BOX, 11, pk)
    b = ics.gaussian_field(8, BOX, 11, pk)
    c = ics.gaussian_field(8, BOX, 12, pk)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


# --- 2LPT (§2.1) ------------------------------------------------------------------------

def test_zeldovich_plane_wave_exact_and_no_2lpt_source():
    n, amp = 16, 0.3
    dk = plane_wave_field(n, [((1, 0, 0), amp)])
    psi1, psi2 = ics.lpt_displacements(dk, BOX)
    k1 = 2 * math.pi / BOX
    qx = np.arange(n) * BOX / n
    expect = -(amp / k1) * np.sin(k1 * qx)                    # div Psi1 = -delta (Eq. za)
    assert np.abs(psi1[0] - expect[None, None, :]).max() < 1e-12 * abs(amp / k1)
    assert np.abs(psi1[1]).max() < 1e-14 and np.abs(psi1[2]).max() < 1e-14
    assert np.abs(psi2).max() < 1e-12                           # one plane wave: S = 0


def test_2lpt_two_mode_source_analytic():
    # delta = A cos(k1.q) + B cos(k2.q), k1 = (c,0,0), k2 = (a,b,0):
    # S = phi_xx phi_yy - phi_xy^2 = A B b^2/|k2|^2 cos(k1.q) cos(k2.q); Psi2 = grad phi2, lap phi2 = S.
    n, A, B = 8, 0.2, 0.15
    dk = plane_wave_field(n, [((1, 0, 0), A), ((1, 2, 0), B)])
    _, psi2 = ics.lpt_displacements(dk, BOX)
    kf = 2 * math.pi / BOX
    k1 = np.array([1.0, 0, 0]) * kf
    k2 = np.array([1.0, 2.0, 0]) * kf
    coef = A * B * k2[1] ** 2 / (k2 @ k2) / 2
    g = np.arange(n) * BOX / n
    qz, qy, qx = np.meshgrid(g, g, g, indexing="ij")
    expect = np.zeros((3, n, n, n))
    for kk in (k1 + k2, k1 - k2):             # cos a cos b = (cos(a+b) + cos(a-b)) / 2
        phase = kk[0] * qx + kk[1] * qy + kk[2] * qz
        for j in range(3):                    # phi2 = -coef cos/|K|^2 -> grad = coef K sin / |K|^2
            expect[j] += coef * kk[j] * np.sin(phase) / (kk @ kk)
    assert np.abs(psi2 - expect).max() < 1e-12 * np.abs(expect).max()


# --- Fixed-point CIC (§2.4 step 1) ---------------------------------------------------------

def bruteforce_deposit(u, nm):
    rho = np.zeros((nm, nm, nm), dtype=np.int64)
    for p in u:
        cell, frac = [], []
        for d in range(3):
            c = math.floor(p[d])
            fq = int(np.rint((p[d] - c) * 32768))
            if fq == 32768:
                c, fq = c + 1, 0
            cell.append(c % nm)
            frac.append(fq)
        for dz, dy, dx in itertools.product((0, 1), repeat=3):
            w = 1
            for d, o in zip(range(3), (dx, dy, dz)):
                w *= frac[d] if o else 32768 - frac[d]
            rho[(cell[2] + dz) % nm, (cell[1] + dy) % nm, (cell[0] + dx) % nm] += w
    return rho


def test_cic_deposit_bruteforce_and_mass():
    nm = 8
    rng = np.random.default_rng(4)
    u = rng.uniform(0, nm, size=(50, 3))
    u[0] = [0.0, 7.9999999, 3.5]            # carry (rounds up to the next cell, wraps)
    u[1] = [2.0, 2.0, 2.0]                  # on a node
    u[2] = [1.0 + 0.5 / 32768, 4.25, 6.0]   # exact half-step tie -> round half to even
    rho = pm.cic_deposit(u, nm)
    assert np.array_equal(rho, bruteforce_deposit(u, nm))
    assert rho.sum() == len(u) << 45
    single = pm.cic_deposit(u[1:2], nm)
    assert single[2, 2, 2] == 1 << 45 and np.count_nonzero(single) == 1


def test_cic_quantise_tie_and_carry():
    c, fq = pm.quantise(np.array([[1.0 + 0.5 / 32768, 1.0 + 1.5 / 32768, 7.99999999]]), 8)
    assert list(fq[0]) == [0, 2, 0] and list(c[0]) == [1, 1, 0]


# --- PM force (§2.4 steps 2-4) ---------------------------------------------------------------

def test_zero_self_force_single_particle():
    nm = 16
    rng = np.random.default_rng(5)
    for _ in range(4):
        x = rng.uniform(0, BOX, size=(1, 3))
        f, _ = pm.pm_accel(x, BOX, nm, nm)
        assert np.abs(f).max() < 1e-12 * BOX / nm


def test_pair_antisymmetry_and_momentum_conservation():
    nm = 16
    rng = np.random.default_rng(6)
    x = rng.uniform(0, BOX, size=(2, 3))
    f, _ = pm.pm_accel(x, BOX, nm, nm)
    assert np.abs(f[0] + f[1]).max() < 1e-12 * np.abs(f).max()
    x = rng.uniform(0, BOX, size=(40, 3))
    f, _ = pm.pm_accel(x, BOX, nm, nm)
    assert np.abs(f.sum(axis=0)).max() < 1e-11 * np.abs(f).max()


@pytest.mark.parametrize("sep", [5.0, 7.0])
def test_newtonian_limit_pair(sep):
    # Far from the mesh scale the pair force approaches -M r_hat / (4 pi r^2), M = (L/N_p)^3 per particle.
    nm = 64
    box = float(nm)                       # cell = 1
    d = np.array([1.0, 0.7, 0.4])
    d /= np.linalg.norm(d)
    x = np.array([[20.3, 21.1, 22.7], [0, 0, 0]])
    x[1] = x[0] + sep * d
    f, _ = pm.pm_accel(x, box, nm, nm)
    expect = sep ** -2 / (4 * math.pi) * d            # particle 0 is pulled toward particle 1
    assert np.linalg.norm(f[0] - expect) < 0.03 * np.linalg.norm(expect)


def test_force_and_lpt_spectra_vanish_on_the_nyquist_planes():
    # Every spectral operator is zero on modes with any index at N/2 (the stencils stay odd and the
    # fields real): the transforms of the force meshes and LPT displacements have no coefficient there.
    nm = 16
    rng = np.random.default_rng(12)
    rho = pm.cic_deposit(rng.uniform(0, nm, size=(300, 3)), nm)
    force = pm.force_mesh(pm.density_contrast(rho, 8, nm), BOX, 1)
    _, _, _, nyq = ics.wavevectors(nm, BOX)
    for j in range(3):
        fk = fft.fftn(force[j])
        assert np.abs(fk[nyq]).max() < 1e-12 * np.abs(fk).max(), j
    dk = ics.gaussian_field(nm, BOX, 3, cosmology.linear_pk(0.3, 0.7, 0.96, 0.8))
    for field in ics.lpt_displacements(dk, BOX):
        for j in range(3):
            fk = fft.fftn(field[j])
            assert np.abs(fk[nyq]).max() < 1e-12 * np.abs(fk).max(), j


def test_mesh_force_of_a_sinusoid_is_exact():
    nm, amp = 16, 0.1
    k1 = 2 * math.pi / BOX
    xg = np.arange(nm) * BOX / nm
    delta = np.broadcast_to(amp * np.cos(k1 * xg), (nm, nm, nm)).copy()
    force = pm.force_mesh(delta, BOX, deconv=0)
    assert np.abs(force[0] - (-(amp / k1) * np.sin(k1 * xg))).max() < 1e-12 * amp / k1
    # With deconv = 1 the mode is divided by W(k1) = sinc^2(pi/N).
    w = (math.sin(math.pi / nm) / (math.pi / nm)) ** 2
    force1 = pm.force_mesh(delta, BOX, deconv=1)
    assert np.abs(force1[0] * w - force[0]).max() < 1e-12 * amp / k1


def test_uniform_lattice_has_zero_contrast_at_mesh_ratio_two():
    # The Lagrangian lattice sits half a PM cell off the mesh nodes. With N_m = 2 N_p each particle
    # splits equally over 8 cells and every cell receives exactly 1/8 of one particle, so the mass
    # per cell times the particle mass (N_m/N_p)^3 = 8 cells is exactly the mean: delta = 0 everywhere.
    # The same holds on the coarse meshes of §7.3 (N_m = N_p / 2, N_p / 4): 8 and 64 particles' worth
    # of weight per cell, each particle of mass 1/8 and 1/64 cells.
    for np_, nm in ((8, 16), (4, 4), (16, 8), (16, 4)):
        q = ics.lagrangian_grid(np_, BOX, nm)
        rho = pm.cic_deposit(q * (nm / BOX), nm)
        assert np.all(rho == rho.flat[0]) and rho.sum() == np_ ** 3 << 45
        assert np.abs(pm.density_contrast(rho, np_, nm)).max() == 0.0
    # Any positions: the contrast averages to zero (mass conservation with the particle mass above).
    rng = np.random.default_rng(9)
    u = rng.uniform(0, 16, size=(8 ** 3, 3))
    assert abs(pm.density_contrast(pm.cic_deposit(u, 16), 8, 16).mean()) < 1e-15


@pytest.mark.parametrize("sep", [5.0, 7.0])
def test_newtonian_limit_pair_at_mesh_ratio_two(sep):
    # With N_m = 2 N_p one particle carries (N_m/N_p)^3 = 8 cell volumes of mass: the pair force far
    # from the mesh scale approaches -8 r_hat / (4 pi r^2) in cell units (Gauss's law).
    nm = 64
    box = float(nm)
    d = np.array([0.3, 1.0, 0.6])
    d /= np.linalg.norm(d)
    x = np.array([[30.6, 12.2, 40.9], [0, 0, 0]])
    x[1] = x[0] + sep * d
    f, _ = pm.pm_accel(x, box, nm // 2, nm)
    expect = 8.0 * sep ** -2 / (4 * math.pi) * d
    assert np.linalg.norm(f[0] - expect) < 0.03 * np.linalg.norm(expect)
    assert np.linalg.norm(f[1] + expect) < 0.03 * np.linalg.norm(expect)


# --- COLA / PM stepping (§2.3) -------------------------------------------------------------

def pancake_error(np_, nm, n_steps, cola_on, stepping="modified", amp=0.5, deconv=1):
    r = cola.Run(BOX, np_, nm, 0.3, 9.0, 0.0, n_steps, stepping=stepping, cola=cola_on, deconv=deconv)
    a = amp / r.table["D1"][-1]
    r.set_displacements(*ics.lpt_displacements(plane_wave_field(np_, [((1, 0, 0), a)]), BOX))
    if cola_on:
        assert not r.p.any()                     # residual momentum starts at zero
    r.run()
    exact = r.table["D1"][-1] * r.psi1           # x = q + D1 Psi1 before shell crossing
    return np.sqrt(np.mean((r.displacement() - exact) ** 2)) / np.abs(exact).max()


def test_pancake_cola_ten_steps():
    # 1-D Zel'dovich solution is exact before shell crossing; the remaining error is the PM
    # discreteness of 32 sheets (measured 9.8e-3 at 32^3, 3.8e-3 at 64^3).
    assert pancake_error(32, 32, 10, True) < 1.5e-2


def test_pancake_cola_at_mesh_ratio_two():
    # N_m = 2 N_p, the ratio of the benchmarked runs: the mass normalisation (N_m/N_p)^3 enters the
    # force. Without the CIC deconvolution the 32 displaced sheets are followed to 1.9e-2 rms; with it
    # (the default) the sheets' own graininess near the mesh Nyquist frequency is amplified by 1/W:
    # 4.8e-2 measured, 2.7e-2 at 64 sheets on a 128 mesh (PM discreteness, converging).
    assert pancake_error(32, 64, 10, True, deconv=0) < 2.5e-2
    assert pancake_error(32, 64, 10, True) < 6e-2


def test_finalize_total_momentum_of_the_pancake():
    # Before shell crossing the exact 1-D solution is x = q + D1 Psi1, so the total momentum
    # p = a^3 E dx/da at a_N is P1(a_N) Psi1 (Psi2 = 0): finalize must return it, to the PM
    # discreteness of the positions (1.0e-2 measured at 32 sheets).
    amp = 0.5
    r = cola.Run(BOX, 32, 32, 0.3, 9.0, 0.0, 10)
    a = amp / r.table["D1"][-1]
    r.set_displacements(*ics.lpt_displacements(plane_wave_field(32, [((1, 0, 0), a)]), BOX))
    r.run()
    p = r.finalize()
    exact = r.table["P1"][-1] * r.psi1
    assert np.sqrt(np.mean((p - exact) ** 2)) < 1.5e-2 * np.abs(exact).max()
    assert np.abs(p[:, 1:]).max() < 1e-12 * np.abs(exact).max()


def test_finalize_adds_the_lpt_frame_momentum():
    # COLA moves particles as x = x_res + D1(a) Psi1 + D2(a) Psi2 (§2.3), so the total momentum
    # p = a^3 E dx/da is the residual one plus a^3 E (dD1/da Psi1 + dD2/da Psi2). The derivatives
    # are taken here by central differences of the growth factors (pinned by the EdS closed forms
    # and the Heath integral), not from the momenta P1, P2 that finalize uses.
    om, box, np_ = 0.3, 64.0, 8
    rng = np.random.default_rng(17)
    r = cola.Run(box, np_, 16, om, 9.0, 0.5, 4)
    r.set_displacements(rng.standard_normal((3, np_, np_, np_)), 0.6 * rng.standard_normal((3, np_, np_, np_)))
    r.run()
    p_total = r.finalize()
    a, h = r.table["a"][-1], 1e-3
    d1p, d2p, _, _ = cosmology.growth(np.array([a + h]), om)
    d1m, d2m, _, _ = cosmology.growth(np.array([a - h]), om)
    a3e = a ** 3 * cosmology.hubble_e(a, om)
    expect = a3e * ((d1p - d1m) / (2 * h) * r.psi1 + (d2p - d2m) / (2 * h) * r.psi2)
    assert np.abs(p_total - r.p - expect).max() < 1e-5 * np.abs(expect).max()


def lpt_acceleration_coefficients(a, om):
    """(c1, c2) per scale factor a (array), with the acceleration of the exact LPT trajectory
    x = q + D1 Psi1 + D2 Psi2 equal to c1 Psi1 + c2 Psi2 in the force units of the kick: the equation
    of motion dp/da = 1.5 Om F / (a^2 E) with p = a^3 E dx/da (§2.3) gives
    F = a^2 E / (1.5 Om) d/da [a^3 E dD/da] per LPT order. The two derivatives are nested central
    differences of the growth factors alone."""
    a = np.asarray(a, dtype=np.float64)
    h = 2e-3 * a
    d1, d2, _, _ = cosmology.growth(np.concatenate([a - 2 * h, a, a + 2 * h]), om)
    e = cosmology.hubble_e

    def outer(d):
        d = d.reshape(3, -1)
        lo = (a - h) ** 3 * e(a - h, om) * (d[1] - d[0]) / (2 * h)
        hi = (a + h) ** 3 * e(a + h, om) * (d[2] - d[1]) / (2 * h)
        return a * a * e(a, om) / (1.5 * om) * (hi - lo) / (2 * h)
    return outer(d1), outer(d2)


class LptForceRun(cola.Run):
    """A run whose force is the acceleration of the exact LPT trajectory at the current a_i."""

    def force(self):
        if not hasattr(self, "_coef"):
            self._coef = lpt_acceleration_coefficients(self.table["a"], self.om)
        i = self.step_index
        return self._coef[0][i] * self.psi1 + self._coef[1][i] * self.psi2


def lpt_momentum(r):
    """a^3 E dx/da of the exact LPT trajectory at a_N, by central differences of the growth factors."""
    a, om = r.table["a"][-1], r.om
    h = 2e-3 * a
    d1p, d2p, _, _ = cosmology.growth(np.array([a + h]), om)
    d1m, d2m, _, _ = cosmology.growth(np.array([a - h]), om)
    return a ** 3 * cosmology.hubble_e(a, om) * ((d1p - d1m) / (2 * h) * r.psi1 + (d2p - d2m) / (2 * h) * r.psi2)


def lpt_trajectory_run(cola_on, n_steps, spacing="lin", stepping="modified", finalize=False):
    """Relative max error of the positions at a_N (and, with finalize, of the final momenta)."""
    om, box, np_ = 0.3, 64.0, 4
    rng = np.random.default_rng(23)
    r = LptForceRun(box, np_, 8, om, 9.0, 0.0, n_steps, spacing=spacing, stepping=stepping, cola=cola_on)
    r.set_displacements(rng.standard_normal((3, np_, np_, np_)), rng.standard_normal((3, np_, np_, np_)))
    r.run()
    t = r.table
    exact = t["D1"][-1] * r.psi1 + t["D2"][-1] * r.psi2
    err = np.abs(r.displacement() - exact).max() / np.abs(exact).max()
    if not finalize:
        return r, err
    p_exact = lpt_momentum(r)
    return r, err, np.abs(r.finalize() - p_exact).max() / np.abs(p_exact).max()


@pytest.mark.parametrize("stepping", ["modified", "quinn"])
def test_cola_follows_the_exact_lpt_trajectory(stepping):
    # Given the exact acceleration of the 2LPT trajectory (Psi2 != 0), COLA's residual force is zero
    # (the LPT terms of the kick are what the growth equations make of the two modes), so the residual
    # momentum stays zero, the particles stay on x = q + D1 Psi1 + D2 Psi2 after any number of steps,
    # and finalize returns p = a^3 E dx/da at a_N (derivatives by central differences, not P1, P2).
    r, err = lpt_trajectory_run(True, 10, stepping=stepping)
    assert err < 1e-5
    assert np.abs(r.p).max() < 1e-5 * np.abs(r.psi1).max()
    p_total = r.finalize()
    assert np.abs(r.p).max() < 1e-5 * np.abs(r.psi1).max()
    expect = lpt_momentum(r)
    assert np.abs(p_total - expect).max() < 1e-5 * np.abs(expect).max()


def test_plain_pm_converges_to_the_exact_lpt_trajectory():
    # COLA off (§7.1): the same exact acceleration, integrated by the kick and drift coefficients alone
    # from the 2LPT momentum, converges to the LPT trajectory as the steps shrink (leapfrog: second
    # order in the step), for linear and logarithmic spacing in a.
    # The closing half kick of finalize synchronises the momentum with the positions at a_N, so the
    # final momentum converges at second order as well.
    for spacing, stepping in itertools.product(("lin", "log"), ("modified", "quinn")):
        runs = [lpt_trajectory_run(False, n, spacing, stepping, finalize=True) for n in (20, 40, 80)]
        for k in (1, 2):
            errs = [run[k] for run in runs]
            assert errs[2] < errs[1] < errs[0] < 2e-2, (spacing, stepping, k, errs)
            assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0, (spacing, stepping, k, errs)


def test_pancake_plain_pm_converges():
    # COLA off: the kick normalisation alone must reproduce linear growth (50 steps: 8.8e-3).
    assert pancake_error(32, 32, 50, False) < 1.5e-2
    assert pancake_error(32, 32, 50, False, stepping="quinn") < 1.5e-2


def test_quinn_and_modified_stepping_converge():
    pk = cosmology.linear_pk(0.3, 0.7, 0.96, 0.8)
    out = {}
    for st in ("quinn", "modified"):
        r = cola.Run(BOX, 8, 8, 0.3, 9.0, 0.0, 200, stepping=st)
        r.make_ics(5, pk)
        r.run()
        out[st] = r.displacement()
    scale = np.abs(out["quinn"]).max()
    assert np.abs(out["quinn"] - out["modified"]).max() < 2e-3 * scale


# --- Power spectrum (§7.1) ---------------------------------------------------------------

def test_power_parseval_and_mode_count():
    n = 12
    rng = np.random.default_rng(8)
    delta = rng.standard_normal((n, n, n))
    dk = fft.fftn(delta)
    kx, ky, kz, nyq = ics.wavevectors(n, BOX)
    dk[nyq] = 0                                 # band-limit so every mode falls in a bin
    dk[0, 0, 0] = 0                             # and remove the mean, which no bin holds
    delta = fft.ifftn(dk).real
    kf = 2 * math.pi / BOX
    kmin, kmax = kf, kf * n                     # above sqrt(3) (n/2 - 1) kf
    kmean, pb, cnt = power.binned_power(dk, BOX, 10, kmin, kmax, window=False)
    total = np.nansum(pb * cnt) * n ** 6 / BOX ** 3
    assert abs(total / (n ** 3 * (delta ** 2).sum()) - 1) < 1e-12      # Parseval
    # Brute-force mode count over the integer lattice.
    edges = kmin * (kmax / kmin) ** (np.arange(11) / 10)
    brute = np.zeros(10, int)
    s = range(-n // 2 + 1, n // 2)
    for i, j, k in itertools.product(s, s, s):
        km = kf * math.sqrt(i * i + j * j + k * k)
        for b in range(10):
            if edges[b] <= km < edges[b + 1]:
                brute[b] += 1
    assert np.array_equal(cnt, brute)


def test_power_single_mode_and_cross_correlation():
    n = 16
    dk = plane_wave_field(n, [((2, 1, 0), 0.1)])
    kf = 2 * math.pi / BOX
    kmean, pb, cnt = power.binned_power(dk, BOX, 20, kf, kf * n / 2, window=False)
    b = np.flatnonzero(np.nan_to_num(pb) > 0)
    assert len(b) == 1
    # Two modes (+-k) of |delta_k|^2 = (0.1 N^3 / 2)^2 each: P = L^3 0.01 / 4 per mode.
    assert abs(pb[b[0]] * cnt[b[0]] / 2 / (BOX ** 3 * 0.01 / 4) - 1) < 1e-12
    r = power.cross_correlation(dk, 3.0 * dk, BOX, 20, kf, kf * n / 2)
    assert abs(r[b[0]] - 1) < 1e-12
    r = power.cross_correlation(dk, -dk, BOX, 20, kf, kf * n / 2)
    assert abs(r[b[0]] + 1) < 1e-12


def test_power_cic_window_of_a_planted_mode():
    # One planted mode n = (3, -2, 5) with all three indices non-zero (and its conjugate): the
    # windowed estimator must give L^3 (A/2)^2 / W(n)^2 with W = prod_i sinc^2(pi n_i / N) (§7.1),
    # the CIC window divided out twice in power (once per delta_k).
    n, amp = 16, 0.1
    m = (3, -2, 5)
    dk = plane_wave_field(n, [(m, amp)])
    kf = 2 * math.pi / BOX
    w = 1.0
    for mi in m:
        x = math.pi * mi / n
        w *= (math.sin(x) / x) ** 2
    kmean, pb, cnt = power.binned_power(dk, BOX, 20, kf, kf * n / 2, window=True)
    b = np.flatnonzero(cnt > 0)
    sel = b[np.nan_to_num(pb[b]) > 0]
    assert len(sel) == 1
    i = sel[0]
    assert abs(pb[i] * cnt[i] / 2 / (BOX ** 3 * (amp / 2) ** 2 / w ** 2) - 1) < 1e-12
    # and without the window the bare |delta_k|^2 normalisation
    _, pb0, _ = power.binned_power(dk, BOX, 20, kf, kf * n / 2, window=False)
    assert abs(pb0[i] * cnt[i] / 2 / (BOX ** 3 * (amp / 2) ** 2) - 1) < 1e-12


def test_planar_force_reduces_the_3d_operator_to_one_axis():
    # A density that varies along x only has modes with n_y = n_z = 0: the 3-D force mesh is the
    # 1-D solution along x, constant in y and z, and the other two components vanish.
    from oracle import pm as opm
    nm, box = 16, 40.0
    rng = np.random.default_rng(3)
    d1 = rng.standard_normal(nm)
    delta = np.broadcast_to(d1[None, None, :], (nm, nm, nm)).copy()
    for deconv in (0, 1, 2):
        f3 = opm.force_mesh(delta, box, deconv)
        f1 = opm.planar_force_1d(d1, box, deconv)
        assert np.allclose(f3[0], f1[None, None, :], atol=1e-12)
        assert np.abs(f3[1]).max() < 1e-12 and np.abs(f3[2]).max() < 1e-12
    # numpy's FFT as the primitive gives the same operator
    delta = rng.standard_normal((nm, nm, nm))
    assert np.allclose(opm.force_mesh(delta, box, 1, fft="numpy"), opm.force_mesh(delta, box, 1), atol=1e-10)


def test_numpy_fft_primitive_gives_the_same_run():
    # The fft="numpy" option swaps only the transform primitive: same ICs, steps and P(k).
    kw = dict(box=64.0, np_=8, nm=16, om=0.3, z_init=9.0, z_final=0.0, n_steps=3)
    pk = cosmology.linear_pk(0.3, 0.7, 0.96, 0.8)
    a, b = cola.Run(**kw), cola.Run(**kw, fft="numpy")
    a.make_ics(5, pk)
    b.make_ics(5, pk)
    a.run()
    b.run()
    assert np.max(np.abs(a.x - b.x)) < 1e-9
    pa = power.power_from_positions(a.x, 64.0, 8, 16, 8)
    pb = power.power_from_positions(b.x, 64.0, 8, 16, 8, fft="numpy")
    assert np.allclose(pa[1], pb[1], rtol=1e-9, equal_nan=True)


# --- Redshift space (§7.1) --------------------------------------------------------------------------

def test_redshift_space_displacement_by_hand():
    # Observer at the box centre, particle at centre + (3, 4, 0) Mpc/h, peculiar velocity (500, 0, 0) km/s
    # at a = 0.5: v_los = 300 km/s along (0.6, 0.8, 0); H(a) = 100 E(a) km/s per Mpc/h; the particle
    # moves by v_los / (a H) along the line of sight. Momenta in the method's units: v = 100 p / a km/s.
    box, a, om = 100.0, 0.5, 0.3
    x = np.array([[53.0, 54.0, 50.0]])
    p = np.array([[500.0 * a / 100.0, 0.0, 0.0]])
    h_kms = 100.0 * math.sqrt(om / a ** 3 + 1 - om)
    shift = 300.0 / (a * h_kms)
    s = power.redshift_space(x, p, a, om, box)
    assert np.abs(s[0] - (x[0] + shift * np.array([0.6, 0.8, 0.0]))).max() < 1e-12
    # plane-parallel along y: the x velocity does not move it; along x it moves by 500 / (a H)
    assert np.abs(power.redshift_space(x, p, a, om, box, los=1) - x).max() < 1e-12
    sx = power.redshift_space(x, p, a, om, box, los=0)
    assert abs(sx[0, 0] - (53.0 + 500.0 / (a * h_kms))) < 1e-12
    # periodic wrap, and no motion without velocity
    xe = np.array([[99.9, 1.0, 2.0]])
    assert power.redshift_space(xe, np.array([[1.0, 0, 0]]), a, om, box, los=0)[0, 0] < 5.0
    assert np.array_equal(power.redshift_space(x, 0 * p, a, om, box), x)


def test_redshift_space_kaiser_factor_in_the_linear_regime():
    # Zel'dovich particles (Psi2 = 0) at z = 49 with the growing-mode momentum p = P1 Psi1: along the
    # axis the redshift-space displacement is D1 (Psi + f Psi_z z^), so every low-k mode of the density
    # is multiplied by 1 + f mu^2 (Kaiser 1987), f = dln D1 / dln a = P1 / (a^3 E D1 / a) (§7.1).
    n, box, om = 32, 256.0, 0.3
    a = 0.02
    d1, _, p1, _ = cosmology.growth(np.array([a]), om)
    f = p1[0] / (a ** 2 * cosmology.hubble_e(a, om) * d1[0])
    pk = cosmology.linear_pk(om, 0.7, 0.96, 0.8)
    dk = ics.gaussian_field(n, box, 21, pk)
    psi1, _ = ics.lpt_displacements(dk, box)
    q = ics.lagrangian_grid(n, box, n)
    psi = ics.per_particle(psi1)
    x = np.mod(q + d1[0] * psi, box)
    s = power.redshift_space(x, p1[0] * psi, a, om, box, los=2)
    dr = fft.fftn(pm.density_contrast(pm.cic_deposit(x * n / box, n), n, n))
    ds = fft.fftn(pm.density_contrast(pm.cic_deposit(s * n / box, n), n, n))
    kx, ky, kz, nyq = ics.wavevectors(n, box)
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    sel = (k > 0) & (k < 4 * 2 * math.pi / box) & ~nyq
    mu2 = kz[sel] ** 2 / k[sel] ** 2
    ratio = (ds[sel] / dr[sel]).real
    assert abs(f - 1.0) < 0.01                       # matter dominated at z = 49
    assert np.abs(ratio - (1 + f * mu2)).max() < 0.02


# --- Local primordial non-Gaussianity (§5) -----------------------------------------------------------

def _d_md(om):
    return cosmology.growth_matter_era(om)


def test_matter_era_growth_normalisation():
    # EdS: D1 = a exactly; LCDM: within 1% of the Carroll, Press & Turner (1992) fit
    # g = 5/2 Om / (Om^(4/7) - OL + (1 + Om/2)(1 + OL/70)).
    assert abs(cosmology.growth_matter_era(1.0) - 1.0) < 1e-10
    for om in (0.25, 0.3, 0.5):
        ol = 1 - om
        cpt = 2.5 * om / (om ** (4 / 7) - ol + (1 + om / 2) * (1 + ol / 70))
        assert abs(cosmology.growth_matter_era(om) / cpt - 1) < 1e-2


def test_fnl_zero_is_the_gaussian_field_and_the_change_is_linear_in_fnl():
    n, om, h = 16, 0.3, 0.7
    pk = cosmology.linear_pk(om, h, 0.96, 0.8)
    dk = ics.gaussian_field(n, BOX, 5, pk)
    dmd = _d_md(om)
    d0 = ics.local_fnl_field(dk, BOX, 0.0, om, h, dmd)
    assert np.abs(d0 - dk).max() < 1e-12 * np.abs(dk).max()
    d1 = ics.local_fnl_field(dk, BOX, 100.0, om, h, dmd)
    d2 = ics.local_fnl_field(dk, BOX, 200.0, om, h, dmd)
    assert np.abs(d1 - dk).max() > 1e-6 * np.abs(dk).max()          # it does something
    assert np.abs((d2 - dk) - 2 * (d1 - dk)).max() < 1e-9 * np.abs(d1 - dk).max()
    # the change is f_NL M FFT(phi^2) on every mode but k = 0: the square of the real-space potential
    m = ics.potential_to_density(n, BOX, om, h, dmd)
    phi_k = np.where(m > 0, dk / np.where(m > 0, m, 1.0), 0.0)
    phi = fft.ifftn(phi_k).real
    sq = m * fft.fftn(phi * phi)
    _, _, _, nyq = ics.wavevectors(n, BOX)
    sq[nyq] = 0.0
    assert np.abs((d1 - dk) - 100.0 * sq).max() < 1e-9 * np.abs(sq).max() * 100.0


def test_primordial_potential_amplitude_is_physical():
    # With sigma_8 = 0.8, the potential implied by M(k) has the order of the observed primordial
    # curvature amplitude: P_Phi k^3 / (2 pi^2) = (9/25) A_s (k / k_*)^(n_s - 1) at k_* = 0.05 / Mpc
    # (Phi = 3/5 zeta in matter domination), A_s ~ 2.1e-9 from CMB fits with CAMB spectra. BBKS without
    # baryons has about 1.5x more power than such spectra where sigma_8 is fixed (k ~ 0.1-0.3 h/Mpc),
    # so the same sigma_8 implies about half of that A_s (9.5e-10 here). The window rejects a dropped
    # 2/3 (4.2e-10), a dropped 1/Om (1e-8) or a dropped growth to z = 0 (5.8e-10).
    om, h, ns = 0.3, 0.7, 0.96
    pk = cosmology.linear_pk(om, h, ns, 0.8)
    kstar = 0.05 / h                                            # h/Mpc
    k = np.array([kstar])
    t = cosmology.t_bbks(k, om, h)[0]
    m = 2.0 / 3.0 * (kstar * ics.HUBBLE_DISTANCE) ** 2 * t * _d_md(om) / om
    p_phi = pk(k)[0] / m ** 2
    a_s = p_phi * kstar ** 3 / (2 * math.pi ** 2) * 25.0 / 9.0
    assert 7e-10 < a_s < 2.5e-9, a_s


# --- Lightcone (§6) ------------------------------------------------------------------------------------

def test_comoving_distance_eds_closed_form():
    from oracle import lightcone
    # EdS: int_a^1 da / (a^2 a^-3/2) = 2 (1 - sqrt(a))
    for a in (0.25, 0.5, 0.9):
        assert abs(lightcone.comoving_distance(a, 1.0) / (2 * lightcone.HUBBLE_DISTANCE * (1 - math.sqrt(a))) - 1) < 1e-12


def _lonely_particle_run(r_obs, stepping="modified", cola_on=True, n_steps=10):
    """One particle at distance r_obs (Mpc/h) from the observer, no displacement: it feels no force
    (zero self-force) and stays put, so it leaves the lightcone when R_L(a) = r_obs."""
    from oracle import lightcone
    box = 2000.0
    r = lightcone.LightconeRun(box, 1, 4, 0.3, 9.0, 0.0, n_steps, stepping=stepping, cola=cola_on,
                               origin=(0.0, 0.0, 0.0), z_max=1.0)
    r.set_displacements(np.zeros((3, 1, 1, 1)), np.zeros((3, 1, 1, 1)))
    r.x = np.array([[r_obs, 0.0, 0.0]])
    r.run()
    return r


def test_lightcone_exit_of_a_particle_at_rest():
    # The exit time is the interpolation of Eq. eq:lightconeinterp; against the exact root of
    # R_L(a) = R it is off by the curvature of R_L within the step only (<0.5% in a, as in §6.1.1),
    # and exact at a step boundary; the output position is the particle's own.
    from oracle import lightcone
    from scipy import optimize
    for r_obs in (500.0, 1234.5, 1900.0):
        r = _lonely_particle_run(r_obs)
        out = r.lightcone()
        assert len(out) == 1
        exact = optimize.brentq(lambda a: lightcone.comoving_distance(a, 0.3) - r_obs, 0.3, 1.0, xtol=1e-14)
        assert abs(out[0, 3] / exact - 1) < 5e-3
        assert np.abs(out[0, :3] - [r_obs, 0, 0]).max() < 1e-9
    a = r.table["a"]
    rl = lightcone.comoving_distance(a[6], 0.3)
    out = _lonely_particle_run(rl * (1 - 1e-12)).lightcone()
    assert abs(out[0, 3] - a[6]) < 1e-9


def test_lightcone_drift_to_the_exit_time():
    # Plain PM, one particle with constant momentum (no force): between boundaries it moves by
    # p int_{a_i}^{a_L} da / (a^3 E) (Quinn drift, Eq. 16 at a_L); the output lies on that path and on
    # the interpolated radius.
    from oracle import lightcone
    r = lightcone.LightconeRun(3000.0, 1, 4, 0.3, 9.0, 0.0, 10, stepping="quinn", cola=False,
                               origin=(0.0, 0.0, 0.0), z_max=2.0)
    r.set_displacements(np.zeros((3, 1, 1, 1)), np.zeros((3, 1, 1, 1)))
    x0 = np.array([1500.0, 300.0, 200.0])
    r.x = x0[None, :].copy()
    r.p = np.array([[-200.0, 50.0, 0.0]])
    a = r.table["a"]
    r.run()
    out = r.lightcone()
    assert len(out) == 1
    al = out[0, 3]
    i = int(np.searchsorted(a, al)) - 1
    xi = x0 + r.p[0] * sum(cosmology.drift_coeff(a[j], a[j + 1], 0.0, 0.3, "quinn") for j in range(i))
    s, _ = integrate.quad(lambda v: 1.0 / (v ** 3 * cosmology.hubble_e(v, 0.3)), a[i], al, epsrel=1e-13)
    assert np.abs(out[0, :3] - (xi + r.p[0] * s)).max() < 1e-8 * np.abs(xi).max()
    assert np.abs(out[0, 4:7] - r.p[0]).max() < 1e-12


def test_every_image_inside_the_start_radius_leaves_exactly_once():
    # With z_final = 0 the lightcone shrinks to the observer, so every particle image inside the
    # lightcone at its start leaves during the run, once; images outside never enter (v << c).
    from oracle import lightcone
    pk = cosmology.linear_pk(0.3, 0.7, 0.96, 0.8)
    box, np_ = 300.0, 8
    r = lightcone.LightconeRun(box, np_, 16, 0.3, 9.0, 0.0, 8, origin=(20.0, 150.0, 280.0), z_max=0.2,
                               rep_lo=(-1, -1, 0), rep_hi=(1, 1, 1))
    r.make_ics(4, pk)
    r.run(r.first)
    rl = lightcone.comoving_distance(r.table["a"][r.first], 0.3)
    inside = 0
    for rep in r.reps:
        d = r.x + rep * box - r.origin
        inside += int(np.sum(np.sqrt(np.sum(d * d, axis=1)) <= rl))
    r.run()
    out = r.lightcone()
    assert inside > 100 and len(out) == inside
    # one output per (particle, image): the image is the output position minus the drift, within half a box
    keys = {(int(row[7]), tuple(np.floor((row[:3] - r.x[int(row[7])] + box / 2) / box).astype(int))) for row in out}
    assert len(keys) == len(out)
