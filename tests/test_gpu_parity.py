"""GPU path vs the FP64 oracle, element by element, through the C ABI.

Bars: bit-exact for the int64 density mesh (integer work) and the mode counts; forces,
positions and momenta within 1e-4 rms relative; P(k) within 1e-3 per bin for independent
runs and 1e-4 on shared positions. Sizes span several FFT tiles with ragged tails and
mixed radices (N_m = 96, 160, 192).
"""
import math

import numpy as np
import pytest

from oracle import cola as ocola, cosmology as ocosmo, ics as oics, pm as opm, power as opower
from paper_1506_03737_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_1506_03737_gb300 import colapm
    return colapm


class Sim:
    def __init__(self, C, **kw):
        self.C = C
        self.p = C.default_params(**kw)
        self.ctx = C.colapm_create(self.p)
        self.np, self.nm, self.box = self.p.np, self.p.nm, self.p.box

    def close(self):
        self.C.colapm_destroy(self.ctx)

    def state(self):
        n = self.np ** 3
        cell = np.empty((n, 3), np.int32)
        off = np.empty((n, 3), np.float32)
        mom = np.empty((n, 3), np.float32)
        self.C.colapm_get_state(self.ctx, cell, off, mom)
        return cell, off, mom

    def lpt(self):
        n = self.np ** 3
        a, b = np.empty(3 * n, np.float32), np.empty(3 * n, np.float32)
        self.C.colapm_get_lpt(self.ctx, a, b)
        return a.reshape(3, self.np, self.np, self.np), b.reshape(3, self.np, self.np, self.np)

    def density(self):
        m = np.empty(self.nm ** 3, np.int64)
        self.C.colapm_get_density(self.ctx, m)
        return m.reshape(self.nm, self.nm, self.nm)

    def force(self):
        f = np.empty(3 * self.nm ** 3, np.float32)
        self.C.colapm_get_force(self.ctx, f)
        return f.reshape(3, self.nm, self.nm, self.nm)


def mesh_coords(cell, off):
    return cell.astype(np.float64) + off.astype(np.float64)


def oracle_run(sim, **kw):
    p = sim.p
    r = ocola.Run(p.box, p.np, p.nm, p.cosmo.omega_m, p.z_init, p.z_final, p.n_steps,
                  spacing="log" if p.spacing else "lin", stepping="quinn" if p.stepping else "modified",
                  nlpt=p.nlpt, cola=bool(p.cola), deconv=p.deconv, **kw)
    return r


def rel_rms(a, b):
    return float(np.sqrt(np.mean((np.asarray(a, np.float64) - b) ** 2)) / np.sqrt(np.mean(np.asarray(b) ** 2)))


# --- initial conditions ------------------------------------------------------------------

@pytest.mark.parametrize("np_,seed", [(32, 1), (64, 9)])
def test_gaussian_field_matches_oracle(C, np_, seed):
    s = Sim(C, np=np_, nm=np_, box=256.0, seed=seed)
    try:
        dk = np.empty(np_ ** 3, np.float32)
        C.colapm_get_gaussian_field(s.ctx, dk)
        gpu = dk.view(np.complex64).reshape(np_, np_, np_ // 2).astype(np.complex128)
        pk = ocosmo.linear_pk(0.3, 0.7, 0.96, 0.8)
        ref = oics.gaussian_field(np_, 256.0, seed, pk)[:, :, : np_ // 2]
        assert np.abs(gpu - ref).max() < 1e-5 * np.abs(ref).max()
        assert np.array_equal(gpu == 0, ref == 0)
    finally:
        s.close()


@pytest.mark.parametrize("np_", [32, 64])
def test_local_fnl_initial_field_matches_oracle(C, np_):
    # §5: local f_NL on the primordial potential; the GPU runs its transforms on the Stockham engine.
    box, seed = 256.0, 9
    s = Sim(C, np=np_, nm=np_, box=box, seed=seed)
    try:
        half = lambda: np.empty(np_ ** 3, np.float32)                    # noqa: E731
        g0 = half()
        C.colapm_get_gaussian_field(s.ctx, g0)
        C.colapm_set_fnl(s.ctx, 0.0)
        g00 = half()
        C.colapm_get_gaussian_field(s.ctx, g00)
        assert np.array_equal(g0, g00)
        pk = ocosmo.linear_pk(0.3, 0.7, 0.96, 0.8)
        dk = oics.gaussian_field(np_, box, seed, pk)
        dmd = ocosmo.growth_matter_era(0.3)
        gau = g0.view(np.complex64).reshape(np_, np_, np_ // 2).astype(np.complex128)
        for fnl in (300.0, -3000.0):
            C.colapm_set_fnl(s.ctx, fnl)
            g = half()
            C.colapm_get_gaussian_field(s.ctx, g)
            gpu = g.view(np.complex64).reshape(np_, np_, np_ // 2).astype(np.complex128)
            ref = oics.local_fnl_field(dk, box, fnl, 0.3, 0.7, dmd)
            assert np.abs(gpu - ref[:, :, : np_ // 2]).max() < 1e-5 * np.abs(ref).max()
            ng_gpu, ng_ref = gpu - gau, (ref - dk)[:, :, : np_ // 2]
            assert np.abs(ng_gpu - ng_ref).max() < 2e-3 * np.abs(ng_ref).max(), fnl
        # the ICs of the last f_NL: LPT displacements from the oracle's non-Gaussian field
        C.colapm_make_ics(s.ctx)
        g1, g2 = s.lpt()
        p1, p2 = oics.lpt_displacements(ref, box)
        assert rel_rms(g1, p1) < 1e-5 and rel_rms(g2, p2) < 1e-4
        with pytest.raises(C.ColapmError) as e:
            C.colapm_set_fnl(s.ctx, float("nan"))
        assert e.value.code == -1
    finally:
        s.close()


@pytest.mark.parametrize("np_,nm", [(32, 64), (64, 64)])
def test_lpt_displacements_and_initial_positions(C, np_, nm):
    s = Sim(C, np=np_, nm=nm, box=256.0, seed=4)
    try:
        C.colapm_make_ics(s.ctx)
        g1, g2 = s.lpt()
        pk = ocosmo.linear_pk(0.3, 0.7, 0.96, 0.8)
        r = oracle_run(s)
        dk = r.make_ics(4, pk)
        psi1, psi2 = oics.lpt_displacements(dk, s.box)
        assert rel_rms(g1, psi1) < 1e-5
        assert rel_rms(g2, psi2) < 1e-4
        cell, off, mom = s.state()
        u = mesh_coords(cell, off)
        ref_u = np.mod(r.x * nm / s.box, nm)
        d = u - ref_u
        d -= nm * np.rint(d / nm)
        assert np.sqrt(np.mean(d ** 2)) < 1e-4 * np.sqrt(np.mean((r.displacement() * nm / s.box) ** 2))
        assert not mom.any()                                   # COLA: residual momentum starts at 0
    finally:
        s.close()


# --- deposit -------------------------------------------------------------------------------

@pytest.mark.parametrize("np_,nm,kind", [(32, 64, "random"), (32, 96, "random"), (64, 64, "clustered"),
                                         (32, 160, "random"), (64, 32, "random"), (64, 16, "clustered")])
def test_density_bit_exact(C, np_, nm, kind):
    s = Sim(C, np=np_, nm=nm, box=200.0)
    try:
        C.colapm_make_ics(s.ctx)
        gen = workloads.random_state if kind == "random" else workloads.clustered_state
        cell, off, _ = gen(np_, nm, 11)
        C.colapm_set_state(s.ctx, cell, off, None)
        gpu = s.density()
        ref = opm.cic_deposit(mesh_coords(cell, off), nm)
        assert np.array_equal(gpu, ref)
        assert int(gpu.astype(np.uint64).sum()) == np_ ** 3 << 45   # 2^63 for 64^3: sum unsigned
        assert np.array_equal(s.density(), gpu)                # deterministic across runs
    finally:
        s.close()


# --- force ---------------------------------------------------------------------------------

@pytest.mark.parametrize("np_,nm,deconv", [(32, 64, 1), (32, 96, 1), (64, 128, 0), (32, 64, 2), (96, 192, 1),
                                           (64, 32, 1)])
def test_force_mesh_matches_oracle(C, np_, nm, deconv):
    s = Sim(C, np=np_, nm=nm, box=300.0, deconv=deconv)
    try:
        C.colapm_make_ics(s.ctx)
        cell, off, _ = workloads.clustered_state(np_, nm, 3)
        C.colapm_set_state(s.ctx, cell, off, None)
        gpu = s.force()
        rho = opm.cic_deposit(mesh_coords(cell, off), nm)
        ref = opm.force_mesh(opm.density_contrast(rho, np_, nm), s.box, deconv) * (nm / s.box)
        for j in range(3):
            assert rel_rms(gpu[j], ref[j]) < 1e-4, j
    finally:
        s.close()


@pytest.mark.parametrize("np_,nm", [(32, 64), (32, 96), (64, 128), (32, 160), (96, 192)])
@pytest.mark.parametrize("two_stage", [1, 0])
def test_force_engines_match_oracle(C, np_, nm, two_stage):
    """Both FFT engines against the oracle at the power-of-two and mixed-radix sizes of the batch:
    the two-stage register plans (second radix 8, 10, 12 by the prime-factor split) and the
    multi-stage Stockham plans, each in every pass, with the whole step chain behind it."""
    s = Sim(C, np=np_, nm=nm, box=250.0)
    try:
        C.colapm_set_engine(s.ctx, 0, two_stage, 256)
        C.colapm_make_ics(s.ctx)
        cell, off, _ = workloads.clustered_state(np_, nm, 7)
        C.colapm_set_state(s.ctx, cell, off, None)
        gpu = s.force()
        rho = opm.cic_deposit(mesh_coords(cell, off), nm)
        ref = opm.force_mesh(opm.density_contrast(rho, np_, nm), s.box, 1) * (nm / s.box)
        for j in range(3):
            assert rel_rms(gpu[j], ref[j]) < 1e-4, j
        k, p, cnt = C.colapm_power(s.ctx, 20)
        kr, pr, nr = opower.power_from_positions(mesh_coords(cell, off) * (s.box / nm), s.box, np_, nm, 20,
                                                 fft="numpy")
        assert np.array_equal(cnt, nr)
        ok = nr > 0
        assert np.max(np.abs(p[ok] / pr[ok] - 1)) < 1e-4
    finally:
        s.close()


# --- one step from a shared state ----------------------------------------------------------

@pytest.mark.parametrize("cola_on,stepping,spacing", [(1, 0, 0), (0, 0, 0), (1, 1, 0), (1, 0, 1), (0, 1, 1)])
def test_single_step_matches_oracle(C, cola_on, stepping, spacing):
    np_, nm = 32, 64
    s = Sim(C, np=np_, nm=nm, box=256.0, cola=cola_on, stepping=stepping, spacing=spacing, seed=5)
    try:
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, 3)                       # evolve a little, then compare one step
        cell, off, mom = s.state()
        g1, g2 = s.lpt()
        r = oracle_run(s)
        r.set_displacements(g1.astype(np.float64), g2.astype(np.float64))
        r.x = mesh_coords(cell, off) * s.box / nm
        r.p = mom.astype(np.float64) * s.box / nm
        r.step_index = 3
        r.step()
        C.colapm_step(s.ctx, 1)
        cell2, off2, mom2 = s.state()
        d = mesh_coords(cell2, off2) * s.box / nm - r.x
        d -= s.box * np.rint(d / s.box)
        move = mesh_coords(cell2, off2) - mesh_coords(cell, off)
        move -= nm * np.rint(move / nm)
        assert np.sqrt(np.mean(d ** 2)) < 1e-4 * np.sqrt(np.mean((move * s.box / nm) ** 2))
        assert rel_rms(mom2 * s.box / nm, r.p) < 1e-4
    finally:
        s.close()


# --- full runs ------------------------------------------------------------------------------

def test_full_run_cola_32p_64m(C):
    kw = workloads.run_params("cola_32p_64m_256mpc")
    s = Sim(C, **kw)
    try:
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, -1)
        cell, off, mom = s.state()
        r = oracle_run(s)
        r.make_ics(kw["seed"], ocosmo.linear_pk(0.3, 0.7, 0.96, 0.8))
        r.run()
        d = mesh_coords(cell, off) * s.box / s.nm - r.x
        d -= s.box * np.rint(d / s.box)
        disp = np.sqrt(np.mean(r.displacement() ** 2))
        assert np.sqrt(np.mean(d ** 2)) < 1e-4 * disp
        k, pk, nmodes = C.colapm_power(s.ctx, 100)
        kr, pr, nr = opower.power_from_positions(r.x, s.box, s.np, s.nm, 100)
        assert np.array_equal(nmodes, nr)
        ok = nr > 0
        assert np.nanmax(np.abs(pk[ok] / pr[ok] - 1)) < 1e-3
        assert np.nanmax(np.abs(k[ok] / kr[ok] - 1)) < 1e-6    # per-mode |k| in FP32, sums in FP64
    finally:
        s.close()


@pytest.mark.parametrize("np_,nm", [(64, 32), (64, 16)])
def test_full_run_on_a_coarse_mesh(C, np_, nm):
    # §7.3's coarse force meshes (N_m = N_p / 2, N_p / 4): the lattice sits at i N_m / N_p + 1/2 cells.
    kw = workloads.run_params("cola_32p_64m_256mpc", np=np_, nm=nm, seed=17)
    s = Sim(C, **kw)
    try:
        C.colapm_make_ics(s.ctx)
        cell0, off0, _ = s.state()
        r = oracle_run(s)
        r.make_ics(17, ocosmo.linear_pk(0.3, 0.7, 0.96, 0.8))
        d0 = mesh_coords(cell0, off0) * s.box / nm - r.x
        d0 -= s.box * np.rint(d0 / s.box)
        assert np.sqrt(np.mean(d0 ** 2)) < 1e-4 * np.sqrt(np.mean(r.displacement() ** 2))
        C.colapm_step(s.ctx, -1)
        cell, off, mom = s.state()
        r.run()
        d = mesh_coords(cell, off) * s.box / nm - r.x
        d -= s.box * np.rint(d / s.box)
        assert np.sqrt(np.mean(d ** 2)) < 1e-4 * np.sqrt(np.mean(r.displacement() ** 2))
        psi = np.empty((np_ ** 3, 3), np.float32)
        C.colapm_get_displacement(s.ctx, psi)
        assert np.sqrt(np.mean((psi - r.displacement()) ** 2)) < 1e-4 * np.sqrt(np.mean(r.displacement() ** 2))
        k, pk, nmodes = C.colapm_power(s.ctx, 20)
        kr, pr, nr = opower.power_from_positions(r.x, s.box, np_, nm, 20)
        assert np.array_equal(nmodes, nr)
        ok = nr > 0
        assert np.nanmax(np.abs(pk[ok] / pr[ok] - 1)) < 1e-3
    finally:
        s.close()


@pytest.mark.parametrize("nbins,kmin,kmax", [(100, 0.0, 0.0), (37, 0.05, 0.4), (12, 0.0, 2.0)])
def test_power_on_shared_positions(C, nbins, kmin, kmax):
    np_, nm = 32, 64
    s = Sim(C, np=np_, nm=nm, box=256.0, seed=8)
    try:
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, -1)
        cell, off, _ = s.state()
        k, pk, nmodes = C.colapm_power(s.ctx, nbins, kmin, kmax)
        x = mesh_coords(cell, off) * s.box / nm
        kr, pr, nr = opower.power_from_positions(x, s.box, np_, nm, nbins, kmin or None, kmax or None)
        assert np.array_equal(nmodes, nr)
        ok = nr > 0
        assert np.max(np.abs(pk[ok] / pr[ok] - 1)) < 1e-4
    finally:
        s.close()


@pytest.mark.parametrize("cola_on", [1, 0])
def test_redshift_space_power_matches_oracle(C, cola_on):
    # §7.1: positions moved by v_los / (a H) along the line of sight (radial from the box centre, or
    # plane-parallel), on the GPU's finalized state shared with the oracle.
    np_, nm, box = 32, 64, 256.0
    s = Sim(C, np=np_, nm=nm, box=box, seed=31, cola=cola_on)
    try:
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, -1)
        with pytest.raises(C.ColapmError) as e:
            C.colapm_power_rsd(s.ctx, -1, 20)               # velocities are final only after finalize
        assert e.value.code == -6
        C.colapm_finalize(s.ctx)
        cell, off, mom = s.state()
        x = mesh_coords(cell, off) * (box / nm)
        p = mom.astype(np.float64) * (box / nm)
        _, pr_real, _ = C.colapm_power(s.ctx, 40)
        for los in (-1, 0, 2):
            k, pk, cnt = C.colapm_power_rsd(s.ctx, los, 40)
            xs = opower.redshift_space(x, p, 1.0, 0.3, box, los)
            kr, pr, nr = opower.power_from_positions(xs, box, np_, nm, 40)
            assert np.array_equal(cnt, nr)
            ok = nr > 0
            assert np.max(np.abs(pk[ok] / pr[ok] - 1)) < 1e-4, los
            assert np.max(np.abs(pk[ok] / pr_real[ok] - 1)) > 1e-2      # redshift space differs
        with pytest.raises(C.ColapmError) as e:
            C.colapm_power_rsd(s.ctx, 3, 20)
        assert e.value.code == -1
    finally:
        s.close()


def test_cross_correlation_matches_oracle(C):
    # Two fields of the same seed, one COLA and one plain PM: correlated at low k, less so near the
    # mesh scale. The library bins Re(delta_a delta_b^*) from |delta_a + delta_b|^2 - |delta_a|^2 -
    # |delta_b|^2; the oracle bins the products directly (§7.1).
    np_, nm, box = 32, 64, 256.0
    a, b = Sim(C, np=np_, nm=nm, box=box, seed=8), Sim(C, np=np_, nm=nm, box=box, seed=8, cola=0, n_steps=4)
    try:
        for s in (a, b):
            C.colapm_make_ics(s.ctx)
            C.colapm_step(s.ctx, -1)
        dks = []
        for s in (a, b):
            cell, off, _ = s.state()
            rho = opm.cic_deposit(mesh_coords(cell, off), nm)
            dks.append(np.fft.fftn(opm.density_contrast(rho, np_, nm)))
        for nbins, kmin, kmax in ((40, 0.0, 0.0), (12, 0.05, 0.5)):
            k, r, cnt = C.colapm_cross_correlation(a.ctx, b.ctx, nbins, kmin, kmax)
            kf = 2 * math.pi / box
            lo, hi = kmin or kf, kmax or math.pi * nm / box
            rr = opower.cross_correlation(dks[0], dks[1], box, nbins, lo, hi)
            _, _, nr = opower.binned_power(dks[0], box, nbins, lo, hi, window=False)
            assert np.array_equal(cnt, nr)
            ok = nr > 0
            assert np.max(np.abs(r[ok] - rr[ok])) < 1e-5
            assert np.isnan(r[~ok]).all()
        assert np.nanmin(r) < 0.999 and np.nanmax(r) > 0.9     # a non-trivial test: r spans a range
        _, r1, _ = C.colapm_cross_correlation(a.ctx, a.ctx, 12)
        assert np.nanmax(np.abs(r1 - 1)) < 1e-6
        with pytest.raises(C.ColapmError) as e:
            other = Sim(C, np=np_, nm=2 * nm, box=box)
            try:
                C.colapm_make_ics(other.ctx)
                C.colapm_cross_correlation(a.ctx, other.ctx, 12)
            finally:
                other.close()
        assert e.value.code == -1
    finally:
        a.close()
        b.close()


def test_finalize_adds_lpt_momentum(C):
    s = Sim(C, np=32, nm=64, box=256.0, n_steps=4, seed=6)
    try:
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, -1)
        cell, off, mom = s.state()
        g1, g2 = s.lpt()
        C.colapm_finalize(s.ctx)
        pos, momf = np.empty((32 ** 3, 3), np.float32), np.empty((32 ** 3, 3), np.float32)
        C.colapm_get_particles(s.ctx, pos, momf)
        r = oracle_run(s)
        r.set_displacements(g1.astype(np.float64), g2.astype(np.float64))
        r.x = mesh_coords(cell, off) * s.box / s.nm
        r.p = mom.astype(np.float64) * s.box / s.nm
        r.step_index = 4
        ref = r.finalize()
        assert rel_rms(momf, ref) < 1e-4
    finally:
        s.close()


# --- particle order ------------------------------------------------------------------------------

@pytest.mark.parametrize("np_,nm,every,tiles", [(32, 64, 1, 0), (64, 128, 3, 0), (32, 96, 2, 0), (32, 64, 1, 2),
                                                 (64, 128, 1, 4), (64, 128, 2, 8), (32, 96, 1, 4), (64, 128, 1, -4)])
def test_cell_order_changes_no_result(C, np_, nm, every, tiles):
    """Reordering the particle arrays by cell (by rows, or tile by tile with the tiled deposit) is
    invisible: every step is per particle or an exact integer sum, so runs with and without it give
    bit-identical catalogues, states, LPT fields, densities and finalized momenta, in particle-id
    order, and the same spectra up to the order of their atomic FP64 bin sums."""
    kw = dict(np=np_, nm=nm, box=200.0, seed=13, n_steps=6)
    a, b = Sim(C, **kw), Sim(C, **kw)
    try:
        C.colapm_set_sort(b.ctx, every)
        if tiles < 0:
            C.colapm_set_sort_tiles(b.ctx, -tiles)     # tile-major order, plain deposit
        else:
            C.colapm_set_deposit_tiles(b.ctx, tiles)
        for s in (a, b):
            C.colapm_make_ics(s.ctx)
            C.colapm_step(s.ctx, 4)
        for x, y in zip(a.state(), b.state()):
            assert np.array_equal(x, y)
        for x, y in zip(a.lpt(), b.lpt()):
            assert np.array_equal(x, y)
        for s in (a, b):
            C.colapm_step(s.ctx, -1)
        n = np_ ** 3
        pa, ma = np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)
        pb, mb = np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)
        C.colapm_get_particles(a.ctx, pa, ma)
        C.colapm_get_particles(b.ctx, pb, mb)
        assert np.array_equal(pa, pb) and np.array_equal(ma, mb)
        assert np.array_equal(a.density(), b.density())
        ka, pka, na = C.colapm_power(a.ctx, 30)
        kb, pkb, nb = C.colapm_power(b.ctx, 30)
        assert np.array_equal(na, nb)   # P(k): up to the order of the atomic FP64 bin sums
        assert np.allclose(pka, pkb, rtol=1e-12, atol=0.0, equal_nan=True)
        psi_a, psi_b = np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)
        C.colapm_get_displacement(a.ctx, psi_a)
        C.colapm_get_displacement(b.ctx, psi_b)
        assert np.array_equal(psi_a, psi_b)
        for s in (a, b):
            C.colapm_finalize(s.ctx)
        C.colapm_get_particles(a.ctx, None, ma)
        C.colapm_get_particles(b.ctx, None, mb)
        assert np.array_equal(ma, mb)
    finally:
        a.close()
        b.close()


@pytest.mark.parametrize("tiles", [0, 2, 4, 8])
def test_tiled_deposit_bit_exact_on_clustered_state(C, tiles):
    """The tiled deposit (each tile and its halo summed in shared memory) on a clustered state in
    tile order, right after the sort and after particles have moved out of their tiles: the int64
    mesh equals the oracle's deposit of the same positions exactly."""
    np_, nm = 64, 128
    s = Sim(C, np=np_, nm=nm, box=200.0, seed=3, n_steps=6)
    try:
        C.colapm_set_sort(s.ctx, 1)
        C.colapm_set_deposit_tiles(s.ctx, tiles)
        cfg = C.colapm_get_config(s.ctx)
        assert cfg["deposit_tiled"] == (tiles > 0) and (tiles == 0 or cfg["sort_tiles"] == tiles)
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, 1)
        cell, off, _ = workloads.clustered_state(np_, nm, 17)
        C.colapm_set_state(s.ctx, cell, off, None)
        for _ in range(2):
            C.colapm_step(s.ctx, 1)             # reorders (tile key) before the step, then moves the particles
            gpu = s.density()                   # deposit of the moved particles, still in tile order
            cell2, off2, _ = s.state()
            assert np.array_equal(gpu, opm.cic_deposit(mesh_coords(cell2, off2), nm))
        for bad in (3, 16, -2, 1):
            with pytest.raises(C.ColapmError):
                C.colapm_set_deposit_tiles(s.ctx, bad)
        for bad in (0, 3, 16):
            with pytest.raises(C.ColapmError):
                C.colapm_set_sort_tiles(s.ctx, bad)
    finally:
        s.close()


def test_cell_order_checkpoint_and_async_export(C):
    kw = dict(np=32, nm=64, box=256.0, seed=14, n_steps=8)
    a, b = Sim(C, **kw), Sim(C, **kw)
    try:
        C.colapm_set_sort(a.ctx, 1)
        C.colapm_make_ics(a.ctx)
        C.colapm_step(a.ctx, 5)                       # arrays in cell order here
        buf = C.colapm_save_state(a.ctx)              # saved in id order
        C.colapm_step(a.ctx, 1)                       # sorts again
        C.colapm_load_state(b.ctx, buf)
        C.colapm_step(b.ctx, 1)
        for x, y in zip(a.state(), b.state()):
            assert np.array_equal(x, y)
        import torch
        n = 32 ** 3
        C.colapm_step(a.ctx, 1)
        ref = np.empty((n, 3), np.float32)
        C.colapm_get_particles(a.ctx, ref, None)
        pos = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
        C.colapm_step(b.ctx, 1)
        C.colapm_get_particles_async(a.ctx, pos, None)
        C.colapm_wait_particles(a.ctx)
        assert np.array_equal(pos.numpy(), ref)
        with pytest.raises(C.ColapmError) as e:
            C.colapm_set_sort(a.ctx, -1)
        assert e.value.code == -1
    finally:
        a.close()
        b.close()


# --- error paths and state I/O ----------------------------------------------------------------

def test_error_codes(C):
    with pytest.raises(C.ColapmError) as e:
        C.colapm_create(C.default_params(np=33))
    assert e.value.code == -1
    with pytest.raises(C.ColapmError) as e:
        C.colapm_create(C.default_params(np=64, nm=96))          # nm not a multiple of np
    assert e.value.code == -1
    s = Sim(C, np=16, nm=32)
    try:
        with pytest.raises(C.ColapmError) as e:
            C.colapm_step(s.ctx, 1)                                # before ICs
        assert e.value.code == -6
        with pytest.raises(C.ColapmError) as e:
            C.colapm_get_particles_async(s.ctx, np.empty((16 ** 3, 3), np.float32), None)
        assert e.value.code == -6
        C.colapm_wait_particles(s.ctx)                             # nothing pending: returns at once
        C.colapm_make_ics(s.ctx)
        cell, off, _ = workloads.random_state(16, 32, 1)
        off[10, 1] = 1.0                                          # out of range
        with pytest.raises(C.ColapmError) as e:
            C.colapm_set_state(s.ctx, cell, off, None)
        assert e.value.code == -1
        with pytest.raises(C.ColapmError) as e:
            C.colapm_step(s.ctx, 11)
        assert e.value.code == -6
    finally:
        s.close()


def test_fixed_point_overflow_is_reported(C):
    # 2^18 particles on one node put 2^63 into one cell: the top bit is set and the FFT pass flags it.
    s = Sim(C, np=64, nm=64)
    try:
        C.colapm_make_ics(s.ctx)
        n = 64 ** 3
        C.colapm_set_state(s.ctx, np.zeros((n, 3), np.int32), np.zeros((n, 3), np.float32), None)
        f = np.empty(3 * 64 ** 3, np.float32)
        with pytest.raises(C.ColapmError) as e:
            C.colapm_get_force(s.ctx, f)
        assert e.value.code == -4
    finally:
        s.close()


def test_checkpoint_resume_is_bit_exact(C):
    kw = dict(np=32, nm=64, box=256.0, seed=12)
    a, b = Sim(C, **kw), Sim(C, **kw)
    try:
        C.colapm_make_ics(a.ctx)
        C.colapm_step(a.ctx, 4)
        buf = C.colapm_save_state(a.ctx)
        C.colapm_step(a.ctx, -1)
        C.colapm_load_state(b.ctx, buf)
        assert C.colapm_steps_done(b.ctx) == 4
        C.colapm_step(b.ctx, -1)
        assert np.array_equal(a.density(), b.density())
        sa, sb = a.state(), b.state()
        for x, y in zip(sa, sb):
            assert np.array_equal(x, y)
    finally:
        a.close()
        b.close()


def test_phase_timing_counts(C):
    """Each COLA step runs every step phase once (the x inverse timed on its own); reading clears."""
    s = Sim(C, np=32, nm=64, box=256.0, n_steps=4)
    try:
        C.colapm_set_timing(s.ctx, True)
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, 2)
        ms, n = C.colapm_get_timing(s.ctx)
        assert set(ms) == set(C.PHASES)
        for ph in ("deposit", "fft_fwd", "poisson", "fft_inv", "fft_inv_x", "gather"):
            assert n[ph] == 2 and ms[ph] > 0.0, ph
        assert n["ics"] == 1 and n["power"] == 0
        kd = np.empty(16)
        C.colapm_power(s.ctx, 16, 0.0, 0.0, kd, np.empty(16), np.empty(16, np.int64))
        ms, n = C.colapm_get_timing(s.ctx)
        assert n["power"] == 1 and n["deposit"] == 0 and n["fft_fwd"] == 0   # P(k) timed as one phase
        ms2, n2 = C.colapm_get_timing(s.ctx)
        assert all(v == 0 for v in n2.values()) and all(v == 0.0 for v in ms2.values())
    finally:
        s.close()


def test_async_catalogue_copy_matches_sync(C):
    """colapm_get_particles_async delivers the catalogue of the moment it was called, even when the
    caller steps the particles on before waiting; a second call reuses the staging array."""
    import torch
    s = Sim(C, np=32, nm=64, box=256.0, n_steps=4, seed=5)
    try:
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, 1)
        n = s.np ** 3
        ref_p, ref_m = np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)
        C.colapm_get_particles(s.ctx, ref_p, ref_m)
        pos = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
        mom = torch.empty((n, 3), dtype=torch.float32, pin_memory=True)
        C.colapm_get_particles_async(s.ctx, pos, mom)
        C.colapm_step(s.ctx, 1)                      # moves the particles while the copy may run
        C.colapm_wait_particles(s.ctx)
        assert np.array_equal(pos.numpy(), ref_p) and np.array_equal(mom.numpy(), ref_m)
        ref2_p = np.empty((n, 3), np.float32)
        C.colapm_get_particles(s.ctx, ref2_p, None)
        assert not np.array_equal(ref2_p, ref_p)
        C.colapm_get_particles_async(s.ctx, pos, None)
        C.colapm_wait_particles(s.ctx)
        assert np.array_equal(pos.numpy(), ref2_p)
    finally:
        s.close()



# --- past lightcone (§6) ----------------------------------------------------------------------------

@pytest.mark.parametrize("sort_every,cola_on", [(0, 1), (3, 1), (0, 0)])
def test_lightcone_matches_oracle(C, sort_every, cola_on):
    from oracle import lightcone as olc
    np_, nm, box = 16, 32, 256.0
    origin, z_max, lo, hi = (30.0, 128.0, 200.0), 0.3, (-1, -1, 0), (1, 1, 1)
    s = Sim(C, np=np_, nm=nm, box=box, seed=3, cola=cola_on)
    try:
        C.colapm_set_sort(s.ctx, sort_every)
        C.colapm_set_lightcone(s.ctx, origin, z_max, lo, hi, capacity=200000)
        C.colapm_make_ics(s.ctx)
        g1, g2 = s.lpt()
        C.colapm_step(s.ctx, -1)
        count, rows = C.colapm_get_lightcone(s.ctx)
        assert count == len(rows) > 500
        r = olc.LightconeRun(box, np_, nm, 0.3, 9.0, 0.0, 10, cola=bool(cola_on), origin=origin, z_max=z_max,
                             rep_lo=lo, rep_hi=hi)
        r.set_displacements(g1.astype(np.float64), g2.astype(np.float64))
        r.run()
        ref = r.lightcone()
        # pair the rows of every particle by position; all but a handful of marginal exits agree
        by_id = {}
        for row in ref:
            by_id.setdefault(int(row[7]), []).append(row)
        matched, dpos, da, dmom = 0, [], [], []
        for g in rows:
            cand = by_id.get(int(g["id"]), [])
            if not cand:
                continue
            gp = np.array([g["x"], g["y"], g["z"]], np.float64)
            k = int(np.argmin([np.linalg.norm(c[:3] - gp) for c in cand]))
            c = cand.pop(k)
            matched += 1
            dpos.append(np.linalg.norm(c[:3] - gp))
            da.append(abs(c[3] - g["a"]))
            dmom.append(np.linalg.norm(c[4:7] - [g["px"], g["py"], g["pz"]]) / max(np.linalg.norm(c[4:7]), 1e-3))
        assert len(ref) - matched <= 3 and len(rows) - matched <= 3
        assert np.max(dpos) < 2e-2 and np.median(dpos) < 2e-3      # Mpc/h
        assert np.max(da) < 1e-5
        assert np.median(dmom) < 1e-4
        # a new realisation starts a new lightcone
        C.colapm_make_ics(s.ctx)
        assert C.colapm_get_lightcone(s.ctx)[0] == 0
    finally:
        s.close()


def test_lightcone_capacity_and_arguments(C):
    s = Sim(C, np=16, nm=32, box=256.0, seed=3)
    try:
        with pytest.raises(C.ColapmError) as e:
            C.colapm_get_lightcone(s.ctx)                              # none set
        assert e.value.code == -6
        with pytest.raises(C.ColapmError) as e:
            C.colapm_set_lightcone(s.ctx, (0, 0, 0), -0.5, capacity=10)   # starts after z_final
        assert e.value.code == -1
        C.colapm_set_lightcone(s.ctx, (128.0, 128.0, 128.0), 0.5, (-1, -1, -1), (1, 1, 1), capacity=50)
        C.colapm_make_ics(s.ctx)
        C.colapm_step(s.ctx, -1)
        with pytest.raises(C.ColapmError) as e:
            C.colapm_get_lightcone(s.ctx)
        assert e.value.code == -4                                      # more images than rows
        C.colapm_set_lightcone(s.ctx, None)
    finally:
        s.close()
