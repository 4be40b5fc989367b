"""GPU vs the FP64 oracle at the sizes the benchmark runs, through the C ABI, default engine.

The 256^3 / 512^3 and 512^3 / 1024^3 workloads run code that the small parity cases do not reach:
the two-stage IC transforms (z-pass modes LPT1 / LPT2 for N_p = 256 and 512), the blocked
power-spectrum binning (N_m = 512, 1024), the blocked force passes on a state with modes off the
axes, mixed-radix meshes of 320 and 384, and cell indices up to 2^30 in the deposit. The oracle
uses numpy's FFT as its transform primitive here (pinned against its own FFT, which is pinned
against the DFT definition); everything else is the same FP64 code as in the small cases.

Where the oracle's whole-mesh arrays would not fit the host, the comparison is on sampled outputs
the oracle computes one region at a time (the deposit at 1024^3), or the test is skipped with the
memory it needs (the full 512^3-particle ICs and the 1024^3 P(k)), never weakened.

Bars as in the small cases: density bit-exact; forces 1e-4 rms relative; Psi1 1e-5 and Psi2
1e-4 rms relative; positions 1e-4 of the rms displacement; P(k) 1e-4 per bin on shared
positions with exact mode counts.
"""
import numpy as np
import pytest

from oracle import cosmology as ocosmo, ics as oics, pm as opm, power as opower
from paper_1506_03737_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def C():
    from paper_1506_03737_gb300 import colapm
    return colapm


def host_gb_available():
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) / 2 ** 20
    return 0.0


def need_host_gb(gb):
    have = host_gb_available()
    if have < gb:
        pytest.skip(f"the FP64 oracle needs about {gb} GB of host memory here, {have:.0f} GB available")


def rel_rms(a, b):
    a = np.asarray(a, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2)) / np.sqrt(np.mean(np.asarray(b, np.float64) ** 2)))


def create(C, **kw):
    return C.colapm_create(C.default_params(**kw))


def state(C, ctx, n):
    cell = np.empty((n, 3), np.int32)
    off = np.empty((n, 3), np.float32)
    C.colapm_get_state(ctx, cell, off, None)
    return cell, off


# --- 2LPT initial conditions with the two-stage transforms ------------------------------------

@pytest.mark.parametrize("name,host_gb", [("cola_256p_512m_512mpc", 12), ("cola_512p_1024m_1024mpc", 90)])
def test_ics_at_full_size(C, name, host_gb):
    need_host_gb(host_gb)
    kw = workloads.run_params(name)
    np_, nm, box, seed = kw["np"], kw["nm"], kw["box"], kw["seed"]
    n = np_ ** 3
    ctx = C.colapm_create(C.default_params(**kw))
    try:
        C.colapm_make_ics(ctx)
        g1 = np.empty(3 * n, np.float32)
        g2 = np.empty(3 * n, np.float32)
        C.colapm_get_lpt(ctx, g1, g2)
        cell, off = state(C, ctx, n)
    finally:
        C.colapm_destroy(ctx)
    pk = ocosmo.linear_pk(kw["omega_m"], kw["h"], kw["n_s"], kw["sigma8"])
    dk = oics.gaussian_field(np_, box, seed, pk)
    psi1, psi2 = oics.lpt_displacements(dk, box, fft="numpy")
    del dk
    g1 = g1.reshape(3, np_, np_, np_)
    g2 = g2.reshape(3, np_, np_, np_)
    for j in range(3):
        assert rel_rms(g1[j], psi1[j]) < 1e-5, j
        assert rel_rms(g2[j], psi2[j]) < 1e-4, j
    # positions x = q + D1(a0) Psi1 + D2(a0) Psi2 (mesh units) against the GPU's cell + offset
    t = ocosmo.timestep_table(kw["omega_m"], kw["z_init"], kw["z_final"], kw["n_steps"])
    d1, d2 = t["D1"][0], t["D2"][0]
    q = oics.lagrangian_grid(np_, box, nm)
    to_mesh = nm / box
    err2 = disp2 = 0.0
    for j in range(3):
        disp = (d1 * psi1[j].ravel() + d2 * psi2[j].ravel()) * to_mesh
        ref = np.mod(q[:, j] * to_mesh + disp, nm)
        d = cell[:, j] + off[:, j].astype(np.float64) - ref
        d -= nm * np.rint(d / nm)
        err2 += float(np.sum(d * d))
        disp2 += float(np.sum(disp * disp))
    assert np.sqrt(err2 / disp2) < 1e-4


# --- power spectrum with the blocked binning ---------------------------------------------------

@pytest.mark.parametrize("name,host_gb", [("cola_256p_512m_512mpc", 24), ("cola_512p_1024m_1024mpc", 190)])
def test_power_at_full_size_on_shared_positions(C, name, host_gb):
    need_host_gb(host_gb)
    kw = workloads.run_params(name)
    np_, nm, box = kw["np"], kw["nm"], kw["box"]
    ctx = C.colapm_create(C.default_params(**kw))
    try:
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, -1)
        k, pk, cnt = C.colapm_power(ctx, 100)
        cell, off = state(C, ctx, np_ ** 3)
    finally:
        C.colapm_destroy(ctx)
    x = (cell + off.astype(np.float64)) * (box / nm)
    del cell, off
    kr, pr, nr = opower.power_from_positions(x, box, np_, nm, 100, fft="numpy")
    assert np.array_equal(cnt, nr)
    ok = nr > 0
    assert np.max(np.abs(pk[ok] / pr[ok] - 1)) < 1e-4
    assert np.max(np.abs(k[ok] / kr[ok] - 1)) < 1e-6


@pytest.mark.parametrize("name,host_gb", [("cola_256p_512m_512mpc", 24), ("cola_512p_1024m_1024mpc", 190)])
def test_redshift_space_power_at_full_size(C, name, host_gb):
    need_host_gb(host_gb)
    kw = workloads.run_params(name)
    np_, nm, box = kw["np"], kw["nm"], kw["box"]
    n = np_ ** 3
    ctx = C.colapm_create(C.default_params(**kw))
    try:
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, -1)
        C.colapm_finalize(ctx)
        k, pk, cnt = C.colapm_power_rsd(ctx, -1, 100)
        cell, off, mom = np.empty((n, 3), np.int32), np.empty((n, 3), np.float32), np.empty((n, 3), np.float32)
        C.colapm_get_state(ctx, cell, off, mom)
    finally:
        C.colapm_destroy(ctx)
    x = (cell + off.astype(np.float64)) * (box / nm)
    del cell, off
    xs = opower.redshift_space(x, mom.astype(np.float64) * (box / nm), 1.0, kw["omega_m"], box, -1)
    del x, mom
    kr, pr, nr = opower.power_from_positions(xs, box, np_, nm, 100, fft="numpy")
    assert np.array_equal(cnt, nr)
    ok = nr > 0
    assert np.max(np.abs(pk[ok] / pr[ok] - 1)) < 1e-4


# --- force on a clustered 3-D state --------------------------------------------------------------

@pytest.mark.parametrize("np_,nm,box", [(256, 512, 512.0), (160, 320, 300.0), (192, 384, 400.0)])
def test_force_on_clustered_state_at_full_size(C, np_, nm, box):
    # Clumps put power in every mode of the mesh (all three indices non-zero), unlike planar slabs.
    need_host_gb(30)
    ctx = create(C, np=np_, nm=nm, box=box)
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
    del cell, off
    ref = opm.force_mesh(opm.density_contrast(rho, np_, nm), box, 1, fft="numpy") * (nm / box)
    for j in range(3):
        assert rel_rms(f[j], ref[j]) < 1e-4, j


# --- deposit at 1024^3 after ten steps --------------------------------------------------------------

def test_deposit_bit_exact_at_1024_after_ten_steps(C):
    """The bench workload after its ten steps (clustered): every cell of several 96^3 regions -- the
    densest one, one straddling the periodic corner (linear cell indices up to 2^30 - 1) and a random
    one -- equals the oracle's deposit of the particles that can reach it, and the whole mesh holds
    exactly N_p^3 particles."""
    need_host_gb(24)
    kw = workloads.run_params("cola_512p_1024m_1024mpc")
    np_, nm = kw["np"], kw["nm"]
    n = np_ ** 3
    ctx = C.colapm_create(C.default_params(**kw))
    try:
        C.colapm_make_ics(ctx)
        C.colapm_step(ctx, -1)
        rho = np.empty(nm ** 3, np.int64)
        C.colapm_get_density(ctx, rho)
        cell, off = state(C, ctx, n)
    finally:
        C.colapm_destroy(ctx)
    assert (rho >= 0).all()
    # exact total mass: the cells are below 2^63, so 32-bit halves sum without overflow in 64 bits
    total = (int((rho >> 32).sum(dtype=np.int64)) << 32) + int((rho & 0xFFFFFFFF).sum(dtype=np.int64))
    assert total == n << 45
    rho = rho.reshape(nm, nm, nm)
    m = 96
    peak = np.unravel_index(int(np.argmax(rho)), rho.shape)[::-1]          # (x, y, z) of the densest cell
    rng = np.random.default_rng(41)
    origins = [tuple((int(c) - m // 2) % nm for c in peak), (nm - m // 2,) * 3,
               tuple(int(v) for v in rng.integers(0, nm, 3))]
    for o in origins:
        # particles whose raw cell lies in [o - 2, o + m + 1] per axis (periodic) reach every cell of
        # [o, o + m - 1]; shift them to a sub-mesh of m + 8 cells, where nothing wraps
        rel = (cell.astype(np.int64) - (np.array(o) - 2)) % nm
        sel = np.all(rel < m + 4, axis=1)
        u = rel[sel] + off[sel].astype(np.float64)
        sub = opm.cic_deposit(u, m + 8)                                   # [z][y][x]
        want = sub[2:m + 2, 2:m + 2, 2:m + 2]
        iz, iy, ix = [(o[a] + np.arange(m)) % nm for a in (2, 1, 0)]
        got = rho[np.ix_(iz, iy, ix)]
        assert np.array_equal(got, want), o
        assert got.sum() > 0
