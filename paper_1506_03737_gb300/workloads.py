"""Named workloads and seeded synthetic inputs.

The workloads are the configurations the library is measured on: flat LCDM with a BBKS
linear spectrum (Omega_m 0.3, h 0.7, n_s 0.96, sigma_8 0.8), 2LPT initial conditions at
z = 9 and 10 modified (nLPT = -2.5) COLA steps linear in a to z = 0. The paper's own runs
use CAMB spectra (§7); the BBKS Gaussian fields stand in for them.

The generators here only draw seeded random inputs (particle states for parity tests);
they hold none of the method's arithmetic.
"""
import numpy as np

COSMO = dict(omega_m=0.3, omega_b=0.05, h=0.7, n_s=0.96, sigma8=0.8)

WORKLOADS = {
    "cola_32p_64m_256mpc": dict(np=32, nm=64, box=256.0, seed=1),
    "cola_256p_512m_512mpc": dict(np=256, nm=512, box=512.0, seed=2),
    "cola_512p_1024m_1024mpc": dict(np=512, nm=1024, box=1024.0, seed=3),
}


def run_params(name, **over):
    """Keyword arguments for ``colapm.default_params`` of a named workload."""
    kw = dict(COSMO)
    kw.update(WORKLOADS[name])
    kw.update(dict(z_init=9.0, z_final=0.0, n_steps=10, spacing=0, stepping=0, nlpt=-2.5, cola=1, deconv=1))
    kw.update(over)
    return kw


def random_state(np_, nm, seed, edge_cases=True):
    """Random particle state: int32 cells (N,3) in [0, nm), float32 offsets (N,3) in [0, 1),
    float32 momenta (N,3). With ``edge_cases`` the first particles sit on nodes, on exact
    half-steps of the 2^-15 grid, just below 1 (rounding up to the next cell) and at the
    last cell (wrapping)."""
    rng = np.random.default_rng(seed)
    n = np_ ** 3
    cell = rng.integers(0, nm, size=(n, 3), dtype=np.int32)
    off = rng.random((n, 3), dtype=np.float32)
    mom = rng.standard_normal((n, 3)).astype(np.float32)
    if edge_cases and n >= 8:
        off[0] = 0.0
        off[1] = np.float32(0.5 / 32768)
        off[2] = np.float32(1.5 / 32768)
        off[3] = np.nextafter(np.float32(1.0), np.float32(0.0))
        off[4] = np.float32(1.0 - 0.5 / 32768)
        cell[5] = nm - 1
        off[5] = np.float32(0.99999)
        cell[6] = 0
        off[7] = np.float32(0.25)
    return cell, off, mom


def clustered_state(np_, nm, seed, frac=0.3, width=2.0):
    """Like ``random_state`` but with a fraction of particles packed in a few dense clumps,
    as in late-time halos."""
    rng = np.random.default_rng(seed)
    cell, off, mom = random_state(np_, nm, seed, edge_cases=False)
    n = cell.shape[0]
    k = int(frac * n)
    centres = rng.uniform(0, nm, size=(8, 3))
    pick = rng.integers(0, 8, size=k)
    pos = np.mod(centres[pick] + rng.normal(0, width, size=(k, 3)), nm)
    c = np.floor(pos).astype(np.int32) % nm
    cell[:k] = c
    off[:k] = np.clip((pos - np.floor(pos)).astype(np.float32), 0, np.nextafter(np.float32(1), np.float32(0)))
    return cell, off, mom
