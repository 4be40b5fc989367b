"""Oracle (test infrastructure only): Gaussian initial field and 2LPT displacements.

§5: the initial-conditions generator computes the first- and second-order
Lagrangian displacements at the points of a uniform particle grid. §2.1: with
x = q - D1 grad(phi1) + D2 grad(phi2), lap(phi1) = delta_L and
lap(phi2) = sum_{i>j} (phi1_ii phi1_jj - phi1_ij^2). Hence, with the convention
f(x) = (1/N^3) sum_k f_k exp(i k.x) (so grad -> i k, lap -> -k^2):

    Psi1_k   =  i k delta_k / k^2          (Psi1 = -grad phi1, div Psi1 = -delta_L: Eq. za)
    phi_ij,k =  k_i k_j delta_k / k^2      (second derivatives of phi1)
    S        =  sum_{i>j} (phi_ii phi_jj - phi_ij^2)   in real space
    Psi2_k   = -i k S_k / k^2              (Psi2 = +grad phi2)

and x = q + D1 Psi1 + D2 Psi2 with D2 < 0. Every spectral multiplier is zero at
k = 0 and on modes with any index at the Nyquist frequency N/2.

Gaussian field: for each mode of the half grid (k_x index in [0, N/2)), one
Philox4x32-10 draw keyed by (seed) with counter = full-grid mode index
m = ix + N (iy + N iz) gives two uniforms u1, u2; Box-Muller gives
g = sqrt(-2 ln u1) exp(2 pi i u2) / sqrt(2), and delta_k = N^3 sqrt(P(k)/L^3) g, so
<|delta_k|^2> = N^6 P(k) / L^3. On the k_x = 0 plane the mode with the larger
index of each conjugate pair is the conjugate of its partner.
"""
import math

import numpy as np

from .fft import fftn, ifftn
from .philox import MASK, philox4x32_10, uniform_open


def signed_index(n):
    """Signed wavenumber index of FFT bin i: i for i < n/2, i - n otherwise."""
    i = np.arange(n)
    return np.where(i < n // 2, i, i - n)


def wavevectors(n, box):
    """Return (kx, ky, kz, nyq) on the full [z][y][x] grid, k in h/Mpc; nyq marks any index == N/2."""
    s = signed_index(n).astype(np.float64)
    kf = 2.0 * math.pi / box
    kz, ky, kx = np.meshgrid(s * kf, s * kf, s * kf, indexing="ij")
    i = np.arange(n)
    ny1 = (i == n // 2) if n % 2 == 0 else np.zeros(n, bool)
    nz_, ny_, nx_ = np.meshgrid(ny1, ny1, ny1, indexing="ij")
    return kx, ky, kz, (nz_ | ny_ | nx_)


def mode_uniforms(n, seed):
    """(u1, u2) for every mode of the half grid [iz][iy][ix], ix < N/2."""
    h = n // 2
    iz, iy, ix = np.meshgrid(np.arange(n, dtype=np.uint64), np.arange(n, dtype=np.uint64),
                             np.arange(h, dtype=np.uint64), indexing="ij")
    m = (iz * np.uint64(n) + iy) * np.uint64(n) + ix
    s = np.uint64(seed)
    r0, r1, _, _ = philox4x32_10(m & MASK, m >> np.uint64(32), 0, 0, s & MASK, s >> np.uint64(32))
    return uniform_open(r0), uniform_open(r1)


def gaussian_field(n, box, seed, pk):
    """Full complex N^3 array delta_k [iz][iy][ix] of a Hermitian Gaussian field with power P(k)."""
    h = n // 2
    u1, u2 = mode_uniforms(n, seed)
    g = np.sqrt(-2.0 * np.log(u1)) * np.exp(2j * math.pi * u2) / math.sqrt(2.0)

    s = signed_index(n)
    nz, ny, nx = np.meshgrid(s, s, s[:h], indexing="ij")
    n2 = (nx * nx + ny * ny + nz * nz).astype(np.float64)
    k = 2.0 * math.pi * np.sqrt(n2) / box
    with np.errstate(divide="ignore", invalid="ignore"):
        amp = n ** 3 * np.sqrt(np.where(n2 > 0, pk(np.where(n2 > 0, k, 1.0)), 0.0) / box ** 3)
    half = amp * g
    i = np.arange(n)
    iz, iy = np.meshgrid(i, i, indexing="ij")
    nyq_plane = (iz == h) | (iy == h)
    half[nyq_plane] = 0.0

    # Hermitian symmetry on the kx = 0 plane.
    pz, py = (n - iz) % n, (n - iy) % n
    m_self = iz * n + iy
    m_part = pz * n + py
    non_canon = m_self > m_part
    plane = half[:, :, 0].copy()
    plane[non_canon] = np.conj(plane[pz[non_canon], py[non_canon]])
    half[:, :, 0] = plane

    full = np.zeros((n, n, n), dtype=np.complex128)
    full[:, :, :h] = half
    xs = np.arange(h + 1, n)
    neg = (-i) % n
    full[:, :, h + 1:] = np.conj(full[np.ix_(neg, neg, n - xs)])
    return full


# Hubble distance c / H0 in Mpc/h (H0 = 100 h km/s/Mpc, c = 299792.458 km/s).
HUBBLE_DISTANCE = 2997.92458


def potential_to_density(n, box, om, h, d_md):
    """M(k) on the full [z][y][x] grid: delta_k(z = 0) = M(k) Phi_k for the primordial potential Phi
    in matter domination (the Poisson equation with the transfer function and the growth from the
    matter era to z = 0): M = (2/3) (k c / H0)^2 T_BBKS(k) d_md / Om, with d_md the z = 0 growth
    factor normalised to a in matter domination. Zero at k = 0. Sign: Phi and delta have the same
    sign (Phi is minus the Newtonian potential, the convention in which f_NL > 0 skews the density
    positively)."""
    from .cosmology import t_bbks
    kx, ky, kz, _ = wavevectors(n, box)
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    m = np.zeros_like(k)
    ok = k > 0
    m[ok] = 2.0 / 3.0 * (k[ok] * HUBBLE_DISTANCE) ** 2 * t_bbks(k[ok], om, h) * d_md / om
    return m


def local_fnl_field(delta_k, box, fnl, om, h, d_md, fft=None):
    """Local primordial non-Gaussianity (§5): the Gaussian field delta_k = M phi_k defines the Gaussian
    potential phi; in real space Phi = phi + f_NL (phi^2 - <phi^2>) (<> the box average), and the
    initial density is M Phi_k, zero at k = 0 and on the Nyquist planes. f_NL = 0 returns delta_k."""
    fftn_, ifftn_ = (np.fft.fftn, np.fft.ifftn) if fft == "numpy" else (fftn, ifftn)
    n = delta_k.shape[0]
    m = potential_to_density(n, box, om, h, d_md)
    phi_k = np.zeros_like(delta_k)
    ok = m > 0
    phi_k[ok] = delta_k[ok] / m[ok]
    phi = ifftn_(phi_k).real
    big_phi = phi + fnl * (phi * phi - np.mean(phi * phi))
    out = m * fftn_(big_phi)
    _, _, _, nyq = wavevectors(n, box)
    out[nyq] = 0.0
    return out


def lpt_displacements(delta_k, box, fft=None):
    """Return (Psi1, Psi2), each (3, N, N, N) real [component x,y,z][iz][iy][ix], in Mpc/h.

    fft="numpy" takes numpy's FFT as the transform primitive (large grids); the operators are the same."""
    fftn_, ifftn_ = (np.fft.fftn, np.fft.ifftn) if fft == "numpy" else (fftn, ifftn)
    kx, ky, kz, nyq = wavevectors(delta_k.shape[0], box)
    kvec = (kx, ky, kz)
    k2 = kx * kx + ky * ky + kz * kz
    inv = np.zeros_like(k2)
    ok = (k2 > 0) & ~nyq
    inv[ok] = 1.0 / k2[ok]

    psi1 = np.stack([ifftn_(1j * kvec[j] * delta_k * inv).real for j in range(3)])
    phi = {}
    for a in range(3):
        for b in range(a, 3):
            phi[a, b] = ifftn_(kvec[a] * kvec[b] * delta_k * inv).real
    src = (phi[0, 0] * phi[1, 1] + phi[0, 0] * phi[2, 2] + phi[1, 1] * phi[2, 2]
           - phi[0, 1] ** 2 - phi[0, 2] ** 2 - phi[1, 2] ** 2)
    src_k = fftn_(src)
    psi2 = np.stack([ifftn_(-1j * kvec[j] * src_k * inv).real for j in range(3)])
    return psi1, psi2


def lagrangian_grid(n, box, nm=None):
    """q for particle id p = ix + N (iy + N iz), shape (N^3, 3), columns (x, y, z), Mpc/h.

    The lattice of spacing L/N is offset by half a PM cell, L/(2 N_m), from the mesh nodes
    (§5 places the particles on a uniform grid without fixing its offset). On a node the CIC
    kernel has its kink, and with N_m = 2 N_p a node-centred lattice resonates with the
    2-cell ringing of the Nyquist-truncated force kernel.
    """
    nm = n if nm is None else nm
    i = (np.arange(n, dtype=np.float64) + 0.5 * n / nm) * (box / n)
    qz, qy, qx = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)


def per_particle(field):
    """(3, N, N, N) displacement field -> (N^3, 3) in particle-id order."""
    return np.stack([field[j].ravel() for j in range(3)], axis=1)
