"""Oracle (test infrastructure only): the particle-mesh force of §2.4.

Steps (§2.4): (1) Cloud-in-Cell assignment of the particles to an N_m^3 mesh;
(2) FFT of the density contrast and the comoving Poisson equation in Fourier space;
(3) spectral gradient, deconvolution of the CIC window, inverse FFT per axis;
(4) CIC interpolation of the mesh force back to each particle.

Mesh nodes sit at integer multiples of the cell size Delta = L / N_m; arrays are
[iz][iy][ix]. A particle at mesh coordinate u = x / Delta has base cell floor(u)
and fraction f = u - floor(u) per axis.

Fixed-point CIC (the definition shared by the oracle and the GPU path): the
fraction is quantised as f_q = rint(f * 2^15) (round half to even); if f_q = 2^15
the base cell moves up by one and f_q = 0. The axis weights are (2^15 - f_q, f_q)
and a corner's weight is their int64 product (scale 2^45), so the total mass on the
mesh is exactly N_p^3 * 2^45. The gather uses the same quantised weights / 2^45, so
deposit and interpolation share one stencil (which is what makes the self-force vanish).

Poisson (§2.4 step 2, and the grad(Phi) expression of §2.2): with
delta = rho * (N_m/N_p)^3 * 2^-45 - 1, the mesh force F = -grad(psi), lap(psi) = delta,
is F_j(k) = i k_j delta_k / (k^2 W(k)^d), W(k) = prod_i sinc^2(pi n_i / N_m), where
d = 1 deconvolves the CIC window once (§2.4 step 3; d = 0 and d = 2 are options).
F is zero at k = 0 and on every mode with any index at N_m/2. The factor
1.5 Om_m0 / a of the paper's Poisson equation is carried by the kick coefficient.
"""
import math

import numpy as np

from .fft import fft_axis, fftn, ifftn
from .ics import wavevectors, signed_index

QBITS = 15
QONE = 1 << QBITS


def quantise(u, nm):
    """Fixed-point CIC base cell (int64, (P,3)) and fraction f_q in [0, 2^15) from mesh coords u (P,3)."""
    u = np.asarray(u, dtype=np.float64)
    c = np.floor(u).astype(np.int64)
    fq = np.rint((u - c) * QONE).astype(np.int64)
    carry = fq == QONE
    c[carry] += 1
    fq[carry] = 0
    return c % nm, fq


def _corners(c, fq, nm):
    """Yield (flat mesh index, int64 weight) for the 8 CIC corners."""
    w = [(QONE - fq), fq]
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                idx = ((((c[:, 2] + dz) % nm) * nm + (c[:, 1] + dy) % nm) * nm + (c[:, 0] + dx) % nm)
                yield idx, w[dx][:, 0] * w[dy][:, 1] * w[dz][:, 2]


def cic_deposit(u, nm):
    """int64 fixed-point CIC mass on the N_m^3 mesh, [iz][iy][ix] (§2.4 step 1)."""
    c, fq = quantise(u, nm)
    rho = np.zeros(nm ** 3, dtype=np.int64)
    for idx, w in _corners(c, fq, nm):
        np.add.at(rho, idx, w)
    return rho.reshape(nm, nm, nm)


def density_contrast(rho, np_, nm):
    """delta = rho * (N_m/N_p)^3 * 2^-45 - 1 in FP64."""
    return rho.astype(np.float64) * (float(nm) / np_) ** 3 * 2.0 ** -45 - 1.0


def cic_window(nm):
    """W(n) = prod_i sinc^2(pi n_i / N_m) on the full [z][y][x] grid."""
    s = signed_index(nm).astype(np.float64)
    x = math.pi * s / nm
    with np.errstate(divide="ignore", invalid="ignore"):
        sinc = np.where(s == 0, 1.0, np.sin(x) / np.where(s == 0, 1.0, x))
    s2 = sinc * sinc
    wz, wy, wx = np.meshgrid(s2, s2, s2, indexing="ij")
    return wx * wy * wz


def force_mesh(delta, box, deconv=1, fft=None):
    """Three real meshes F_j = -d psi / d x_j (Mpc/h), lap psi = delta (§2.4 steps 2-3).

    fft="numpy" takes numpy's FFT as the transform primitive (for meshes where the oracle's own
    FFT, pinned against the DFT definition, is too slow); the operator is the same."""
    nm = delta.shape[0]
    kx, ky, kz, nyq = wavevectors(nm, box)
    k2 = kx * kx + ky * ky + kz * kz
    mult = np.zeros_like(k2)
    ok = (k2 > 0) & ~nyq
    win = cic_window(nm) ** deconv
    mult[ok] = 1.0 / (k2[ok] * win[ok])
    fwd, inv = (np.fft.fftn, np.fft.ifftn) if fft == "numpy" else (fftn, ifftn)
    dk = fwd(delta)
    return np.stack([inv(1j * kv * dk * mult).real for kv in (kx, ky, kz)])


def planar_force_1d(delta_1d, box, deconv=1):
    """Force along the axis of a density that varies along one axis only (§2.4 steps 2-3 reduced
    to one dimension: only modes with the other two indices zero are present, so k^2 = k_a^2 and
    the CIC window is the single factor sinc^2(pi n_a / N); the Nyquist index is excluded)."""
    nm = delta_1d.shape[0]
    s = signed_index(nm).astype(np.float64)
    k = s * 2.0 * math.pi / box
    x = math.pi * s / nm
    with np.errstate(divide="ignore", invalid="ignore"):
        sinc = np.where(s == 0, 1.0, np.sin(x) / np.where(s == 0, 1.0, x))
    win = (sinc * sinc) ** deconv
    mult = np.zeros(nm)
    ok = (s != 0) & (np.arange(nm) != nm // 2)
    mult[ok] = 1.0 / (k[ok] * k[ok] * win[ok])
    dk = fft_axis(np.asarray(delta_1d, dtype=np.complex128), 0, -1)
    return (fft_axis(1j * k * dk * mult, 0, +1) / nm).real


def cic_gather(force, u):
    """Interpolate the (3, N, N, N) mesh force to mesh coordinates u (P,3) with the deposit stencil (§2.4 step 4)."""
    nm = force.shape[1]
    c, fq = quantise(u, nm)
    out = np.zeros((u.shape[0], 3))
    flat = force.reshape(3, -1)
    for idx, w in _corners(c, fq, nm):
        wf = w.astype(np.float64) * 2.0 ** -45
        for j in range(3):
            out[:, j] += wf * flat[j][idx]
    return out


def pm_accel(x, box, np_, nm, deconv=1, fft=None):
    """Mesh force F (Mpc/h) at particle positions x (Mpc/h, (P,3)), and the int64 density used."""
    u = np.mod(np.asarray(x, dtype=np.float64) * (nm / box), nm)
    rho = cic_deposit(u, nm)
    force = force_mesh(density_contrast(rho, np_, nm), box, deconv, fft)
    return cic_gather(force, u) , rho
