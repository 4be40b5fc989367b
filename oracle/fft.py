"""Oracle (test infrastructure only): the oracle's own discrete Fourier transforms.

The paper computes its transforms with FFTW-3 (§2.4 step 2, §4.3); the oracle does
not use a library FFT. Convention: forward X[k] = sum_n x[n] exp(-2 pi i k n / N),
inverse with exp(+2 pi i k n / N) and the 1/N applied by ``ifftn``.

``dft_bruteforce`` is the O(N^2) definition; ``fft_axis`` is a textbook recursive
decimation-in-time Cooley-Tukey over the prime factors of N (any N), with twiddle
angles reduced exactly in integers before the trigonometric call.
"""
import numpy as np


def _twiddle(num, n, sign):
    """exp(sign * 2 pi i * num / n) with num reduced modulo n in integer arithmetic."""
    num = np.asarray(num) % n
    return np.exp(sign * 2j * np.pi * (num / n))


def dft_bruteforce(a, axis=-1, sign=-1):
    """Direct O(N^2) DFT along one axis (the definition)."""
    a = np.asarray(a, dtype=np.complex128)
    n = a.shape[axis]
    j = np.arange(n)
    mat = _twiddle(np.outer(j, j), n, sign)
    moved = np.moveaxis(a, axis, -1)
    return np.moveaxis(moved @ mat.T, -1, axis)


def _smallest_prime_factor(n):
    f = 2
    while f * f <= n:
        if n % f == 0:
            return f
        f += 1
    return n


def _ct_last(a, sign):
    """Recursive Cooley-Tukey along the last (contiguous) axis."""
    n = a.shape[-1]
    if n == 1:
        return a.copy()
    r = _smallest_prime_factor(n)
    m = n // r
    subs = [_ct_last(np.ascontiguousarray(a[..., j::r]), sign) for j in range(r)]
    k = np.arange(m)
    out = np.empty(a.shape, dtype=np.complex128)
    for q in range(r):
        acc = np.zeros(a.shape[:-1] + (m,), dtype=np.complex128)
        for j in range(r):
            acc += _twiddle(j * (k + q * m), n, sign) * subs[j]
        out[..., q * m:(q + 1) * m] = acc
    return out


def fft_axis(a, axis=-1, sign=-1):
    """FFT along ``axis`` (unnormalised in both directions)."""
    a = np.asarray(a, dtype=np.complex128)
    moved = np.ascontiguousarray(np.moveaxis(a, axis, -1))
    return np.moveaxis(_ct_last(moved, sign), -1, axis)


def fftn(a):
    """Forward 3-D (or n-D) transform over all axes."""
    out = np.asarray(a, dtype=np.complex128)
    for ax in range(out.ndim):
        out = fft_axis(out, ax, -1)
    return out


def ifftn(a):
    """Inverse n-D transform including the 1/N^d normalisation."""
    out = np.asarray(a, dtype=np.complex128)
    for ax in range(out.ndim):
        out = fft_axis(out, ax, +1)
    return out / out.size
