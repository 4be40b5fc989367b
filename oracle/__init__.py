"""FP64 CPU oracle for the COLA particle-mesh method (Howlett, Manera & Percival,
"L-PICOLA: A parallel code for fast dark matter simulation").

THIS PACKAGE IS TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py`` may import it. The product
path (``paper_1506_03737_gb300`` and its CUDA library) never imports, links or
calls anything here, and nothing here imports the product path.

It is a plain, slow, obviously correct restatement of what the method computes,
written from the paper's equations in the paper's order and notation:

* ``cosmology`` -- E(a), growth factors D1/D2 (§2.1, Eq. eq:2LPTgrowth and the
  growth ODE they solve), the Kick-Drift-Kick coefficients (§2.3, the Quinn
  integrals and Eq. eq:modifiedt), BBKS linear P(k) with sigma_8 normalisation.
* ``philox`` -- the Philox4x32-10 counter-based generator (Salmon et al. 2011),
  written from its published definition; the GPU path carries its own copy.
* ``fft`` -- its own mixed-radix FFT and a brute-force DFT (§2.4 step 2 uses
  FFTW-3; the oracle does not).
* ``ics`` -- Gaussian field and 2LPT displacements (§2.1, Eqs. za, 2lpt and the
  two Lagrangian-potential Poisson equations; §5).
* ``pm`` -- fixed-point Cloud-in-Cell deposit, Poisson solve with spectral
  gradient and CIC deconvolution, CIC force interpolation (§2.4 steps 1-4).
* ``cola`` -- COLA kick/drift (§2.3, Eqs. eq:vcola and eq:rcola), plain PM
  stepping (Eq. eq:rstandard), the full run.
* ``power`` -- binned periodic-box power spectrum and cross-correlation (§7.1).

Everything is FP64 except where the method itself is defined on integers (the
fixed-point CIC weights and the Philox stream).
"""
