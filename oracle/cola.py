"""Oracle (test infrastructure only): COLA and plain-PM Kick-Drift-Kick stepping (§2.2-§2.3).

COLA (Eq. eq:cola) splits the motion into the stored LPT displacements scaled by
the growth factors and a residual, and discretises the residual with the kick and
drift of Eqs. eq:vcola and eq:rcola:

    p_res <- p_res + K_i [F(x_i) - D1(a_i) Psi1 - (D2(a_i) - D1(a_i)^2) Psi2]
    x     <- x + S_i p_res + (D1(a_{i+1}) - D1(a_i)) Psi1 + (D2(a_{i+1}) - D2(a_i)) Psi2

with K_i (which includes 1.5 Om) and S_i from ``cosmology.timestep_table``. The
bracket is -T[Psi_res] of §2.3 per unit 1.5 Om/(a^2 E): the LPT terms are the
accelerations the growth ODEs give the two LPT modes. The residual momentum starts
at zero (§2.3: the initial velocity is that of the LPT frame, removed before the
first step and added back at the end).

Plain PM (COLA switched off, §7.1) uses the same loop with the LPT terms dropped
(Eqs. eq:vcola with grad(phi) and eq:rstandard), starting from the 2LPT momentum
p = P1(a0) Psi1 + P2(a0) Psi2.

Positions are FP64 in Mpc/h, wrapped into [0, L).
"""
import numpy as np

from . import cosmology, ics, pm


def wrap(x, box):
    """Periodic wrap into [0, L): np.mod returns L itself for tiny negative x, which is mapped to 0."""
    x = np.mod(x, box)
    x[x >= box] -= box
    return x


class Run:
    """State of one simulation in the oracle (all FP64, particle-id order)."""

    def __init__(self, box, np_, nm, om, z_init, z_final, n_steps, spacing="lin",
                 stepping="modified", nlpt=-2.5, cola=True, deconv=1, fft=None):
        """fft="numpy": numpy's FFT as the transform primitive (large meshes); same operators."""
        self.fft = fft
        self.box, self.np_, self.nm = float(box), int(np_), int(nm)
        self.om, self.cola, self.deconv = float(om), bool(cola), int(deconv)
        self.stepping, self.nlpt = stepping, nlpt
        self.table = cosmology.timestep_table(om, z_init, z_final, n_steps, spacing, stepping, nlpt)
        self.n_steps = int(n_steps)
        self.step_index = 0
        self.x = self.p = self.psi1 = self.psi2 = self.q = None

    # --- initial conditions (§5) ------------------------------------------------------
    def set_displacements(self, psi1, psi2):
        """psi1, psi2: (3, N_p, N_p, N_p) fields in Mpc/h on the Lagrangian grid."""
        t = self.table
        self.q = ics.lagrangian_grid(self.np_, self.box, self.nm)
        self.psi1 = ics.per_particle(psi1)
        self.psi2 = ics.per_particle(psi2)
        self.x = wrap(self.q + t["D1"][0] * self.psi1 + t["D2"][0] * self.psi2, self.box)
        if self.cola:
            self.p = np.zeros_like(self.x)
        else:
            self.p = t["P1"][0] * self.psi1 + t["P2"][0] * self.psi2
        self.step_index = 0

    def make_ics(self, seed, pk):
        delta_k = ics.gaussian_field(self.np_, self.box, seed, pk)
        psi1, psi2 = ics.lpt_displacements(delta_k, self.box, self.fft)
        self.set_displacements(psi1, psi2)
        return delta_k

    # --- one Kick-Drift step ------------------------------------------------------------
    def force(self):
        f, _ = pm.pm_accel(self.x, self.box, self.np_, self.nm, self.deconv, self.fft)
        return f

    def kick(self, coeff, d1, d2, force):
        acc = force
        if self.cola:
            acc = force - d1 * self.psi1 - (d2 - d1 * d1) * self.psi2
        self.p = self.p + coeff * acc

    def step(self):
        t, i = self.table, self.step_index
        force = self.force()
        self.kick(t["kick"][i], t["D1"][i], t["D2"][i], force)
        dx = t["drift"][i] * self.p
        if self.cola:
            dx = dx + t["dD1"][i] * self.psi1 + t["dD2"][i] * self.psi2
        self.x = wrap(self.x + dx, self.box)
        self.step_index += 1
        return force

    def run(self, k=None):
        k = self.n_steps - self.step_index if k is None else k
        for _ in range(k):
            self.step()

    def finalize(self):
        """Closing half kick to a_N, then total momentum p = p_res + P1 Psi1 + P2 Psi2 (COLA) (§2.3)."""
        t = self.table
        n = self.n_steps
        force = self.force()
        self.kick(t["kick_final"], t["D1"][n], t["D2"][n], force)
        if self.cola:
            return self.p + t["P1"][n] * self.psi1 + t["P2"][n] * self.psi2
        return self.p.copy()

    def displacement(self):
        """x - q with the minimum-image convention."""
        d = self.x - self.q
        return d - self.box * np.rint(d / self.box)
