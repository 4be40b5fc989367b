"""Oracle (test infrastructure only): the past lightcone built during the run (§6).

An observer sits at `origin` (Mpc/h); the lightcone radius at scale factor a is the comoving
distance R_L(a) = c int_a^1 da' / (a'^2 H(a')) (Mpc/h with H0 = 100 h km/s/Mpc). The box may be
replicated: every particle has images x + R L for integer vectors R in the given ranges. From the
first step boundary at or after a(z_max) on, an image leaves the lightcone during the drift from
a_i to a_{i+1} when R_p,i <= R_L,i and R_p,i+1 > R_L,i+1 (R_p its distance to the origin). Its exit
time is the linear interpolation of both radii across the step (Eq. eq:lightconeinterp):

    a_L = a_i + (a_{i+1} - a_i)(R_L,i - R_p,i) / ((R_p,i+1 - R_p,i) - (R_L,i+1 - R_L,i))

and it is output at the position the COLA drift gives at a_L (the drift of Eq. eq:rcola with every
coefficient taken over [a_i, a_L]) with the momentum of the kick-drift-kick step (the residual
momentum at a_{i+1/2}) plus, for COLA, the LPT frame momentum P1(a_L) Psi1 + P2(a_L) Psi2.
The trajectory of an image is continuous across the drift (no periodic wrap inside a step).
"""
import numpy as np
from scipy import integrate

from . import cola, cosmology

HUBBLE_DISTANCE = 2997.92458   # c / H0 in Mpc/h


def comoving_distance(a, om):
    """R_L(a) = (c / H0) int_a^1 da' / (a'^2 E(a')), Mpc/h."""
    def f(x):
        return 1.0 / (x * x * cosmology.hubble_e(x, om))
    val, _ = integrate.quad(f, a, 1.0, epsabs=0.0, epsrel=1e-13, limit=200)
    return HUBBLE_DISTANCE * val


def replicate_offsets(rep_lo, rep_hi):
    """Integer replicate vectors R with rep_lo[j] <= R_j <= rep_hi[j]."""
    r = [np.arange(rep_lo[j], rep_hi[j] + 1) for j in range(3)]
    g = np.meshgrid(*r, indexing="ij")
    return np.stack([x.ravel() for x in g], axis=1)


class LightconeRun(cola.Run):
    """A run that records the lightcone: `origin` (3,) Mpc/h, `z_max` the redshift where it starts,
    replicate ranges rep_lo, rep_hi (3 ints each). `out` holds rows (x, y, z, a_L, px, py, pz, id)."""

    def __init__(self, *args, origin=(0.0, 0.0, 0.0), z_max=1.0, rep_lo=(0, 0, 0), rep_hi=(0, 0, 0), **kw):
        super().__init__(*args, **kw)
        self.origin = np.asarray(origin, dtype=np.float64)
        a = self.table["a"]
        a_start = 1.0 / (1.0 + z_max)
        self.first = int(np.searchsorted(a, a_start - 1e-12))    # first step boundary at or after it
        self.reps = replicate_offsets(rep_lo, rep_hi)
        self.out = []

    def step(self):
        t, i = self.table, self.step_index
        force = self.force()
        self.kick(t["kick"][i], t["D1"][i], t["D2"][i], force)
        dx = t["drift"][i] * self.p
        if self.cola:
            dx = dx + t["dD1"][i] * self.psi1 + t["dD2"][i] * self.psi2
        if i >= self.first:
            self._record(i, dx)
        self.x = cola.wrap(self.x + dx, self.box)
        self.step_index += 1
        return force

    def _record(self, i, dx):
        t = self.table
        a0, a1 = t["a"][i], t["a"][i + 1]
        rl0, rl1 = comoving_distance(a0, self.om), comoving_distance(a1, self.om)
        hits = []   # (particle, a_L, replicate)
        for rep in self.reps:
            r0 = self.x + rep * self.box - self.origin
            rp0 = np.sqrt(np.sum(r0 * r0, axis=1))
            r1 = r0 + dx
            rp1 = np.sqrt(np.sum(r1 * r1, axis=1))
            for p in np.flatnonzero((rp0 <= rl0) & (rp1 > rl1)):
                al = a0 + (a1 - a0) * (rl0 - rp0[p]) / ((rp1[p] - rp0[p]) - (rl1 - rl0))
                hits.append((p, al, rep))
        if hits:
            self._exit_states(i, hits)

    def _exit_states(self, i, hits):
        """Positions and momenta of the images at their exit times within step i (§6, Eq. 16)."""
        t = self.table
        a0, amid = t["a"][i], t["a_half"][i]
        als = np.array([h[1] for h in hits])
        d1, d2, p1, p2 = cosmology.growth(als, self.om)
        for k, (p, al, rep) in enumerate(hits):
            s = cosmology.drift_coeff(a0, al, amid, self.om, self.stepping, self.nlpt)
            x = self.x[p] + s * self.p[p]
            mom = self.p[p].copy()
            if self.cola:
                x = x + (d1[k] - t["D1"][i]) * self.psi1[p] + (d2[k] - t["D2"][i]) * self.psi2[p]
                mom = mom + p1[k] * self.psi1[p] + p2[k] * self.psi2[p]
            self.out.append(np.concatenate([x + rep * self.box, [al], mom, [p]]))

    def lightcone(self):
        """(N, 8) array of the output rows, sorted by (id, x, y, z)."""
        if not self.out:
            return np.zeros((0, 8))
        o = np.array(self.out)
        return o[np.lexsort((o[:, 2], o[:, 1], o[:, 0], o[:, 7]))]
