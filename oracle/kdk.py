"""Adaptive Kick-Drift-Kick stepping (Sec. 3.4), oracle side.

Test infrastructure only (see the package docstring).  Plain numpy in
float64, written from the paper's description:

* Drift D(t1; t2): x += p * int_{t1}^{t2} dt / a^2;
  Kick  K(t1; t2): p += (-grad phi) * int_{t1}^{t2} dt / a
  (the symplectic pair of operators of the cosmic scheme the paper adopts).
* KDK: a half-step kick, a full-step drift, a half-step kick.
* Adaptive steps: a particle's step must not exceed
  t_acc = sqrt(2 eta eps / |a|); a step that is too long is halved, so every
  step is the top step divided by a power of two (its level), and particles
  of different levels meet at the ends of the coarser steps.

Readings taken here (the paper is silent or garbled on each):

* Criterion.  The printed form 2 eta eps / sqrt(|a|) is dimensionally
  garbled; the criterion is Gadget-2's t_acc = sqrt(2 eta eps / |a|).  The
  level of a particle is the smallest k in [0, max_level] with
  (dt / 2^k)^2 |a| <= 2 eta eps (max_level when none), decided in FP64 as
  written: lhs = dt * dt * |a|, then lhs *= 0.25 per level.
* Block steps.  One top step of length dt is an integer timeline of
  T = 2^max_level ticks.  A particle on level k has steps of T / 2^k ticks.
  At the top step's start every particle takes its level from its current
  acceleration and an opening half kick.  Then, event by event (the
  earliest end of any particle's current step): all particles drift to the
  event (velocities are constant between kicks), the force is recomputed
  for all, the particles whose step ends there take their closing half
  kick and, unless the top step is over, a new level (refined until its
  step length divides the elapsed ticks, so steps stay aligned) and an
  opening half kick.
* Force.  The total force of the split: the short-range PP sum
  (``force.accel``) plus, with a mesh, the long-range PM part
  (``pm.accel``).
* Clocks.  Newtonian: the time variable is t, drift and kick factors are
  t2 - t1.  Flat Lambda-CDM: the time variable is the scale factor a,
  D = int da / (a^3 H(a)), K = int da / (a^2 H(a)),
  H(a) = H0 sqrt(Omega_m a^-3 + Omega_L); the criterion's t_acc is
  converted to a step in a by multiplying with a H(a) at the step's start.
* Positions stay in [0, L): after each drift a coordinate outside the box
  becomes x - L floor(x / L) (a result equal to L maps to 0).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate

from . import force, pm

CLOCK_NEWTON = 0
CLOCK_LCDM = 1


class Clock:
    """Drift and kick factors of the time variable."""

    def __init__(self, kind=CLOCK_NEWTON, H0=1.0, omega_m=1.0, omega_l=0.0):
        self.kind, self.H0, self.om, self.ol = kind, H0, omega_m, omega_l

    def hubble(self, a):
        return self.H0 * math.sqrt(self.om / a ** 3 + self.ol)

    def drift(self, t1, t2):
        if self.kind == CLOCK_NEWTON or t1 == t2:
            return t2 - t1
        return integrate.quad(lambda a: 1.0 / (a ** 3 * self.hubble(a)), t1, t2, epsabs=0, epsrel=1e-13)[0]

    def kick(self, t1, t2):
        if self.kind == CLOCK_NEWTON or t1 == t2:
            return t2 - t1
        return integrate.quad(lambda a: 1.0 / (a ** 2 * self.hubble(a)), t1, t2, epsabs=0, epsrel=1e-13)[0]

    def step_scale(self, t):
        """Factor from a physical time step to a step of the time variable."""
        return 1.0 if self.kind == CLOCK_NEWTON else t * self.hubble(t)


def step_levels(acc, dt, eta, eps, max_level):
    """Level of each particle: smallest k <= max_level with
    (dt / 2^k)^2 |a| <= 2 eta eps (Gadget-2's t_acc criterion)."""
    acc = np.asarray(acc, np.float64)
    amag = np.sqrt(acc[:, 0] * acc[:, 0] + acc[:, 1] * acc[:, 1] + acc[:, 2] * acc[:, 2])
    lhs = dt * dt * amag
    thr = 2.0 * eta * eps
    k = np.zeros(len(amag), np.int64)
    for _ in range(max_level):
        more = lhs > thr
        if not more.any():
            break
        k[more] += 1
        lhs = np.where(more, lhs * 0.25, lhs)
    return k


def wrap(x, L):
    inside = (x >= 0.0) & (x < L)
    xw = np.where(inside, x, x - L * np.floor(x / L))
    return np.where(xw >= L, 0.0, xw)


class Sim:
    """Particles advanced by adaptive KDK block steps under the split force."""

    def __init__(self, pos, mom, mass, L, G, eps, rs, rcut, n_mesh, dt, eta, max_level, t0=0.0,
                 clock: Clock | None = None, eps_step=None):
        self.x = wrap(np.array(pos, np.float64), L)
        self.p = np.array(mom, np.float64)
        self.m = np.asarray(mass, np.float64)
        self.L, self.G, self.eps, self.rs, self.rcut, self.n_mesh = L, G, eps, rs, rcut, n_mesh
        self.dt, self.eta, self.max_level = dt, eta, max_level
        self.eps_step = eps if eps_step is None else eps_step
        self.t = t0
        self.clock = clock or Clock()
        self.force_passes = 0
        self.level = np.zeros(len(self.x), np.int64)
        self.acc = self.total_force(self.x)

    def total_force(self, x):
        """Short-range PP plus (n_mesh > 0) long-range PM acceleration."""
        self.force_passes += 1
        a = force.accel(x, self.m, self.L, self.G, self.eps, self.rs, self.rcut).acc
        if self.n_mesh:
            a = a + pm.accel(x, self.m, self.L, self.G, self.rs, self.n_mesh).acc
        return a

    def _levels(self, t):
        """Levels from the current accelerations at time t: the criterion's
        physical step is dt / (a H) in the Lambda-CDM clock."""
        return step_levels(self.acc, self.dt / self.clock.step_scale(t), self.eta, self.eps_step, self.max_level)

    def top_step(self):
        """One top step of length dt (Sec. 3.4's KDK with halved steps)."""
        T = 1 << self.max_level
        h = self.dt / T
        t0 = self.t
        tt = lambda tick: t0 + tick * h        # noqa: E731
        k = self._levels(t0)
        start = np.zeros(len(self.x), np.int64)
        for lv in np.unique(k):
            sel = k == lv
            self.p[sel] += self.acc[sel] * self.clock.kick(t0, tt((T >> lv) / 2))
        tick = 0
        while tick < T:
            nxt = int(np.min(start + (T >> k)))
            self.x = wrap(self.x + self.p * self.clock.drift(tt(tick), tt(nxt)), self.L)
            tick = nxt
            self.acc = self.total_force(self.x)
            ending = start + (T >> k) == tick
            for lv in np.unique(k[ending]):
                sel = ending & (k == lv)
                self.p[sel] += self.acc[sel] * self.clock.kick(tt(tick - (T >> lv) / 2), tt(tick))
            if tick < T:
                kn = self._levels(tt(tick))
                kn = np.where(ending, kn, k)
                while True:
                    bad = ending & (tick % (T >> kn) != 0)
                    if not bad.any():
                        break
                    kn = np.where(bad, kn + 1, kn)
                k = kn
                start = np.where(ending, tick, start)
                for lv in np.unique(k[ending]):
                    sel = ending & (k == lv)
                    self.p[sel] += self.acc[sel] * self.clock.kick(tt(tick), tt(tick + (T >> lv) / 2))
        self.level = k
        self.t = t0 + self.dt
