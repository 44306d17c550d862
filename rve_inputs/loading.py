"""Macroscopic loading histories (inputs of each increment).

Component index c = 3*i + j of the row-major 3x3 tensor.  `mask[c] = 1`
marks a stress-controlled component (its average first Piola-Kirchhoff
stress is prescribed by `Pbar`), `mask[c] = 0` a strain-controlled one (its
average deformation gradient is prescribed by `Fbar`).
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class LoadHistory:
    dt: np.ndarray  # [nsteps]
    Fbar: np.ndarray  # [nsteps][9]
    mask: np.ndarray  # [nsteps][9] uint8
    Pbar: np.ndarray  # [nsteps][9]
    cycle_start: np.ndarray  # [nsteps] bool: FIP accumulators restart here

    @property
    def nsteps(self):
        return int(self.dt.shape[0])

    def head(self, k):
        return LoadHistory(self.dt[:k], self.Fbar[:k], self.mask[:k], self.Pbar[:k], self.cycle_start[:k])


def isochoric(F11):
    """Quasi-uniaxial isochoric macroscopic deformation gradient
    diag(F, F^-1/2, F^-1/2) (Eq. eqFt)."""
    F = np.zeros(9)
    F[0] = F11
    F[4] = F[8] = 1.0 / np.sqrt(F11)
    return F


def cyclic_history(eps, cycles, incr_per_quarter=20, period=4.0):
    """Fully reversed (R = -1) triangular strain cycles of amplitude `eps`:
    F11 = 1 + e(t) with e going 0 -> +eps -> 0 -> -eps -> 0 in each period,
    all nine components strain-controlled."""
    nq = 4 * incr_per_quarter
    n = cycles * nq
    dt = np.full(n, period / nq)
    t = (np.arange(n) + 1) * (period / nq)
    tc = np.mod(t, period) / period  # phase in [0, 1)
    tc[np.isclose(tc, 0.0)] = 0.0
    e = np.where(tc <= 0.25, 4 * tc, np.where(tc <= 0.75, 2 - 4 * tc, 4 * tc - 4)) * eps
    # exact end-of-cycle zeros
    e[np.mod(np.arange(n) + 1, nq) == 0] = 0.0
    Fbar = np.stack([isochoric(1.0 + ei) for ei in e])
    mask = np.zeros((n, 9), dtype=np.uint8)
    Pbar = np.zeros((n, 9))
    cs = np.mod(np.arange(n), nq) == 0
    return LoadHistory(dt, Fbar, mask, Pbar, cs)


def ramp_history(F11_final=1.01, nsteps=5, dt=1.0):
    """F11 ramped linearly from 1 to F11_final in `nsteps` equal steps, the
    other components at zero average stress.  Zero average stress on all
    eight other components leaves a rigid rotation about the loading axis
    free (P(QF) = Q P(F) keeps a uniaxial P when Q turns about x), so F32 is
    held at 0 instead of P32; the solution then has <P32> = 0 as well."""
    Fbar = np.zeros((nsteps, 9))
    Fbar[:, 0] = 1.0 + (F11_final - 1.0) * (np.arange(nsteps) + 1) / nsteps
    Fbar[:, 4] = Fbar[:, 8] = 1.0
    mask = np.ones((nsteps, 9), dtype=np.uint8)
    mask[:, 0] = 0
    mask[:, 7] = 0
    Pbar = np.zeros((nsteps, 9))
    cs = np.zeros(nsteps, dtype=bool)
    cs[0] = True
    return LoadHistory(np.full(nsteps, dt), Fbar, mask, Pbar, cs)
