"""Observables of the paper's results section (Sec. 5) from the library's measurements.

Host arithmetic on measurement outputs only (the measurements themselves run on
the GPU: ``Ensemble.sweep(qhist=...)`` / ``Ensemble.measure`` and
``Ensemble.measure_planes``).  Definitions (standard; the paper shows the
curves without printing the formulas):

* overlap of site i between the two copies: q_i = S^1_i S^2_i, q = (1/N) sum_i q_i;
  a measurement with n differing sites has q = 1 - 2 n / N;
* Binder ratio g = (3 - <q^4> / <q^2>^2) / 2;
* Fourier mode of a site field f_i at k = (2 pi / L) e_a:
  f(k) = (1/N) sum_i f_i exp(i k . r_i) = (1/N) sum_p exp(2 pi i p / L) F_p, with F_p
  the sum of f over the plane of index p along axis a;
* susceptibility chi(k) = N <|f(k)|^2> (averaged over the three axes for k != 0);
* second-moment correlation length xi = sqrt(chi(0) / chi(k_min) - 1) / (2 sin(pi / L)).
f is the overlap q_i for the spin glass and the magnetisation m_i = S_i for the
ferromagnet.
"""
from __future__ import annotations

import math

import numpy as np


def q_values(N: int) -> np.ndarray:
    """q for each bin n = 0..N of an overlap histogram."""
    return 1.0 - 2.0 * np.arange(N + 1, dtype=np.float64) / N


def binder_ratio(hist, N: int) -> np.ndarray:
    """Binder ratio per row of a q histogram ([..., N + 1] counts of n differing sites)."""
    h = np.asarray(hist, dtype=np.float64)
    q2 = q_values(N) ** 2
    w = h.sum(axis=-1)
    m2 = (h * q2).sum(axis=-1) / w
    m4 = (h * q2 * q2).sum(axis=-1) / w
    return 0.5 * (3.0 - m4 / (m2 * m2))


def overlap_plane_sums(counts, L: int) -> np.ndarray:
    """Plane sums of q_i from per-plane counts of differing sites (mode 0): L^2 - 2 n_p."""
    return float(L * L) - 2.0 * np.asarray(counts, dtype=np.float64)


def magnetisation_plane_sums(counts, L: int) -> np.ndarray:
    """Plane sums of S_i from per-plane counts of up spins (mode 1): 2 u_p - L^2."""
    return 2.0 * np.asarray(counts, dtype=np.float64) - float(L * L)


def fourier_squares(plane_sums, L: int):
    """|f(0)|^2 and |f(k_min)|^2 (mean over the three axes) per sample.

    plane_sums: [..., 3, L] (axis, plane); returns two arrays of shape [...]."""
    F = np.asarray(plane_sums, dtype=np.float64)
    N = float(L) ** 3
    phase = np.exp(2j * math.pi * np.arange(L) / L)
    f0 = F[..., 0, :].sum(axis=-1) / N
    fk = (F * phase).sum(axis=-1) / N
    return f0 * f0, (np.abs(fk) ** 2).mean(axis=-1)


def correlation_length(chi0, chik, L: int):
    """Second-moment correlation length from chi(0) and chi(k_min)."""
    ratio = np.asarray(chi0, dtype=np.float64) / np.asarray(chik, dtype=np.float64)
    return np.sqrt(np.maximum(ratio - 1.0, 0.0)) / (2.0 * math.sin(math.pi / L))


def susceptibilities(plane_sums, L: int, axis=None):
    """chi(0) and chi(k_min) = N <|f(k)|^2>, averaged over `axis` of the samples
    (default: every sample axis, i.e. all but the trailing [3, L])."""
    s0, sk = fourier_squares(plane_sums, L)
    N = float(L) ** 3
    if axis is None:
        axis = tuple(range(s0.ndim))
    return N * s0.mean(axis=axis), N * sk.mean(axis=axis)
