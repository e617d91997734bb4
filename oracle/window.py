"""Flat window filter (Section 2.3, Eq. 9-10), FP64.

G is a Gaussian multiplied, in time, by the Dirichlet kernel of a frequency box of
half-width 3L/4, i.e. in frequency a box convolved with a Gaussian (reading R4).
It is truncated to |j| <= h and normalised so that sum_j G_j = 1, which makes the
spectrum G'^_0 = 1.

G'^_k = sum_{|j| <= h} G_j omega_N^{k j} = sum_j G_j cos(2 pi k j / N)  (real, even),
the DFT of the truncated window, with the paper's omega_N = exp(-2 pi i / N) and
without the 1/N of Eq. 2 (the bucket value of an isolated tone is G'^_{bL-u} X_f).

Pinned by: Eq. 9 itself (|1 - G'^_k| <= delta on |k| <= L/2, |G'^_k| <= delta on
|k| >= L, checked at every k for small N), and a brute-force direct sum.
"""

import math

import numpy as np

from .plan import window_halfwidth


def window_time(N, B, delta):
    """Time-domain window G_j for j = -h..h (array of length w = 2h + 1) and h."""
    L = N // B
    h, s_t = window_halfwidth(N, B, delta)
    M = (3 * L) // 4                      # box covers frequencies |k| <= M
    j = np.arange(-h, h + 1, dtype=np.int64)
    g = np.exp(-0.5 * (j / s_t) ** 2)
    # Dirichlet kernel sum_{|k|<=M} e^{2 pi i k j / N} = sin(pi (2M+1) j / N) / sin(pi j / N),
    # with the integer arguments reduced mod 2N first so the sines are accurate.
    num = np.sin(np.pi * (((2 * M + 1) * j) % (2 * N)) / N)
    den = np.sin(np.pi * (j % (2 * N)) / N)
    D = np.where(j == 0, float(2 * M + 1), num / np.where(j == 0, 1.0, den))
    G = g * D
    G = G / G.sum()
    return G, h


def window_spectrum_full(N, G, h):
    """G'^_k for all k in [0, N) via one length-N FFT of the zero-padded window."""
    Gz = np.zeros(N, dtype=np.float64)
    j = np.arange(-h, h + 1, dtype=np.int64)
    Gz[j % N] = G
    return np.fft.fft(Gz).real


class WindowCache:
    """G and G'^_k (|k| <= 3L/2) per bucket count B, computed on first use."""

    def __init__(self, N, delta):
        self.N = N
        self.delta = delta
        self._c = {}

    def get(self, B):
        if B not in self._c:
            G, h = window_time(self.N, B, self.delta)
            L = self.N // B
            full = window_spectrum_full(self.N, G, h)
            self._c[B] = (G, h, full[: (3 * L) // 2 + 1].copy())
        return self._c[B]
