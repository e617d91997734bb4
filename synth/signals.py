"""Synthetic K-sparse test signals (Section 4.1 set-up), seeded.

K frequencies drawn uniformly without replacement from [0, N), magnitude 1 and a
uniform phase on [0, 2 pi); the time signal is x_n = sum_f X_f exp(+2 pi i f n / N),
i.e. the inverse of the DFT of Eq. 2.  In the general sparse case circular white
Gaussian noise is added in the time domain with per-sample variance
(sum_f |X_f|^2) * 10^(-SNR/10), so SNR compares per-sample powers.

Draws use numpy's ``Generator(Philox(seed))``.  The signal is stored as complex64
(what the GPU reads); tests widen exactly those values to complex128 for the oracle.
"""

from dataclasses import dataclass

import numpy as np


@dataclass
class SparseSignal:
    N: int
    K: int
    freqs: np.ndarray      # sorted int64, length K
    values: np.ndarray     # complex128, X_f at freqs
    x: np.ndarray          # complex64 time signal, length N (None if not synthesised)
    snr_db: float          # None = noiseless


def spectrum(N, K, seed):
    """(sorted freqs, values) of a unit-magnitude, uniform-phase K-sparse spectrum."""
    rng = np.random.Generator(np.random.Philox(seed))
    f = np.sort(rng.choice(N, size=K, replace=False).astype(np.int64))
    ph = rng.uniform(0.0, 2.0 * np.pi, size=K)
    return f, np.exp(1j * ph), rng


def snr_noise_std(values, snr_db):
    """Per-component std of complex noise giving the requested per-sample SNR."""
    var = float(np.sum(np.abs(values) ** 2)) * 10.0 ** (-snr_db / 10.0)
    return np.sqrt(var / 2.0)


def sparse_signal(N, K, seed, snr_db=None):
    """Seeded K-sparse signal, synthesised on the CPU with numpy (exact, portable)."""
    f, v, rng = spectrum(N, K, seed)
    X = np.zeros(N, dtype=np.complex128)
    X[f] = v
    x = np.fft.ifft(X) * N
    if snr_db is not None:
        s = snr_noise_std(v, snr_db)
        x = x + s * (rng.standard_normal(N) + 1j * rng.standard_normal(N))
    return SparseSignal(N=N, K=K, freqs=f, values=v, x=x.astype(np.complex64), snr_db=snr_db)


def batch_spectra(N, K, seeds):
    """Spectra only (no time signal) for a batch; the caller synthesises on a device."""
    out = []
    for sd in seeds:
        f, v, _ = spectrum(N, K, sd)
        out.append((f, v))
    return out


def uneven_sizes(nsig, seed, n_range=(16, 22), k_range=(10, 2000), snr_range=(10.0, 40.0)):
    """Sizes of a batch of signals of uneven length and sparsity: N = 2^n with n uniform on
    the integers of n_range (N log-uniform over the powers of two), K = round(exp(U[ln k_lo,
    ln k_hi])) capped at N/64, SNR uniform on snr_range in dB (None: noiseless).
    Returns (Ns int64 array, Ks int64 array, list of SNRs)."""
    rng = np.random.Generator(np.random.Philox(seed))
    n = rng.integers(n_range[0], n_range[1] + 1, size=nsig)
    Ns = np.left_shift(np.int64(1), n.astype(np.int64))
    K = np.rint(np.exp(rng.uniform(np.log(k_range[0]), np.log(k_range[1]), size=nsig))).astype(np.int64)
    Ks = np.minimum(K, Ns // 64)
    if snr_range is None:
        snrs = [None] * nsig
    else:
        snrs = [float(s) for s in rng.uniform(snr_range[0], snr_range[1], size=nsig)]
    return Ns, Ks, snrs


def signal_seed(seed, i):
    """Seed of signal i of a batch drawn with seed `seed`."""
    return (int(seed) << 20) + int(i)


def device_signal(N, K, seed, snr_db, device, out=None):
    """The spectrum of sparse_signal(N, K, seed) synthesised on a CUDA device with torch:
    complex128 inverse DFT times N, plus (snr_db not None) circular Gaussian noise of the same
    variance drawn from torch's generator seeded with `seed` (not numpy's stream, so the noise
    differs from sparse_signal's), stored as complex64 into `out` (or a new tensor).
    Returns (x, freqs, values)."""
    import torch
    f, v, _ = spectrum(N, K, seed)
    X = torch.zeros(N, dtype=torch.complex128, device=device)
    X[torch.from_numpy(f).to(device)] = torch.from_numpy(v).to(device)
    x = torch.fft.ifft(X) * N
    if snr_db is not None:
        g = torch.Generator(device=device)
        g.manual_seed(int(seed))
        std = float(snr_noise_std(v, snr_db))
        nr = torch.randn(N, generator=g, device=device, dtype=torch.float64)
        ni = torch.randn(N, generator=g, device=device, dtype=torch.float64)
        x = x + std * torch.complex(nr, ni)
    if out is None:
        out = torch.empty(N, dtype=torch.complex64, device=device)
    out.copy_(x.to(torch.complex64))
    return out, f, v
