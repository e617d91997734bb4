"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

Holds none of the transform's arithmetic: it only draws spectra and noise and
synthesises time signals from them.
"""

from .signals import SparseSignal, sparse_signal, snr_noise_std, batch_spectra  # noqa: F401
