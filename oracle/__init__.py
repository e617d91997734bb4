"""Plain, slow FP64 CPU oracle for sFFT4.0 (Li, Jiang and Chen, "On Performance of
Multiscale Sparse Fast Fourier Transform Algorithm", arXiv 2011.05698).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import, call or run
anything in this package.  The product path (the CUDA library and its Python
binding) never imports it and shares no code, table or constant generator with it.

Modules
-------
philox   Philox4x64-10 counter-based generator (Salmon et al., SC'11), written from
         its published definition; draws sigma and the base offset of each iteration.
plan     Static iteration schedule, multiscale levels, offsets tau and vote
         thresholds (Sections 3.1-3.3, Lemma 2).
window   Flat window G and its spectrum G'^ (Section 2.3, Eq. 9-10).
sfft4    Bucketization (Lemma 1, Eq. 13), update (Section 3.1), large-bucket
         selection, multiscale location (Section 3.2, Eq. 15-19), median estimation
         (Eq. 14), merge and final top-K.

Parity status of each function is stated in its docstring; every function here is
pinned by a ``-m "not gpu"`` test against something other than itself (brute-force
DFTs, closed forms, numpy's Philox, exhaustive single tones, exact support recovery).
"""

from . import philox, plan, window, sfft4  # noqa: F401
