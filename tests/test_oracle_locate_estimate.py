"""Pins of the oracle's location, vote and estimate steps (no GPU).

Three things are checked against definitions written out here, independently of the oracle:

* the median estimate (Eq. 14 applied to every round, reading R12): per-round values with
  planted outliers, odd and even round counts, against a brute-force sorted middle;
* the magnitude half of a vote (reading R10, the consequence of Eq. 14-15 that a lone tone
  has the same bucket magnitude in every round): one round's |yhat_s|^2 planted just inside
  and just outside mag_tol |yhat_0|^2 must change the vote count by exactly one;
* the fixed-point multiscale location (Section 3.2, Eq. 15-19, Fig. 3-4; readings R6-R10),
  against a plain FP64 restatement: float phases in turns, float block centres
  u_min + (j + 1/2) r with r = Lbar / l, a direct argmin over the l blocks and over the
  integers of the final level, float vote windows.  The two must agree on every candidate
  whose decisions are not within 2^-20 turns (or a relative 1e-5 in magnitude) of a tie.
"""

import math

import numpy as np
import pytest

from oracle import plan as P, sfft4, window as W

FRAGILE_UNITS = 1 << 12    # 2^-20 turns in the oracle's 2^-32-turn units
FRAGILE_REL = 1e-5


# ----------------------------------------------------------------- median estimate -------
def _sorted_middle(vals):
    """The median written out: the middle of the sorted values, or the mean of the two
    middle values for an even count."""
    s = sorted(vals)
    n = len(s)
    return s[n // 2] if n % 2 else 0.5 * (s[n // 2 - 1] + s[n // 2])


def _planted_buckets(vr, u, b, it, N, sigma, offsets, Ghat):
    """Bucket rows of a lone tone at u whose round-r value is vr[r]: the forward model of
    Lemma 1 for one coefficient, yhat_r[b] = G'^_{bL-u} v_r exp(2 pi i (f o_r mod N) / N),
    f = sigma^-1 u mod N (pinned by the bucketization identity test)."""
    f = (pow(int(sigma), -1, N) * int(u)) % N
    k = sfft4.signed_offset(b * it.L - u, N)
    Y = np.zeros((len(offsets), it.B), dtype=np.complex128)
    for r, o in enumerate(offsets):
        Y[r, b] = vr[r] * Ghat[abs(k)] * np.exp(2j * np.pi * ((f * o) % N) / N)
    return Y, f


@pytest.mark.parametrize("R", [3, 4, 5, 6, 7, 8, 9])
def test_median_estimate_with_planted_outliers(R):
    """Reading R12: v = median_r Re(v_r) + i median_r Im(v_r), with v_r the Eq. 14 estimate of
    round r; for even R the mean of the two middle values.  The per-round values carry planted
    outliers, so the mean, a median of |v_r|, a median over the wrong middle and a median
    taken before the phase correction all differ from the expected value."""
    N, B = 2**14, 64
    it = P.make_iteration(1, N, 14, B, 4, P.quantize_q(0.5), 1e-8)
    _, _, Ghat = W.WindowCache(N, 1e-8).get(B)
    rng = np.random.default_rng(100 + R)
    for trial in range(40):
        sigma = 2 * int(rng.integers(0, N // 2)) + 1
        offsets = [int(o) for o in rng.integers(0, N, size=R)]
        b = int(rng.integers(0, B))
        u = (b * it.L + int(rng.integers(-it.L, it.L))) % N
        # most rounds near 1 + 2i, a minority far away (outliers), distinct real and imaginary
        # parts so the two medians come from different rounds
        vr = 1.0 + 2.0j + 0.05 * (rng.standard_normal(R) + 1j * rng.standard_normal(R))
        nout = (R - 1) // 2
        sgn = complex(rng.choice([-1, 1]), rng.choice([-1, 1]))
        for r in rng.choice(R, size=nout, replace=False):
            vr[r] = complex(sgn.real * rng.uniform(20, 60), sgn.imag * rng.uniform(20, 60))
        Y, f = _planted_buckets(vr, u, b, it, N, sigma, offsets, Ghat)
        fo, v, vr_back = sfft4.estimate(Y, [b], np.array([u]), sigma, offsets, it, N, Ghat)
        assert int(fo[0]) == f
        want = complex(_sorted_middle(vr.real.tolist()), _sorted_middle(vr.imag.tolist()))
        assert abs(v[0] - want) <= 1e-12 * abs(want), (trial, v[0], want)
        assert np.max(np.abs(vr_back[:, 0] - vr)) <= 1e-12 * np.max(np.abs(vr))
        # the planted values make the alternatives visibly different
        assert abs(np.mean(vr) - want) > 1.0


def test_median_estimate_even_count_takes_both_middles():
    """Even R: the mean of the two middle values, not either one alone."""
    N, B = 2**12, 32
    it = P.make_iteration(1, N, 12, B, 4, P.quantize_q(0.5), 1e-8)
    _, _, Ghat = W.WindowCache(N, 1e-8).get(B)
    vr = np.array([1 + 10j, 3 - 2j, 2 + 6j, 10 + 0j])
    offsets = [0, 17, 301, 1999]
    Y, _ = _planted_buckets(vr, 5 * it.L + 3, 5, it, N, 77, offsets, Ghat)
    _, v, _ = sfft4.estimate(Y, [5], np.array([5 * it.L + 3]), 77, offsets, it, N, Ghat)
    assert abs(v[0] - (2.5 + 3.0j)) < 1e-12


# ----------------------------------------------------------------- magnitude vote --------
def _lone_tone(u, it, N, rng, errs=None):
    """Bucket values of one candidate (rounds 0..S) for a lone tone at u: unit magnitude and
    the phases u tau_s / N (+ errs[s - 1]) turns relative to round 0."""
    y = np.empty(it.R, dtype=np.complex128)
    y[0] = np.exp(2j * np.pi * rng.uniform())
    for s in range(1, it.R):
        ph = ((u * it.tau[s]) % N) / N + (0.0 if errs is None else errs[s - 1])
        y[s] = y[0] * np.exp(2j * np.pi * ph)
    return y


@pytest.mark.parametrize("N,B,l,q", [(2**14, 64, 4, 0.5), (2**16, 64, 16, 1.0), (2**20, 128, 16, 1.0)])
def test_magnitude_vote_threshold(N, B, l, q):
    """Reading R10: level s votes only if | |yhat_s|^2 - |yhat_0|^2 | <= mag_tol |yhat_0|^2.
    A lone tone with exact phases gets all S votes; scaling one round's squared magnitude
    to (1 +- mag_tol (1 - eps)) |yhat_0|^2 keeps them, to (1 +- mag_tol (1 + eps)) |yhat_0|^2
    loses exactly one.  The location itself is unaffected (it reads phases only)."""
    n = N.bit_length() - 1
    qn = P.quantize_q(q)
    it = P.make_iteration(1, N, n, B, l, qn, 1e-8)
    mag_tol, eps = 0.5, 1e-3
    rng = np.random.default_rng(N + l)
    b = 7
    for trial in range(12):
        u = (b * it.L + int(rng.integers(-it.L // 2, it.L // 2))) % N
        y = _lone_tone(u, it, N, rng)
        s_hit = int(rng.integers(1, it.S + 1))
        for side in (1.0, -1.0):
            for inside, want in ((1.0 - eps, it.S), (1.0 + eps, it.S - 1)):
                yy = y.copy()
                yy[s_hit] *= math.sqrt(1.0 + side * mag_tol * inside)
                Yb = np.zeros((it.R, B), dtype=np.complex128)
                Yb[:, b] = yy
                loc = sfft4.locate(Yb, np.array([b]), it, N, n, l, qn, mag_tol)
                assert int(loc["ustar"][0]) == u
                assert int(loc["votes"][0]) == want, (trial, side, inside, int(loc["votes"][0]))


# ----------------------------------------------------------------- plain FP64 location ---
def _turns(c):
    """Phase of c in turns, in [0, 1), FP64."""
    return (np.angle(c) / (2.0 * np.pi)) % 1.0


def _cdist(a, b):
    """Distance of two phases (turns) on the circle."""
    d = (a - b) % 1.0
    return min(d, 1.0 - d)


def _centre_phase(umin, j, Lb, ts, l, N):
    """Phase (turns) of the centre u_min + (j + 1/2) Lbar / l of block j times tau / N, mod 1;
    the integer parts are reduced exactly before the division so the float keeps its
    precision."""
    a = ((umin * ts) % N) / N
    c = (((2 * j + 1) * Lb * ts) % (2 * l * N)) / (2 * l * N)
    return (a + c) % 1.0


def plain_locate_one(y, b, it, N, l, q, mag_tol):
    """Section 3.2 in FP64 for one candidate bucket b with round values y[0..S]:
    block levels choose the block whose centre phase is nearest to phi_s (ties to the lower
    block) and move to the extended block [u_min + (j - q/2) r, ...); the final level takes the
    nearest of the Lbar_S integers; votes compare phi_s with u* tau_s / N within the extended
    half-block (1 + q) r tau_s / (2N) (block levels) or half the spacing tau_S / (2N) (final),
    and the squared magnitude with round 0's."""
    S, L, B = it.S, it.L, it.B
    phi = [_turns(y[s] * np.conj(y[0])) for s in range(1, S + 1)]
    umin = b * L - L
    for s in range(1, S):
        Lb, ts = it.Lbar[s - 1], it.tau[s]
        d = [_cdist(phi[s - 1], _centre_phase(umin, j, Lb, ts, l, N)) for j in range(l)]
        j = int(np.argmin(d))
        umin = umin + math.floor(((j - q / 2.0) * Lb) / l)
    Lb, ts = it.Lbar[S - 1], it.tau[S]
    d = [_cdist(phi[S - 1], (((umin + i) * ts) % N) / N) for i in range(Lb)]
    ustar = (umin + int(np.argmin(d))) % N
    m0 = abs(y[0]) ** 2
    votes = 0
    for s in range(1, S + 1):
        Lb, ts = it.Lbar[s - 1], it.tau[s]
        H = (1.0 + q) * Lb * ts / (2.0 * l * N) if s < S else ts / (2.0 * N)
        ok_phase = _cdist(phi[s - 1], ((ustar * ts) % N) / N) <= H
        ok_mag = abs(abs(y[s]) ** 2 - m0) <= mag_tol * m0
        votes += int(ok_phase and ok_mag)
    own = ((ustar + L // 2) // L) % B == b
    return ustar, votes, own


def _adversarial_phases(u_true, b, it, N, l, q, rng, delta):
    """Round values whose phase at each block level sits delta turns from the midpoint of two
    adjacent block centres (on the side of the block holding u_true, if any), and at the final
    level delta from the midpoint of two adjacent candidates: every argmin has a margin of
    2 delta, the smallest the cross-check admits."""
    S, L = it.S, it.L
    y = np.empty(it.R, dtype=np.complex128)
    y[0] = np.exp(2j * np.pi * rng.uniform()) * rng.uniform(0.5, 2.0)
    umin = b * L - L
    for s in range(1, S):
        Lb, ts = it.Lbar[s - 1], it.tau[s]
        r = Lb / l
        j = int(min(l - 2, max(0, math.floor((u_true - umin) / r))))
        c0 = _centre_phase(umin, j, Lb, ts, l, N)
        c1 = _centre_phase(umin, j + 1, Lb, ts, l, N)
        gap = (c1 - c0) % 1.0
        side = rng.choice([-1.0, 1.0])
        ph = (c0 + 0.5 * gap + side * delta) % 1.0
        y[s] = y[0] * np.exp(2j * np.pi * ph)
        jj = j if side < 0 else j + 1
        umin = umin + math.floor(((jj - q / 2.0) * Lb) / l)
    Lb, ts = it.Lbar[S - 1], it.tau[S]
    i = int(rng.integers(0, max(1, Lb - 1)))
    e0 = (((umin + i) * ts) % N) / N
    e1 = (((umin + i + 1) * ts) % N) / N
    gap = (e1 - e0) % 1.0
    y[S] = y[0] * np.exp(2j * np.pi * ((e0 + 0.5 * gap + rng.choice([-1.0, 1.0]) * delta) % 1.0))
    return y


CASES = [(2**14, 64, 4, 0.5), (2**16, 64, 16, 1.0), (2**16, 16, 8, 1.5), (2**14, 64, 3, 0.25),
         (2**20, 128, 16, 1.0), (2**22, 1024, 16, 1.0), (2**12, 16, 32, 2.0)]


@pytest.mark.parametrize("N,B,l,q", CASES)
def test_fixed_point_locate_matches_plain_fp64(N, B, l, q):
    """The oracle's location works on phases held as 2^-32 turns with block centres rounded
    from exact rationals; a plain FP64 restatement of Section 3.2 must give the same u*, votes
    and ownership on every candidate whose decisions are not within 2^-20 turns of a tie.
    Inputs: lone tones with phase errors around the Eq. 19 tolerance, random bucket values,
    and phases planted 2^-19 .. 2^-12 turns from block and candidate midpoints."""
    n = N.bit_length() - 1
    qn = P.quantize_q(q)
    qq = qn / float(P.Q_DEN)
    it = P.make_iteration(1, N, n, B, l, qn, 1e-8)
    mag_tol = 0.5
    rng = np.random.default_rng(n * 100 + l)
    cols, bs = [], []
    tol = np.array([qq * it.Lbar[s - 1] * it.tau[s] / (2.0 * l * N) if s < it.S else it.tau[s] / (2.0 * N)
                    for s in range(1, it.S + 1)])
    edge_buckets = [0, B - 1, 1, B // 2]
    for k in range(240):
        b = edge_buckets[k % 4] if k < 16 else int(rng.integers(0, B))
        u = (b * it.L + int(rng.integers(-it.L, it.L))) % N
        kind = k % 3
        if kind == 0:
            errs = rng.uniform(-1.6, 1.6, it.S) * tol
            y = _lone_tone(u, it, N, rng, errs)
            y[1:] *= np.sqrt(1.0 + rng.uniform(-0.7, 0.7, it.S))
        elif kind == 1:
            y = rng.standard_normal(it.R) + 1j * rng.standard_normal(it.R)
        else:
            delta = 2.0 ** -float(rng.integers(12, 20))
            y = _adversarial_phases(u, b, it, N, l, qq, rng, delta)
        cols.append(y)
        bs.append(b)
    # several candidates share a bucket index: place each in its own copy of the arrays
    agree = robust = 0
    for y, b in zip(cols, bs):
        Yb = np.zeros((it.R, B), dtype=np.complex128)
        Yb[:, b] = y
        loc = sfft4.locate(Yb, np.array([b]), it, N, n, l, qn, mag_tol)
        if loc["margin"][0] < FRAGILE_UNITS or loc["mag_margin"][0] < FRAGILE_REL:
            continue
        robust += 1
        us, v, own = plain_locate_one(y, b, it, N, l, qq, mag_tol)
        assert int(loc["ustar"][0]) == us, (b, int(loc["ustar"][0]), us)
        assert int(loc["votes"][0]) == v, (b, int(loc["votes"][0]), v)
        assert bool(loc["own"][0]) == bool(own)
        agree += 1
    assert robust >= 0.8 * len(cols), robust


def test_plain_fp64_locate_recovers_lone_tones():
    """The plain restatement itself locates lone tones with errors inside Eq. 19 exactly
    (so agreement with it is agreement with a working location, not with a shared bug)."""
    N, B, l, q = 2**16, 64, 16, 1.0
    qn = P.quantize_q(q)
    it = P.make_iteration(1, N, 16, B, l, qn, 1e-8)
    tol = np.array([q * it.Lbar[s - 1] * it.tau[s] / (2.0 * l * N) if s < it.S else it.tau[s] / (2.0 * N)
                    for s in range(1, it.S + 1)])
    rng = np.random.default_rng(9)
    b = 11
    for u in range(b * it.L - it.L, b * it.L + it.L, 29):
        y = _lone_tone(u % N, it, N, rng, rng.uniform(-0.9, 0.9, it.S) * tol)
        us, v, own = plain_locate_one(y, b, it, N, l, q, 0.5)
        assert us == u % N and v == it.S
        assert own == (((u % N) + it.L // 2) // it.L % B == b)


def test_location_exact_ties_go_to_lower_index():
    """Reading R7/R9: an exact tie between two blocks (or two final-level integers) goes to the
    lower index.  At N = 2^22, B = 1024, l = 16, q = 1 the block size of level 1 is r = 512 and
    the final level's spacing is tau_S / N = 1/4 turn, so the midpoints between adjacent block
    centres, u_min + (j + 1) r, and between adjacent candidates are exact in 2^-32-turn units.
    A lone tone at u near the start of its block j gets level 1's phase planted on the
    midpoint between blocks j and j + 1: the tie must pick j (block j + 1's extended region no
    longer holds u, so the upper choice would lose the tone).  Its final-level phase planted
    between u and u + 1 must give u."""
    N, B, l, q = 2**22, 1024, 16, 1.0
    n, qn = 22, P.quantize_q(q)
    it = P.make_iteration(1, N, n, B, l, qn, 1e-8)
    S, L = it.S, it.L
    r = it.Lbar[0] // l
    assert it.Lbar[0] % l == 0 and it.tau[S] * 4 == N
    rng = np.random.default_rng(21)
    for trial in range(20):
        b = int(rng.integers(0, B))
        umin = b * L - L
        j = int(rng.integers(0, l - 1))
        u = umin + j * r + int(rng.integers(1, r // 8))
        y = _lone_tone(u % N, it, N, rng)
        Yb = np.zeros((it.R, B), dtype=np.complex128)
        # level 1 on the midpoint between the centres of blocks j and j + 1
        mid = ((umin + (j + 1) * r) * it.tau[1]) % N
        y1 = y.copy()
        y1[1] = y1[0] * np.exp(2j * np.pi * mid / N)
        Yb[:, b] = y1
        loc = sfft4.locate(Yb, np.array([b]), it, N, n, l, qn, 0.5)
        assert int(loc["jstar"][0][0]) == j, trial
        assert int(loc["ustar"][0]) == u % N
        # final level on the midpoint between the candidates u and u + 1
        yS = y.copy()
        ph = (((u % N) * it.tau[S]) % N) / N + it.tau[S] / (2.0 * N)
        yS[S] = yS[0] * np.exp(2j * np.pi * ph)
        Yb[:, b] = yS
        loc = sfft4.locate(Yb, np.array([b]), it, N, n, l, qn, 0.5)
        assert int(loc["ustar"][0]) == u % N, trial
