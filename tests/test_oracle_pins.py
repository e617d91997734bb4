"""Pins of the FP64 oracle against things other than itself (no GPU).

Each test checks one oracle function against a definition written out independently
(brute-force O(N^2) DFTs, direct sums), a third-party implementation (numpy's
Philox), the paper's own bounds (Eq. 9, Eq. 18-19) and worked numbers, or exact
recovery of known sparse spectra.
"""

import math
import os

import numpy as np
import pytest

from oracle import philox, plan as P, sfft4, window as W
from synth import sparse_signal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----------
@pytest.mark.parametrize("key,counter", [((0, 0), (0, 0, 0, 0)), ((5, 0), (7, 3, 1, 0)),
                                         ((2**64 - 1, 12345), (2**63, 1, 2, 3))])
def test_philox_matches_numpy(key, counter):
    # numpy increments the 256-bit counter before producing a block.
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array(counter, dtype=np.uint64))
    ref = [int(v) for v in bg.random_raw(8)]
    c = list(counter)
    got = []
    for _ in range(2):
        # 256-bit increment with carry
        i = 0
        while True:
            c[i] = (c[i] + 1) & philox.MASK64
            if c[i] != 0 or i == 3:
                break
            i += 1
        got.extend(philox.philox4x64_10(c, key))
    assert got == ref


def test_permutation_draw_is_odd_and_in_range():
    for N in (256, 2**14, 2**22, 2**26):
        for m in range(1, 6):
            s, a = philox.permutation_draw(123, 7, m, N)
            assert s % 2 == 1 and 0 < s < N and 0 <= a < N
            assert math.gcd(s, N) == 1


# ---------------------------------------------------------------- window ----------
def _ghat_direct(G, h, N, ks):
    """sum_{|j|<=h} G_j exp(-2 pi i k j / N), written out term by term (complex)."""
    j = np.arange(-h, h + 1)
    ks = np.asarray(ks)
    ang = -2.0 * np.pi * (np.outer(ks, j) % N) / N
    return (np.exp(1j * ang) * G[None, :]).sum(axis=1)


@pytest.mark.parametrize("N,B,delta", [(2**12, 16, 1e-8), (2**14, 64, 1e-8), (2**16, 256, 1e-6),
                                       (2**16, 16, 1e-8)])
def test_window_eq9_flatness_every_k(N, B, delta):
    """Eq. 9: |G'^ - 1| <= delta on |k| <= L/2 and |G'^| <= delta on |k| >= L, all k."""
    G, h = W.window_time(N, B, delta)
    L = N // B
    full = W.window_spectrum_full(N, G, h)
    k = np.arange(N)
    ks = np.where(k >= N // 2, k - N, k)
    assert abs(G.sum() - 1.0) < 1e-14
    assert np.max(np.abs(1.0 - full[np.abs(ks) <= L // 2])) <= delta
    assert np.max(np.abs(full[np.abs(ks) >= L])) <= delta
    assert np.all(np.abs(full) <= 1.0 + delta)
    # time support w = 2h + 1 = O(B log(1/delta)), as the paper states for the flat window
    assert 2 * h + 1 < 50 * B * math.log10(1.0 / delta) / 8.0


def test_window_spectrum_matches_direct_sum():
    N, B, delta = 2**14, 64, 1e-8
    G, h = W.window_time(N, B, delta)
    full = W.window_spectrum_full(N, G, h)
    ks = np.array([0, 1, 7, 100, 255, 256, 300, 383, 384, 511, 1000, 8191, 8192, 16383])
    d = _ghat_direct(G, h, N, ks)
    assert np.max(np.abs(d.imag)) < 1e-13
    assert np.max(np.abs(d.real - full[ks])) < 1e-13


def test_window_halfwidth_is_about_44_buckets():
    # w ~ 44.3 B at delta = 1e-8 (Gaussian tail truncated at delta)
    for B in (16, 64, 1024, 4096):
        h, _ = P.window_halfwidth(2**26, B, 1e-8)
        assert abs((2 * h + 1) / B - 44.29) < 0.05 + 3.0 / B   # ceil() adds < 2 samples


# ---------------------------------------------------------------- permutation -----
def _dft(x):
    """Eq. 2 written out: X_i = (1/N) sum_j x_j omega^{ij}, omega = exp(-2 pi i / N)."""
    N = x.shape[0]
    j = np.arange(N)
    F = np.exp(-2j * np.pi * (np.outer(j, j) % N) / N) / N
    return F @ x


def test_permutation_spectrum_eq8_all_sigma():
    """Gather form x'_t = x[(sigma t + o) mod N] has X'_u = X_{sigma^-1 u} e^{2 pi i (sigma^-1 u) o / N}."""
    N = 256
    rng = np.random.default_rng(0)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = _dft(x)
    t = np.arange(N)
    for sigma in range(1, N, 2):
        o = (37 * sigma + 11) % N
        xp = x[(sigma * t + o) % N]
        Xp = _dft(xp)
        sinv = pow(sigma, -1, N)
        u = np.arange(N)
        f = (sinv * u) % N
        expect = X[f] * np.exp(2j * np.pi * ((f * o) % N) / N)
        assert np.max(np.abs(Xp - expect)) < 1e-12


# ---------------------------------------------------------------- bucketization ---
@pytest.mark.parametrize("N,B", [(2**10, 16), (2**12, 32), (2**12, 64)])
def test_bucketize_lemma1_identity(N, B):
    """Lemma 1 with the exact window spectrum: yhat[b] = sum_f X_f G'^_{bL - sigma f} e^{2 pi i f o / N}."""
    rng = np.random.default_rng(N + B)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    X = _dft(x)                                  # Eq. 2, so x_n = sum_f X_f e^{+2 pi i f n / N}
    L = N // B
    G, h = W.window_time(N, B, 1e-8)
    Gfull = _ghat_direct(G, h, N, np.arange(N))  # complex, no symmetry assumed
    sigma, a = 2 * 57 + 1, 901 % N
    offs = [(a + sigma * t) % N for t in (0, 5, 77)]
    Y = sfft4.bucketize(x, N, B, G, h, sigma, offs)
    f = np.arange(N)
    for s, o in enumerate(offs):
        for b in range(B):
            k = (b * L - sigma * f) % N
            expect = np.sum(X * Gfull[k] * np.exp(2j * np.pi * ((f * o) % N) / N))
            assert abs(Y[s, b] - expect) < 1e-10 * max(1.0, abs(expect))


@pytest.mark.parametrize("N,B,K", [(2**12, 32, 6), (2**14, 64, 12)])
def test_update_removes_exact_coefficients(N, B, K):
    """Reading R13: subtracting the true coefficients of a noiseless K-sparse signal from
    buckets b-1, b, b+1 of every round (G'^_{b'L-u} v e^{2 pi i f o / N}) leaves only the
    window's leakage beyond the neighbours (each |G'^_k| <= delta there).  A wrong phase sign,
    a missing neighbour bucket or a wrong round offset leaves residuals of the buckets' own
    size; with half of the coefficients removed, the other half must remain untouched."""
    sig = sparse_signal(N, K, 3, None)
    x = sig.x.astype(np.complex128)
    L = N // B
    G, h, Ghat = W.WindowCache(N, 1e-8).get(B)
    sigma, a = 2 * 83 + 1, 1234 % N
    offs = [(a + sigma * t) % N for t in (0, 7, 301, 4099 % N)]
    Y = sfft4.bucketize(x, N, B, G, h, sigma, offs)
    scale = np.max(np.abs(Y))
    full = sfft4.FoundSet()
    for f, v in zip(sig.freqs, sig.values):
        full.merge(int(f), complex(v), 0, 1)
    assert np.max(np.abs(sfft4.update(Y, full, N, B, L, sigma, offs, Ghat))) <= 1e-6 * scale
    # removing half of the coefficients equals the bucketization of the other half alone
    half = sfft4.FoundSet()
    for f, v in list(zip(sig.freqs, sig.values))[: K // 2]:
        half.merge(int(f), complex(v), 0, 1)
    rest = np.zeros(N, dtype=np.complex128)
    n = np.arange(N)
    for f, v in list(zip(sig.freqs, sig.values))[K // 2:]:
        rest += v * np.exp(2j * np.pi * ((f * n) % N) / N)
    Yrest = sfft4.bucketize(rest, N, B, G, h, sigma, offs)
    assert np.max(np.abs(sfft4.update(Y, half, N, B, L, sigma, offs, Ghat) - Yrest)) <= 1e-6 * scale


@pytest.mark.parametrize("N,B", [(256, 16), (1024, 32), (4096, 256)])
def test_bucket_of_nearest_centre_ties_up(N, B):
    """Reading R5: u falls in bucket b when u lies in [(2b-1)L/2, (2b+1)L/2) (mod N), i.e.
    b L is the nearest bucket centre on the circle and a half-way u goes to the upper
    bucket.  Checked for every u against a brute-force nearest-centre search."""
    L = N // B
    u = np.arange(N, dtype=np.int64)
    got = sfft4.bucket_of(u, L, B)
    centres = np.arange(B, dtype=np.int64) * L
    for uu in range(N):
        d = (uu - centres) % N
        d = np.where(d >= N - d, d - N, d)          # signed distance in [-N/2, N/2)
        best = np.flatnonzero(np.abs(d) == np.abs(d).min())
        # the nearest centre; at a half-way u the upper bucket (its centre lies above u)
        want = best[0] if len(best) == 1 else [b for b in best if d[b] < 0][0]
        assert got[uu] == want, (uu, got[uu], want)


def test_select_top_energy_ties_to_lower_bucket():
    """Reading R11: the candidates are the n_c buckets of largest |yhat_0|^2 (equal keys: the
    lower bucket first), keeping only those strictly above the floor theta; returned sorted.
    Checked on keys with planted ties against a brute-force sort."""
    rng = np.random.default_rng(7)
    for trial in range(200):
        B = int(rng.choice([16, 32, 64]))
        # values with exact squared magnitudes, so that equal keys are exact ties
        vals = np.array([0, 1, -1, 1j, -1j, 1 + 1j, 2, -2j, 1 - 1j, 0.5, 3j, -1.5 + 2j])
        Y0 = rng.choice(vals, size=B).astype(np.complex128)
        key = Y0.real ** 2 + Y0.imag ** 2
        n_c = int(rng.integers(1, B + 1))
        theta = float(rng.choice([0.0, 0.2, 1.0, 4.0]))
        got, _ = sfft4.select(Y0, n_c, theta)
        order = sorted(range(B), key=lambda b: (-key[b], b))
        want = sorted(b for b in order[:n_c] if key[b] > theta)
        assert [int(b) for b in got] == want, (trial, list(got), want)


def test_unique_samples_counts_union():
    it = P.make_iteration(1, 2**22, 22, 1024, 16, 256, 1e-8)
    brute = set()
    for t in it.tau:
        brute.update(range(t - it.h, t + it.h + 1))
    assert sfft4.unique_samples(it, 2**22) == len(brute)


# ---------------------------------------------------------------- levels ----------
@pytest.mark.parametrize("L,l,q", [(8192, 16, 1.0), (4096, 4, 0.5), (2**22, 16, 1.0), (200, 8, 1.5),
                                   (64, 3, 0.25), (10000, 32, 2.0)])
def test_levels_region_contains_extended_block(L, l, q):
    """Every integer of the extended block [u_min + (j - q/2) r, u_min + (j + 1 + q/2) r)
    lies inside the next region [u_min', u_min' + Lbar_{s+1})  (Section 3.2, Fig. 4)."""
    qn = P.quantize_q(q)
    lv = P.levels(L, l, qn)
    qq = qn / 256.0
    for s in range(len(lv) - 1):
        Lb, Ln = lv[s], lv[s + 1]
        assert Ln < Lb
        r = Lb / l
        for umin in (-Lb, 0, 12345):
            for j in range(l):
                new = umin + ((2 * j * 256 - qn) * Lb) // (2 * l * 256)
                lo = umin + (j - qq / 2) * r
                hi = umin + (j + 1 + qq / 2) * r
                ints = [u for u in range(math.ceil(lo), math.ceil(hi))]
                assert all(new <= u < new + Ln for u in ints)
    assert lv[-1] <= l or P.levels(lv[-1], l, qn) == [lv[-1]]


def test_levels_config3_values():
    # N = 2^22, B = 1024: region 2L = 8192; l = 16, q = 1
    assert P.levels(8192, 16, 256) == [8192, 1025, 130, 18, 4]
    it = P.make_iteration(1, 2**22, 22, 2048, 16, 256, 1e-8)
    assert it.Lbar == [4096, 513, 66, 10]
    assert it.tau == [0, 2**22 // 4352, 2**22 // 546, 2**22 // 71, 2**22 // 10]


def test_schedule_invariants():
    for K, B1 in [(16, 64), (100, 128), (1000, 2048), (4000, 4096), (1, 16)]:
        sch = P.schedule(K, B1)
        Bs = [b for b, _ in sch]
        Ks = [k for _, k in sch]
        assert all(b & (b - 1) == 0 and P.B_MIN <= b <= B1 for b in Bs)
        assert all(Bs[i] >= Bs[i + 1] for i in range(len(Bs) - 1))
        assert all(Ks[i] >= Ks[i + 1] for i in range(len(Ks) - 1))
        assert Ks[0] == K and Bs[0] == min(B1, max(P.B_MIN, P.pow2ceil(B1)))


def test_plan_validation():
    with pytest.raises(ValueError):
        P.make_plan(1000, 4, 16, 1.0, 0)          # N not a power of two
    with pytest.raises(ValueError):
        P.make_plan(2**14, 300, 16, 1.0, 0)       # K > N / 64
    with pytest.raises(ValueError):
        P.make_plan(2**14, 16, 2, 1.0, 0)         # l <= q + 1
    pl = P.make_plan(2**22, 1000, 16, 1.0, 0)
    assert pl.B1 == 2048


# ---------------------------------------------------------------- location --------
def _synthetic_buckets(u, it, N, errs, rng):
    """Y[s] of a lone tone at u: unit magnitude, phase u tau_s / N + err_s turns."""
    Y = np.empty((it.R, 1), dtype=np.complex128)
    Y[0, 0] = np.exp(2j * np.pi * rng.uniform())
    for s in range(1, it.R):
        ph = ((u * it.tau[s]) % N) / N + errs[s - 1]
        Y[s, 0] = Y[0, 0] * np.exp(2j * np.pi * ph)
    return Y


def _guaranteed_tol(it, N, l, qn):
    """Largest phase error (turns) each level tolerates by Eq. 19 (block levels) or half
    the candidate spacing (final level)."""
    tol = []
    for s in range(1, it.S + 1):
        Lb, ts = it.Lbar[s - 1], it.tau[s]
        if s < it.S:
            tol.append(qn / 256.0 * Lb * ts / (2.0 * l * N))
        else:
            tol.append(ts / (2.0 * N))
    return np.array(tol)


@pytest.mark.parametrize("N,B,l,q", [(2**14, 64, 4, 0.5), (2**16, 64, 16, 1.0), (2**16, 16, 8, 1.5)])
def test_location_exact_under_eq19_phase_errors(N, B, l, q):
    """Inside the Eq. 19 bound the multiscale location returns u exactly, with all votes."""
    n = N.bit_length() - 1
    qn = P.quantize_q(q)
    it = P.make_iteration(1, N, n, B, l, qn, 1e-8)
    tol = _guaranteed_tol(it, N, l, qn)
    rng = np.random.default_rng(1)
    b = 3
    L = it.L
    for u in range(b * L - L, b * L + L, max(1, L // 97)):
        errs = rng.uniform(-0.95, 0.95, it.S) * tol
        Y = _synthetic_buckets(u % N, it, N, errs, rng)
        Yb = np.zeros((it.R, B), dtype=np.complex128)
        Yb[:, b] = Y[:, 0]
        loc = sfft4.locate(Yb, np.array([b]), it, N, n, l, qn, 0.5)
        assert loc["ustar"][0] == u % N
        assert loc["votes"][0] == it.S


def test_location_fails_beyond_extension():
    """Negative control: errors beyond the extended block make location fail sometimes."""
    N, B, l, q = 2**16, 64, 16, 1.0
    n, qn = 16, P.quantize_q(q)
    it = P.make_iteration(1, N, n, B, l, qn, 1e-8)
    rng = np.random.default_rng(2)
    fails = 0
    for u in range(0, 2 * it.L, 37):
        errs = np.full(it.S, 1.6 * (1 + q) / (2 * l))
        Y = _synthetic_buckets(u % N, it, N, errs, rng)
        Yb = np.zeros((it.R, B), dtype=np.complex128)
        Yb[:, 1] = Y[:, 0]
        loc = sfft4.locate(Yb, np.array([1]), it, N, n, l, qn, 0.5)
        fails += int(loc["ustar"][0] != u % N or loc["votes"][0] < it.S)
    assert fails > 0


def _read_golden():
    rows, example = [], None
    with open(os.path.join(GOLDEN, "eq18_19_worked_numbers.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "example":
                example = tuple(float(p) for p in parts[1:])
            else:
                rows.append((float(parts[0]), int(parts[1])))
    return rows, example


def test_golden_eq18_eq19_worked_numbers():
    """Section 3.2's printed numbers: l limits from Eq. 18 are safe (l <= pi / dPhi up to
    the paper's rounding) and Eq. 19 gives q >= 0.4 for dPhi = 0.3, l = 4."""
    rows, (dphi, l, qmin) = _read_golden()
    for d, lp in rows:
        assert math.pi / d >= 0.95 * lp
    assert abs(dphi * l / math.pi - qmin) < 0.05


@pytest.mark.parametrize("use_row", [0, 1, 2, 3])
def test_golden_location_at_printed_parameters(use_row):
    """At each printed (dPhi, l), location is exact under |dPhi| radians of phase error at
    every level once q meets Eq. 19 (q r / 2 >= du) for this build's offsets tau; that q
    stays close to the paper's q = dPhi l / pi (0.4 in the printed l = 4 example)."""
    rows, (dphi_ex, l_ex, q_ex) = _read_golden()
    dphi, l = (dphi_ex, int(l_ex)) if use_row == 0 else rows[use_row]
    N, B = 2**18, 64
    n = 18
    err_turns = dphi / (2 * math.pi)
    q = None
    for q8 in range(1, 8 * 32):
        qn = P.quantize_q(q8 / 8.0)
        if l * 256 <= 256 + qn:
            break
        it = P.make_iteration(1, N, n, B, l, qn, 1e-8)
        if np.all(_guaranteed_tol(it, N, l, qn) > err_turns):
            q = q8 / 8.0
            break
    if q is None:
        pytest.skip("printed l too small for an extension")
    q_paper = dphi * l / math.pi
    assert q <= 1.25 * q_paper + 0.125
    if use_row == 0:
        assert abs(q_paper - q_ex) < 0.05
    rng = np.random.default_rng(3)
    for u in range(5 * it.L - it.L, 5 * it.L + it.L, max(1, it.L // 53)):
        errs = rng.choice([-1.0, 1.0], it.S) * err_turns
        Y = _synthetic_buckets(u % N, it, N, errs, rng)
        Yb = np.zeros((it.R, B), dtype=np.complex128)
        Yb[:, 5] = Y[:, 0]
        loc = sfft4.locate(Yb, np.array([5]), it, N, n, l, qn, 0.5)
        assert loc["ustar"][0] == u % N


# ---------------------------------------------------------------- whole transform -
def test_single_tone_every_frequency():
    """Every f in [0, N): a lone tone is located exactly, estimated to 1e-9, with all votes."""
    N, K = 2**11, 1
    rng = np.random.default_rng(4)
    n = np.arange(N)
    for f in range(N):
        X = np.exp(2j * np.pi * rng.uniform())
        x = X * np.exp(2j * np.pi * ((f * n) % N) / N)
        pl = P.make_plan(N, K, 4, 0.5, seed=f)
        r = sfft4.run(x, pl)
        assert r["nfound"] == 1 and r["f"][0] == f
        assert abs(r["v"][0] - X) < 1e-9
        assert r["votes"][0] == pl.iters[r["iter"][0] - 1].S


def test_median_estimate_even_rounds():
    vr = np.array([[1 + 1j], [3 + 0j], [2 + 5j], [10 - 2j]])
    v = np.median(vr.real, axis=0) + 1j * np.median(vr.imag, axis=0)
    assert v[0] == 2.5 + 0.5j


def test_finalize_top_k_ties_to_lower_frequency():
    """Reading R16: the output is the K entries of largest |v| (equal magnitudes: the lower
    frequency first), sorted by frequency, with their votes.  Checked on found sets with
    exact planted ties against a brute-force sort."""
    rng = np.random.default_rng(11)
    vals = np.array([1, -1, 1j, 2, -2j, 1 + 1j, 0.5, 3, -3j, 0.25j])
    for trial in range(200):
        n = int(rng.integers(1, 40))
        fs = sfft4.FoundSet()
        for f in rng.choice(4096, size=n, replace=False):
            fs.merge(int(f), complex(rng.choice(vals)), int(rng.integers(0, 5)), 1)
        K = int(rng.integers(1, 50))
        out = sfft4.finalize(fs, K)
        entries = sorted(zip(fs.f, fs.v, fs.votes), key=lambda e: (-abs(e[1]), e[0]))[:K]
        entries.sort(key=lambda e: e[0])
        assert out["f"].tolist() == [e[0] for e in entries], trial
        assert out["v"].tolist() == [e[1] for e in entries], trial
        assert out["votes"].tolist() == [e[2] for e in entries], trial
        assert out["nfound"] == len(entries)


def test_merge_adds_repeated_frequency():
    fs = sfft4.FoundSet()
    fs.merge(5, 1 + 1j, 4, 1)
    fs.merge(9, 2j, 3, 1)
    fs.merge(5, -1 - 1j, 2, 3)
    assert fs.f == [5, 9] and fs.v[0] == 0 and fs.votes[0] == 4 and fs.iter[0] == 1
    out = sfft4.finalize(fs, 1)
    assert out["f"].tolist() == [9]


@pytest.mark.parametrize("N,K,B1,l,q,seeds", [(2**14, 16, 64, 4, 0.5, range(6)),
                                              (2**20, 100, 128, 16, 1.0, range(3)),
                                              (2**22, 1000, 0, 16, 1.0, range(1))])
def test_exact_support_noiseless(N, K, B1, l, q, seeds):
    """Noiseless exactly K-sparse input: the output is the generator's support and values."""
    for seed in seeds:
        sig = sparse_signal(N, K, seed)
        pl = P.make_plan(N, K, l, q, seed=seed, B1=B1)
        r = sfft4.run(sig.x.astype(np.complex128), pl)
        assert np.array_equal(r["f"], sig.freqs)
        # the input is complex64, so values carry ~1e-7 relative input rounding
        rel = np.linalg.norm(r["v"] - sig.values) / np.linalg.norm(sig.values)
        assert rel < 1e-4


def test_generator_snr_and_support():
    sig = sparse_signal(2**16, 50, 7, snr_db=20.0)
    assert sig.freqs.shape == (50,) and np.unique(sig.freqs).size == 50
    clean = sparse_signal(2**16, 50, 7)
    noise = sig.x.astype(np.complex128) - clean.x.astype(np.complex128)
    snr = 10 * np.log10(np.mean(np.abs(clean.x) ** 2) / np.mean(np.abs(noise) ** 2))
    assert abs(snr - 20.0) < 0.2
    # the clean signal's spectrum (Eq. 2) is the drawn K-sparse spectrum
    X = np.fft.fft(clean.x.astype(np.complex128)) / clean.N
    assert np.max(np.abs(X[clean.freqs] - clean.values)) < 1e-6
    mask = np.ones(clean.N, bool)
    mask[clean.freqs] = False
    assert np.max(np.abs(X[mask])) < 1e-6


@pytest.mark.parametrize("N,K,want_B1", [(2**14, 256, 128), (2**16, 600, 512), (2**16, 1024, 512)])
def test_dense_default_B1_fits_window_and_recovers(N, K, want_B1):
    """K > N/256: the default B1 is the largest power of two whose window fits in N/2 (the
    window of N/64 buckets would not), and the longer static schedule still recovers the
    generator's support exactly."""
    pl = P.make_plan(N, K, 16, 1.0, seed=1)
    assert pl.B1 == want_B1
    assert 2 * P.window_halfwidth(N, 2 * pl.B1, pl.delta)[0] + 1 > N // 2
    assert all(2 * it.h + 1 <= N // 2 for it in pl.iters)
    sig = sparse_signal(N, K, 3)
    r = sfft4.run(sig.x.astype(np.complex128), pl)
    assert np.array_equal(r["f"], sig.freqs)


def test_uneven_sizes_recipe():
    """The uneven-batch size generator: N powers of two in [2^16, 2^22], K in [10, 2000]
    capped at N/64, SNR in [10, 40] dB; every drawn size has a valid default plan."""
    from synth.signals import uneven_sizes
    Ns, Ks, snrs = uneven_sizes(512, 7)
    assert np.all((Ns & (Ns - 1)) == 0) and Ns.min() >= 2**16 and Ns.max() <= 2**22
    assert np.all(Ks >= 10) and np.all(Ks <= 2000) and np.all(Ks <= Ns // 64)
    assert min(snrs) >= 10.0 and max(snrs) <= 40.0
    assert len(set(Ns.tolist())) == 7
    for N, K in sorted(set(zip(Ns.tolist(), Ks.tolist()))):
        P.make_plan(N, K, 16, 1.0, seed=0)


@pytest.mark.parametrize("N,K,l,q", [(2**14, 16, 4, 0.5), (2**20, 100, 16, 1.0)])
def test_two_round_location_exact_when_collisions_are_rare(N, K, l, q):
    """The two-round (sFFT3.0) location: rounds tau = 0, 1, the phase of yhat_1 / yhat_0 is
    u / N; with its default 8 K buckets noiseless signals are recovered exactly."""
    pl = P.make_plan(N, K, l, q, seed=4, location="two_round")
    assert all(it.R == 2 and it.tau == [0, 1] and it.Lbar == [2 * it.L] for it in pl.iters)
    assert pl.B1 == min(4096, N // 64, P.pow2ceil(8 * K))
    for seed in range(2):
        sig = sparse_signal(N, K, seed)
        r = sfft4.run(sig.x.astype(np.complex128), P.make_plan(N, K, l, q, seed=seed, location="two_round"))
        assert np.array_equal(r["f"], sig.freqs)


def test_two_round_location_needs_few_collisions():
    """With 2 K buckets (collisions common) the two-round location accepts mixtures of
    colliding tones that the multiscale levels reject: multiscale stays exact, two-round
    does not (the robustness difference between the two location schemes)."""
    N, K = 2**20, 100
    sig = sparse_signal(N, K, 0)
    ms = sfft4.run(sig.x.astype(np.complex128), P.make_plan(N, K, 16, 1.0, seed=0, B1=128))
    tr = sfft4.run(sig.x.astype(np.complex128), P.make_plan(N, K, 16, 1.0, seed=0, B1=128, location="two_round"))
    assert np.array_equal(ms["f"], sig.freqs)
    assert not np.array_equal(tr["f"], sig.freqs)


def test_two_round_single_tones():
    N = 2**11
    pl = P.make_plan(N, 1, 4, 0.5, seed=2, location="two_round")
    rng = np.random.default_rng(5)
    n = np.arange(N)
    for f in list(rng.choice(N, 40, replace=False)) + [0, N - 1]:
        X = np.exp(2j * np.pi * rng.uniform())
        x = X * np.exp(2j * np.pi * ((f * n) % N) / N)
        r = sfft4.run(x, pl)
        assert list(r["f"]) == [f] and abs(r["v"][0] - X) < 1e-9


def test_two_round_location_limit():
    with pytest.raises(ValueError):
        P.make_plan(2**21, 100, 16, 1.0, seed=0, location="two_round")
