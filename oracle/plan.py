"""Static parameters of an sFFT4.0 transform (oracle side; FP64 / exact integers).

Follows Section 3.1 (iterations m with K_m, B_m, L_m = N/B_m, w_m, R_m), Section 3.2
(multiscale location: l blocks per level, extension q, L_{s+1} = L_s (q+1)/l,
tau ~ N/L_s) and Lemma 2.  Where the paper is silent or inconsistent the reading
taken is the one listed in the design notes (readings R4, R6, R8-R11, R14):

* q is quantised to q_n / 256 (exact integer region arithmetic).
* The search region of a bucket is 2L wide (pass band plus transition bands), so
  nominal level lengths are Lbar_1 = 2L, Lbar_{s+1} = ceil((q+1) Lbar_s / l) + 1 while
  Lbar_s > l and the length still shrinks; the last length is the final (integer)
  level.  tau_s = floor(N / (Lbar_s + ceil(q Lbar_s / l))) on block levels and
  floor(N / Lbar_S) on the final level; round 0 has tau_0 = 0 (the reference round).
* The schedule is fixed at plan time: B_m = clamp(pow2ceil(ceil(beta * K_m)),
  16, B_1) with beta = B_1 / K, K_1 = K and K_{m+1} = K_m (1 - exp(-2 K_m / B_m)),
  iterated until K_m < 1/2, then two extra iterations at the last B.  Default
  B_1 = pow2ceil(2K) (capped at min(4096, N/64)).

Pinned by tests: level containment (every integer of an extended block lies in
the next region), tau/threshold closed forms, and the schedule's invariants.
"""

import math
from dataclasses import dataclass, field

Q_DEN = 256          # q is stored as q_n / Q_DEN
B_MIN = 16           # smallest bucket count used by the schedule
GAMMA = 2.0          # isolation model: P(isolated) = exp(-GAMMA * rem / B)
EXTRA_ITERS = 2


def pow2ceil(v):
    """Smallest power of two >= v (v >= 1)."""
    p = 1
    while p < v:
        p <<= 1
    return p


def quantize_q(q):
    """q -> q_n with q = q_n / 256, rounding half up."""
    return int(math.floor(q * Q_DEN + 0.5))


def erfcinv(y):
    """Inverse complementary error function for 0 < y < 1 (scipy's routine)."""
    from scipy.special import erfcinv as _e
    return float(_e(y))


def window_halfwidth(N, B, delta):
    """Half-width h of the flat window (w = 2h + 1), reading R4 of Eq. 9.

    Frequency box half-width 3L/4 convolved with a Gaussian of standard deviation
    s_f = L / (4 sqrt(2) erfcinv(delta)); in time the Gaussian has standard deviation
    s_t = N / (2 pi s_f) = B * 4 sqrt(2) erfcinv(delta) / (2 pi) and is truncated where
    it falls to delta: h = ceil(s_t * sqrt(2 ln(1/delta))).
    """
    c = 4.0 * math.sqrt(2.0) * erfcinv(delta)
    s_t = B * c / (2.0 * math.pi)
    return int(math.ceil(s_t * math.sqrt(2.0 * math.log(1.0 / delta)))), s_t


def levels(L, l, qn):
    """Nominal level lengths [Lbar_1 .. Lbar_S] (Section 3.2, Fig. 4; reading R6)."""
    out = [L]
    while out[-1] > l:
        nxt = -(-((Q_DEN + qn) * out[-1]) // (l * Q_DEN)) + 1   # ceil((q+1) Lbar / l) + 1
        if nxt >= out[-1]:
            break
        out.append(nxt)
    return out


@dataclass
class Iteration:
    m: int                 # 1-based iteration index
    B: int                 # buckets B_m
    L: int                 # bucket length L_m = N / B_m
    h: int                 # window half-width, w = 2h + 1
    Lbar: list             # nominal lengths of levels 1..S
    tau: list              # offsets tau_0 = 0, tau_1..tau_S (length R = S + 1)
    H: list                # vote thresholds of levels 1..S in 2^-32 turns
    n_c: int = 0           # candidate buckets examined: min(B, ceil(c * max(K_m, 1)))

    @property
    def S(self):
        return len(self.Lbar)

    @property
    def R(self):
        return len(self.Lbar) + 1


@dataclass
class Plan:
    N: int
    n: int
    K: int
    l: int
    qn: int
    seed: int
    delta: float
    B1: int
    select_factor: float
    min_votes: int         # 0 = all levels must vote (S of the iteration)
    sig_floor: float       # candidate floor, relative to max |yhat_0|^2 of iteration 1
    mag_tol: float         # |yhat_s|^2 consistency tolerance of a vote (Eq. 14-15)
    iters: list = field(default_factory=list)
    location: str = "multiscale"   # or "two_round" (sFFT3.0: rounds tau = 0, 1)


def schedule(K, B1, max_iters=64):
    """Static schedule [(B_m, K_m)] (reading R14 of Section 3.1).

    K_m is the expected number of coefficients still to find in iteration m (the
    paper's expected sparsity K_m), B_m the bucket count sized from it."""
    beta = B1 / K
    rem = float(K)
    out = []
    while len(out) < max_iters:
        B = pow2ceil(int(math.ceil(beta * rem)))
        B = max(B_MIN, min(B1, B))
        out.append((B, rem))
        rem = rem * (1.0 - math.exp(-GAMMA * rem / B))
        if rem < 0.5:
            break
    for _ in range(EXTRA_ITERS):
        if len(out) < max_iters:
            out.append((out[-1][0], rem))
    return out


def make_iteration(m, N, n, B, l, qn, delta, location="multiscale"):
    L = N // B
    h, _ = window_halfwidth(N, B, delta)
    if location == "two_round":
        # sFFT3.0 location in the same iterative framework (Section 3.1: R_m = 2): rounds
        # tau = 0 and 1, so the phase of yhat_1 / yhat_0 is u / N itself; the 2L integers of
        # the search region compete as a final level with spacing 1 / N.  A lone tone's phase
        # sits on an integer up to rounding, so the vote takes 1/8 of the spacing (half of it
        # would accept every phase, i.e. every mixture of colliding tones)
        return Iteration(m=m, B=B, L=L, h=h, Lbar=[2 * L], tau=[0, 1], H=[(1 << (32 - n)) // 8])
    # The search region of bucket b is [bL - L, bL + L): the pass band plus both halves
    # of the transition band (L/2 < |k| < L) where the (L/N, L/2N) window still leaks.
    Lbar = levels(2 * L, l, qn)
    S = len(Lbar)
    # Block levels: the phase circle spans the region plus one extension width q r, so a
    # tone pushed past either end of the region by an error within Eq. 19 does not alias
    # to the opposite end.  Final level: candidates spaced tau / N apart over the circle.
    tau = [0]
    for s, Lb in enumerate(Lbar):
        if s < S - 1:
            tau.append(N // (Lb + -(-(qn * Lb) // (l * Q_DEN))))
        else:
            tau.append(N // Lb)
    H = []
    for s in range(1, S + 1):
        Lb, ts = Lbar[s - 1], tau[s]
        if s < S:
            # half-width of the extended block in phase: (1+q) Lbar tau / (2 l N) turns
            H.append(((Q_DEN + qn) * Lb * ts << (32 - n)) // (2 * l * Q_DEN))
        else:
            # final integer level: half the candidate spacing, tau / (2N) turns
            H.append((ts << (32 - n)) // 2)
    return Iteration(m=m, B=B, L=L, h=h, Lbar=Lbar, tau=tau, H=H)


def make_plan(N, K, l, q, seed, B1=0, delta=1e-8, select_factor=2.0, min_votes=0,
              sig_floor=1e-10, mag_tol=0.5, max_iters=64, location="multiscale"):
    """Validate and build the static plan (same checks as the library's sfft4_plan)."""
    if N < 256 or N & (N - 1) or N > (1 << 30):
        raise ValueError("N must be a power of two in [2^8, 2^30]")
    n = N.bit_length() - 1
    qn = quantize_q(q)
    if K < 1 or K > N // 64:
        raise ValueError("need 1 <= K <= N/64")
    if l < 2 or l > 32 or qn < 0 or l * Q_DEN <= Q_DEN + qn:
        raise ValueError("need 2 <= l <= 32, q >= 0 and l > q + 1")
    if not (0.0 < delta < 0.5):
        raise ValueError("need 0 < delta < 1/2")
    if location not in ("multiscale", "two_round"):
        raise ValueError("location must be 'multiscale' or 'two_round'")
    if location == "two_round" and N > (1 << 20):
        # the library's FP32 bucket arrays resolve the 1/(8N)-turn vote window up to 2^20
        raise ValueError("two-round location needs N <= 2^20")

    if B1 == 0:
        # two-round location tolerates few collisions: default 8 K buckets instead of 2 K
        B1 = max(B_MIN, min(4096, N // 64, pow2ceil((8 if location == "two_round" else 2) * K)))
        # reading R14: halve the default until the window of B1 buckets fits in N/2
        while B1 > B_MIN and 2 * window_halfwidth(N, B1, delta)[0] + 1 > N // 2:
            B1 //= 2
    if B1 < B_MIN or B1 & (B1 - 1) or B1 > N // 64 or B1 > 4096:
        raise ValueError("B1 must be a power of two in [16, min(4096, N/64)]")
    its = []
    for i, (B, Km) in enumerate(schedule(K, B1, max_iters)):
        it = make_iteration(i + 1, N, n, B, l, qn, delta, location)
        it.n_c = min(B, int(math.ceil(select_factor * max(Km, 1.0))))
        its.append(it)
    for it in its:
        if 2 * it.h + 1 > N // 2:
            raise ValueError("window wider than N/2")
    return Plan(N=N, n=n, K=K, l=l, qn=qn, seed=seed, delta=delta, B1=B1,
                select_factor=select_factor, min_votes=min_votes, sig_floor=sig_floor,
                mag_tol=mag_tol, iters=its, location=location)
