"""Helpers shared by the GPU parity tests: fragile-decision detection and the replay that
explains where a GPU run and the oracle part (the oracle's decode, fed the GPU's own bucket
arrays and found set, must reproduce the GPU at the first iteration where they differ, up to
decisions of the replay itself within a fragile margin)."""

import numpy as np

from oracle import philox, plan as OP, sfft4 as O, window as OW

FRAGILE_TURNS = 1 << 12      # 2^-20 turns: FP32 phases of FP32 buckets resolve ~100 units
FRAGILE_REL = 1e-5           # relative margin of magnitude and selection decisions


def fragile(tr):
    """True when a decision of this oracle iteration sits within a fragile margin."""
    if tr["sel_margin"] < FRAGILE_REL:
        return True
    loc = tr["loc"]
    return loc is not None and (np.any(loc["margin"] < FRAGILE_TURNS) or np.any(loc["mag_margin"] < FRAGILE_REL))


def replay_explains(out, rt, f_gpu, sigma, N):
    """True when the oracle's replay of one iteration (found set `out`, trace `rt`, decoded
    from the GPU's own bucket arrays) reproduces the GPU's found set `f_gpu`, or differs from
    it only where the replay itself decided within a fragile margin.  The two decoders then
    saw identical inputs and parted at a decision closer to its threshold than the FP32
    arithmetic of the GPU resolves: a candidate's location or vote within FRAGILE_TURNS of a
    block boundary or of H_s, or its magnitude test within FRAGILE_REL; or a selection within
    FRAGILE_REL of the n_c-th bucket or of theta (one bucket swapped: at most two
    frequencies differ)."""
    got = [int(x) for x in f_gpu]
    if list(out.f) == got:
        return True
    diff = set(int(x) for x in out.f) ^ set(got)
    if rt["sel_margin"] < FRAGILE_REL and len(diff) <= 2:
        return True
    loc = rt["loc"]
    if loc is None:
        return False
    fr = (pow(int(sigma), -1, N) * loc["ustar"]) % N
    for e in diff:
        k = np.flatnonzero(fr == e)
        if k.size == 0 or not np.any((loc["margin"][k] < FRAGILE_TURNS) | (loc["mag_margin"][k] < FRAGILE_REL)):
            return False
    return True


def found_set_from(f, v, vt):
    fs = O.FoundSet()
    for fi, vi, vo in zip(f, v, vt):
        fs.merge(int(fi), complex(vi), int(vo), 0)
    return fs


def explain_divergence(p, r, N, K, l, q, seed, B1=0, signal=0):
    """Walk the iterations of the GPU trace (plan made with trace=True, tracing batch index
    `signal`) and the oracle trace of that signal (run with signal=`signal`); at the first
    iteration whose found sets differ, the oracle must have had a fragile decision and its
    decode fed the GPU's own buckets must reproduce the GPU's found set.  Returns that
    iteration (or None when the traces never part)."""
    op = OP.make_plan(N, K, l, q, seed=seed, B1=B1)
    wc = OW.WindowCache(N, op.delta)
    prev = O.FoundSet()
    for tr in r["traces"]:
        Y, f, v, vt = p.trace(tr["m"])
        fo = tr["found_after"]
        if list(fo.f) == [int(x) for x in f]:
            prev = found_set_from(f, v, vt)
            continue
        assert fragile(tr), ("divergence without a fragile margin", tr["m"])
        it = op.iters[tr["m"] - 1]
        sigma, a = philox.permutation_draw(seed, signal, it.m, N)
        _, _, Ghat = wc.get(it.B)
        out, rt = O.decode_iteration(Y.astype(np.complex128), prev, it, op, sigma, a, r["theta"], Ghat)
        assert replay_explains(out, rt, f, sigma, N), ("replay does not reproduce the GPU", tr["m"])
        return tr["m"]
    return None


def assert_oracle_parity(f, v, vt, r, explain, value_tol):
    """The bar of a GPU result (f, v, vt: support, values, votes) against the oracle's run of
    the same signal, r (run with trace=True):

    * support and votes equal to the oracle's, values within `value_tol` relative l2; or
    * the runs part, and `explain()` (a traced GPU run of the same signal through
      explain_divergence) shows that they part first at a fragile oracle decision that the
      oracle's own decode, replayed on the GPU's bucket arrays, reproduces.  From that
      iteration on the two runs continue from different found sets, so what follows is only
      checked for sanity: nearly the same support, values close on the common part.

    Returns the iteration of an explained divergence, or None."""
    if np.array_equal(f, r["f"]) and np.array_equal(vt, r["votes"]):
        rel = np.linalg.norm(v - r["v"]) / max(np.linalg.norm(r["v"]), 1e-300)
        assert rel <= value_tol, rel
        return None
    m = explain()
    assert m is not None, "the final results differ but the traces never part"
    common = np.intersect1d(f, r["f"])
    assert common.size >= 0.95 * max(len(f), len(r["f"]))
    gi, oi = np.searchsorted(f, common), np.searchsorted(r["f"], common)
    assert np.linalg.norm(v[gi] - r["v"][oi]) <= 1e-2 * np.linalg.norm(r["v"][oi])
    return m
