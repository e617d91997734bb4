"""The replay criterion of the GPU parity tests (parity_helpers.replay_explains), on planted
replays: it accepts a found set that differs from the GPU's only through candidates whose
replayed decisions sit within a fragile margin, and rejects every other difference."""

import numpy as np

from oracle import sfft4 as O

import parity_helpers as PH

N = 2**16
SIGMA = 12345                       # odd, so invertible mod N
SINV = pow(SIGMA, -1, N)


def found(fs):
    s = O.FoundSet()
    for f in fs:
        s.merge(int(f), 1.0 + 0j, 1, 1)
    return s


def replay(freqs, margins, mag_margins, sel_margin=1.0):
    """A replay trace whose candidates locate to `freqs` (u* = sigma f mod N)."""
    u = (SIGMA * np.asarray(freqs, np.int64)) % N
    assert np.array_equal((SINV * u) % N, np.asarray(freqs) % N)
    return {"sel_margin": sel_margin,
            "loc": {"ustar": u, "margin": np.asarray(margins, np.int64),
                    "mag_margin": np.asarray(mag_margins, np.float64)}}


def test_identical_found_sets():
    rt = replay([5, 9], [1 << 20, 1 << 20], [1.0, 1.0])
    assert PH.replay_explains(found([5, 9, 40]), rt, [5, 9, 40], SIGMA, N)


def test_extra_tone_from_fragile_vote_accepted():
    # the replay accepts 9 at 300 units (2^-32 turns) from a threshold: fragile
    rt = replay([5, 9], [1 << 20, 300], [1.0, 1.0])
    assert PH.replay_explains(found([5, 9, 40]), rt, [5, 40], SIGMA, N)
    # the GPU has a tone the replay rejected at a fragile magnitude test
    rt = replay([5, 9], [1 << 20, 1 << 20], [1.0, 3e-6])
    assert PH.replay_explains(found([5, 40]), rt, [5, 9, 40], SIGMA, N)


def test_difference_at_a_firm_decision_rejected():
    rt = replay([5, 9], [1 << 20, PH.FRAGILE_TURNS + 1], [1.0, 1.0])
    assert not PH.replay_explains(found([5, 9, 40]), rt, [5, 40], SIGMA, N)
    rt = replay([5, 9], [1 << 20, 1 << 20], [1.0, 2 * PH.FRAGILE_REL])
    assert not PH.replay_explains(found([5, 40]), rt, [5, 9, 40], SIGMA, N)


def test_difference_outside_the_candidates_rejected():
    # 77 is no candidate of the replay: nothing in this iteration explains it
    rt = replay([5, 9], [300, 300], [1e-9, 1e-9])
    assert not PH.replay_explains(found([5, 9, 40]), rt, [5, 9, 40, 77], SIGMA, N)


def test_fragile_selection_swaps_at_most_one_bucket():
    rt = replay([5], [1 << 20], [1.0], sel_margin=1e-7)
    assert PH.replay_explains(found([5, 40]), rt, [5, 40, 77], SIGMA, N)
    assert PH.replay_explains(found([5, 40, 12]), rt, [5, 40, 77], SIGMA, N)
    assert not PH.replay_explains(found([5, 40, 12, 13]), rt, [5, 40, 77], SIGMA, N)
    # the same differences with a firm selection are rejected
    rt = replay([5], [1 << 20], [1.0], sel_margin=0.5)
    assert not PH.replay_explains(found([5, 40]), rt, [5, 40, 77], SIGMA, N)
