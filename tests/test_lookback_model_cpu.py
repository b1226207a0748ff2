"""CPU model of the decoupled look-back protocol the sort passes and the
filter use (the exclusive prefix of per-tile counts over earlier tiles,
Merrill and Garland's single-pass scan), as the kernels walk it: a window of
W words read per memory round trip, taken in order through its first
inclusive prefix, stopping at its first unpublished word and polling that
word again.  Tiles start in ticket order and publish their aggregate, then
(after their own walk) their inclusive prefix; the interleaving of all these
steps is random.  The walk must give every tile the serial exclusive prefix
and, as the sort's checked pass needs, the last key of the nearest earlier
tile with a non-empty run.  A model of the protocol, not of the CUDA code:
the GPU parity tests cover the kernels."""
import random

import pytest

AGG, PRE = "A", "P"


def simulate(counts, keys, window, seed):
    rnd = random.Random(seed)
    T = len(counts)
    words = [None] * T           # None | (flag, count, key)
    state = [None] * T           # per tile: None (not started) or its walk state
    result = [None] * T
    started = 0
    while any(r is None for r in result):
        # runnable: the next tile to start (tickets in order) or any tile in its walk
        choices = [t for t in range(T) if state[t] is not None and result[t] is None]
        if started < T:
            choices.append(-1)
        pick = rnd.choice(choices)
        if pick == -1:
            t = started
            started += 1
            c, k = counts[t], keys[t]
            if t == 0:
                words[0] = (PRE, c, k if c else None)
                result[0] = (0, None)
                state[0] = "done"
            else:
                words[t] = (AGG, c, k if c else None)
                state[t] = {"j": t - 1, "excl": 0, "found": False, "pred": None}
            continue
        t = pick
        s = state[t]
        # one round trip: read the window's words (each read is one atomic snapshot)
        j = s["j"]
        win = [words[j - u] if j - u >= 0 else (PRE, 0, None) for u in range(window)]
        done = False
        u = 0
        while u < window:
            w = win[u]
            if w is None:
                break
            flag, c, k = w
            if not s["found"] and c > 0:
                s["found"], s["pred"] = True, k
            s["excl"] += c
            if flag == PRE:
                done = True
                break
            u += 1
        if done:
            c, k = counts[t], keys[t]
            carry = k if c else s["pred"]
            words[t] = (PRE, s["excl"] + c, carry)
            result[t] = (s["excl"], s["pred"] if s["found"] else None)
        else:
            s["j"] = j - u       # u < window: that word is polled again; else move on
    return result


@pytest.mark.parametrize("window", [1, 2, 4, 32])
@pytest.mark.parametrize("seed", range(6))
def test_windowed_lookback_matches_serial_scan(window, seed):
    rnd = random.Random(100 + seed)
    T = 150
    counts = [0 if rnd.random() < 0.3 else rnd.randint(1, 50) for _ in range(T)]
    keys = [rnd.randint(-1000, 1000) for _ in range(T)]
    res = simulate(counts, keys, window, seed)
    run = 0
    last = None
    for t in range(T):
        excl, pred = res[t]
        assert excl == run, (t, excl, run)
        assert pred == last, (t, pred, last)
        run += counts[t]
        if counts[t]:
            last = keys[t]


def test_planted_mistake_is_caught():
    """A walk that skips the stalled word instead of polling it again (a
    plausible slip in the window logic) must fail the check."""
    counts = [3] * 40
    keys = list(range(40))
    bad = False
    for seed in range(20):
        rnd = random.Random(seed)
        T = len(counts)
        words = [None] * T
        excls = []
        # tiles publish aggregates in a random order; tile 0 its prefix
        order = list(range(T))
        rnd.shuffle(order)
        for t in order[: T // 2]:
            words[t] = (AGG, counts[t], keys[t])
        words[0] = (PRE, counts[0], keys[0])
        for t in range(1, T):
            j, excl = t - 1, 0
            while j >= 0:
                w = words[j]
                if w is None:          # the slip: skip instead of waiting
                    j -= 1
                    continue
                excl += w[1]
                if w[0] == PRE:
                    break
                j -= 1
            excls.append(excl)
        bad |= any(e != 3 * (t + 1) for t, e in enumerate(excls))
    assert bad
