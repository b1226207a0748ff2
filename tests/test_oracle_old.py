"""Pins of the oracle's `old` (Sec. 4, Listing 3: Current = old Current):
the plain definition (first unit whose bits differ) by brute force, and the
fingerprint that stands for `old` by properties fixed by its definition --
the empty value, the effect of one changed unit (a closed form in SplitMix64,
itself pinned to published outputs), injectivity in every unit (brute force
over all 2^16 values of a 16-bit unit), and position dependence."""
import itertools

import numpy as np

import oracle

M64 = (1 << 64) - 1


def test_first_changed_brute_force():
    base = np.array([1.5, -0.0, np.nan, 3.0, 0.0, -2.0, 7.0, 1e-40], np.float32)
    assert oracle.first_changed(base, base.copy()) == -1
    for i in range(8):
        b = base.copy()
        b.view(np.uint32)[i] ^= 1                       # one bit of one unit
        assert oracle.first_changed(base, b) == i
    for i, j in itertools.combinations(range(8), 2):
        b = base.copy()
        b.view(np.uint32)[i] ^= 0x80000000
        b.view(np.uint32)[j] ^= 0x80000000
        assert oracle.first_changed(base, b) == i       # the smaller index wins
    # bits, not values: -0 differs from +0, a NaN equals its own bits
    z = np.array([0.0], np.float32)
    assert oracle.first_changed(z, -z) == 0
    n1 = np.array([np.nan], np.float32)
    assert oracle.first_changed(n1, n1.copy()) == -1
    # 16-bit units (bf16 / fp16 data)
    h = np.arange(8, dtype=np.float16)
    h2 = h.copy()
    h2[5] = 9
    assert oracle.first_changed(h, h2) == 5


def test_fingerprint_empty_and_one_unit():
    assert oracle.fingerprint_old(np.zeros(0, np.float32)) == (0, 0)
    for w in [0, 1, 0xDEADBEEF, 0xFFFFFFFF]:
        x = np.array([w], np.uint32)
        h = oracle.splitmix64(w)
        assert oracle.fingerprint_old(x) == (h, ((h >> 32) * (h & 0xFFFFFFFF)) & M64)


def test_fingerprint_one_changed_unit_closed_form():
    """Changing unit i from w to w' moves F1 by mix(i 2^32 + w') - mix(i 2^32 + w)."""
    g = np.random.default_rng(5)
    x = g.integers(0, 2 ** 32, 37, dtype=np.uint64).astype(np.uint32)
    f1, _ = oracle.fingerprint_old(x)
    for i in [0, 1, 17, 36]:
        y = x.copy()
        y[i] = np.uint32(int(x[i]) ^ 0x12345)
        g1, _ = oracle.fingerprint_old(y)
        d = (oracle.splitmix64((i << 32) | int(y[i])) -
             oracle.splitmix64((i << 32) | int(x[i]))) & M64
        assert (g1 - f1) & M64 == d


def test_fingerprint_injective_in_a_unit_brute_force():
    x = np.array([3, 1, 4, 1], np.float16)
    seen = set()
    v = x.view(np.uint16)
    for w in range(1 << 16):
        v[2] = w
        seen.add(oracle.fingerprint_old(x)[0])
    assert len(seen) == 1 << 16


def test_fingerprint_depends_on_positions():
    x = np.array([1.0, 2.0, 3.0, 4.0], np.float32)
    y = x[[1, 0, 2, 3]].copy()
    assert oracle.fingerprint_old(x) != oracle.fingerprint_old(y)
    # 64-bit elements are two 32-bit units
    d = np.array([1.0, 2.0], np.float64)
    assert oracle.fingerprint_old(d) == oracle.fingerprint_old(d.view(np.uint32))
