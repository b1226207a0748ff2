"""Pins for the oracle's sort and sort contracts (Listing 4), matrix product
(Sec. 3.4), Freivalds check, Gaussian elimination (Sec. 5 / Listing 6 read as
GEPP), the batched chain and the MLP cost model.  CPU only.

Independent references: brute force over permutations, Python's sorted(),
exact integer and rational arithmetic (fractions), Leibniz's determinant
formula, numpy's float64 matmul, central finite differences, hand-computed
values and the published SplitMix64 outputs.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

f32 = np.float32


# --------------------------------------------------------------------------
# sort
# --------------------------------------------------------------------------

def test_sort_brute_force_permutations():
    g = np.random.default_rng(0)
    for n in range(0, 8):
        for _ in range(5):
            x = g.integers(-5, 5, n).astype(np.int32)
            # the sorted arrangement is the one permutation with no descent
            cands = {p for p in itertools.permutations(x.tolist())
                     if all(p[i] <= p[i + 1] for i in range(len(p) - 1))}
            assert len(cands) <= 1
            out = oracle.sort_i32(x)
            if n:
                assert tuple(out.tolist()) in cands


def test_sort_matches_python_sorted_full_range():
    x = inputs.sort_keys_uniform(100000, seed=99)
    assert oracle.sort_i32(x).tolist() == sorted(x.tolist())
    ext = np.array([2**31 - 1, -2**31, 0, -1, 1, -2**31, 2**31 - 1], np.int32)
    assert oracle.sort_i32(ext).tolist() == sorted(ext.tolist())


def test_sort_distinct_variant_counts():
    x = inputs.sort_keys_distinct(50000)
    out = oracle.sort_i32(x)
    assert len(np.unique(x)) <= 256
    vals, cnt = np.unique(x, return_counts=True)
    vals2, cnt2 = np.unique(out, return_counts=True)
    assert np.array_equal(vals, vals2) and np.array_equal(cnt, cnt2)
    assert oracle.first_unsorted_i32(out) == -1


def test_first_unsorted_planted():
    x = np.arange(1000, dtype=np.int32)
    assert oracle.first_unsorted_i32(x) == -1
    y = x.copy()
    y[500], y[501] = y[501], y[500]
    assert oracle.first_unsorted_i32(y) == 500
    y = x.copy()
    y[999] = -7
    y[10] = 10**6
    assert oracle.first_unsorted_i32(y) == 10
    assert oracle.first_unsorted_i32(np.zeros(0, np.int32)) == -1
    assert oracle.first_unsorted_i32(np.zeros(1, np.int32)) == -1


def test_same_multiset():
    x = inputs.sort_keys_uniform(5000, seed=5)
    s = oracle.sort_i32(x)
    assert oracle.same_multiset_i32(x, s)
    t = s.copy()
    t[17] += 1
    assert not oracle.same_multiset_i32(x, t)
    t = s.copy()
    t[3], t[4000] = t[4000], t[3]       # a swap keeps the multiset
    assert oracle.same_multiset_i32(x, t)
    assert not oracle.same_multiset_i32(x, s[:-1])


# --------------------------------------------------------------------------
# matrix product
# --------------------------------------------------------------------------

def test_matmul_identity_and_permutation_exact():
    A, B = inputs.matmul_inputs(64)
    I = np.eye(64, dtype=f32)
    assert np.array_equal(oracle.matmul_f64(I, B), B.astype(np.float64))
    perm = np.random.default_rng(1).permutation(64)
    P = np.eye(64, dtype=f32)[perm]
    assert np.array_equal(oracle.matmul_f64(P, A), A[perm].astype(np.float64))
    assert np.array_equal(oracle.matmul_f64(A, P.T), A[:, perm].astype(np.float64))


def test_matmul_small_integers_exact():
    g = np.random.default_rng(2)
    A = g.integers(-8, 9, (16, 24))
    B = g.integers(-8, 9, (24, 12))
    ref = [[sum(int(A[i, k]) * int(B[k, j]) for k in range(24)) for j in range(12)]
           for i in range(16)]
    assert np.array_equal(oracle.matmul_f64(A.astype(f32), B.astype(f32)), np.array(ref))


def test_matmul_vs_numpy_and_rows():
    A, B = inputs.matmul_inputs(96)
    C = oracle.matmul_f64(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64)
    assert np.max(np.abs(C - ref)) <= 1e-12 * np.max(np.abs(ref))
    rows = np.array([0, 95, 17])
    assert np.array_equal(oracle.matmul_rows_f64(A, B, rows), C[rows])


# --------------------------------------------------------------------------
# Freivalds
# --------------------------------------------------------------------------

def test_splitmix64_published_outputs():
    gamma = 0x9E3779B97F4A7C15
    # the first two outputs of SplitMix64 seeded with 0
    assert oracle.splitmix64(gamma) == 0xE220A8397B1DCDAF
    assert oracle.splitmix64((2 * gamma) % 2**64) == 0x6E789E6AA1B965F4


def test_rademacher_balance():
    r = oracle.rademacher(6, 0, 20000)
    assert set(np.unique(r)) == {-1.0, 1.0}
    assert abs(r.mean()) < 0.03
    assert not np.array_equal(r, oracle.rademacher(6, 1, 20000))


def test_freivalds_exact_product_passes_and_corruption_is_found():
    g = np.random.default_rng(3)
    n = 48
    A = g.integers(-4, 5, (n, n)).astype(f32)
    B = g.integers(-4, 5, (n, n)).astype(f32)
    C = (A.astype(np.int64) @ B.astype(np.int64)).astype(f32)
    first, gap, tau = oracle.freivalds(A, B, C, seed=6)
    assert first == -1 and np.all(gap == 0)
    for row in [0, 31, n - 1]:
        D = C.copy()
        D[row, 7] += 4 * tau[row]            # beyond the tolerance for any sign
        first, _, _ = oracle.freivalds(A, B, D, seed=6)
        assert first == row
    D = C.copy()
    D[40, 1] += 4 * tau[40]
    D[12, 2] += 4 * tau[12]
    assert oracle.freivalds(A, B, D, seed=6)[0] == 12


def test_freivalds_rounded_product_within_tolerance():
    A, B = inputs.matmul_inputs(128)
    C = (A.astype(np.float64) @ B.astype(np.float64)).astype(f32)
    first, gap, tau = oracle.freivalds(A, B, C, seed=6, u_eff=2.0 ** -24 * math.sqrt(128))
    assert first == -1
    assert np.max(gap / tau) < 0.5


# --------------------------------------------------------------------------
# Gaussian elimination with partial pivoting
# --------------------------------------------------------------------------

def frac_gepp(A):
    """Exact rational GEPP with the same pivot rule (largest |a_ik|, lowest
    index on ties)."""
    n = len(A)
    M = [[Fraction(v) for v in row] for row in A]
    piv = []
    for k in range(n):
        p = max(range(k, n), key=lambda i: (abs(M[i][k]), -i))
        piv.append(p)
        M[k], M[p] = M[p], M[k]
        for i in range(k + 1, n):
            l = M[i][k] / M[k][k]
            M[i][k] = l
            for j in range(k + 1, n):
                M[i][j] -= l * M[k][j]
    return M, piv


def leibniz_det(A):
    n = len(A)
    total = 0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        term = 1
        for i in range(n):
            term *= int(A[i][p[i]])
        total += -term if inv % 2 else term
    return total


def test_gepp_matches_exact_rationals():
    g = np.random.default_rng(4)
    for n in range(1, 7):
        A = g.integers(-9, 10, (n, n))
        while round(np.linalg.det(A)) == 0:
            A = g.integers(-9, 10, (n, n))
        LU, piv, info = oracle.gepp_f64(A.astype(np.float64))
        M, piv_ref = frac_gepp(A.tolist())
        assert info == 0 and piv.tolist() == piv_ref
        for i in range(n):
            for j in range(n):
                assert abs(LU[i, j] - float(M[i][j])) <= 1e-12 * (1 + abs(float(M[i][j])))


def test_det_vs_leibniz_n8():
    g = np.random.default_rng(5)
    A = g.integers(-5, 6, (8, 8))
    LU, piv, info = oracle.gepp_f64(A.astype(np.float64))
    d = oracle.det_f64(LU, piv)
    ref = leibniz_det(A.tolist())
    assert abs(d - ref) <= 1e-9 * max(1, abs(ref))


def test_pivot_tie_lowest_index_and_zero_pivot():
    A = np.array([[1.0, 2.0, 0.0], [-3.0, 1.0, 1.0], [3.0, 0.0, 2.0]])
    _, piv, _ = oracle.gepp_f64(A)
    assert piv[0] == 1            # |-3| == |3|: the lower index wins
    S = np.array([[1.0, 2.0], [2.0, 4.0]])
    _, _, info = oracle.gepp_f64(S)
    assert info == 2              # exactly singular: zero pivot at step 1


def test_vandermonde_integer_solution():
    for n in range(2, 7):
        t = np.arange(1, n + 1, dtype=np.float64)
        V = np.vander(t, increasing=True).astype(f32)
        xs = np.arange(1, n + 1, dtype=np.float64) * np.where(np.arange(n) % 2, -1, 1)
        b = np.array([sum(int(V[i, j]) * int(xs[j]) for j in range(n)) for i in range(n)],
                     dtype=np.float64)
        x = oracle.solve(V, b)
        cond = np.linalg.cond(V.astype(np.float64))
        assert np.max(np.abs(x - xs)) <= 1e-15 * cond * np.max(np.abs(xs)) * 10


def test_diag_dominant_solution_is_ones():
    A, b = inputs.gepp_inputs(256)
    x = oracle.solve(A, b)
    assert np.max(np.abs(x - 1.0)) <= 1e-13
    _, piv, _ = oracle.gepp_f64(A.astype(np.float64))
    assert np.array_equal(piv, np.arange(256))   # dominance: no row swaps


# --------------------------------------------------------------------------
# batched chain
# --------------------------------------------------------------------------

MAP = [("x", 0), ("x", 0), ("c", 1.0), ("fma",)]          # x*x + 1, one rounding
PRE = [("x", 0), ("c", 1.0), ("ge",)]                     # y >= 1
FILT = [("x", 0), ("c", 1.5), ("gt",)]                    # y > 1.5


def round_f32(q: Fraction) -> np.float32:
    """Correctly rounded (nearest, ties to even) binary32 of a rational."""
    c = np.float32(float(q))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        d = abs(Fraction(float(cand)) - q)
        even = (int(np.array(cand).view(np.uint32)) & 1) == 0
        if best is None or d < best[0] or (d == best[0] and even):
            best = (d, cand)
    return best[1]


def exact_fma(a, b, c):
    return round_f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def test_batch_chain_brute_force():
    g = np.random.default_rng(6)
    L = np.array([0, 1, 5, 64, 3, 100])
    off = inputs.batch_offsets(L)
    x = inputs.uniform_pm1(g, int(off[-1]))
    x[off[3] + 10] = np.nan
    sums, fv, kept = oracle.batch_chain(MAP, PRE, FILT, x, off)
    for s in range(len(L)):
        seg = x[off[s]:off[s + 1]]
        y = [exact_fma(v, v, 1.0) if not np.isnan(v) else np.float32(np.nan) for v in seg]
        ks = [float(v) for v in y if v > 1.5]
        assert kept[s] == len(ks)
        assert abs(sums[s] - math.fsum(ks)) <= 1e-12 * (1 + len(ks))
        viol = [i for i, v in enumerate(y) if not (v >= 1)]
        assert fv[s] == (viol[0] if viol else -1)
    assert fv[3] == 10


def test_batch_chain_statistics():
    L = np.full(50, 20000)
    off = inputs.batch_offsets(L)
    x = inputs.batch_data(int(off[-1]))
    sums, fv, kept = oracle.batch_chain(MAP, PRE, FILT, x, off)
    # E[(x^2+1) 1{x^2 > 1/2}] for x ~ U[-1,1] = int_{sqrt(.5)}^1 (x^2+1) dx
    r = math.sqrt(0.5)
    expect = (1 / 3 + 1) - (r ** 3 / 3 + r)
    assert abs(sums.sum() / off[-1] - expect) < 2e-3
    assert abs(kept.sum() / off[-1] - (1 - r)) < 2e-3
    assert np.all(fv == -1)


# --------------------------------------------------------------------------
# MLP
# --------------------------------------------------------------------------

def test_mlp_hand_computed():
    d_in, H = 2, 2
    # W1 = [[1, -1], [2, 0]], b1 = [0, -1], W2 = [[1, 1], [-1, 0]], b2 = [0, 0.5],
    # W3 = [3, -2], b3 = 0.25
    P = np.array([1, -1, 2, 0, 0, -1, 1, 1, -1, 0, 0, 0.5, 3, -2, 0.25], np.float64)
    X = np.array([[1.0, 0.5], [-1.0, 2.0]])
    # x0: z1 = [0.5, 1], h1 = [0.5, 1]; z2 = [1.5, 0], h2 = [1.5, 0]; y = 4.5 + 0.25
    # x1: z1 = [-3, -3], h1 = 0; z2 = [0, 0.5], h2 = [0, 0.5]; y = -1 + 0.25
    y = oracle.mlp_forward(P, X, d_in, H)
    assert np.allclose(y, [4.75, -0.75], rtol=0, atol=1e-15)
    loss, G = oracle.mlp_loss_grad(P, X, np.array([4.0, 0.0]), d_in, H)
    assert abs(loss - (0.75 ** 2 + 0.75 ** 2) / 2) < 1e-15
    assert abs(G[-1] - (2 * 0.75 - 2 * 0.75) / 2) < 1e-15     # d loss / d b3


def test_mlp_gradient_vs_finite_differences():
    d_in = 6
    P = inputs.mlp_init(d_in, 64, seed=3)
    g = np.random.default_rng(8)
    X = g.standard_normal((32, d_in))
    y = g.standard_normal(32)
    _, G = oracle.mlp_loss_grad(P, X, y, d_in)
    h = 1e-6
    idx = g.choice(len(P), 60, replace=False)
    for i in idx:
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (oracle.mlp_loss_grad(Pp, X, y, d_in)[0] -
              oracle.mlp_loss_grad(Pm, X, y, d_in)[0]) / (2 * h)
        assert abs(fd - G[i]) <= 1e-6 * max(1.0, abs(G[i])) + 1e-8


def test_adam_first_step_hand_computed():
    P = np.array([1.0, -2.0])
    G = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    oracle.adam_step(P, G, m, v, 1, lr=0.1)
    # bias-corrected first step moves each weight by lr * g / (|g| + eps')
    assert np.allclose(P, [0.9, -1.9], atol=1e-6)
    assert np.allclose(m, [0.05, -0.025]) and np.allclose(v, [0.00025, 0.0000625])


# ---- transpose and matrix-vector products (Sec. 3.4, Listing 1) ----

def test_transpose_brute_force_and_involution():
    g = np.random.default_rng(21)
    for r, c in [(1, 1), (1, 7), (7, 1), (3, 5), (16, 9)]:
        A = g.standard_normal((r, c)).astype(np.float32)
        At = oracle.transpose_f32(A)
        assert At.shape == (c, r)
        for i in range(r):
            for j in range(c):
                assert At[j, i] == A[i, j]
        assert np.array_equal(oracle.transpose_f32(At), A)   # (A^T)^T = A


def test_matvec_closed_forms():
    g = np.random.default_rng(22)
    n = 37
    x = g.standard_normal(n).astype(np.float32)
    # identity: y = x exactly; permutation P: y = P x exactly
    assert np.array_equal(oracle.matvec_f64(np.eye(n, dtype=np.float32), x), x.astype(np.float64))
    p = g.permutation(n)
    P = np.eye(n, dtype=np.float32)[p]
    assert np.array_equal(oracle.matvec_f64(P, x), x[p].astype(np.float64))
    # all-ones vector: y_i = row sums (small integers: exact)
    A = g.integers(-9, 10, (5, 8)).astype(np.float32)
    assert np.array_equal(oracle.matvec_f64(A, np.ones(8, np.float32)), A.sum(axis=1))
    assert np.array_equal(oracle.vecmat_f64(np.ones(5, np.float32), A), A.sum(axis=0))
    # e_k picks row k (left) / column k (right)
    ek = np.zeros(8, np.float32); ek[3] = 1
    assert np.array_equal(oracle.matvec_f64(A, ek), A[:, 3])
    e2 = np.zeros(5, np.float32); e2[2] = 1
    assert np.array_equal(oracle.vecmat_f64(e2, A), A[2])


def test_matvec_vecmat_vs_numpy_and_duality():
    g = np.random.default_rng(23)
    A = g.standard_normal((50, 70)).astype(np.float32)
    x = g.standard_normal(70).astype(np.float32)
    v = g.standard_normal(50).astype(np.float32)
    assert np.allclose(oracle.matvec_f64(A, x), A.astype(np.float64) @ x.astype(np.float64),
                       rtol=1e-12, atol=1e-12)
    assert np.allclose(oracle.vecmat_f64(v, A), v.astype(np.float64) @ A.astype(np.float64),
                       rtol=1e-12, atol=1e-12)
    # x^T A = (A^T x)^T: the left product equals the right product of the transpose
    assert np.array_equal(oracle.vecmat_f64(v, A), oracle.matvec_f64(oracle.transpose_f32(A), v))


# ---- binary32 keys (Listing 4 sorts REAL_32) ----

def _f32(bits):
    return np.array(bits, dtype=np.uint32).view(np.float32)


# the totalOrder of IEEE 754 (Sec. 5.10) on these bit patterns, written out
# by hand: -NaN(big payload), -NaN(small), -inf, -2.5, -tiny, -0, +0, +tiny,
# 1.0, +inf, +NaN(small), +NaN(big)
TOTAL_ORDER = [0xFFC00005, 0xFFC00001, 0xFF800000, 0xC0200000, 0x80000001, 0x80000000,
               0x00000000, 0x00000001, 0x3F800000, 0x7F800000, 0x7FC00001, 0x7FC00005]


def test_sort_f32_total_order_special_values():
    want = _f32(TOTAL_ORDER).view(np.uint32)
    g = np.random.default_rng(31)
    for _ in range(200):
        x = _f32(TOTAL_ORDER)[g.permutation(len(TOTAL_ORDER))]
        assert np.array_equal(oracle.sort_f32(x).view(np.uint32), want)


def test_sort_f32_brute_force_small():
    # all permutations of 7 keys with repeats and both zeros: one output
    base = _f32([0x80000000, 0x00000000, 0x3F800000, 0x3F800000, 0xBF800000, 0x7F800000,
                 0x7FC00000])
    want = None
    for p in itertools.permutations(range(7)):
        got = oracle.sort_f32(base[list(p)]).view(np.uint32)
        if want is None:
            want = got
            assert list(got) == [0xBF800000, 0x80000000, 0x00000000, 0x3F800000, 0x3F800000,
                                 0x7F800000, 0x7FC00000]
        assert np.array_equal(got, want)


def test_sort_f32_matches_numpy_on_finite_nonzero():
    g = np.random.default_rng(32)
    x = (g.standard_normal(100000) * 1e3).astype(np.float32)
    x[x == 0] = 1.0
    assert np.array_equal(oracle.sort_f32(x), np.sort(x))
    assert oracle.first_unsorted_f32(oracle.sort_f32(x)) == -1


def test_first_unsorted_f32_ieee():
    x = np.array([1.0, 2.0, 2.0, 5.0, 3.0, 4.0], np.float32)
    assert oracle.first_unsorted_f32(x) == 3
    # NaN compares false and +0 / -0 compare equal: neither is a violation
    assert oracle.first_unsorted_f32(np.array([1.0, np.nan, 0.5], np.float32)) == -1
    assert oracle.first_unsorted_f32(_f32([0x00000000, 0x80000000])) == -1
    assert oracle.first_unsorted_f32(np.array([], np.float32)) == -1
