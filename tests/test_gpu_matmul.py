"""GPU parity of matrix `multiply` (Sec. 3.4) in its three forms -- binary32
SIMT, bf16 and fp16 operands on the tensor cores with binary32 accumulation --
and of its Freivalds postcondition, through the C ABI.

Normwise error eta = |C - C*|_F / |C*|_F against the binary64 oracle:
binary32 <= 1e-5; fp16 operands <= 2e-3; bf16 operands <= 8e-3 (operand
rounding u = 2^-11 / 2^-8 dominates; expected about u*sqrt(2/3)).  Small
integer matrices are exact in every form, so they must match bit for bit."""
import math

import numpy as np
import pytest

import oracle
from paper_1410_6685_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = {0: 1e-5, 1: 8e-3, 2: 2e-3}


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    yield sg, ctx, torch
    sg.sg_destroy(ctx)


def gemm(env, A, B, prec, flush=True):
    sg, ctx, torch = env
    ta = torch.from_numpy(np.ascontiguousarray(A, dtype=np.float32)).cuda()
    tb = torch.from_numpy(np.ascontiguousarray(B, dtype=np.float32)).cuda()
    ma, mb = sg.wrap_tensor(ctx, ta), sg.wrap_tensor(ctx, tb)
    mc = sg.sg_matmul(ctx, ma, mb, prec)
    if flush:
        sg.sg_flush(ctx)
    return mc, (ta, tb, ma, mb)


def read(env, m, M, N):
    sg, ctx, _ = env
    return sg.sg_matrix_read(ctx, m, np.empty((M, N), np.float32))


def eta(C, ref):
    return np.linalg.norm(C.astype(np.float64) - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("shape", [(1, 1, 1), (7, 13, 5), (128, 256, 64), (129, 257, 65),
                                   (300, 500, 200), (512, 512, 512)])
def test_matmul_normwise_error(env, prec, shape):
    M, K, N = shape
    g = np.random.default_rng(M * 7 + N)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((K, N)).astype(np.float32)
    mc, keep = gemm(env, A, B, prec)
    C = read(env, mc, M, N)
    assert eta(C, oracle.matmul_f64(A, B)) <= TOL[prec]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_matmul_small_integers_exact(env, prec):
    g = np.random.default_rng(11)
    M, K, N = 200, 320, 300
    A = g.integers(-8, 9, (M, K)).astype(np.float32)
    B = g.integers(-8, 9, (K, N)).astype(np.float32)
    mc, keep = gemm(env, A, B, prec)
    assert np.array_equal(read(env, mc, M, N), oracle.matmul_f64(A, B).astype(np.float32))


@pytest.mark.parametrize("prec", [0, 1])
def test_identity_and_permutation(env, prec):
    n = 256
    A, B = inputs.matmul_inputs(n)
    # bf16-representable values so the product is exact in every form
    if prec:
        A = (A.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32)
    I = np.eye(n, dtype=np.float32)
    mc, keep = gemm(env, I, A, prec)
    assert np.array_equal(read(env, mc, n, n), A)
    P = np.eye(n, dtype=np.float32)[np.random.default_rng(2).permutation(n)]
    mc, keep = gemm(env, A, P, prec)
    assert np.array_equal(read(env, mc, n, n), oracle.matmul_f64(A, P).astype(np.float32))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_workload_1024(env, prec):
    """The matmul workload at N = 1024, N(0,1) entries."""
    n = 1024
    A, B = inputs.matmul_inputs(n)
    mc, keep = gemm(env, A, B, prec)   # the built-in Freivalds check must pass
    C = read(env, mc, n, n)
    assert eta(C, oracle.matmul_f64(A, B)) <= TOL[prec]


_ROWS_CACHE = {}


def oracle_rows(n, nrows=512):
    """Binary64 oracle rows of C = A B for the matmul workload at size n, on
    `nrows` seeded random rows (the full binary64 product at 8192 is 5.5e11
    multiply-adds).  Row blocks go to the C oracle from a thread pool; each
    call computes its rows exactly as the single-threaded oracle does."""
    key = (n, nrows)
    if key not in _ROWS_CACHE:
        from concurrent.futures import ThreadPoolExecutor
        import os
        A, B = inputs.matmul_inputs(n)
        rows = np.sort(np.random.default_rng(3).choice(n, nrows, replace=False))
        parts = np.array_split(rows, min(16, os.cpu_count() or 1))
        with ThreadPoolExecutor(len(parts)) as ex:
            refs = list(ex.map(lambda r: oracle.matmul_rows_f64(A, B, r), parts))
        _ROWS_CACHE[key] = (A, B, rows, np.concatenate(refs))
    return _ROWS_CACHE[key]


@pytest.mark.parametrize("prec", [0, 1, 2])
@pytest.mark.parametrize("n", [4096, 8192])
def test_workload_sampled_rows(env, n, prec):
    """The matmul workload at N = 4096 and 8192 in all three forms (binary32
    SIMT, bf16 and fp16 operands on the tensor cores), through the same call
    whose built-in Freivalds postcondition must pass; eta on 512 seeded rows
    against the binary64 oracle."""
    A, B, rows, ref = oracle_rows(n)
    mc, keep = gemm(env, A, B, prec)
    C = read(env, mc, n, n)
    env[0].sg_matrix_release(mc)
    assert eta(C[rows], ref) <= TOL[prec]


def test_freivalds_flags_planted_row(env):
    """User-attached ensure(C = A B) on matrices given by the caller."""
    sg, ctx, torch = env
    n = 512
    A, B = inputs.matmul_inputs(n)
    C = (A.astype(np.float64) @ B.astype(np.float64)).astype(np.float32)
    u_eff = 2.0 ** -24 * math.sqrt(n)
    first, gap, tau = oracle.freivalds(A, B, C, seed=6, nvec=4, c=8.0, u_eff=u_eff)
    assert first == -1
    for row in [0, 311, n - 1]:
        D = C.copy()
        D[row, 17] += np.float32(4 * tau[row])
        assert oracle.freivalds(A, B, D, seed=6, nvec=4, c=8.0, u_eff=u_eff)[0] == row
        ta, tb, td = (torch.from_numpy(x).cuda() for x in (A, B, D))
        ma, mb, md = (sg.wrap_tensor(ctx, t) for t in (ta, tb, td))
        sg.sg_ensure(ctx, md, sg.contract(sg.SG_C_FREIVALDS, other=[ma, mb], seed=6, nvec=4,
                                          tol=8.0))
        with pytest.raises(sg.SgError) as e:
            sg.sg_flush(ctx)
        assert e.value.status == sg.SG_ERR_POSTCONDITION
        v = sg.sg_last_violation(ctx)
        assert v.kind == sg.SG_C_FREIVALDS and v.first_index == row
    # the clean product passes, and the GPU's worst ratio is close to the oracle's
    ta, tb, tc = (torch.from_numpy(x).cuda() for x in (A, B, C))
    ma, mb, mc = (sg.wrap_tensor(ctx, t) for t in (ta, tb, tc))
    sg.sg_ensure(ctx, mc, sg.contract(sg.SG_C_FREIVALDS, other=[ma, mb], seed=6, nvec=4, tol=8.0))
    sg.sg_flush(ctx)


def test_contract_modes_matmul(env):
    sg, ctx, _ = env
    n = 256
    A, B = inputs.matmul_inputs(n)
    sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_OFF)
    try:
        mc, keep = gemm(env, A, B, 1, flush=False)
        assert "freivalds" not in sg.sg_plan_describe(ctx)
        sg.sg_flush(ctx)
    finally:
        sg.sg_set_contract_mode(ctx, sg.SG_CONTRACTS_PRE_POST)
    mc, keep = gemm(env, A, B, 1, flush=False)
    assert "freivalds" in sg.sg_plan_describe(ctx)
    sg.sg_flush(ctx)


def test_fused_check_in_plan(env):
    """The built-in Freivalds check of a square tensor-core product is folded
    into the product (casts + epilogue); the binary32 product keeps the
    stand-alone check, and so does a product with fusion switched off."""
    sg, ctx, _ = env
    A, B = inputs.matmul_inputs(256)
    for prec, fused in [(1, True), (2, True), (0, False)]:
        mc, keep = gemm(env, A, B, prec, flush=False)
        d = sg.sg_plan_describe(ctx)
        assert ("+freivalds(fused)" in d) == fused, d
        assert ("freivalds n=256" in d) == (not fused), d
        sg.sg_flush(ctx)
    sg.sg_set_fusion(ctx, sg.SG_FUSE_OFF)
    try:
        mc, keep = gemm(env, A, B, 1, flush=False)
        assert "freivalds n=256" in sg.sg_plan_describe(ctx)
        sg.sg_flush(ctx)
    finally:
        sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("n", [512, 1000])
@pytest.mark.parametrize("fusion", [True, False])
def test_builtin_check_flags_planted_element(env, prec, n, fusion):
    """An error planted in one product element (host-chosen, applied by the
    kernel's epilogue before the store) is reported by the built-in
    postcondition at its row, in the fused and the stand-alone forms; the
    oracle, given the product read back, names the same row."""
    sg, ctx, _ = env
    A, B = inputs.matmul_inputs(n)
    u_eff = (2.0 ** -8 if prec == 1 else 2.0 ** -10) + 2.0 ** -24 * math.sqrt(n)
    mc, keep = gemm(env, A, B, prec)
    C0 = read(env, mc, n, n)
    first, gap, tau = oracle.freivalds(A, B, C0, seed=6, nvec=4, c=8.0, u_eff=u_eff)
    assert first == -1
    sg.sg_set_fusion(ctx, sg.SG_FUSE_ON if fusion else sg.SG_FUSE_OFF)
    try:
        for row, col in [(0, 0), (n // 3, n - 1), (n - 1, 17)]:
            delta = np.float32(4 * tau[row])
            sg.sg_debug_inject_matmul(ctx, row, col, float(delta))
            mc, keep = gemm(env, A, B, prec, flush=False)
            with pytest.raises(sg.SgError) as e:
                sg.sg_flush(ctx)
            assert e.value.status == sg.SG_ERR_POSTCONDITION
            v = sg.sg_last_violation(ctx)
            assert v.kind == sg.SG_C_FREIVALDS and v.first_index == row
            assert oracle.freivalds(A, B, C0 + np.where(
                (np.arange(n)[:, None] == row) & (np.arange(n)[None, :] == col), delta,
                np.float32(0)), seed=6, nvec=4, c=8.0, u_eff=u_eff)[0] == row
    finally:
        sg.sg_set_fusion(ctx, sg.SG_FUSE_ON)
    # the injection is consumed: the next product is clean again
    mc, keep = gemm(env, A, B, prec)
    assert np.array_equal(read(env, mc, n, n), C0)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("shape", [(129, 257, 65), (300, 500, 700), (1024, 1024, 1024)])
def test_portable_one_cta_product(env, prec, shape):
    """The one-CTA tensor-core product (the form for devices without CTA
    pairs), forced through the testing switch: within the operand-rounding
    bound of the oracle, and within binary32 accumulation distance of the
    CTA-pair form (both accumulate the same bf16/fp16 products in binary32)."""
    sg, ctx, _ = env
    M, K, N = shape
    g = np.random.default_rng(M + 3 * N)
    A = g.standard_normal((M, K)).astype(np.float32)
    B = g.standard_normal((K, N)).astype(np.float32)
    mc, keep = gemm(env, A, B, prec)
    fast = read(env, mc, M, N)
    sg.sg_matrix_release(mc)
    sg.sg_debug_portable_kernels(ctx, True)
    try:
        mc, keep2 = gemm(env, A, B, prec)
        one = read(env, mc, M, N)
        sg.sg_matrix_release(mc)
    finally:
        sg.sg_debug_portable_kernels(ctx, False)
    ref = oracle.matmul_f64(A, B)
    assert eta(one, ref) <= TOL[prec]
    assert eta(one, fast.astype(np.float64)) <= 1e-5
