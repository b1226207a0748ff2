"""GPU parity of matrix `transpose` and the matrix-vector products
`right_multiply` / `left_multiply` (Sec. 3.4; Listing 1 chains transpose and
right_multiply), through the C ABI.  The transpose is bit-exact; the products
are compared with the binary64 oracle within the binary32 summation bound
(terms + 8) 2^-24 sum |a x| stated in the header."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1), (7, 13), (64, 64), (65, 127), (1000, 3), (3, 1000), (513, 2048), (2048, 1031), (300, 3076),
          (300, 4096), (1000, 5002), (4099, 4608)]


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1410_6685_gb300 import safegpu as sg
    ctx = sg.sg_init(0, torch.cuda.current_stream().cuda_stream)
    yield sg, ctx, torch
    sg.sg_destroy(ctx)


def dev(env, a):
    sg, ctx, torch = env
    t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    return sg.wrap_tensor(ctx, t), t


def bound(A, x, left):
    terms = A.shape[0] if left else A.shape[1]
    ax = np.abs(A.astype(np.float64))
    s = (np.abs(x) @ ax) if left else (ax @ np.abs(x))
    return (terms + 8) * 2.0 ** -24 * s + 1e-30


@pytest.mark.parametrize("shape", SHAPES)
def test_transpose_bit_exact(env, shape):
    sg, ctx, _ = env
    A = np.random.default_rng(shape[0] * 7 + shape[1]).standard_normal(shape).astype(np.float32)
    mA, keep = dev(env, A)
    mt = sg.sg_transpose(ctx, mA)
    got = sg.sg_matrix_read(ctx, mt, np.empty((shape[1], shape[0]), np.float32))
    sg.sg_matrix_release(mt)
    assert np.array_equal(got, oracle.transpose_f32(A))


@pytest.mark.parametrize("shape", SHAPES)
def test_matvec_and_vecmat(env, shape):
    sg, ctx, _ = env
    g = np.random.default_rng(shape[0] * 11 + shape[1])
    A = g.standard_normal(shape).astype(np.float32)
    x = g.standard_normal(shape[1]).astype(np.float32)
    v = g.standard_normal(shape[0]).astype(np.float32)
    mA, k1 = dev(env, A)
    vx, k2 = dev(env, x)
    vv, k3 = dev(env, v)
    y = sg.sg_matvec(ctx, mA, vx)
    got = sg.sg_vector_read(ctx, y, np.empty(shape[0], np.float32))
    sg.sg_vector_release(y)
    ref = oracle.matvec_f64(A, x)
    assert np.all(np.abs(got - ref) <= bound(A, x, False))
    z = sg.sg_vecmat(ctx, vv, mA)
    got = sg.sg_vector_read(ctx, z, np.empty(shape[1], np.float32))
    sg.sg_vector_release(z)
    ref = oracle.vecmat_f64(v, A)
    assert np.all(np.abs(got - ref) <= bound(A, v, True))


def test_listing1_transpose_folded_into_left_product(env):
    """matrix.transpose.right_multiply(vector) (Listing 1): with the transpose's
    handle released the plan has no transpose pass and gives x^T A bit for bit;
    with the handle kept the transpose is materialised and read back."""
    sg, ctx, _ = env
    g = np.random.default_rng(3)
    A = g.standard_normal((777, 1536)).astype(np.float32)
    v = g.standard_normal(777).astype(np.float32)
    mA, k1 = dev(env, A)
    vv, k2 = dev(env, v)
    z = sg.sg_vecmat(ctx, vv, mA)
    direct = sg.sg_vector_read(ctx, z, np.empty(1536, np.float32))
    sg.sg_vector_release(z)
    mt = sg.sg_transpose(ctx, mA)
    y = sg.sg_matvec(ctx, mt, vv)
    sg.sg_matrix_release(mt)
    plan = sg.sg_plan_describe(ctx)
    assert "transpose" not in plan.replace("transpose folded", "") and "vecmat 777x1536" in plan, plan
    got = sg.sg_vector_read(ctx, y, np.empty(1536, np.float32))
    sg.sg_vector_release(y)
    assert np.array_equal(got, direct)
    assert np.all(np.abs(got - oracle.vecmat_f64(v, A)) <= bound(A, v, True))
    # handle kept: transpose materialised, right product on it
    mt = sg.sg_transpose(ctx, mA)
    y = sg.sg_matvec(ctx, mt, vv)
    plan = sg.sg_plan_describe(ctx)
    assert "transpose 777x1536" in plan and "matvec 1536x777" in plan, plan
    got = sg.sg_vector_read(ctx, y, np.empty(1536, np.float32))
    assert np.array_equal(sg.sg_matrix_read(ctx, mt, np.empty((1536, 777), np.float32)), A.T)
    assert np.all(np.abs(got - oracle.vecmat_f64(v, A)) <= bound(A, v, True))
    sg.sg_vector_release(y)
    sg.sg_matrix_release(mt)


def test_shape_precondition(env):
    sg, ctx, _ = env
    mA, k1 = dev(env, np.zeros((4, 5), np.float32))
    vx, k2 = dev(env, np.zeros(4, np.float32))
    with pytest.raises(sg.SgError) as e:
        sg.sg_matvec(ctx, mA, vx)
    assert e.value.status == sg.SG_ERR_SHAPE
    vy, k3 = dev(env, np.zeros(5, np.float32))
    with pytest.raises(sg.SgError) as e:
        sg.sg_vecmat(ctx, vy, mA)
    assert e.value.status == sg.SG_ERR_SHAPE


def test_full_size_transpose_and_products_sampled(env):
    """8192 x 8192 (the paper's transpose benchmark scale, 6.7e7 elements):
    the transpose checked exactly on sampled rows, the products on sampled
    entries against the oracle."""
    sg, ctx, torch = env
    n = 8192
    g = torch.Generator(device="cuda").manual_seed(12)
    tA = torch.randn(n, n, device="cuda", generator=g)
    tx = torch.randn(n, device="cuda", generator=g)
    mA, vx = sg.wrap_tensor(ctx, tA), sg.wrap_tensor(ctx, tx)
    mt = sg.sg_transpose(ctx, mA)
    At = sg.sg_matrix_read(ctx, mt, np.empty((n, n), np.float32))
    sg.sg_matrix_release(mt)
    A = tA.cpu().numpy()
    x = tx.cpu().numpy()
    rows = np.random.default_rng(1).choice(n, 16, replace=False)
    for r in rows:
        assert np.array_equal(At[r], A[:, r])
    y = sg.sg_matvec(ctx, mA, vx)
    yv = sg.sg_vector_read(ctx, y, np.empty(n, np.float32))
    sg.sg_vector_release(y)
    ref = oracle.matvec_f64(A[rows], x)
    assert np.all(np.abs(yv[rows] - ref) <= bound(A[rows], x, False))
    # x^T A at full size (the clustered left product): every entry
    z = sg.sg_vecmat(ctx, vx, mA)
    zv = sg.sg_vector_read(ctx, z, np.empty(n, np.float32))
    sg.sg_vector_release(z)
    assert np.all(np.abs(zv - oracle.vecmat_f64(x, A)) <= bound(A, x, True))
