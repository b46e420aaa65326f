"""The INT8 digit form on the legacy integer tensor path (mma.sync m16n8k32 s8),
through the C ABI, against the oracle's INT8 form.

Level products bit for bit (ragged tiles and k, the top digit at its largest,
a k past one int32 segment), the recombined product equal to the exact kept
sum rounded once, the automatic count from halved spreads, default products
within the componentwise bound, and the plain fallback's bits.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from gpu_util import bound_ok, fixed_shift

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

I8 = em.OFFSET_INT8


@pytest.fixture(scope="module")
def mm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2408_15384_gb300 as mm
    from paper_2408_15384_gb300 import build
    build.build()
    return mm


@pytest.fixture(scope="module")
def h(mm):
    with mm.Handle(0) as hh:
        yield hh


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def top_of_binade(A):
    """Each row's largest entry the largest double below a power of two (the
    INT8 form's top digit reaches 64 there)."""
    A = A.copy()
    for i in range(A.shape[0]):
        A[i, (7 * i) % A.shape[1]] = math.ldexp(1.0 - 2.0 ** -53, i % 7 - 3) * (-1 if i % 2 else 1)
    return A


@pytest.mark.parametrize("m,n,k,s", [(130, 70, 300, 5), (257, 129, 1000, 6), (64, 64, 33, 3), (31, 9, 500, 7)])
def test_int8_level_products_bit_exact(h, m, n, k, s):
    A = top_of_binade(inputs.row_scaled(m, k, 10 + k))
    B = np.ascontiguousarray(top_of_binade(inputs.col_scaled(k, n, 20 + k).T).T)
    _, sA = em.fp64_slices_A(A, s, offset=I8)
    _, sB = em.fp64_slices_B(B, s, offset=I8)
    L_ref = em.level_products(sA, sB, s)
    assert np.array_equal(h.debug_levels_int8(dev(A), dev(B), s).cpu().numpy(), L_ref)


def test_int8_level_products_past_one_segment(h):
    # k = 17000: more than 512 K blocks of 32, the int32 sums fold mid-level
    m, n, k, s = 40, 24, 17000, 5
    A = inputs.row_scaled(m, k, 5)
    B = inputs.col_scaled(k, n, 5)
    _, sA = em.fp64_slices_A(A, s, offset=I8)
    _, sB = em.fp64_slices_B(B, s, offset=I8)
    assert np.array_equal(h.debug_levels_int8(dev(A), dev(B), s).cpu().numpy(), em.level_products(sA, sB, s))


@pytest.mark.parametrize("s", [4, 5])
def test_int8_product_is_the_exact_kept_sum_rounded_once(h, mm, s):
    m, n, k = 200, 150, 900
    A = inputs.row_scaled(m, k, 30 + s)
    B = inputs.col_scaled(k, n, 30 + s)
    assert fixed_shift(s, k) == 0
    Ad, Bd = dev(A), dev(B)
    h.set_option(mm.OPT_INT8_SLICES, 1)
    h.set_option(mm.OPT_SLICES, s)
    try:
        C = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
        assert h.sync() == 0
    finally:
        h.set_option(mm.OPT_SLICES, 0)
        h.set_option(mm.OPT_INT8_SLICES, 0)
    assert np.array_equal(C.cpu().numpy(), em.gemm_fp64_emu(A, B, s, offset=I8))


@pytest.mark.parametrize("dist,m,n,k", [("scaled", 300, 260, 700), ("normal", 128, 96, 4100), ("cauchy", 64, 48, 900)])
def test_int8_default_within_bound(h, mm, dist, m, n, k):
    gen = {"scaled": lambda r, c, sd, st: (inputs.row_scaled(r, c, sd) if st == 1 else inputs.col_scaled(r, c, sd)),
           "normal": lambda r, c, sd, st: inputs.box_muller(r, c, sd, st),
           "cauchy": lambda r, c, sd, st: inputs.cauchy(r, c, sd, st)}[dist]
    A = gen(m, k, 50 + k, 1)
    B = gen(k, n, 50 + k, 2)
    Ad, Bd = dev(A), dev(B)
    h.set_option(mm.OPT_INT8_SLICES, 1)
    try:
        C = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
        assert h.sync() == 0
    finally:
        h.set_option(mm.OPT_INT8_SLICES, 0)
    got = C.cpu().numpy()
    assert bound_ok(got, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(k, "fp64_emu"))
    s = em.slice_count_int8(A, B)
    if s == em.S_PLAIN:
        Cp = h.gemm(Ad, Bd, precision=mm.FP64)
        assert h.sync() == 0
        assert np.array_equal(got, Cp.cpu().numpy())
    elif fixed_shift(s, k) == 0 and s <= em.S_MAX:
        # far from a threshold of the rule here: the same count as the oracle's
        assert np.array_equal(got, em.gemm_fp64_emu(A, B, s, offset=I8))
