"""The automatic FP64-accuracy slice count on the device against the oracle.

The device forms each row's and column's spread in float from a one-pass
scan; the oracle sums exactly. The smallest spreads must agree to float
rounding, and the slice count must be the oracle's, except where the oracle's
own spreads sit within that rounding of a threshold of the rule (then either
neighbouring count is correct). The products are then checked within the
componentwise bound on every output, and the plain FP64 fallback against the
plain kernel bit for bit.
"""
import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from gpu_util import bound_ok, max_ratio

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-4   # float sums of up to a few thousand terms per thread, and mantissas cut to 23 bits


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
    # the digit form for single products too, so that grouped and single
    # products are compared on the same form (grouped ones always take it)
    with mm.Handle(0) as hh:
        hh.set_option(mm.OPT_FP64_SCHEME, 1)
        yield hh


def _case(name, m, n, k, seed):
    if name == "uniform":
        return inputs.uniform(m, k, seed, 1), inputs.uniform(k, n, seed, 2)
    if name == "scaled":
        return inputs.row_scaled(m, k, seed), inputs.col_scaled(k, n, seed)
    if name == "normal":
        return inputs.box_muller(m, k, seed, 1), inputs.box_muller(k, n, seed, 2)
    if name == "t3":
        return inputs.student_t3(m, k, seed, 1), inputs.student_t3(k, n, seed, 2)
    if name == "spread":
        return inputs.wide_spread(m, k, seed, 1), inputs.wide_spread(k, n, seed, 2)
    if name == "cauchy":
        return inputs.cauchy(m, k, seed, 1), inputs.cauchy(k, n, seed, 2)
    if name == "special":
        # zero rows and columns, an all-subnormal row and column, a single-entry row
        A = inputs.uniform(m, k, seed, 1)
        B = inputs.uniform(k, n, seed, 2)
        A[3] = 0.0
        B[:, 5] = 0.0
        A[7] = inputs.uniform(1, k, seed, 3)[0] * 2.0 ** -1040
        B[:, 2] = inputs.uniform(k, 1, seed, 4)[:, 0] * 2.0 ** -1050
        A[9] = 0.0
        A[9, k // 2] = -3.5
        return A, B
    raise KeyError(name)


def oracle_spreads(A, B):
    a = em.row_spread(A, em.row_exponents(A, 2)).min()
    b = em.col_spread(B, em.col_exponents(B, 2)).min()
    return float(a), float(b)


def count_is_consistent(k, s_dev, a, b):
    """s_dev is the oracle's count, or a count the rule gives within REL of the oracle's spreads."""
    allowed = {em.slice_count_from_spread(k, a * f, b * g) for f in (1 - REL, 1, 1 + REL) for g in (1 - REL, 1, 1 + REL)}
    return s_dev in allowed


CASES = [("uniform", 70, 90, 700), ("scaled", 130, 50, 4100), ("normal", 40, 300, 1500), ("t3", 64, 64, 2000),
         ("spread", 33, 129, 777), ("cauchy", 50, 40, 900), ("special", 20, 24, 513), ("normal", 9, 7, 96)]


@pytest.mark.parametrize("name,m,n,k", CASES)
def test_device_count_and_spreads_match_the_oracle(h, mm, name, m, n, k):
    A, B = _case(name, m, n, k, 11 + k)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    s, a_dev, b_dev = h.debug_slice_count(Ad, Bd)
    a, b = oracle_spreads(A, B)
    assert abs(a_dev - a) <= REL * a and abs(b_dev - b) <= REL * b, (a_dev, a, b_dev, b)
    assert count_is_consistent(k, s, a, b), (s, em.slice_count_from_spread(k, a, b))
    # the product with that count, every output within the bound
    C = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
    assert h.sync() == 0
    ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
    g = em.gamma(k, "fp64_emu")
    got = C.cpu().numpy()
    # outputs in the subnormal range (the all-subnormal row and column) carry
    # the absolute rounding of gradual underflow: each of the oracle's k
    # products and sums, and the emulation's one rounding, may add up to
    # 2^-1075, so the componentwise bound gets that absolute term
    eta = (k + 1) * 2.0 ** -1074
    err = np.abs(got - ref)
    assert np.all(err <= g * D + eta), max_ratio(got, ref, D, g)
    if s == em.S_PLAIN:
        # the fallback is the plain FP64 kernel: the same bits as MM_FP64
        Cp = h.gemm(Ad, Bd, precision=mm.FP64)
        assert h.sync() == 0
        assert np.array_equal(got, Cp.cpu().numpy())


def test_count_follows_the_data_not_k(h, mm):
    # the same k, rows of different spread: uniform takes fewer slices than normal
    k = 4096
    Au, Bu = _case("scaled", 16, 16, k, 5)
    An, Bn = _case("normal", 16, 16, k, 5)
    su = h.debug_slice_count(torch.from_numpy(Au).cuda(), torch.from_numpy(Bu).cuda())[0]
    sn = h.debug_slice_count(torch.from_numpy(An).cuda(), torch.from_numpy(Bn).cuda())[0]
    assert (su, sn) == (5, 6)


def test_fixed_count_option_still_applies(h, mm):
    # MM_OPT_SLICES fixes s for every product: the level products' count shows it
    A, B = _case("normal", 24, 20, 300, 3)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    h.set_option(mm.OPT_SLICES, 4)
    try:
        C4 = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
        assert h.sync() == 0
    finally:
        h.set_option(mm.OPT_SLICES, 0)
    assert np.array_equal(C4.cpu().numpy(), em.gemm_fp64_emu(A, B, 4))


def test_grouped_problems_decide_their_own_counts(h, mm):
    # one group mixing uniform, normal and Cauchy problems: each problem gets
    # the count its own data asks for, the same bits as mm_gemm on it alone
    probs = []
    for i, (name, m, n, k) in enumerate([("uniform", 40, 60, 3000), ("normal", 70, 30, 3000),
                                         ("cauchy", 33, 45, 800), ("spread", 128, 130, 200),
                                         ("uniform", 5, 7, 3)]):
        A, B = _case(name, m, n, k, 90 + i)
        probs.append((A, B, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                      torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")))
    h.grouped([(a, b, c) for _, _, a, b, c in probs], precision=mm.FP64_EMU)
    assert h.sync() == 0
    for A, B, Ad, Bd, Cd in probs:
        alone = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
        assert h.sync() == 0
        assert np.array_equal(Cd.cpu().numpy(), alone.cpu().numpy())
        g = em.gamma(A.shape[1], "fp64_emu")
        assert bound_ok(Cd.cpu().numpy(), oracle.gemm(A, B), oracle.absprod(A, B), g)
