"""Grouped products (one persistent launch per stage, replayed from a CUDA graph)
against the single-product path and the CPU oracle.

FP64 and FP64-accuracy results are bit-identical to mm_gemm on each problem
(same kernels, same slice counts, exact integer recombination); FP32-accuracy
results meet their bound against the oracle. Graph replay with new
descriptors, re-capture on growth, and edge problems (k = 0, empty, k <= 4)
are covered.
"""
import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from gpu_util import bound_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def make_set(count, lo, hi, seed):
    dims = inputs.problem_set(count, lo, hi, seed)
    probs = []
    for i, (m, n, k) in enumerate(dims):
        A = inputs.row_scaled(int(m), int(k), seed * 1000 + i)
        B = inputs.col_scaled(int(k), int(n), seed * 1000 + i)
        probs.append((A, B))
    return probs


def to_dev(probs):
    out = []
    for A, B in probs:
        Ad = torch.from_numpy(A).cuda()
        Bd = torch.from_numpy(B).cuda()
        Cd = torch.full((A.shape[0], B.shape[1]), np.nan, dtype=torch.float64, device="cuda")
        out.append((Ad, Bd, Cd))
    return out


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_grouped_matches_single(h, mm, prec):
    probs = make_set(40, 1, 300, 7 + prec)
    dp = to_dev(probs)
    h.grouped(dp, precision=prec)
    assert h.sync() == 0
    for (A, B), (Ad, Bd, Cd) in zip(probs, dp):
        Cs = h.gemm(Ad, Bd, precision=prec)
        assert h.sync() == 0
        Cg = Cd.cpu().numpy()
        if prec in (0, 1):
            assert np.array_equal(Cg, Cs.cpu().numpy())
        k = A.shape[1]
        mode = {0: "fp64", 1: "fp64_emu", 2: "fp32_emu"}[prec]
        assert bound_ok(Cg, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(k, mode))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_graph_replay_new_descriptors_and_recapture(h, mm, prec):
    # same count and precision: the captured graph is replayed with new data
    for rnd in range(3):
        probs = make_set(24, 8, 200 if rnd < 2 else 700, 50 + rnd + 10 * prec)
        dp = to_dev(probs)
        h.grouped(dp, precision=prec)
        assert h.sync() == 0
        mode = {0: "fp64", 1: "fp64_emu", 2: "fp32_emu"}[prec]
        for (A, B), (_, _, Cd) in list(zip(probs, dp))[::5]:
            assert bound_ok(Cd.cpu().numpy(), oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(A.shape[1], mode))


def test_grouped_edge_problems(h, mm):
    shapes = [(5, 7, 0), (0, 4, 3), (6, 0, 2), (9, 11, 3), (33, 17, 4), (70, 90, 130), (1, 1, 1)]
    for prec in (0, 1, 2):
        dp, ref = [], []
        for i, (m, n, k) in enumerate(shapes):
            A = inputs.row_scaled(m, k, 3 + i) if m and k else np.zeros((m, k))
            B = inputs.col_scaled(k, n, 3 + i) if n and k else np.zeros((k, n))
            Ad = torch.from_numpy(np.ascontiguousarray(A)).cuda()
            Bd = torch.from_numpy(np.ascontiguousarray(B)).cuda()
            Cd = torch.full((m, n), 5.0, dtype=torch.float64, device="cuda")
            dp.append((Ad, Bd, Cd))
            ref.append((A, B))
        h.grouped(dp, precision=prec)
        assert h.sync() == 0
        mode = {0: "fp64", 1: "fp64_emu", 2: "fp32_emu"}[prec]
        for (A, B), (_, _, Cd) in zip(ref, dp):
            C = Cd.cpu().numpy()
            if C.size == 0:
                continue
            if A.shape[1] == 0:
                assert np.all(C == 0.0)
            else:
                assert bound_ok(C, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(A.shape[1], mode))


def test_grouped_workload_shape_bit_identical(h, mm):
    # the grouped workload's shape mix (dims log-uniform on [32, 1024]), fewer problems
    dims = inputs.problem_set(96, 32, 1024, 4)
    dp = []
    for i, (m, n, k) in enumerate(dims):
        Ad = torch.empty((int(m), int(k)), dtype=torch.float64, device="cuda")
        Bd = torch.empty((int(k), int(n)), dtype=torch.float64, device="cuda")
        mm.fill_uniform(Ad, 4000 + i, inputs.STREAM_A)
        mm.fill_uniform(Bd, 4000 + i, inputs.STREAM_B)
        dp.append((Ad, Bd, torch.empty((int(m), int(n)), dtype=torch.float64, device="cuda")))
    for prec in (0, 1):
        h.grouped(dp, precision=prec)
        assert h.sync() == 0
        for Ad, Bd, Cd in dp[::7]:
            Cs = h.gemm(Ad, Bd, precision=prec)
            assert torch.equal(Cs, Cd)
    Ad, Bd, Cd = dp[3]
    A, B = Ad.cpu().numpy(), Bd.cpu().numpy()
    assert bound_ok(Cd.cpu().numpy(), oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(A.shape[1], "fp64_emu"))


def test_grouped_argument_errors(h, mm):
    X = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(mm.MMError):
        h.grouped([(X, X, X)], precision=1)   # C overlaps A and B
    assert h.lib.mm_gemm_grouped(h.h, -1, None, 0, None) == 2
    assert h.lib.mm_gemm_grouped(h.h, 0, None, 0, None) == 0
