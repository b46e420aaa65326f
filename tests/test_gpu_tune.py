"""The launch-configuration autotuner: tuned entries per shape bucket, results
unchanged by tuning (FP64-accuracy bit for bit), the grouped path on every tile
width it can pick, and the table's save / load round trip.
"""
import os

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


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run(h, A, B, prec):
    C = h.gemm(dev(A), dev(B), precision=prec)
    assert h.sync() == 0
    return C.cpu().numpy()


def test_autotune_single_fp64_emu_same_bits(mm):
    m, n, k = 700, 600, 900
    A = inputs.row_scaled(m, k, 61)
    B = inputs.col_scaled(k, n, 61)
    with mm.Handle(0) as h0:
        ref = run(h0, A, B, mm.FP64_EMU)
        assert h0.tune_lookup(mm.FP64_EMU, m, n, k) is None      # autotuning is off by default
    with mm.Handle(0) as h:
        h.set_option(mm.OPT_AUTOTUNE, 1)
        C1 = run(h, A, B, mm.FP64_EMU)
        entry = h.tune_lookup(mm.FP64_EMU, m, n, k)
        assert entry is not None
        bn, cg, _ = entry
        assert bn in (128, 192, 240, 256) and cg in (1, 2)
        # a later product of the same bucket uses the entry: one split pass (the
        # fused scan of both operands, the column spreads, row and column
        # slicing), one slice GEMM (k = 900 admits only s = 6 or 7, one kernel
        # for both) and the plain-FP64 fallback launch, which returns at once;
        # m n k is below 2^33, so the modular form is not among the candidates
        n0 = h.stats()
        C2 = run(h, A, B, mm.FP64_EMU)
        assert h.stats() - n0 == 6
        assert h.tune_lookup(mm.FP64_EMU, 720, 620, 1000) == entry   # same bucket
    assert np.array_equal(C1, ref) and np.array_equal(C2, ref)


def test_autotune_plain_and_fp32(mm):
    m, n, k = 300, 280, 500
    A = inputs.uniform(m, k, 62, inputs.STREAM_A)
    B = inputs.uniform(k, n, 62, inputs.STREAM_B)
    C_ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
    with mm.Handle(0) as h:
        h.set_option(mm.OPT_AUTOTUNE, 1)
        C = run(h, A, B, mm.FP64)
        assert h.tune_lookup(mm.FP64, m, n, k)[2] in (1, 2)
        assert bound_ok(C, C_ref, D, em.gamma(k, "fp64"))
        C = run(h, A, B, mm.FP32_EMU)
        bn, cg, _ = h.tune_lookup(mm.FP32_EMU, m, n, k)
        assert (bn, cg) in ((128, 1), (256, 1), (256, 2))
        assert bound_ok(C, C_ref, D, em.gamma(k, "fp32_emu"))


def make_group(count, lo, hi, seed):
    dims = inputs.problem_set(count, lo, hi, seed)
    probs = []
    for i, (m, n, k) in enumerate(dims):
        A = inputs.row_scaled(int(m), int(k), seed * 100 + i)
        B = inputs.col_scaled(int(k), int(n), seed * 100 + i)
        probs.append((A, B))
    return probs


def run_group(h, probs, prec):
    dp = []
    for A, B in probs:
        dp.append((dev(A), dev(B), torch.full((A.shape[0], B.shape[1]), np.nan, dtype=torch.float64, device="cuda")))
    h.grouped(dp, precision=prec)
    assert h.sync() == 0
    return [C.cpu().numpy() for _, _, C in dp]


def group_bucket(probs):
    d = np.mean([np.cbrt(A.shape[0] * B.shape[1] * max(A.shape[1], 1)) for A, B in probs])
    return len(probs), int(round(d))


def test_autotune_grouped_same_bits(mm):
    probs = make_group(30, 16, 400, 63)
    with mm.Handle(0) as h0:
        ref = [run(h0, A, B, mm.FP64_EMU) for A, B in probs]
    with mm.Handle(0) as h:
        h.set_option(mm.OPT_AUTOTUNE, 1)
        out = run_group(h, probs, mm.FP64_EMU)
        cnt, d = group_bucket(probs)
        entry = h.tune_lookup(mm.FP64_EMU, cnt, d, grouped=True)
        assert entry is not None and entry[0] in (128, 256) and entry[1] == 1
        again = run_group(h, probs, mm.FP64_EMU)
    for C, Cr, C2 in zip(out, ref, again):
        assert np.array_equal(C, Cr) and np.array_equal(C2, Cr)


@pytest.mark.parametrize("prec", [1, 2])
def test_grouped_wide_tiles_from_loaded_table(mm, tmp_path, prec):
    # force the 256-wide grouped kernels through a loaded table entry
    probs = make_group(24, 16, 600, 64 + prec)
    cnt, d = group_bucket(probs)
    b_cnt, b_d = int(np.ceil(np.log2(cnt))), int(np.ceil(np.log2(d)))
    path = tmp_path / "tune.txt"
    path.write_text("# mm tune table v1: kind precision b0 b1 b2 bn cg kern ms\n"
                    f"1 {prec} {b_cnt} {b_d} 0 256 1 0 1.0\n")
    with mm.Handle(0) as h:
        ref = [run(h, A, B, prec) for A, B in probs]
        h.tune_load(str(path))
        assert h.tune_lookup(prec, cnt, d, grouped=True) == (256, 1, 0)
        out = run_group(h, probs, prec)
    for (A, B), C, Cr in zip(probs, out, ref):
        k = A.shape[1]
        if prec == mm.FP64_EMU:
            assert np.array_equal(C, Cr)
        mode = "fp64_emu" if prec == mm.FP64_EMU else "fp32_emu"
        assert bound_ok(C, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(k, mode))


def test_tune_table_save_load(mm, tmp_path):
    m, n, k = 260, 300, 200
    A = inputs.row_scaled(m, k, 65)
    B = inputs.col_scaled(k, n, 65)
    path = str(tmp_path / "table.txt")
    with mm.Handle(0) as h:
        h.set_option(mm.OPT_AUTOTUNE, 1)
        run(h, A, B, mm.FP64_EMU)
        entry = h.tune_lookup(mm.FP64_EMU, m, n, k)
        h.tune_save(path)
    text = open(path).read().splitlines()
    assert text[0].startswith("# mm tune table v1") and len(text) == 2
    with mm.Handle(0) as h2:
        assert h2.tune_lookup(mm.FP64_EMU, m, n, k) is None
        h2.tune_load(path)
        assert h2.tune_lookup(mm.FP64_EMU, m, n, k) == entry
        with pytest.raises(mm.MMError) as ei:
            h2.tune_load(str(tmp_path / "missing.txt"))
        assert ei.value.status == mm.NOT_FOUND
        bad = tmp_path / "bad.txt"
        bad.write_text("# mm tune table v1\n0 1 9 9 9 200 1 0 1.0\n")     # 200 columns: no such kernel
        with pytest.raises(mm.MMError) as ei:
            h2.tune_load(str(bad))
        assert ei.value.status == mm.INVALID_ARG
        assert h2.tune_lookup(mm.FP64_EMU, 2 ** 9, 2 ** 9, 2 ** 9) is None
