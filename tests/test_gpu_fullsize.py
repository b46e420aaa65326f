"""Parity at the workloads' full sizes, in the launch configuration the
benchmark uses (default options), on outputs the oracle computes row by row:

* 512^3 plain FP64, uniform[-1,1): every output;
* plain FP64 at 1024 .. 8192: sampled rows;
* split-precision inputs (uniform[-1,1) * 2^e per row of A / column of B) at
  4096 and 8192 in both emulated modes and the plain mode: sampled rows;
* a grouped batch of 512 products with dimensions log-uniform on [32, 1024]
  in all three modes: sampled rows of every problem, all outputs of some;
* a served stream of requests with dimensions log-uniform on [64, 4096],
  FP64/FP32-accuracy 50:50, under the 40 GB budget: sampled rows of each.
Inputs are made on the device by the seeded filler (bit-identical to the
input module, checked in test_gpu_gemm) and copied back for the oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from gpu_util import bound_ok, max_ratio

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODE = {0: "fp64", 1: "fp64_emu", 2: "fp32_emu"}


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
    with mm.Handle(0, budget_bytes=40 << 30) as hh:
        yield hh


def sample_rows(m, seed, count=6):
    rows = {0, m - 1, m // 2}
    extra = inputs.int_uniform(0, m - 1, count, seed, inputs.STREAM_DIMS)
    rows.update(int(r) for r in extra)
    return sorted(rows)


def device_inputs(mm, N, seed, scaled):
    A = torch.empty((N, N), dtype=torch.float64, device="cuda")
    B = torch.empty_like(A)
    if scaled:
        mm.fill_uniform(A, seed, inputs.STREAM_A, 1, inputs.STREAM_EXP_A)
        mm.fill_uniform(B, seed, inputs.STREAM_B, 2, inputs.STREAM_EXP_B)
    else:
        mm.fill_uniform(A, seed, inputs.STREAM_A)
        mm.fill_uniform(B, seed, inputs.STREAM_B)
    torch.cuda.synchronize()
    return A, B


_REF = {}


def _oracle_rows(Ah, Bh, rows):
    key = ("r", id(Ah), id(Bh), tuple(rows))
    if key not in _REF:
        _REF.clear()
        _REF[key] = (oracle.gemm_rows_par(Ah, Bh, rows), oracle.absprod_rows_par(Ah, Bh, rows))
    return _REF[key]


def check_rows(C, Ah, Bh, rows, mode, frac=1.0):
    k = Ah.shape[1]
    got = C[rows].cpu().numpy()
    ref, D = _oracle_rows(Ah, Bh, rows)
    g = frac * em.gamma(k, mode)
    assert bound_ok(got, ref, D, g), max_ratio(got, ref, D, g)


def check_cols(C, Ah, Bh, cols, mode, frac=1.0):
    # columns of A*B are the rows of the oracle's product of A with those columns of B
    k = Ah.shape[1]
    got = C[:, cols].cpu().numpy()
    Bc = np.ascontiguousarray(Bh[:, cols])
    all_rows = list(range(Ah.shape[0]))
    ref = oracle.gemm_rows_par(Ah, Bc, all_rows)
    D = oracle.absprod_rows_par(Ah, Bc, all_rows)
    g = frac * em.gamma(k, mode)
    assert bound_ok(got, ref, D, g), max_ratio(got, ref, D, g)


def test_config_512_plain_every_output(h, mm):
    A, B = device_inputs(mm, 512, 1, False)
    C = h.gemm(A, B, precision=mm.FP64)
    assert h.sync() == 0
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    assert np.array_equal(Ah, inputs.uniform(512, 512, 1, inputs.STREAM_A))
    assert bound_ok(C.cpu().numpy(), oracle.gemm(Ah, Bh), oracle.absprod(Ah, Bh), em.gamma(512, "fp64"))


@pytest.mark.parametrize("N", [1024, 2048, 4096, 8192])
def test_config_plain_sweep_sampled(h, mm, N):
    seed = 2 + int(np.log2(N))
    A, B = device_inputs(mm, N, seed, False)
    C = h.gemm(A, B, precision=mm.FP64)
    assert h.sync() == 0
    check_rows(C, A.cpu().numpy(), B.cpu().numpy(), sample_rows(N, seed, 3), "fp64")


@pytest.mark.parametrize("N", [4096, 8192])
def test_config_split_precision_sampled(h, mm, N):
    # 64 sampled rows and 64 sampled columns of every mode's result
    A, B = device_inputs(mm, N, 3, True)
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    rows = sample_rows(N, 3 + N, 61)
    cols = sample_rows(N, 4 + N, 61)
    for prec in (mm.FP64_EMU, mm.FP32_EMU, mm.FP64):
        C = h.gemm(A, B, precision=prec)
        assert h.sync() == 0
        check_rows(C, Ah, Bh, rows, MODE[prec])
        check_cols(C, Ah, Bh, cols, MODE[prec])
        del C


def test_uniform_workload_takes_five_slices_on_the_device(h, mm):
    # the benchmark workload keeps s = 5 under the automatic count
    A, B = device_inputs(mm, 8192, 3, True)
    s, a, b = h.debug_slice_count(A, B)
    assert s == 5, (s, a, b)


@pytest.mark.parametrize("N", [4096, 8192])
def test_default_options_normal_inputs_within_bound(h, mm, N):
    """The paper's Box-Muller normal entries (Sec. IV) at k = 4096 and 8192 with
    default options: 64 sampled rows within the bound (the automatic count
    takes s = 6 here, where a count from k alone gave 5 and left the bound)."""
    A = inputs.box_muller(N, N, 40 + N, inputs.STREAM_A)
    B = inputs.box_muller(N, N, 40 + N, inputs.STREAM_B)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    s, _, _ = h.debug_slice_count(Ad, Bd)
    assert s == 6
    C = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
    assert h.sync() == 0
    check_rows(C, A, B, sample_rows(N, 41 + N, 61), "fp64_emu")


@pytest.mark.parametrize("dist,N", [("t3", 4096), ("spread", 2048), ("cauchy", 1024)])
def test_default_options_heavy_tailed_within_bound(h, mm, dist, N):
    """Heavy tails (Student-t with 3 degrees of freedom; entries spread over 16
    octaves within each row; Cauchy) with default options: within the bound on
    sampled rows; Cauchy rows need more than 7 slices and take the plain FP64
    kernel."""
    gen = {"t3": inputs.student_t3, "spread": inputs.wide_spread, "cauchy": inputs.cauchy}[dist]
    A = gen(N, N, 60 + N, inputs.STREAM_A)
    B = gen(N, N, 60 + N, inputs.STREAM_B)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    s, _, _ = h.debug_slice_count(Ad, Bd)
    assert s >= 6
    if dist == "cauchy":
        assert s == 8
    C = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
    assert h.sync() == 0
    check_rows(C, A, B, sample_rows(N, 61 + N, 29), "fp64_emu")


def grouped_set(count, lo, hi, seed):
    dims = inputs.problem_set(count, lo, hi, seed)
    return [(int(m), int(n), int(k)) for m, n, k in dims]


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_config_grouped_512(h, mm, prec):
    dims = grouped_set(512, 32, 1024, 4)
    host, dev = [], []
    for i, (m, n, k) in enumerate(dims):
        A = inputs.uniform(m, k, 4000 + i, inputs.STREAM_A)
        B = inputs.uniform(k, n, 4000 + i, inputs.STREAM_B)
        host.append((A, B))
        dev.append((torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(),
                    torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")))
    h.grouped(dev, precision=prec)
    assert h.sync() == 0
    for i, ((A, B), (_, _, Cd)) in enumerate(zip(host, dev)):
        C = Cd.cpu().numpy()
        k = A.shape[1]
        if i % 64 == 0:
            assert bound_ok(C, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(k, MODE[prec])), i
        else:
            rows = [0, A.shape[0] - 1]
            assert bound_ok(C[rows], oracle.gemm_rows(A, B, rows), oracle.absprod_rows(A, B, rows),
                            em.gamma(k, MODE[prec])), i


def test_config_serve_stream(h, mm):
    count = 160
    dims = grouped_set(count, 64, 4096, 5)
    classes = inputs.unit(5, inputs.STREAM_CLASS, count) < 0.5
    reqs = []
    for i, (m, n, k) in enumerate(dims):
        A = torch.empty((m, k), dtype=torch.float64, device="cuda")
        B = torch.empty((k, n), dtype=torch.float64, device="cuda")
        mm.fill_uniform(A, 5000 + i, inputs.STREAM_A)
        mm.fill_uniform(B, 5000 + i, inputs.STREAM_B)
        C = torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")
        reqs.append((A, B, C, mm.FP64_EMU if classes[i] else mm.FP32_EMU))
    torch.cuda.synchronize()
    tickets = [h.serve_submit(A, B, C, precision=p, tag=i) for i, (A, B, C, p) in enumerate(reqs)]
    h.serve_drain()
    for i, t in enumerate(tickets):
        rc, st = h.serve_poll(t)
        assert rc == 0 and st.user_tag == i
    for i, (A, B, C, p) in enumerate(reqs):
        if i % 4:
            continue
        Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
        check_rows(C, Ah, Bh, [0, A.shape[0] - 1], MODE[p])


@pytest.mark.parametrize("N", [32, 64, 128, 256, 512, 1024])
def test_paper_sizes_box_muller_every_output(h, mm, N):
    # the paper's sizes (Sec. IV) with its Box-Muller normal entries
    A = inputs.box_muller(N, N, 7 + N, inputs.STREAM_A)
    B = inputs.box_muller(N, N, 7 + N, inputs.STREAM_B)
    ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    for prec in (mm.FP64, mm.FP64_EMU, mm.FP32_EMU):
        C = h.gemm(Ad, Bd, precision=prec)
        assert h.sync() == 0
        assert bound_ok(C.cpu().numpy(), ref, D, em.gamma(N, MODE[prec])), (N, prec)
    # the automatic slice count keeps half the bound on normal rows
    C = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
    assert h.sync() == 0
    assert bound_ok(C.cpu().numpy(), ref, D, 0.5 * em.gamma(N, "fp64_emu")), N
