"""The allocation-free entry point mm_gemm_emu_static, through the C ABI.

Some callers cannot call cudaMalloc (host callbacks, allocator hooks, loops that
must not pay its implicit synchronisation, processes whose device memory is
reserved up front). mm_gemm_emu_static serves them from one fixed scratch array
in the library image. These checks compare it with mm_gemm on two calls in a row
(different shapes and data, so stale scratch contents from the first call would
show), within the tolerance the other GPU tests use: 4k*2^-53 |A||B| for
FP64-accuracy (where the two must in fact agree bit for bit) and 4k*2^-24 |A||B|
for FP32-accuracy, and each against the CPU oracle within the same bound.
This file runs last so a failure here does not hide the rest.
"""
import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

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


def call_static(lib, A, B, prec):
    m, k = A.shape
    n = B.shape[1]
    C = torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.mm_gemm_emu_static(m, n, k, A.data_ptr(), k, B.data_ptr(), n, C.data_ptr(), n, prec, stream)
    torch.cuda.synchronize()
    return rc, C


# shapes that cover the paths: the automatic slice count at s = 6 and 7 and at
# s = 5 (k >= 4096, where the 128-wide kernel folds while mm_gemm's wider
# tiles recombine by byte carry), the plain-FP64 fallback (Cauchy rows), the
# FP64 kernel for k <= 4, and k = 0
CASES = [(300, 260, 700, 1, "scaled"), (130, 70, 1500, 2, "scaled"), (128, 128, 4096, 3, "scaled"),
         (128, 96, 5000, 4, "scaled"), (64, 80, 600, 5, "cauchy"), (40, 30, 3, 6, "scaled"), (33, 17, 0, 7, "scaled")]


def _operands(m, n, k, seed, kind):
    if kind == "cauchy":
        return inputs.cauchy(m, k, seed, inputs.STREAM_A), inputs.cauchy(k, n, seed, inputs.STREAM_B)
    return inputs.row_scaled(m, k, seed), inputs.col_scaled(k, n, seed)


@pytest.mark.parametrize("prec,mode", [(1, "fp64_emu"), (2, "fp32_emu")])
def test_static_scratch_matches_mm_gemm_twice(mm, prec, mode):
    with mm.Handle(0) as h:
        # the allocation-free call takes the digit form; so does this handle
        h.set_option(mm.OPT_FP64_SCHEME, 1)
        for m, n, k, seed, kind in CASES:
            A, B = _operands(m, n, k, seed, kind)
            Ad = torch.from_numpy(A).cuda()
            Bd = torch.from_numpy(B).cuda()
            for _ in range(2):   # the second call meets the first one's scratch contents
                rc, Cs = call_static(h.lib, Ad, Bd, prec)
                assert rc == 0
                assert h.lib.mm_gemm_emu_static_status(torch.cuda.current_stream().cuda_stream) == 0
                Cg = h.gemm(Ad, Bd, precision=prec)
                assert h.sync() == 0
                cs, cg = Cs.cpu().numpy(), Cg.cpu().numpy()
                if k == 0:
                    assert np.all(cs == 0.0) and np.all(cg == 0.0)
                    continue
                # both against the oracle within the mode's bound ...
                ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
                assert np.all(np.abs(cs - ref) <= em.gamma(k, mode) * D), (m, n, k, kind)
                assert np.all(np.abs(cs - cg) <= em.gamma(k, mode) * D)
                # ... and FP64-accuracy bit for bit with mm_gemm
                if prec == 1:
                    assert np.array_equal(cs, cg), (m, n, k, kind)


def test_static_scratch_rejects_oversize(mm):
    lib = mm._lib.load()
    A = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    B = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    rc, _ = call_static(lib, A, B, 1)
    assert rc == 3  # MM_ERR_BUDGET: larger than the fixed scratch
    assert lib.mm_gemm_emu_static(8, 8, 8, None, 8, None, 8, None, 8, 0, None) == 2   # plain FP64 is not offered


@pytest.mark.parametrize("prec", [1, 2])
def test_static_status_reports_nonfinite_and_clears(mm, prec):
    lib = mm._lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    A, B = _operands(70, 50, 300, 11, "scaled")
    Bd = torch.from_numpy(B).cuda()

    def run(Am):
        rc, C = call_static(lib, torch.from_numpy(Am).cuda(), Bd, prec)
        assert rc == 0   # the call itself does not wait for its kernels
        return C.cpu().numpy()

    bad = A.copy()
    bad[5, 7] = np.nan
    assert np.all(np.isnan(run(bad)[5]))
    assert lib.mm_gemm_emu_static_status(stream) == 4   # MM_ERR_NONFINITE
    assert lib.mm_gemm_emu_static_status(stream) == 0   # read and cleared
    # the word covers the last call: a clean call clears what an earlier one left
    bad[5, 7] = np.inf
    run(bad)
    run(A)
    assert lib.mm_gemm_emu_static_status(stream) == 0
    # ... also on the paths that take no split (k = 0; FP64-accuracy k <= 4)
    run(bad)
    for k in (0, 3):
        rc, _ = call_static(lib, torch.zeros((8, k), dtype=torch.float64, device="cuda"),
                            torch.zeros((k, 8), dtype=torch.float64, device="cuda"), prec)
        assert rc == 0
        assert lib.mm_gemm_emu_static_status(stream) == 0
        run(bad)
    assert lib.mm_gemm_emu_static_status(stream) == 4
