"""GPU parity of the three precision modes against the CPU oracle, through the C ABI.

* integer and byte work bit for bit: scale exponents, slices (bfloat16 bit
  patterns), the tensor-core level products, the seeded device filler;
* FP64 and FP64-accuracy results within 4k*2^-53 |A||B| of the triple-loop
  oracle, FP32-accuracy within 4k*2^-24 |A||B|; the FP64-accuracy result also
  equals the exactly rounded emulated value of the emulation oracle;
* shapes span several tiles and ragged tails; edge cases: k = 0, empty
  products, k <= 4, odd leading dimensions, non-finite inputs, bad arguments.
"""
import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from gpu_util import bf16_bits_of, bound_ok, fixed_shift, max_ratio

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


@pytest.fixture(scope="module", params=["modular", "digits"])
def h(mm, request):
    # "modular": FP64-accuracy products take the modular form wherever it fits
    # (MM_OPT_FP64_SCHEME = 2; by default only products of m n k >= 2^33 do,
    # larger than these); "digits": the digit form only (= 1)
    with mm.Handle(0) as hh:
        hh.set_option(mm.OPT_FP64_SCHEME, 2 if request.param == "modular" else 1)
        yield hh


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def run(h, A, B, prec, **kw):
    C = h.gemm(dev(A), dev(B), precision=prec, **kw)
    rc = h.sync()
    return C.cpu().numpy(), rc


# ------------------------------------------------------------------ inputs
def test_device_filler_matches_host_generator(mm):
    X = torch.empty((37, 129), dtype=torch.float64, device="cuda")
    mm.fill_uniform(X, seed=9, stream_id=inputs.STREAM_A)
    torch.cuda.synchronize()
    assert np.array_equal(X.cpu().numpy(), inputs.uniform(37, 129, 9, inputs.STREAM_A))
    mm.fill_uniform(X, seed=9, stream_id=inputs.STREAM_A, scale_mode=1, exp_stream_id=inputs.STREAM_EXP_A)
    torch.cuda.synchronize()
    assert np.array_equal(X.cpu().numpy(), inputs.row_scaled(37, 129, 9))
    Y = torch.empty((50, 33), dtype=torch.float64, device="cuda")
    mm.fill_uniform(Y, seed=4, stream_id=inputs.STREAM_B, scale_mode=2, exp_stream_id=inputs.STREAM_EXP_B)
    torch.cuda.synchronize()
    assert np.array_equal(Y.cpu().numpy(), inputs.col_scaled(50, 33, 4))


# ------------------------------------------------------------------ slices
@pytest.mark.parametrize("s", [3, 5, 6, 7])
def test_fp64_slices_bit_exact(h, mm, s):
    A = inputs.row_scaled(70, 133, 20 + s)
    A[3, :] = 0.0
    A[5, 7] = 5e-324
    A[6, 1] = -1e-310
    B = inputs.col_scaled(133, 45, 20 + s)
    B[:, 2] = 0.0
    E_ref, sA = em.fp64_slices_A(A, s)
    F_ref, sB = em.fp64_slices_B(B, s)
    E, slA, rc = h.debug_slices(dev(A), 0, mm.FP64_EMU, s)
    assert rc == 0
    assert np.array_equal(E.cpu().numpy(), E_ref)
    assert np.array_equal(slA.cpu().numpy().view(np.uint16), bf16_bits_of(sA))
    F, slB, rc = h.debug_slices(dev(B), 1, mm.FP64_EMU, s)
    assert rc == 0
    assert np.array_equal(F.cpu().numpy(), F_ref)
    # the library stores B's slices transposed: [s][n][k]
    assert np.array_equal(slB.cpu().numpy().view(np.uint16), bf16_bits_of(np.transpose(sB, (0, 2, 1))))


def test_fp32_slices_bit_exact(h, mm):
    A = inputs.row_scaled(66, 100, 3)
    A[2, 5] = 1e-45          # deep below the row maximum: bfloat16 subnormal slices
    A[4, :] = 0.0
    B = inputs.col_scaled(100, 39, 3)
    E_ref, sA = em.fp32_slices_A(A)
    F_ref, sB = em.fp32_slices_B(B)
    E, slA, rc = h.debug_slices(dev(A), 0, mm.FP32_EMU)
    assert rc == 0
    assert np.array_equal(E.cpu().numpy(), E_ref)
    assert np.array_equal(slA.cpu().numpy().view(np.uint16), bf16_bits_of(sA))
    F, slB, rc = h.debug_slices(dev(B), 1, mm.FP32_EMU)
    assert np.array_equal(F.cpu().numpy(), F_ref)
    assert np.array_equal(slB.cpu().numpy().view(np.uint16), bf16_bits_of(np.transpose(sB, (0, 2, 1))))


def test_golden_digits_on_device(h, mm, golden_dir):
    import json, os
    g = json.load(open(os.path.join(golden_dir, "digits_t8.json")))
    for case in g["cases"]:
        row = np.array([case["row"]], float)
        s = case["s"]
        E, sl, rc = h.debug_slices(dev(row), 0, mm.FP64_EMU, s)
        assert int(E.cpu()[0]) == case["E"]
        want = np.array(case["digits"], dtype=np.int64).T[:, None, :]   # [s][1][cols]
        assert np.array_equal(sl.cpu().numpy().view(np.uint16), bf16_bits_of(want)), case["why"]


# ------------------------------------------------------------ level products
@pytest.mark.parametrize("m,n,k,s", [(136, 150, 1100, 5), (64, 200, 300, 7), (129, 129, 64, 6), (1, 3, 2000, 4)])
def test_level_products_bit_exact(h, m, n, k, s):
    A = inputs.row_scaled(m, k, m + k)
    B = inputs.col_scaled(k, n, n + k)
    _, sA = em.fp64_slices_A(A, s)
    _, sB = em.fp64_slices_B(B, s)
    L_ref = em.level_products(sA, sB, s)
    L = h.debug_levels(dev(A), dev(B), s).cpu().numpy()
    assert np.array_equal(L, L_ref)


def test_level_products_long_k_register_fold(h):
    # level 8 (s = 7) flushes every 128 K; 16000 K passes the 120-chunk fold of the int32 sums
    m, n, k, s = 8, 5, 16000, 7
    A = inputs.row_scaled(m, k, 77)
    B = inputs.col_scaled(k, n, 77)
    _, sA = em.fp64_slices_A(A, s)
    _, sB = em.fp64_slices_B(B, s)
    L_ref = em.level_products(sA, sB, s)
    assert np.array_equal(h.debug_levels(dev(A), dev(B), s).cpu().numpy(), L_ref)


def test_level_products_extreme_digits(h):
    # digits [-127, -128, -128, -128, -128] in every entry of A and B: every
    # slice product is +2^14 and each chunk sum reaches the exactness limit
    # Kc*(d-1)*2^14 = 2^24 of the f32 accumulator
    m, n, k, s = 130, 140, 2048, 5
    R = -(127 * 2 ** 32 + 128 * (2 ** 24 + 2 ** 16 + 2 ** 8 + 1))
    a = R * 2.0 ** -38
    A = np.full((m, k), a)
    B = np.full((k, n), a)
    E, sA = em.fp64_slices_A(A, s)
    assert E[0] == 2 and sA[:, 0, 0].tolist() == [-127, -128, -128, -128, -128]
    _, sB = em.fp64_slices_B(B, s)
    L_ref = em.level_products(sA, sB, s)
    assert np.array_equal(h.debug_levels(dev(A), dev(B), s).cpu().numpy(), L_ref)


# ----------------------------------------------------------- full products
SHAPES = [(1, 1, 5), (37, 45, 7), (128, 128, 64), (130, 270, 300), (257, 129, 1000), (200, 520, 4100)]


@pytest.mark.parametrize("m,n,k", SHAPES)
def test_fp64_emu_within_bound_and_exact(h, mm, m, n, k):
    A = inputs.row_scaled(m, k, 100 + k)
    B = inputs.col_scaled(k, n, 200 + k)
    C, rc = run(h, A, B, mm.FP64_EMU)
    assert rc == 0
    C_ref = oracle.gemm(A, B)
    D = oracle.absprod(A, B)
    assert bound_ok(C, C_ref, D, em.gamma(k, "fp64")), max_ratio(C, C_ref, D, em.gamma(k, "fp64"))
    if k <= 4:
        return
    _, code, bits, _, _, _ = h.debug_fp64_product(dev(A), dev(B))
    want = em.fp64_scheme(A, B, modular=h.get_option(mm.OPT_FP64_SCHEME) == 2)
    if want[0] == "crt":
        # the modular form: the exact integer product of the scaled entries, rounded once
        assert (code, bits) == (mm.CRT_BASE + want[2], want[1])
        rows = list(range(0, m, max(1, m // 16)))[:16]
        assert np.array_equal(C[rows], em.gemm_fp64_crt(A[rows], B, bits, code - mm.CRT_BASE))
        return
    s, _, _ = h.debug_slice_count(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    assert s == em.slice_count(A, B)   # far from the rule's thresholds for these inputs
    assert code == (s if want[0] == "digits" else em.S_PLAIN)
    if s == em.S_PLAIN:
        return
    E, sA = em.fp64_slices_A(A, s)
    F, sB = em.fp64_slices_B(B, s)
    rows = list(range(0, m, max(1, m // 16)))[:16]
    Ce = em.recombine_exact(em.level_products(sA[:, rows], sB, s), E[rows], F, s)
    if fixed_shift(s, k) == 0:
        assert np.array_equal(C[rows], Ce)
    else:
        ulp = np.spacing(np.abs(Ce))
        unit = np.ldexp(1.0, (E[rows][:, None] + F[None, :] - 8 * (s + 1) + fixed_shift(s, k)).astype(int))
        assert np.all(np.abs(C[rows] - Ce) <= 2 * ulp + unit)   # one rounding to the fixed point, one to double


@pytest.mark.parametrize("m,n,k", SHAPES + [(1, 1, 1), (3, 2, 2)])
def test_fp32_emu_within_bound(h, mm, m, n, k):
    A = inputs.row_scaled(m, k, 300 + k)
    B = inputs.col_scaled(k, n, 400 + k)
    C, rc = run(h, A, B, mm.FP32_EMU)
    assert rc == 0
    C_ref = oracle.gemm(A, B)
    D = oracle.absprod(A, B)
    assert bound_ok(C, C_ref, D, em.gamma(k, "fp32")), max_ratio(C, C_ref, D, em.gamma(k, "fp32"))


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 15, 129), (128, 128, 16), (200, 300, 100), (300, 257, 513)])
def test_fp64_within_bound(h, mm, kind, m, n, k):
    h.set_option(mm.OPT_FP64_KERNEL, kind)
    A = inputs.uniform(m, k, 500 + k, inputs.STREAM_A)
    B = inputs.uniform(k, n, 500 + k, inputs.STREAM_B)
    C, rc = run(h, A, B, mm.FP64)
    h.set_option(mm.OPT_FP64_KERNEL, 0)
    assert rc == 0
    C_ref = oracle.gemm(A, B)
    D = oracle.absprod(A, B)
    assert bound_ok(C, C_ref, D, em.gamma(k, "fp64"))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_small_integers_exact_all_modes(h, prec):
    rng = np.random.default_rng(prec)
    A = rng.integers(-8, 9, (150, 700)).astype(float)
    B = rng.integers(-8, 9, (700, 140)).astype(float)
    C, rc = run(h, A, B, prec)
    assert rc == 0
    assert np.array_equal(C, (A.astype(np.int64) @ B.astype(np.int64)).astype(float))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_identity_and_permutation(h, prec):
    rng = np.random.default_rng(5)
    A = rng.integers(-2 ** 20, 2 ** 20, (96, 96)) / 2.0 ** 20
    C, _ = run(h, A, np.eye(96), prec)
    assert np.array_equal(C, A)
    P = np.eye(96)[rng.permutation(96)]
    C, _ = run(h, P, A, prec)
    assert np.all(C == P @ A)


def test_transpose_identity_integers(h, mm):
    rng = np.random.default_rng(8)
    A = rng.integers(-100, 101, (90, 300)).astype(float)
    B = rng.integers(-100, 101, (300, 70)).astype(float)
    for prec in (mm.FP64, mm.FP64_EMU, mm.FP32_EMU):
        C1, _ = run(h, A, B, prec)
        C2, _ = run(h, np.ascontiguousarray(B.T), np.ascontiguousarray(A.T), prec)
        assert np.array_equal(C1, C2.T)


def test_rank_one_closed_form(h, mm):
    rng = np.random.default_rng(9)
    m, n, k = 140, 150, 1000
    u = rng.integers(-64, 65, m) / 64.0
    w = rng.integers(-64, 65, n) / 16.0
    A = np.repeat(u[:, None], k, axis=1)
    B = np.repeat(w[None, :], k, axis=0)
    for prec in (mm.FP64, mm.FP64_EMU, mm.FP32_EMU):
        C, _ = run(h, A, B, prec)
        assert np.array_equal(C, k * np.outer(u, w))


# --------------------------------------------------------------- edge cases
def test_k_zero_writes_zeros_and_empty_is_noop(h, mm):
    for prec in (0, 1, 2):
        C = torch.full((5, 6), 7.0, dtype=torch.float64, device="cuda")
        A = torch.empty((5, 0), dtype=torch.float64, device="cuda")
        B = torch.empty((0, 6), dtype=torch.float64, device="cuda")
        rc = h.lib.mm_gemm(h.h, 5, 6, 0, A.data_ptr(), 1, B.data_ptr(), 6, C.data_ptr(), 6, prec, None)
        assert rc == 0 and h.sync() == 0
        assert torch.all(C == 0)
        C2 = torch.full((5, 6), 7.0, dtype=torch.float64, device="cuda")
        assert h.lib.mm_gemm(h.h, 0, 6, 3, None, 3, None, 6, C2.data_ptr(), 6, prec, None) == 0
        assert torch.all(C2 == 7.0)


def test_k_le_4_fp64_emu_uses_fp64_kernel(h, mm):
    A = inputs.row_scaled(33, 3, 1)
    B = inputs.col_scaled(3, 17, 1)
    C, rc = run(h, A, B, mm.FP64_EMU)
    assert bound_ok(C, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(3, "fp64"))


def test_strided_operands(h, mm):
    # leading dimensions larger than the width, odd ones included
    m, n, k = 70, 50, 90
    Abig = inputs.row_scaled(m, k + 7, 3)
    Bbig = inputs.col_scaled(k, n + 3, 3)
    A, B = Abig[:, :k], Bbig[:, :n]
    C_ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
    for prec, mode in ((0, "fp64"), (1, "fp64_emu"), (2, "fp32_emu")):
        Ad, Bd = dev(Abig)[:, :k], dev(Bbig)[:, :n]
        Cbig = torch.full((m, n + 5), 3.0, dtype=torch.float64, device="cuda")
        h.gemm(Ad, Bd, C=Cbig[:, :n], precision=prec)
        assert h.sync() == 0
        Cn = Cbig.cpu().numpy()
        assert bound_ok(Cn[:, :n], C_ref, D, em.gamma(k, mode))
        assert np.all(Cn[:, n:] == 3.0)   # bytes outside the ldc view untouched


def test_nonfinite_inputs(h, mm):
    A = inputs.row_scaled(20, 30, 2)
    B = inputs.col_scaled(30, 10, 2)
    A[4, 7] = np.inf
    B[3, 6] = np.nan
    for prec in (mm.FP64_EMU, mm.FP32_EMU):
        C, rc = run(h, A, B, prec)
        assert rc == 4  # MM_ERR_NONFINITE
        assert np.all(np.isnan(C[4, :])) and np.all(np.isnan(C[:, 6]))
        ok = np.ones_like(C, bool)
        ok[4, :] = False
        ok[:, 6] = False
        assert np.all(np.isfinite(C[ok]))
    assert h.sync() == 0  # status was cleared
    # the error word belongs to the stream: a failing call on one stream and a
    # clean call on another report independently
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    Ad, Bd = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    Ac, Bc = torch.from_numpy(inputs.row_scaled(20, 30, 3)).cuda(), torch.from_numpy(inputs.col_scaled(30, 10, 3)).cuda()
    torch.cuda.synchronize()
    C1 = h.gemm(Ad, Bd, precision=mm.FP64_EMU, stream=s1)
    C2 = h.gemm(Ac, Bc, precision=mm.FP64_EMU, stream=s2)
    assert h.sync(s2) == 0
    assert h.sync(s1) == 4
    assert h.sync(s1) == 0 and h.sync(s2) == 0
    del C1, C2
    C, rc = run(h, A, B, mm.FP64)
    assert rc == 0
    ref = oracle.gemm(A, B)
    assert np.array_equal(np.isnan(C), np.isnan(ref)) and np.array_equal(np.isinf(C), np.isinf(ref))


def test_argument_errors(h):
    h.sync()
    lib, hh = h.lib, h.h
    X = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    Y = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    Z = torch.zeros((8, 8), dtype=torch.float64, device="cuda")
    p = (X.data_ptr(), Y.data_ptr(), Z.data_ptr())
    assert lib.mm_gemm(hh, -1, 8, 8, p[0], 8, p[1], 8, p[2], 8, 0, None) == 2
    assert lib.mm_gemm(hh, 8, 8, 8, p[0], 7, p[1], 8, p[2], 8, 0, None) == 2
    assert lib.mm_gemm(hh, 8, 8, 8, p[0], 8, p[1], 7, p[2], 8, 0, None) == 2
    assert lib.mm_gemm(hh, 8, 8, 8, p[0], 8, p[1], 8, p[2], 7, 0, None) == 2
    assert lib.mm_gemm(hh, 8, 8, 8, p[0], 8, p[1], 8, p[2], 8, 9, None) == 2
    assert lib.mm_gemm(hh, 8, 8, 8, None, 8, p[1], 8, p[2], 8, 0, None) == 2
    assert lib.mm_gemm(hh, 8, 8, 8, p[0], 8, p[1], 8, p[0], 8, 1, None) == 2   # C overlaps A
    assert lib.mm_gemm(None, 8, 8, 8, p[0], 8, p[1], 8, p[2], 8, 0, None) == 2
    assert h.sync() == 0


def test_host_entry_point(h, mm):
    A = inputs.row_scaled(150, 260, 6)
    B = inputs.col_scaled(260, 140, 6)
    C_ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
    for prec, mode in ((0, "fp64"), (1, "fp64_emu"), (2, "fp32_emu")):
        C = h.gemm_host(A, B, precision=prec)
        assert bound_ok(C, C_ref, D, em.gamma(260, mode))


def test_repeatable_bitwise(h, mm):
    A = inputs.row_scaled(300, 500, 12)
    B = inputs.col_scaled(500, 260, 12)
    for prec in (0, 1, 2):
        C1, _ = run(h, A, B, prec)
        C2, _ = run(h, A, B, prec)
        assert np.array_equal(C1, C2)


def test_budget_exceeded(mm):
    with mm.Handle(0, budget_bytes=1 << 20) as hs:
        A = dev(inputs.row_scaled(512, 512, 1))
        B = dev(inputs.col_scaled(512, 512, 1))
        with pytest.raises(mm.MMError) as ei:
            hs.gemm(A, B, precision=mm.FP64_EMU)
        assert ei.value.status == 3


# ---------------------------------------------------------- single vs CTA-pair tiles
@pytest.mark.parametrize("m,n,k", [(300, 260, 1100), (520, 136, 700), (129, 400, 64), (257, 255, 4100)])
def test_cta_pair_and_single_tiles_agree(h, mm, m, n, k):
    A = inputs.row_scaled(m, k, 900 + k)
    B = inputs.col_scaled(k, n, 900 + k)
    out = {}
    for cg in (1, 2):
        h.set_option(mm.OPT_CTA_PAIR, cg)
        try:
            out[(cg, 1)], rc1 = run(h, A, B, mm.FP64_EMU)
            out[(cg, 2)], rc2 = run(h, A, B, mm.FP32_EMU)
        finally:
            h.set_option(mm.OPT_CTA_PAIR, 0)
        assert rc1 == 0 and rc2 == 0
    assert np.array_equal(out[(1, 1)], out[(2, 1)])          # exact integer path: identical bits
    C_ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
    for cg in (1, 2):
        assert bound_ok(out[(cg, 1)], C_ref, D, em.gamma(k, "fp64_emu"))
        assert bound_ok(out[(cg, 2)], C_ref, D, em.gamma(k, "fp32_emu"))


@pytest.mark.parametrize("cg", [1, 2])
def test_level_products_bit_exact_both_tilings(h, mm, cg):
    m, n, k, s = 300, 150, 1100, 5
    A = inputs.row_scaled(m, k, 31)
    B = inputs.col_scaled(k, n, 31)
    _, sA = em.fp64_slices_A(A, s)
    _, sB = em.fp64_slices_B(B, s)
    L_ref = em.level_products(sA, sB, s)
    h.set_option(mm.OPT_CTA_PAIR, cg)
    try:
        L = h.debug_levels(dev(A), dev(B), s).cpu().numpy()
    finally:
        h.set_option(mm.OPT_CTA_PAIR, 0)
    assert np.array_equal(L, L_ref)


@pytest.mark.parametrize("m,n,k", [(200, 300, 50), (150, 520, 300), (130, 257, 3000), (140, 300, 4500)])
def test_tile_widths_agree_bitwise(h, mm, m, n, k):
    # s = 7, 6, 6, 5: the first three have a fixed point below the lowest level
    A = inputs.row_scaled(m, k, 700 + k)
    B = inputs.col_scaled(k, n, 700 + k)
    out = {}
    for cg in (1, 2):
        for bn in (128, 256):
            h.set_option(mm.OPT_CTA_PAIR, cg)
            h.set_option(mm.OPT_TILE_N, bn)
            try:
                out[(cg, bn)], rc = run(h, A, B, mm.FP64_EMU)
            finally:
                h.set_option(mm.OPT_CTA_PAIR, 0)
                h.set_option(mm.OPT_TILE_N, 0)
            assert rc == 0
    first = out[(1, 128)]
    for key, C in out.items():
        assert np.array_equal(C, first), key
    assert bound_ok(first, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(k, "fp64_emu"))


def test_tile_width_option_checked(h, mm):
    with pytest.raises(mm.MMError):
        h.set_option(mm.OPT_TILE_N, 200)
    assert h.get_option(mm.OPT_TILE_N) == 0


# ------------------------------------------------------- failure detection
def test_bounded_wait_times_out_and_context_survives(h, mm):
    # a wait on a barrier nothing arrives at gives up after 50 ms with MM_ERR_TIMEOUT
    assert h.debug_wait_timeout(50) == mm.TIMEOUT
    assert h.sync() == 0                       # the error word was read and cleared
    A = inputs.row_scaled(130, 70, 5)
    B = inputs.col_scaled(70, 90, 5)
    C, rc = run(h, A, B, mm.FP64_EMU)          # the context still computes
    assert rc == 0
    assert bound_ok(C, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(70, "fp64_emu"))
    with pytest.raises(Exception):
        mm._check(h.debug_wait_timeout(0), "wait probe")


def test_long_k_segment_folds_agree_across_tilings(h, mm):
    # k = 24000 (s = 5): level 6 has more than 120 chunks, so its sums are folded
    # mid-level too; the 128-wide (TMEM total) and 256-wide (register sums,
    # folds spread over the following chunks) kernels must agree bit for bit
    m, n, k = 130, 260, 24000
    A = inputs.row_scaled(m, k, 901)
    B = inputs.col_scaled(k, n, 901)
    out = {}
    for bn in (128, 256):
        h.set_option(mm.OPT_TILE_N, bn)
        try:
            out[bn], rc = run(h, A, B, mm.FP64_EMU)
        finally:
            h.set_option(mm.OPT_TILE_N, 0)
        assert rc == 0
    assert np.array_equal(out[128], out[256])
    rows = [0, 64, 129]
    assert bound_ok(out[256][rows], oracle.gemm_rows(A, B, rows), oracle.absprod_rows(A, B, rows),
                    em.gamma(k, "fp64_emu"))


@pytest.mark.parametrize("prec", [1, 2])
def test_host_entry_two_panels_same_bits(h, mm, prec):
    # m >= 2048: the host entry runs two row panels with the copies overlapping
    # the kernels; the result is the device entry's, bit for bit
    m, n, k = 2600, 530, 700
    A = inputs.row_scaled(m, k, 1300 + prec)
    B = inputs.col_scaled(k, n, 1300 + prec)
    Ch = h.gemm_host(A, B, precision=prec)
    Cd, rc = run(h, A, B, prec)
    assert rc == 0
    assert np.array_equal(Ch, Cd)
    rows = [0, 1299, 1300, 2599]
    mode = "fp64_emu" if prec == 1 else "fp32_emu"
    assert bound_ok(Ch[rows], oracle.gemm_rows(A, B, rows), oracle.absprod_rows(A, B, rows), em.gamma(k, mode))
    # a strided host output (ldc > n) lands in place
    big = np.full((m, n + 9), -7.0)
    h.gemm_host(A, B, big[:, :n], precision=prec)
    assert np.array_equal(big[:, :n], Cd) and np.all(big[:, n:] == -7.0)


def _tilings(h, mm, A, B, bns=(128, 256), cgs=(1, 2)):
    out = {}
    for cg in cgs:
        for bn in bns:
            h.set_option(mm.OPT_CTA_PAIR, cg)
            h.set_option(mm.OPT_TILE_N, bn)
            try:
                out[(cg, bn)], rc = run(h, A, B, mm.FP64_EMU)
            finally:
                h.set_option(mm.OPT_CTA_PAIR, 0)
                h.set_option(mm.OPT_TILE_N, 0)
            assert rc == 0
    return out


@pytest.mark.parametrize("s", [3, 4, 5])
def test_byte_carry_forced_slices_exact(h, mm, s):
    # s <= 5 on 256-wide tiles takes the byte-carry recombination (full rows)
    # next to the int64 fold (the partial last tile); the 128-wide kernel keeps
    # the total in TMEM. All agree bit for bit and equal the exact total
    # rounded once (fixed point at 2^0 here).
    m, n, k = 300, 600, 1000
    A = inputs.row_scaled(m, k, 1500 + s)
    B = inputs.col_scaled(k, n, 1500 + s)
    h.set_option(mm.OPT_SLICES, s)
    try:
        out = _tilings(h, mm, A, B)
    finally:
        h.set_option(mm.OPT_SLICES, 0)
    first = out[(1, 128)]
    for key, C in out.items():
        assert np.array_equal(C, first), key
    assert fixed_shift(s, k) == 0
    E, sA = em.fp64_slices_A(A, s)
    F, sB = em.fp64_slices_B(B, s)
    rows = [0, 1, 127, 128, 255, 256, 299]
    Ce = em.recombine_exact(em.level_products(sA[:, rows], sB, s), E[rows], F, s)
    assert np.array_equal(first[rows], Ce)


@pytest.mark.parametrize("k", [23040, 23104])
def test_byte_carry_segment_limit(h, mm, k):
    # s = 5: k = 23040 puts exactly 120 chunks in the top level (byte carry);
    # one more K block (k = 23104) needs a mid-level fold (int64 fold path)
    m, n = 260, 512
    A = inputs.row_scaled(m, k, 1600)
    B = inputs.col_scaled(k, n, 1600)
    assert h.debug_slice_count(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())[0] == 5
    out = _tilings(h, mm, A, B, cgs=(1, 2))
    first = out[(1, 128)]
    for key, C in out.items():
        assert np.array_equal(C, first), (k, key)
    rows = [0, 131, 259]
    assert bound_ok(first[rows], oracle.gemm_rows(A, B, rows), oracle.absprod_rows(A, B, rows),
                    em.gamma(k, "fp64_emu"))


@pytest.mark.parametrize("prec", [1, 2])
def test_clustered_pairs_same_bits(h, mm, prec):
    # CTA pairs in clusters of two on adjacent 256-wide tiles, each CTA loading
    # half of its rows of A for both pairs (TMA multicast): the same bits as
    # plain CTA pairs; an odd tile-column count falls back to pairs
    for m, n, k in ((1000, 2048, 1000), (700, 1280, 300)):
        A = inputs.row_scaled(m, k, 1700 + k)
        B = inputs.col_scaled(k, n, 1700 + k)
        out = {}
        for cp in (2, 3):
            h.set_option(mm.OPT_CTA_PAIR, cp)
            try:
                out[cp], rc = run(h, A, B, prec)
            finally:
                h.set_option(mm.OPT_CTA_PAIR, 0)
            assert rc == 0
        assert np.array_equal(out[2], out[3]), (m, n, k)
    mode = "fp64_emu" if prec == 1 else "fp32_emu"
    A = inputs.row_scaled(700, 300, 2000)
    B = inputs.col_scaled(300, 1280, 2000)
    rows = [0, 350, 699]
    assert bound_ok(out[3][rows], oracle.gemm_rows(A, B, rows), oracle.absprod_rows(A, B, rows), em.gamma(300, mode))
