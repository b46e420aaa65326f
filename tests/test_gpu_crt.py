"""GPU parity of the modular (Chinese-remainder) form of the FP64-accuracy
product against the oracle, through the C ABI.

* the centred residues of the scaled entries, bit for bit (bfloat16 patterns);
* the device's decision (modulus count and bit count) against the oracle's;
* the residue products reduced modulo their moduli (bytes), bit for bit, over
  several tiles with ragged tails, several K chunks and more than one int32
  segment;
* the result, bit for bit against the oracle's exactly rounded value, and
  within 4k 2^-53 |A||B| of the triple-loop oracle; every tiling gives the
  same bits; non-finite inputs.
"""
import numpy as np
import pytest

import oracle
from oracle import emulation as em
from paper_2408_15384_gb300 import inputs

from gpu_util import bf16_bits_of, bound_ok, max_ratio

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-4   # the device's float spreads against the oracle's exact ones


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
    # the modular form wherever it fits, small products included (by default
    # only products of m n k >= 2^33 take it)
    with mm.Handle(0) as hh:
        hh.set_option(mm.OPT_FP64_SCHEME, 2)
        yield hh


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


# ------------------------------------------------------------------ residues
@pytest.mark.parametrize("N,b", [(3, 8), (11, 37), (12, 42), (14, 53)])
def test_residues_bit_exact(h, mm, N, b):
    A = inputs.row_scaled(70, 133, 20 + N)
    A[3, :] = 0.0
    A[5, 7] = 5e-324
    A[6, 1] = -1e-310
    A[8, :] = 2.0 ** 60 * inputs.uniform(1, 133, 5, 3)[0]
    B = inputs.col_scaled(133, 45, 20 + N)
    B[:, 2] = 0.0
    E_ref = em.row_exponents(A, 2)
    rA = em.crt_residues(em.crt_integer_repr(A, E_ref, b), N)
    E, plA, rc = h.debug_crt_residues(dev(A), 0, N, b)
    assert rc == 0
    assert np.array_equal(E.cpu().numpy(), E_ref)
    assert np.array_equal(plA.cpu().numpy().view(np.uint16), bf16_bits_of(rA))
    F_ref = em.col_exponents(B, 2)
    rB = em.crt_residues(em.crt_integer_repr(B.T, F_ref, b), N)        # [N][n][k]: B transposed
    F, plB, rc = h.debug_crt_residues(dev(B), 1, N, b)
    assert rc == 0
    assert np.array_equal(F.cpu().numpy(), F_ref)
    assert np.array_equal(plB.cpu().numpy().view(np.uint16), bf16_bits_of(rB))


def test_golden_residues_on_device(h, mm, golden_dir):
    import json, os
    g = json.load(open(os.path.join(golden_dir, "crt_residues.json")))
    # entries R * 2^-10 with a row maximum 2^10 * 2^-10 = 1 (E = 2): b = 12 gives R back
    for r in g["residues"]:
        l = em.CRT_MODULI.index(r["m"])
        row = np.array([[r["R"] * 2.0 ** -10, 1.0]])
        _, pl, rc = h.debug_crt_residues(dev(row), 0, l + 1, 12)
        assert rc == 0
        assert pl.cpu().numpy().view(np.uint16)[l, 0, 0] == bf16_bits_of([r["rho"]])[0], r


# ------------------------------------------------------------------ decision
def _case(name, m, n, k, seed):
    if name == "scaled":
        return inputs.row_scaled(m, k, seed), inputs.col_scaled(k, n, seed)
    if name == "uniform":
        return inputs.uniform(m, k, seed, 1), inputs.uniform(k, n, seed, 2)
    if name == "normal":
        return inputs.box_muller(m, k, seed, 1), inputs.box_muller(k, n, seed, 2)
    if name == "t3":
        return inputs.student_t3(m, k, seed, 1), inputs.student_t3(k, n, seed, 2)
    if name == "spread":
        return inputs.wide_spread(m, k, seed, 1), inputs.wide_spread(k, n, seed, 2)
    raise KeyError(name)


def _allowed(k, a, b):
    """decision codes the rule gives within REL of the oracle's spreads"""
    out = set()
    for f in (1 - REL, 1, 1 + REL):
        for g in (1 - REL, 1, 1 + REL):
            bN = em.crt_params_from_spread(k, a * f, b * g)
            if bN:
                out.add((16 + bN[1], bN[0]))
            else:
                s = em.slice_count_from_spread(k, a * f, b * g)
                out.add((s, 0))
    return out


PRODUCTS = [("scaled", 300, 520, 2000), ("scaled", 130, 257, 1100), ("uniform", 129, 130, 64),
            ("normal", 257, 300, 700), ("t3", 64, 200, 1500), ("spread", 200, 129, 900), ("scaled", 1, 1, 5),
            ("scaled", 260, 300, 4100)]


@pytest.mark.parametrize("name,m,n,k", PRODUCTS)
def test_products_bit_exact(h, mm, name, m, n, k):
    A, B = _case(name, m, n, k, 7 + k)
    C, code, bits, a_dev, b_dev, res = h.debug_fp64_product(dev(A), dev(B))
    assert h.sync() == 0
    a = float(em.row_spread(A, em.row_exponents(A, 2)).min())
    b = float(em.col_spread(B, em.col_exponents(B, 2)).min())
    assert abs(a_dev - a) <= REL * a and abs(b_dev - b) <= REL * b
    assert (code, bits) in _allowed(k, a, b), (code, bits, em.fp64_scheme(A, B))
    got = C.cpu().numpy()
    ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
    assert bound_ok(got, ref, D, em.gamma(k, "fp64_emu")), max_ratio(got, ref, D, em.gamma(k, "fp64_emu"))
    if code <= mm.CRT_BASE:
        pytest.skip("this product takes the digit form")
    N = code - mm.CRT_BASE
    # every 7th row and the last (rows of every tile, the ragged tail), all columns
    rows = sorted(set(range(0, m, 7)) | {m - 1})
    E, F = em.row_exponents(A, 2), em.col_exponents(B, 2)
    RA = em.crt_integer_repr(A[rows], E[rows], bits)
    RB = em.crt_integer_repr(B.T, F, bits).T
    P = em.crt_products(em.crt_residues(RA, N), em.crt_residues(RB, N))
    want = np.stack([np.mod(P[l], em.CRT_MODULI[l]) for l in range(N)]).astype(np.uint8)
    assert np.array_equal(res.cpu().numpy()[:, rows, :], want)
    rows = rows[:: max(1, len(rows) // 12)]
    assert np.array_equal(got[rows], em.gemm_fp64_crt(A[rows], B, bits, N))


def test_more_than_one_int32_segment(h, mm):
    # k = 130000: 127 K chunks of 1024 a modulus, so each product's int32 sums
    # are reduced once mid-way (every 120 chunks)
    m, n, k = 9, 20, 130000
    A, B = _case("scaled", m, n, k, 77)
    C, code, bits, _, _, res = h.debug_fp64_product(dev(A), dev(B))
    assert h.sync() == 0
    assert code > mm.CRT_BASE
    N = code - mm.CRT_BASE
    E, F = em.row_exponents(A, 2), em.col_exponents(B, 2)
    P = em.crt_products(em.crt_residues(em.crt_integer_repr(A, E, bits), N),
                        em.crt_residues(em.crt_integer_repr(B.T, F, bits).T, N))
    want = np.stack([np.mod(P[l], em.CRT_MODULI[l]) for l in range(N)]).astype(np.uint8)
    assert np.array_equal(res.cpu().numpy(), want)
    assert np.array_equal(C.cpu().numpy(), em.gemm_fp64_crt(A, B, bits, N))


@pytest.mark.parametrize("m,n,k", [(300, 260, 1100), (129, 400, 64), (257, 255, 4100), (520, 136, 700)])
def test_tilings_agree_bitwise(h, mm, m, n, k):
    A, B = _case("scaled", m, n, k, 900 + k)
    out = {}
    for cg in (1, 2):
        for bn in (128, 256):
            h.set_option(mm.OPT_CTA_PAIR, cg)
            h.set_option(mm.OPT_TILE_N, bn)
            try:
                C, code, _, _, _, _ = h.debug_fp64_product(dev(A), dev(B), residues=False)
                assert h.sync() == 0
            finally:
                h.set_option(mm.OPT_CTA_PAIR, 0)
                h.set_option(mm.OPT_TILE_N, 0)
            assert code > mm.CRT_BASE
            out[(cg, bn)] = C.cpu().numpy()
    first = out[(1, 128)]
    for key, C in out.items():
        assert np.array_equal(C, first), key
    assert bound_ok(first, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(k, "fp64_emu"))


def test_nonfinite_inputs(h, mm):
    m, n, k = 140, 150, 900
    A, B = _case("scaled", m, n, k, 5)
    A[7, 11] = np.nan
    B[3, 20] = np.inf
    C = h.gemm(dev(A), dev(B), precision=mm.FP64_EMU)
    assert h.sync() == mm.NONFINITE
    got = C.cpu().numpy()
    assert np.all(np.isnan(got[7, :])) and np.all(np.isnan(got[:, 20]))
    keep_r = [i for i in range(m) if i != 7]
    keep_c = [j for j in range(n) if j != 20]
    A2, B2 = A[keep_r], B[:, keep_c]
    ref, D = oracle.gemm(A2, B2), oracle.absprod(A2, B2)
    assert bound_ok(got[np.ix_(keep_r, keep_c)], ref, D, em.gamma(k, "fp64_emu"))


def test_digit_form_option(h, mm):
    # MM_OPT_FP64_SCHEME = 1: the digit form, whatever the modular form would do
    A, B = _case("scaled", 200, 300, 3000, 12)
    h.set_option(mm.OPT_FP64_SCHEME, 1)
    try:
        C, code, _, _, _, _ = h.debug_fp64_product(dev(A), dev(B), residues=False)
        assert h.sync() == 0
    finally:
        h.set_option(mm.OPT_FP64_SCHEME, 2)
    assert code == em.slice_count(A, B)
    s = code
    E, sA = em.fp64_slices_A(A, s)
    F, sB = em.fp64_slices_B(B, s)
    rows = [0, 77, 199]
    Ce = em.recombine_exact(em.level_products(sA[:, rows], sB, s), E[rows], F, s)
    assert np.array_equal(C.cpu().numpy()[rows], Ce)
    with pytest.raises(mm.MMError):
        h.set_option(mm.OPT_FP64_SCHEME, 3)


def test_workload_takes_twelve_moduli(h, mm):
    # the benchmark workload at M = N = K = 8192: its smallest spreads (near
    # 0.2436) ask for 38 bits, one more than 11 moduli hold at k = 8192, so 12
    # moduli (12 residue products against the digit form's 15), 41 bits
    A = torch.empty((8192, 8192), dtype=torch.float64, device="cuda")
    B = torch.empty((8192, 8192), dtype=torch.float64, device="cuda")
    mm.fill_uniform(A, seed=3, stream_id=inputs.STREAM_A, scale_mode=1, exp_stream_id=inputs.STREAM_EXP_A)
    mm.fill_uniform(B, seed=3, stream_id=inputs.STREAM_B, scale_mode=2, exp_stream_id=inputs.STREAM_EXP_B)
    C, code, bits, a, b, _ = h.debug_fp64_product(A, B, residues=False)
    assert h.sync() == 0
    assert (code - mm.CRT_BASE, bits) == mm.crt_rule(8192, a, b) == (12, 41), (code, bits, a, b)
    rows = [0, 4095, 8191]
    Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
    got = C.cpu().numpy()[rows]
    assert bound_ok(got, oracle.gemm_rows(Ah, Bh, rows), oracle.absprod_rows(Ah, Bh, rows), em.gamma(8192, "fp64_emu"))


def test_subnormal_outputs_bit_exact(h, mm):
    # entries near 2^-530: every product lies below 2^-1022, so the rebuilt
    # integer is rounded once straight to the subnormal grid (and some rows
    # reach down to zero)
    m, n, k = 140, 130, 700
    A = inputs.uniform(m, k, 17, inputs.STREAM_A) * 2.0 ** -530
    B = inputs.uniform(k, n, 17, inputs.STREAM_B) * 2.0 ** -530
    A[5] *= 2.0 ** -40
    C, code, bits, _, _, _ = h.debug_fp64_product(dev(A), dev(B), residues=False)
    assert h.sync() == 0
    assert code > mm.CRT_BASE
    got = C.cpu().numpy()
    assert np.all(np.abs(got) < 2.0 ** -1022) and np.any(got != 0.0)
    rows = [0, 5, 64, 139]
    assert np.array_equal(got[rows], em.gemm_fp64_crt(A[rows], B, bits, code - mm.CRT_BASE))


def test_grouped_modular_form_matches_single(h, mm):
    # a group in the default scheme: problems that take the modular form, one
    # that falls back to the digit form (short sums of wide-spread rows), one
    # that takes the plain kernel (Cauchy rows) and one the single path takes
    # (k <= 4): every result the same bits as mm_gemm on it alone
    specs = [("scaled", 200, 300, 700), ("normal", 130, 70, 1500), ("uniform", 33, 520, 64), ("t3", 90, 90, 300),
             ("spread", 40, 60, 7), ("scaled", 5, 6, 3), ("scaled", 257, 129, 2100)]
    probs = []
    for i, (name, m, n, k) in enumerate(specs):
        A, B = _case(name, m, n, k, 50 + i)
        probs.append((A, B, dev(A), dev(B), torch.full((m, n), np.nan, dtype=torch.float64, device="cuda")))
    A, B = inputs.cauchy(64, 900, 3, 1), inputs.cauchy(900, 40, 3, 2)
    probs.append((A, B, dev(A), dev(B), torch.full((64, 40), np.nan, dtype=torch.float64, device="cuda")))
    h.grouped([(a, b, c) for _, _, a, b, c in probs], precision=mm.FP64_EMU)
    assert h.sync() == 0
    codes = []
    for A, B, Ad, Bd, Cd in probs:
        alone = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
        assert h.sync() == 0
        got = Cd.cpu().numpy()
        assert np.array_equal(got, alone.cpu().numpy())
        k = A.shape[1]
        assert bound_ok(got, oracle.gemm(A, B), oracle.absprod(A, B), em.gamma(k, "fp64_emu"))
        if k > 4:
            codes.append(h.debug_fp64_product(Ad, Bd, residues=False)[1])
    assert any(c > mm.CRT_BASE for c in codes) and any(c <= 7 for c in codes) and 8 in codes, codes


def test_served_requests_take_the_modular_form(h, mm):
    A, B = _case("scaled", 300, 260, 1100, 9)
    Ad, Bd = dev(A), dev(B)
    Cd = torch.full((300, 260), np.nan, dtype=torch.float64, device="cuda")
    t = h.serve_submit(Ad, Bd, Cd, precision=mm.FP64_EMU)
    h.serve_drain()
    rc, _ = h.serve_poll(t)
    assert rc == 0
    alone = h.gemm(Ad, Bd, precision=mm.FP64_EMU)
    assert h.sync() == 0
    assert np.array_equal(Cd.cpu().numpy(), alone.cpu().numpy())
    assert h.debug_fp64_product(Ad, Bd, residues=False)[1] > mm.CRT_BASE


def test_default_scheme_by_size(mm):
    # the default takes the modular form from m n k >= 2^33 on (where it is the
    # faster form), the digit form below
    with mm.Handle(0) as hd:
        assert hd.get_option(mm.OPT_FP64_SCHEME) == 0
        small = _case("scaled", 1000, 1000, 1000, 4)
        big = (inputs.row_scaled(2048, 2048, 4), inputs.col_scaled(2048, 2048, 4))
        for (A, B), modular in ((small, False), (big, True)):
            C, code, bits, _, _, _ = hd.debug_fp64_product(dev(A), dev(B), residues=False)
            assert hd.sync() == 0
            assert (code > mm.CRT_BASE) == modular, (A.shape, code)
            rows = [0, 999]
            assert bound_ok(C.cpu().numpy()[rows], oracle.gemm_rows(A, B, rows), oracle.absprod_rows(A, B, rows),
                            em.gamma(A.shape[1], "fp64_emu"))


# ------------------------------------------------------------- rebuild pass
def _rebuild_case(N, m, n, seed):
    """Integers Y (object array) chosen across [-M/2, M/2): uniform, small,
    0 and +-1, next to +-M/2, exact halves between doubles (ties) and one
    unit off them; their residues as bytes (some as an unreduced
    representative c + m_l < 256); exponents E, F spanning normal,
    subnormal and overflowing results."""
    import random
    rng = random.Random(seed)
    M = em.crt_modulus_product(N)
    lo, hi = -(M // 2), M - M // 2          # Y in [lo, hi)
    lb = (M // 2).bit_length()              # 2^(lb-1) <= M/2
    Y = np.empty((m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            kind = rng.randrange(8)
            if kind == 0:
                y = rng.randrange(lo, hi)
            elif kind == 1:
                y = rng.randrange(max(lo, -2 ** 20), min(hi, 2 ** 20))
            elif kind == 2:
                y = rng.choice((0, 1, -1))
            elif kind == 3:
                y = rng.choice((hi - 1 - rng.randrange(4), lo + rng.randrange(4)))
            elif kind == 4 and lb > 56:
                # (2^52 + r) 2^(t+1) + 2^t: exactly half way between doubles, +-1
                t = rng.randrange(0, lb - 55)
                y = ((2 ** 52 + rng.randrange(2 ** 52)) << (t + 1)) + (1 << t) + rng.choice((0, 0, 1, -1))
                y = y if rng.random() < 0.5 else -y
            else:
                y = rng.randrange(-(1 << rng.randrange(0, lb)), 1 << rng.randrange(0, lb))
            Y[i, j] = y
    res = np.zeros((N, m, n), dtype=np.uint8)
    for l in range(N):
        ml = em.CRT_MODULI[l]
        for i in range(m):
            for j in range(n):
                c = Y[i, j] % ml
                if c + ml < 256 and rng.random() < 0.1:
                    c += ml
                res[l, i, j] = c
    bits = rng.randrange(24, 54)
    E = np.array([rng.randrange(-520, 480) for _ in range(m)], dtype=np.int32)
    F = np.array([rng.randrange(-520, 480) for _ in range(n)], dtype=np.int32)
    E[1] = -1022 - lb + 2 * bits            # rows of subnormal, underflowing and normal results
    E[3] = 1024 - lb + 2 * bits             # rows of overflowing and normal results
    E[9] = -1022 - lb + 2 * bits + 40
    return Y, res, E, F, bits


NONFINITE = -1000000


@pytest.mark.parametrize("N", list(range(1, 15)))
def test_rebuild_pass_every_modulus_count(h, mm, N):
    m, n = 70, 150           # three row blocks of 32 and three column blocks of 64, both ragged
    Y, res, E, F, bits = _rebuild_case(N, m, n, 1000 + N)
    # the oracle's textbook CRT sum gives the chosen integers back
    Yo = em.crt_reconstruct(res)
    assert all(Yo[i, j] == Y[i, j] for i in range(m) for j in range(n))
    En, Fn = E.copy(), F.copy()
    En[5], Fn[6] = NONFINITE, NONFINITE
    got = h.debug_crt_rebuild(torch.from_numpy(res).cuda(), torch.from_numpy(En), torch.from_numpy(Fn), N,
                              bits).cpu().numpy()
    from fractions import Fraction
    big = Fraction(2 ** 1024 - 2 ** 970)   # round-to-nearest overflows at and above this
    fin = np.ones((m, n), dtype=bool)
    fin[5, :] = False
    fin[:, 6] = False
    want = np.zeros((m, n))
    for i in range(m):
        for j in range(n):
            if not fin[i, j]:
                continue
            v = Fraction(int(Yo[i, j])) * Fraction(2) ** (int(E[i]) + int(F[j]) - 2 * bits)
            want[i, j] = (np.inf if v > 0 else -np.inf) if abs(v) >= big else \
                em.crt_round(Yo[i:i + 1, j:j + 1], E[i:i + 1], F[j:j + 1], bits)[0, 0]
    assert np.all(np.isnan(got[~fin]))
    gb, wb = got[fin].view(np.uint64), want[fin].view(np.uint64)
    bad = np.flatnonzero(gb != wb)
    assert bad.size == 0, (bad.size, got[fin][bad[:4]], want[fin][bad[:4]])
    # the cases reach every branch: subnormal and overflowing results, ties
    w = want[fin]
    assert np.any((w != 0) & (np.abs(w) < 2.0 ** -1022)) and np.any(np.isinf(w))
