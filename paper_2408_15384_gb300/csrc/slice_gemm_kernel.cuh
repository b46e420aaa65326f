// slice_gemm_kernel.cuh -- tcgen05 tensor-core product of bfloat16 operand slices, with
// the FP32-accuracy or FP64-accuracy epilogue. Persistent: each CTA (one per
// SM), or CTA pair (cta_group::2, 256-row tiles), walks a list of 128 x BN
// (256 x BN) output tiles, of one product or of a group of products.
//
// Warp roles:
//   warp 0      TMA producer: one A-slice tile (128 x 64) and one B-slice tile
//               (BN x 64, or BN/2 x 64 per CTA of a pair) per slice pair, one or
//               two pairs of the same K block per pipeline step, into a
//               STAGES-deep shared ring.
//   warp 1      allocates TMEM; one thread issues tcgen05.mma (M = 128 or 256,
//               N = BN, K = 16, bf16 x bf16 -> f32) and tcgen05.commit.
//   warps 2..   epilogue: 8 warps, or 12 / 16 when the FP64-accuracy level sums
//               live in registers; warp w reads TMEM lane quadrant w % 4 (row
//               = TMEM lane), the warps of a quadrant split the columns.
// Accumulation chunks alternate between two TMEM slots of BN columns, so the
// tensor cores run the next chunk (or the next tile) while the epilogue drains
// the previous one.
//
// FP32-accuracy (three bfloat16 slices per operand, or two from k = 512): the
// six slice pairs (p, q) with p + q <= 2 (the three with p + q <= 1) accumulate
// into one f32 accumulator, smallest products first; the epilogue scales by
// 2^(E_i + F_j) and stores doubles.
//
// FP64-accuracy (integer slices, levels d = p + q = 2..s+1, Ozaki-style): the
// kernel walks the levels one after the other, smallest first (d = s+1 down
// to 2). Level d sums d-1 slice pairs; with |slice| <= 2^7 each product is at
// most 2^14, so a K-chunk of Kc with Kc * (d-1) <= 1024 sums to at most 2^24
// and the f32 accumulator holds it exactly. The epilogue converts each
// finished chunk to integers and adds it at its level weight w_d = 8(s+1-d).
// The exact total is rounded once (half up) to a fixed point 2^shift
// (shift >= 0 keeps it below 2^62):
//   X = round(sum_{w_d < shift} 2^w_d L_d / 2^shift) + sum_{w_d >= shift} 2^(w_d - shift) L_d,
// the levels below the fixed point summed exactly first. 128-wide tiles keep
// X in TMEM (512 columns = two accumulator slots + the low and high 32-bit
// planes of X). Wider tiles keep int32 level sums in registers and either fold
// them into X held in C's storage (SLICE_FP64EMU) or recombine them by byte
// carry (SLICE_FP64EMU_CARRY, _CARRY7: each level's final low byte stored once,
// the rest carried into the next level's sum). After the last level X is
// converted to double once, scaled by 2^(E_i + F_j - 8(s+1) + shift) and
// stored. Every tiling and every recombination gives the same bits.
//
// The kernel templates and their launchers; slice_gemm.cu (FP32-accuracy and
// the dispatch), slice_gemm_fold.cu (FP64-accuracy int64 fold and level
// output) and slice_gemm_carry.cu (byte carry) instantiate them, so the
// instances compile in parallel.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "kernels.cuh"
#include "ptx.cuh"

namespace mmdev {

static constexpr int BM = 128;
static constexpr int BK = 64;                 // bf16 elements per K block (128 bytes)
static constexpr int SEG_CHUNKS = SLICE_SEG_CHUNKS;   // chunks per int32 level sum

// The modular form's rebuild constants (filled once per device by
// slice_prepare_crt; only the SLICE_CRT instances read them).
static __constant__ CrtTab c_crt;


// CG = CTAs per output tile: 1, or 2 for a CTA pair (cta_group::2) computing a
// 256-row tile, each CTA holding 128 rows of A and BN/2 rows of B in shared
// memory and its 128 rows of the accumulator in its own TMEM. CG = 4: CTA
// pairs as for 2, two pairs to a cluster on horizontally adjacent tiles
// (same rows of A): each CTA loads half of its 128 rows of A and multicasts
// them to its counterpart in the other pair, so A crosses from L2 once for
// both tiles.
template <int BN, int MODE, int CG>
struct Cfg {
  static constexpr int PAIR = (CG >= 2) ? 2 : 1;   // CTAs computing one tile
  // epilogue warps: 8 (two per TMEM lane quadrant). FP64-accuracy tiles wider
  // than 128 keep their columns' int32 level sums in registers: 16 warps for
  // 256 columns (64 sums a thread), 12 for 192 or 240 (64 or 80 sums a thread;
  // 14 warps leave 128 registers a thread)
  // The modular form keeps int32 sums in registers on every tile width (8
  // warps on 128-wide tiles: 64 sums a thread).
  static constexpr bool REG_SUMS = (MODE == SLICE_CRT) || ((BN != 128) && (MODE != SLICE_FP32EMU));
  static constexpr int EPI_WARPS = !REG_SUMS ? 8 : (BN == 256 ? 16 : (BN == 128 ? 8 : 12));
  static constexpr int EPI_WARP0 = 2;
  static constexpr int NUM_THREADS = 32 * (EPI_WARP0 + EPI_WARPS);
  static constexpr int A_BYTES = BM * BK * 2;
  static constexpr int B_BYTES = (BN / PAIR) * BK * 2;
  static constexpr int PAIR_BYTES = A_BYTES + B_BYTES;    // one slice pair's tiles of one K block
  static constexpr int SMEM_LIMIT = 232448 - 1024 - 256;   // max dynamic smem - alignment - static
  // slice pairs a pipeline step carries: two (8 MMAs a step, half the single
  // issuing threads' per-step work) while three such stages fit, else one
  static constexpr int PPS = (SMEM_LIMIT / (2 * PAIR_BYTES) >= 3) ? 2 : 1;
  static constexpr int STAGE_BYTES = PPS * PAIR_BYTES;
  static constexpr int STAGES_FIT = SMEM_LIMIT / STAGE_BYTES;
  static constexpr int STAGES = STAGES_FIT > 10 ? 10 : STAGES_FIT;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
  // two accumulator slots; FP64-accuracy adds the int64 total's planes (BN = 128)
  static constexpr int TMEM_COLS = (MODE == SLICE_FP32EMU || MODE == SLICE_CRT) ? 2 * BN : 512;
  static constexpr int XLO_COL = 2 * BN;
  static constexpr int XHI_COL = 3 * BN;
  static constexpr int COLS_PER_THREAD = BN / (EPI_WARPS / 4);
  static constexpr int TILE_M = BM * PAIR;
};

// K blocks per chunk at level d (d - 1 pairs): Kc * (d-1) <= 1024.
__device__ __forceinline__ int chunk_blocks(int d) {
  int kb = 16 / (d - 1);
  return kb < 1 ? 1 : kb;
}

__device__ __forceinline__ uint64_t dbits(double x) { return static_cast<uint64_t>(__double_as_longlong(x)); }
__device__ __forceinline__ double bitsd(uint64_t b) { return __longlong_as_double(static_cast<long long>(b)); }

// x * 2^e for finite x, exact unless the result leaves the normal range.
__device__ __forceinline__ double scale_pow2(double x, int e) {
  uint64_t b = dbits(x);
  uint64_t ab = b & 0x7FFFFFFFFFFFFFFFull;
  if (ab == 0) return x;
  int ex = static_cast<int>(ab >> 52);
  if (ex > 0 && ex + e >= 1 && ex + e <= 2046) return bitsd(b + (static_cast<uint64_t>(static_cast<int64_t>(e)) << 52));
  // rare: step through exact powers of two (a subnormal result rounds here)
  while (e > 1000) { x *= bitsd(static_cast<uint64_t>(1000 + 1023) << 52); e -= 1000; }
  while (e < -1000) { x *= bitsd(static_cast<uint64_t>(-1000 + 1023) << 52); e += 1000; }
  return x * bitsd(static_cast<uint64_t>(e + 1023) << 52);
}

// exact float -> double with a power-of-two scale
__device__ __forceinline__ double f32_to_f64_scaled(uint32_t fb, int e) {
  uint32_t e8 = (fb >> 23) & 255u;
  if (e8 == 0u || e8 == 255u) return scale_pow2(static_cast<double>(__uint_as_float(fb)), e);
  int ex = static_cast<int>(e8) - 127 + 1023;
  uint64_t sgn = static_cast<uint64_t>(fb >> 31) << 63;
  uint64_t man = static_cast<uint64_t>(fb & 0x7FFFFFu) << 29;
  if (ex + e >= 1 && ex + e <= 2046) return bitsd(sgn | (static_cast<uint64_t>(ex + e) << 52) | man);
  return scale_pow2(bitsd(sgn | (static_cast<uint64_t>(ex) << 52) | man), e);
}

// The double nearest to (-1)^neg * Y * 2^e (ties to even) for a 128-bit
// magnitude Y = yh:yl, in integer arithmetic only (GB300's FP64 pipe is
// narrow): normal results keep 53 bits, subnormal ones the bits down to
// 2^-1074, so every result is rounded once; overflow gives infinity.
__device__ __forceinline__ uint64_t rn_double_bits(uint64_t yh, uint64_t yl, int e, bool neg) {
  const uint64_t sgn = neg ? (1ull << 63) : 0ull;
  if ((yh | yl) == 0ull) return sgn;
  const int lz = yh ? __clzll(static_cast<long long>(yh)) : 64 + __clzll(static_cast<long long>(yl));
  uint64_t nh, nl;   // Y shifted up so its leading bit is bit 127
  if (lz >= 64) {
    nh = yl << (lz - 64);
    nl = 0ull;
  } else if (lz == 0) {
    nh = yh;
    nl = yl;
  } else {
    nh = (yh << lz) | (yl >> (64 - lz));
    nl = yl << lz;
  }
  int L = 127 - lz + e;                              // exponent of the leading bit
  const int keep = L >= -1022 ? 53 : L + 1075;       // significant bits kept
  if (keep < 0) return sgn;                          // below half the least subnormal
  uint64_t q = keep ? (nh >> (64 - keep)) : 0ull;
  const uint64_t rbit = (nh >> (63 - keep)) & 1ull;
  const bool sticky = (nh & ((1ull << (63 - keep)) - 1ull)) != 0ull || nl != 0ull;
  q += (rbit && (sticky || (q & 1ull))) ? 1ull : 0ull;
  if (keep < 53) return sgn | q;                     // subnormal (2^52: the least normal)
  if (q == (1ull << 53)) {
    q >>= 1;
    ++L;
  }
  if (L + 1023 >= 2047) return sgn | 0x7FF0000000000000ull;
  return sgn | (static_cast<uint64_t>(L + 1023) << 52) | (q & 0xFFFFFFFFFFFFFull);
}

struct Step {
  int kb;              // K block
  int pa, pb;          // A and B slice indices of the step's first pair
  int pa2, pb2;        // of its second pair (pa2 < 0: one pair)
  bool first, last;    // first / last step of its chunk
  int dkb;             // K block of the second pair: kb + dkb
};

// The steps of one FP64-accuracy level D: K chunks of KC blocks, in each K
// block the D-1 pairs (p, D-p), PPS of them a step. D is a compile-time
// constant so the pair loop unrolls into straight-line issue with constant
// slice indices; a runtime pair loop costs the single issuing threads about a
// quarter of the tensor rate.
template <int D, int PPS, typename Fn>
__device__ __forceinline__ void walk_level(int nkb, int& chunk, Fn& f) {
  constexpr int KC = (16 / (D - 1)) < 1 ? 1 : 16 / (D - 1);
  for (int kb0 = 0; kb0 < nkb; kb0 += KC, ++chunk) {
    const int kb1 = min(kb0 + KC, nkb);
    for (int kb = kb0; kb < kb1; ++kb) {
#pragma unroll
      for (int p = 1; p < D; p += PPS) {
        const bool two = PPS == 2 && p + 1 < D;
        f(Step{kb, p - 1, D - p - 1, two ? p : -1, two ? D - p - 2 : -1, kb == kb0 && p == 1,
               kb == kb1 - 1 && p + (two ? 1 : 0) == D - 1},
          chunk);
      }
    }
  }
}

// Walk the pipeline steps of one tile in order; f(Step, chunk offset in tile).
// The steps of the modular form: for each modulus l of the unit's range
// [l0, l1), K chunks of 16 blocks (at most 1024 terms of at most 2^14: exact
// f32 sums), one residue pair (l, l) a K block, PPS consecutive K blocks a step.
template <int PPS, typename Fn>
__device__ __forceinline__ void walk_crt(int l0, int l1, int nkb, Fn& f) {
  int chunk = 0;
  for (int l = l0; l < l1; ++l) {
    for (int kb0 = 0; kb0 < nkb; kb0 += 16, ++chunk) {
      const int kb1 = min(kb0 + 16, nkb);
      for (int kb = kb0; kb < kb1; kb += PPS) {
        const bool two = PPS == 2 && kb + 1 < kb1;
        f(Step{kb, l, l, two ? l : -1, two ? l : -1, kb == kb0, kb + (two ? 1 : 0) == kb1 - 1, 1}, chunk);
      }
    }
  }
}

template <int MODE, int PPS, typename Fn>
__device__ __forceinline__ void for_each_step(int s, int nkb, Fn&& f, int l0 = 0, int l1 = 0) {
  if (MODE == SLICE_CRT) {
    walk_crt<PPS>(l0, l1, nkb, f);
  } else if (MODE == SLICE_FP32EMU) {
    // pairs (p, q), p + q <= 2 (three slices) or p + q <= 1 (s = 2), smallest
    // products first (the same order whether a step carries one pair or two)
    for (int kb = 0; kb < nkb; ++kb) {
      if (PPS == 2) {
        if (s >= 3) {
          f(Step{kb, 2, 0, 1, 1, kb == 0, false}, 0);
          f(Step{kb, 0, 2, 1, 0, false, false}, 0);
          f(Step{kb, 0, 1, 0, 0, false, kb == nkb - 1}, 0);
        } else {
          f(Step{kb, 1, 0, 0, 1, kb == 0, false}, 0);
          f(Step{kb, 0, 0, -1, -1, false, kb == nkb - 1}, 0);
        }
      } else {
        if (s >= 3) {
          f(Step{kb, 2, 0, -1, -1, kb == 0, false}, 0);
          f(Step{kb, 1, 1, -1, -1, false, false}, 0);
          f(Step{kb, 0, 2, -1, -1, false, false}, 0);
          f(Step{kb, 1, 0, -1, -1, false, false}, 0);
        } else {
          f(Step{kb, 1, 0, -1, -1, kb == 0, false}, 0);
        }
        f(Step{kb, 0, 1, -1, -1, false, false}, 0);
        f(Step{kb, 0, 0, -1, -1, false, kb == nkb - 1}, 0);
      }
    }
  } else {
    int chunk = 0;
    for (int d = s + 1; d >= 2; --d) {   // smallest level first; s is 3 .. 7
      switch (d) {
        case 8: walk_level<8, PPS>(nkb, chunk, f); break;
        case 7: walk_level<7, PPS>(nkb, chunk, f); break;
        case 6: walk_level<6, PPS>(nkb, chunk, f); break;
        case 5: walk_level<5, PPS>(nkb, chunk, f); break;
        case 4: walk_level<4, PPS>(nkb, chunk, f); break;
        case 3: walk_level<3, PPS>(nkb, chunk, f); break;
        default: walk_level<2, PPS>(nkb, chunk, f); break;
      }
    }
  }
}

template <int MODE>
__device__ __forceinline__ int chunks_per_tile(int s, int nkb) {
  if (MODE == SLICE_FP32EMU) return 1;
  if (MODE == SLICE_CRT) return s * ((nkb + 15) / 16);   // s: the unit's modulus count
  int c = 0;
  for (int d = 2; d <= s + 1; ++d) {
    const int kc = chunk_blocks(d);
    c += (nkb + kc - 1) / kc;
  }
  return c;
}

struct TileJob {
  const SliceProblem* P;
  const CUtensorMap* ta;
  const CUtensorMap* tb;
  int tm, tn;
  int s, fix;    // the problem's slice count and fixed-point shift (modular form: N and b)
  bool skip;     // the problem's slice count is outside this launch's range
};

// A problem's slice count: its automatic count from device memory (written by
// the splitting kernels before this launch), else the host's.
// A decision code above SLICE_CRT_BASE names the modular form: N moduli, its
// bit count in the record's next word.
__device__ __forceinline__ void resolve_slices(const SliceGemmArgs& a, const SliceProblem& P, TileJob& j) {
  if (P.s_dev != nullptr) {
    const int code = *P.s_dev;
    if (code > SLICE_CRT_BASE) {
      j.s = code - SLICE_CRT_BASE;
      j.skip = code < a.s_lo || code > a.s_hi;
      j.fix = P.s_dev[1];
    } else {
      j.s = code;
      j.skip = j.s < a.s_lo || j.s > a.s_hi || j.s > SLICE_S_MAX;
      j.fix = j.skip ? 0 : P.fix_tab[j.s & 7];
    }
  } else {
    j.s = P.s;
    j.fix = P.fix_shift;
    j.skip = false;
  }
}

// The units a launch's walkers take in turn: unit u < nfull is tile u with all
// its moduli; the last, partial round of tiles (single modular-form products
// whose rebuild is a pass of its own) is split by moduli, `parts` units a
// tile, so that round ends after about N / parts moduli instead of N while
// the other walkers would idle. Every role maps a unit the same way.
struct Units {
  int nfull, parts, units;
};
__device__ __forceinline__ Units whole_tiles(int ntiles) { return Units{ntiles, 1, ntiles}; }
__device__ __forceinline__ Units split_tail(int ntiles, int walkers, int N) {
  const int tail = ntiles % walkers;
  int parts = tail > 0 ? walkers / tail : 1;
  if (parts > N) parts = N;
  if (parts < 2) return whole_tiles(ntiles);
  return Units{ntiles - tail, parts, ntiles - tail + tail * parts};
}
__device__ __forceinline__ int unit_tile(const Units& U, int u) {
  return u < U.nfull ? u : U.nfull + (u - U.nfull) / U.parts;
}
// the unit's moduli [l0, l1) of the tile's N
__device__ __forceinline__ void unit_moduli(const Units& U, int u, int N, int& l0, int& l1) {
  if (u < U.nfull) {
    l0 = 0;
    l1 = N;
  } else {
    const int part = (u - U.nfull) % U.parts;
    l0 = part * N / U.parts;
    l1 = (part + 1) * N / U.parts;
  }
}

// col_pairs = 2 (clusters of two CTA pairs): t numbers pairs of horizontally
// adjacent tiles and the cluster's pair `pair_col` takes tile column
// 2 * (pair of columns) + pair_col; single products only.
__device__ __forceinline__ TileJob get_job(const SliceGemmArgs& a, const CUtensorMap* pa, const CUtensorMap* pb,
                                           int t, int col_pairs = 1, int pair_col = 0) {
  TileJob j;
  if (a.probs == nullptr) {
    // raster in groups of 8 tile rows so consecutive tiles share B panels
    const SliceProblem& P = a.single;
    const int GROUP = 8;
    const int tiles_n = P.tiles_n / col_pairs;
    const int in_group = GROUP * tiles_n;
    const int gid = t / in_group;
    const int first_m = gid * GROUP;
    const int gsize = min(P.tiles_m - first_m, GROUP);
    j.tm = first_m + (t % in_group) % gsize;
    j.tn = ((t % in_group) / gsize) * col_pairs + pair_col;
    j.P = &a.single;
    j.ta = pa;
    j.tb = pb;
    resolve_slices(a, P, j);
  } else {
    const TileRef r = a.tiles[t];
    j.P = a.probs + r.prob;
    j.ta = a.tmaps + 2 * r.prob;
    j.tb = a.tmaps + 2 * r.prob + 1;
    j.tm = r.tm;
    j.tn = r.tn;
    resolve_slices(a, *j.P, j);
  }
  return j;
}

// The rebuild constants of N moduli as one output's rebuild reads them: M_N
// as 32-bit words and as two 64-bit words, M_N / 2, the quotient window's
// shift and scale. NW: how many 32-bit words M_N (and every W_l) needs; the
// words above are zero, and with a compile-time NW the arithmetic on them
// folds away.
struct CrtK {
  uint32_t m0, m1, m2, m3;
  uint64_t Ml, Mh, Hl, Hh;
  int wsh;
  float qscale;
};
template <int NW>
__device__ __forceinline__ CrtK crt_k(int N) {
  CrtK k;
  k.m0 = c_crt.M[N][0];
  k.m1 = NW > 1 ? c_crt.M[N][1] : 0u;
  k.m2 = NW > 2 ? c_crt.M[N][2] : 0u;
  k.m3 = NW > 3 ? c_crt.M[N][3] : 0u;
  k.Ml = (static_cast<uint64_t>(k.m1) << 32) | k.m0;
  k.Mh = (static_cast<uint64_t>(k.m3) << 32) | k.m2;
  k.Hl = c_crt.H[N][0];
  k.Hh = NW > 2 ? c_crt.H[N][1] : 0ull;
  k.wsh = c_crt.wsh[N];
  k.qscale = c_crt.qscale[N];
  return k;
}

// One output of a modular-form product from the column sums T0..T3 of
// S = sum_l c_l W_l (T_i: the 64-bit sum of the products of the residues with
// the W_l's 32-bit word i; S < 14 * 2^8 * M < 2^123). q = round(S / M) from a
// float estimate good to 2^-11; Y = S - q M moved into [-M/2, M/2) (one step
// at most) is the exact integer product; it is rounded to double once and
// scaled by 2^e (e = E_i + F_j - 2b). Returns the double's bits.
template <int NW>
__device__ __forceinline__ uint64_t crt_output(uint64_t T0, uint64_t T1, uint64_t T2, uint64_t T3, const CrtK& k,
                                               int e) {
  if (NW < 2) T1 = 0ull;
  if (NW < 3) T2 = 0ull;
  if (NW < 4) T3 = 0ull;
  // carries: S = hi:lo
  const uint64_t t1 = T1 + (T0 >> 32);
  const uint64_t t2 = T2 + (t1 >> 32);
  const uint64_t t3 = T3 + (t2 >> 32);
  const uint64_t lo = (t1 << 32) | (T0 & 0xFFFFFFFFull);
  const uint64_t hi = (t3 << 32) | (t2 & 0xFFFFFFFFull);
  // q = round(S / M) from the window S >> wsh (< 2^32)
  const int wsh = k.wsh;
  const uint64_t win = wsh >= 64 ? (hi >> (wsh - 64)) : (wsh == 0 ? lo : ((lo >> wsh) | (hi << (64 - wsh))));
  const float qf = __uint2float_rn(static_cast<uint32_t>(win)) * k.qscale;
  const uint32_t q = __float_as_uint(qf + 8388608.0f) - 0x4B000000u;   // round to nearest
  // q M in 32-bit words, then Y = S - q M (two's complement, 128 bits)
  const uint64_t p0 = static_cast<uint64_t>(q) * k.m0;
  const uint64_t p1 = static_cast<uint64_t>(q) * k.m1 + (p0 >> 32);
  const uint64_t p2 = static_cast<uint64_t>(q) * k.m2 + (p1 >> 32);
  const uint64_t p3 = static_cast<uint64_t>(q) * k.m3 + (p2 >> 32);
  const uint64_t qml = (p1 << 32) | (p0 & 0xFFFFFFFFull), qmh = (p3 << 32) | (p2 & 0xFFFFFFFFull);
  uint64_t yl = lo - qml;
  uint64_t yh = hi - qmh - (lo < qml ? 1ull : 0ull);
  // Y >= M/2: Y - M; Y < -M/2: Y + M
  const uint64_t th = yh - k.Hh - (yl < k.Hl ? 1ull : 0ull);
  if (static_cast<int64_t>(th) >= 0) {
    const uint64_t nl = yl - k.Ml;
    yh = yh - k.Mh - (yl < k.Ml ? 1ull : 0ull);
    yl = nl;
  } else {
    const uint64_t ul = yl + k.Hl;
    const uint64_t uh = yh + k.Hh + (ul < yl ? 1ull : 0ull);
    if (static_cast<int64_t>(uh) < 0) {
      const uint64_t nl = yl + k.Ml;
      yh = yh + k.Mh + (nl < yl ? 1ull : 0ull);
      yl = nl;
    }
  }
  // |Y| < 2^127: one rounding to double
  const bool neg = static_cast<int64_t>(yh) < 0;
  if (neg) {
    yl = ~yl + 1ull;
    yh = ~yh + (yl == 0ull ? 1ull : 0ull);
  }
  return rn_double_bits(yh, yl, e, neg);
}

// Rebuild of 4 outputs of a modular-form product inside the slice GEMM's
// epilogue: row `row`, columns c4 .. c4 + 3 (c4 a multiple of 4), from the
// residue bytes of its N products (crt_output each; W4: whether M_N needs a
// fourth 32-bit word). Kept out of line: it runs at modulus ends, between
// chunk drains, and gets the whole register budget.
template <bool W4>
static __device__ __noinline__ void crt_rebuild4(const SliceProblem& P, int64_t row, int64_t c4, int N, int bits) {
  constexpr int NW = W4 ? 4 : 3;
  const int64_t n = P.n;
  const int32_t Ei = P.E[row];
  double* const crow = P.C + row * P.ldc;
  const uint8_t* const rb = P.res + row * 8 + (c4 >> 3) * P.ldr + (c4 & 4);
  const CrtK k = crt_k<NW>(N);
  const int ebase = Ei - 2 * bits;
  // every modulus's bytes of the 4 columns, all loads in flight together
  uint32_t wc[CRT_N_MAX];
#pragma unroll
  for (int l = 0; l < CRT_N_MAX; ++l)
    wc[l] = (l < N) ? *reinterpret_cast<const uint32_t*>(rb + static_cast<int64_t>(l) * P.rplane) : 0u;
  uint64_t T[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int i = 0; i < 4; ++i) T[j][i] = 0ull;
#pragma unroll
  for (int l = 0; l < CRT_N_MAX; ++l) {
    if (l < N) {
      const uint32_t W0 = c_crt.W[N][l][0], W1 = c_crt.W[N][l][1], W2 = c_crt.W[N][l][2];
      const uint32_t W3 = W4 ? c_crt.W[N][l][3] : 0u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const uint32_t cl = (wc[l] >> (8 * j)) & 255u;
        T[j][0] += static_cast<uint64_t>(cl) * W0;
        T[j][1] += static_cast<uint64_t>(cl) * W1;
        T[j][2] += static_cast<uint64_t>(cl) * W2;
        if (W4) T[j][3] += static_cast<uint64_t>(cl) * W3;
      }
    }
  }
  const int4 f4 = (c4 + 3 < n && ((reinterpret_cast<uintptr_t>(P.F + c4) & 15u) == 0))
                      ? __ldg(reinterpret_cast<const int4*>(P.F + c4))
                      : make_int4(__ldg(P.F + c4), c4 + 1 < n ? __ldg(P.F + c4 + 1) : 0,
                                  c4 + 2 < n ? __ldg(P.F + c4 + 2) : 0, c4 + 3 < n ? __ldg(P.F + c4 + 3) : 0);
  uint64_t ob[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int32_t Fj = j == 0 ? f4.x : j == 1 ? f4.y : j == 2 ? f4.z : f4.w;
    ob[j] = (Ei == EXP_NONFINITE || Fj == EXP_NONFINITE)
                ? 0x7FF8000000000000ull
                : crt_output<NW>(T[j][0], T[j][1], T[j][2], T[j][3], k, ebase + Fj);
  }
  if (c4 + 3 < n && ((reinterpret_cast<uintptr_t>(crow + c4) & 15u) == 0)) {
    double2* const op = reinterpret_cast<double2*>(crow + c4);
    op[0] = make_double2(__longlong_as_double(static_cast<long long>(ob[0])),
                         __longlong_as_double(static_cast<long long>(ob[1])));
    op[1] = make_double2(__longlong_as_double(static_cast<long long>(ob[2])),
                         __longlong_as_double(static_cast<long long>(ob[3])));
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (c4 + j < n) crow[c4 + j] = __longlong_as_double(static_cast<long long>(ob[j]));
  }
}

template <int BN, int MODE, int CG>
__global__ void __launch_bounds__(Cfg<BN, MODE, CG>::NUM_THREADS, 1)
    slice_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                      const __grid_constant__ SliceGemmArgs args) {
  using C_ = Cfg<BN, MODE, CG>;
  extern __shared__ uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full_bar[C_::STAGES];
  __shared__ __align__(8) uint64_t empty_bar[C_::STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2];
  __shared__ __align__(8) uint64_t acce_bar[2];
  __shared__ __align__(8) uint64_t drain_bar;
  __shared__ uint32_t tmem_base_slot;
  __shared__ volatile uint32_t abort_flag;

  // a single product whose automatic slice count another launch handles:
  // nothing to do (the whole grid returns before any setup)
  if (args.probs == nullptr && args.single.s_dev != nullptr) {
    const int s = *args.single.s_dev;
    if (s < args.s_lo || s > args.s_hi || (s > SLICE_S_MAX && s <= SLICE_CRT_BASE)) return;
  }
  const uint32_t warp = warp_id(), lane = lane_id();
  const uint32_t smem_base = (smem_u32(smem_raw) + 1023u) & ~1023u;
  uint8_t* smem_gen = smem_raw + (smem_base - smem_u32(smem_raw));
  // clusters of two pairs (CG = 4) walk pairs of adjacent tiles, one each
  constexpr int COL_PAIRS = (CG == 4) ? 2 : 1;
  const int ntiles =
      (args.probs == nullptr) ? args.single.tiles_m * (args.single.tiles_n / COL_PAIRS) : *args.ntiles_dev;
  // tile walk: CTAs (CG = 1), CTA pairs (CG = 2) or clusters of two pairs
  // (CG = 4) stride over the tile list
  const uint32_t crank = (CG >= 2) ? cluster_ctarank() : 0u;
  const uint32_t rank = crank & 1u;              // rank within the CTA pair
  const uint32_t pair_rank0 = crank & ~1u;       // cluster rank of the pair's leader
  const int pair_col = static_cast<int>(crank >> 1);   // CG = 4: which tile of the cluster's two
  const int walker = (CG >= 2) ? static_cast<int>(cluster_id_x()) : static_cast<int>(blockIdx.x);
  const int walkers = (CG >= 2) ? static_cast<int>(cluster_count_x()) : static_cast<int>(gridDim.x);
  const bool leader = (rank == 0);
  // a single modular-form product whose rebuild is deferred: the last round
  // of tiles split by moduli (N from the decision record)
  Units U = whole_tiles(ntiles);
  if constexpr (MODE == SLICE_CRT) {
    if (args.probs == nullptr && args.crt_defer) {
      TileJob j0;
      resolve_slices(args, args.single, j0);
      U = split_tail(ntiles, walkers, j0.s);
    }
  }

  WaitCtl wc;
  wc.abort = &abort_flag;
  wc.err = args.err;
  wc.deadline_ns = globaltimer_ns() + args.timeout_ns;

  if (threadIdx.x == 0) {
    for (int i = 0; i < C_::STAGES; ++i) {
      mbar_init(&full_bar[i], 1);
      // CG = 4: both pairs' MMAs read data this CTA's copies wrote
      mbar_init(&empty_bar[i], CG == 4 ? 2 : 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&accf_bar[i], 1);
      mbar_init(&acce_bar[i], C_::EPI_WARPS * C_::PAIR);   // the pair's epilogue warps all report to the leader
    }
    mbar_init(&drain_bar, 1);
    abort_flag = 0u;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0 && args.probs == nullptr) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  if (warp == 1) {
    if constexpr (CG >= 2) {
      tmem_alloc_pair(&tmem_base_slot, C_::TMEM_COLS);   // collective: the same columns in both CTAs
      tmem_relinquish_pair();
    } else {
      tmem_alloc(&tmem_base_slot, C_::TMEM_COLS);
      tmem_relinquish();
    }
  }
  tc_fence_before();
  if constexpr (CG >= 2)
    cluster_sync_all();   // every CTA's barriers exist before any cross-CTA signal
  else
    __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = tmem_base_slot;


  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (int u = walker; u < U.units && ok; u += walkers) {
        const TileJob job = get_job(args, &tmA, &tmB, unit_tile(U, u), COL_PAIRS, pair_col);
        if (job.skip) continue;
        int l0, l1;
        unit_moduli(U, u, job.s, l0, l1);
        const int ya = job.tm * C_::TILE_M + static_cast<int>(rank) * BM;
        const int yb = job.tn * BN + static_cast<int>(rank) * (BN / C_::PAIR);
        for_each_step<MODE, C_::PPS>(job.s, job.P->nkb, [&](const Step& st, int) {
          if (!ok) return;
          const int stage = it % C_::STAGES;
          const uint32_t use = static_cast<uint32_t>(it / C_::STAGES);
          if (!mbar_wait(&empty_bar[stage], (use & 1u) ^ 1u, wc)) { ok = false; return; }
          // the stage holds [A tile | B tile] per slice pair of the step
          const int npairs = (C_::PPS == 2 && st.pa2 >= 0) ? 2 : 1;
          const uint32_t bytes = static_cast<uint32_t>(npairs * C_::PAIR_BYTES);
          uint8_t* const s0 = smem_gen + stage * C_::STAGE_BYTES;
          if constexpr (CG == 4) {
            // the pair's bytes complete on its leader's barrier; this CTA's
            // half of its 128 rows of A also lands in the other pair's
            // counterpart CTA (same rows of A), and that CTA's half lands here
            if (leader) mbar_arrive_expect_tx(&full_bar[stage], 2 * bytes);
            const uint32_t fb = mapa_shared(smem_u32(&full_bar[stage]), pair_rank0);
            const uint16_t mask = static_cast<uint16_t>((1u << rank) | (1u << (rank + 2u)));
            for (int q = 0; q < npairs; ++q) {
              uint8_t* sa = s0 + q * C_::PAIR_BYTES;
              const int kx = (st.kb + (q ? st.dkb : 0)) * BK;
              tma_load_3d_pair_mc(sa + pair_col * (C_::A_BYTES / 2), job.ta, kx, ya + pair_col * (BM / 2),
                                  q ? st.pa2 : st.pa, fb, mask);
              tma_load_3d_pair(sa + C_::A_BYTES, job.tb, kx, yb, q ? st.pb2 : st.pb, fb);
            }
          } else if constexpr (CG >= 2) {
            // both CTAs' bytes complete on the leader's barrier; only the leader arrives
            if (leader) mbar_arrive_expect_tx(&full_bar[stage], 2 * bytes);
            const uint32_t fb = mapa_shared(smem_u32(&full_bar[stage]), 0);
            for (int q = 0; q < npairs; ++q) {
              uint8_t* sa = s0 + q * C_::PAIR_BYTES;
              const int kx = (st.kb + (q ? st.dkb : 0)) * BK;
              tma_load_3d_pair(sa, job.ta, kx, ya, q ? st.pa2 : st.pa, fb);
              tma_load_3d_pair(sa + C_::A_BYTES, job.tb, kx, yb, q ? st.pb2 : st.pb, fb);
            }
          } else {
            mbar_arrive_expect_tx(&full_bar[stage], bytes);
            for (int q = 0; q < npairs; ++q) {
              uint8_t* sa = s0 + q * C_::PAIR_BYTES;
              const int kx = (st.kb + (q ? st.dkb : 0)) * BK;
              tma_load_3d(sa, job.ta, kx, ya, q ? st.pa2 : st.pa, &full_bar[stage]);
              tma_load_3d(sa + C_::A_BYTES, job.tb, kx, yb, q ? st.pb2 : st.pb, &full_bar[stage]);
            }
          }
          ++it;
        }, l0, l1);
      }
      if (!ok) {
        // copies already issued must land before the CTA exits
        const uint64_t dl = globaltimer_ns() + 100000000ull;
        for (int j = (it > C_::STAGES ? it - C_::STAGES : 0); j < it; ++j)
          mbar_wait_quiet(&full_bar[j % C_::STAGES], static_cast<uint32_t>(j / C_::STAGES) & 1u, dl);
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    // ----------------------------------------------------------------- MMA
    if (lane == 0 && leader) {
      const uint32_t idesc = idesc_bf16_f32(C_::TILE_M, BN);
      int it = 0;
      int chunk_base = 0;
      bool ok = true;
      bool issued_any = false;
      for (int u = walker; u < U.units && ok; u += walkers) {
        const TileJob job = get_job(args, &tmA, &tmB, unit_tile(U, u), COL_PAIRS, pair_col);
        if (job.skip) continue;
        int l0, l1;
        unit_moduli(U, u, job.s, l0, l1);
        const int s = job.s, nkb = job.P->nkb;
        for_each_step<MODE, C_::PPS>(s, nkb, [&](const Step& st, int cofs) {
          if (!ok) return;
          const int chunk = chunk_base + cofs;
          const int slot = chunk & 1;
          if (st.first) {
            const uint32_t use = static_cast<uint32_t>(chunk >> 1);
            bool w;
            if constexpr (CG >= 2)
              w = mbar_wait_cluster(&acce_bar[slot], (use & 1u) ^ 1u, wc);
            else
              w = mbar_wait(&acce_bar[slot], (use & 1u) ^ 1u, wc);
            if (!w) { ok = false; return; }
            tc_fence_after();
          }
          const int stage = it % C_::STAGES;
          const uint32_t use = static_cast<uint32_t>(it / C_::STAGES);
          if (!mbar_wait(&full_bar[stage], use & 1u, wc)) { ok = false; return; }
          tc_fence_after();
          const uint32_t dt = tmem_base + static_cast<uint32_t>(slot * BN);
          const int npairs = (C_::PPS == 2 && st.pa2 >= 0) ? 2 : 1;
#pragma unroll
          for (int q = 0; q < C_::PPS; ++q) {
            if (q >= npairs) break;
            const uint32_t sa = smem_base + stage * C_::STAGE_BYTES + q * C_::PAIR_BYTES;
            const uint64_t da = smem_desc_sw128(sa), db = smem_desc_sw128(sa + C_::A_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              // 16 bf16 (32 bytes) further along K inside the 128-byte swizzled rows
              const uint32_t acc = (st.first && q == 0 && kk == 0) ? 0u : 1u;
              if constexpr (CG >= 2)
                umma_bf16_pair(dt, da + static_cast<uint64_t>(kk * 2), db + static_cast<uint64_t>(kk * 2), idesc, acc);
              else
                umma_bf16(dt, da + static_cast<uint64_t>(kk * 2), db + static_cast<uint64_t>(kk * 2), idesc, acc);
            }
          }
          issued_any = true;
          if constexpr (CG == 4) {
            // the stage is free in all four CTAs (each holds data of both pairs' copies)
            umma_commit_pair_mask(&empty_bar[stage], 0xF);
            if (st.last) umma_commit_pair_mask(&accf_bar[slot], static_cast<uint16_t>(3u << (2 * pair_col)));
          } else if constexpr (CG >= 2) {
            umma_commit_pair(&empty_bar[stage]);
            if (st.last) umma_commit_pair(&accf_bar[slot]);
          } else {
            umma_commit(&empty_bar[stage]);
            if (st.last) umma_commit(&accf_bar[slot]);
          }
          ++it;
        }, l0, l1);
        chunk_base += chunks_per_tile<MODE>(MODE == SLICE_CRT ? l1 - l0 : s, nkb);
      }
      if (!ok && issued_any) {
        if constexpr (CG >= 2)
          umma_commit_pair_local(&drain_bar);
        else
          umma_commit(&drain_bar);
        mbar_wait_quiet(&drain_bar, 0u, globaltimer_ns() + 100000000ull);
      }
    }
    __syncwarp();
  } else if (static_cast<int>(warp) >= C_::EPI_WARP0) {
    // ------------------------------------------------------------ epilogue
    const int ew = static_cast<int>(warp) - C_::EPI_WARP0;   // 0 .. EPI_WARPS-1
    const int quad = static_cast<int>(warp & 3u);        // TMEM lane quadrant this warp may access
    const int half = ew >> 2;                            // which share of the tile's columns
    const int row_in_tile = quad * 32 + static_cast<int>(lane);
    const int col_off = half * C_::COLS_PER_THREAD;
    const uint32_t t_lane = static_cast<uint32_t>(quad * 32) << 16;
    int chunk = 0;
    bool ok = true;
    // where this warp reports "slot drained": the leader's barrier
    const uint32_t acce_remote0 = (CG >= 2) ? mapa_shared(smem_u32(&acce_bar[0]), pair_rank0) : 0u;
    const uint32_t acce_remote1 = (CG >= 2) ? mapa_shared(smem_u32(&acce_bar[1]), pair_rank0) : 0u;
    // modular form: a tile's rebuild is deferred and run 4 columns at a time
    // at the following tile's modulus ends, spread evenly over them (pend_t:
    // the tile, -1 for none; pend_g: its next group of 4 columns)
    constexpr int G4 = C_::COLS_PER_THREAD / 4;
    int pend_t = -1, pend_g = 0;
    auto crt_step = [&]() {
      const TileJob pj = get_job(args, &tmA, &tmB, pend_t, COL_PAIRS, pair_col);
      const int64_t prow = static_cast<int64_t>(pj.tm) * C_::TILE_M + static_cast<int64_t>(rank) * BM + row_in_tile;
      const int64_t pc4 = static_cast<int64_t>(pj.tn) * BN + col_off + 4 * pend_g;
      if (prow < pj.P->m && pc4 < pj.P->n) {
        if (pj.s > 12)
          crt_rebuild4<true>(*pj.P, prow, pc4, pj.s, pj.fix);
        else
          crt_rebuild4<false>(*pj.P, prow, pc4, pj.s, pj.fix);
      }
      if (++pend_g == G4) pend_t = -1;
    };
    (void)crt_step;
    for (int u = walker; u < U.units && ok; u += walkers) {
      const int t = unit_tile(U, u);
      const TileJob job = get_job(args, &tmA, &tmB, t, COL_PAIRS, pair_col);
      if (job.skip) continue;
      int l0, l1;
      unit_moduli(U, u, job.s, l0, l1);
      const SliceProblem& P = *job.P;
      const int64_t row = static_cast<int64_t>(job.tm) * C_::TILE_M + static_cast<int64_t>(rank) * BM + row_in_tile;
      const int64_t col0 = static_cast<int64_t>(job.tn) * BN + col_off;
      const int64_t n = P.n;
      const bool row_ok = row < P.m;
      const int32_t Ei = row_ok ? P.E[row] : 0;

      if (MODE == SLICE_FP32EMU) {
        const int slot = chunk & 1;
        if (!mbar_wait(&accf_bar[slot], static_cast<uint32_t>(chunk >> 1) & 1u, wc)) { ok = false; break; }
        tc_fence_after();
        double* crow = P.C + row * P.ldc;
#pragma unroll 1
        for (int cg = 0; cg < C_::COLS_PER_THREAD / 32; ++cg) {
          uint32_t r[32];
          tmem_ld32_sync(tmem_base + t_lane + static_cast<uint32_t>(slot * BN + col_off + cg * 32), r);
          if (row_ok) {
#pragma unroll
            for (int v = 0; v < 32; ++v) {
              const int64_t col = col0 + cg * 32 + v;
              if (col < n) {
                const int32_t Fj = __ldg(P.F + col);
                double out;
                if (Ei == EXP_NONFINITE || Fj == EXP_NONFINITE)
                  out = __longlong_as_double(0x7FF8000000000000ll);
                else
                  out = f32_to_f64_scaled(r[v], Ei + Fj);
                crow[col] = out;
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if constexpr (CG >= 2)
            mbar_arrive_remote(slot ? acce_remote1 : acce_remote0);
          else
            mbar_arrive(&acce_bar[slot]);
        }
        ++chunk;
      } else if constexpr (MODE == SLICE_CRT) {
        // Modular form. For each modulus the thread keeps int32 sums of its
        // columns over the K chunks (reduced modulo m at every int32 segment
        // end: a segment adds at most SEG_CHUNKS 2^24 < 2^31) and stores their
        // remainders in [0, m) as bytes. Grouped launches rebuild the tile's
        // outputs from them (crt_rebuild4) 4 columns at a time at the next
        // tile's modulus ends, so the rebuild overlaps the tensor cores' work;
        // single products (crt_defer) leave it to a pass of its own, which
        // keeps the epilogue warps off the issue slots the MMA thread needs.
        const int N = job.s;
        const int nkb = P.nkb;
        const int nch = (nkb + 15) / 16;
        constexpr int NG = C_::COLS_PER_THREAD / 8;
        constexpr int NQ = C_::COLS_PER_THREAD / 16;
        int32_t lsum[NG][8];
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int v = 0; v < 8; ++v) lsum[g][v] = 0;
        // residue bytes: per plane, blocks of 8 columns, each block the rows'
        // 8-byte records one after the other, so a warp (32 consecutive rows)
        // moves 256 contiguous bytes per access
        uint8_t* const rbase = P.res + row * 8 + (col0 >> 3) * P.ldr;
        // x mod m_l in [0, m) for any int32 x: v = (floor(x / 2^16) + 2^15)
        // (2^16 mod m) + (x mod 2^16) < 2^24 is x + 2^31 modulo m, its quotient
        // floor(v (floor(2^32 / m) + 1) / 2^32) is exact (v / 2^32 < 1/m), and
        // 2^31 mod m comes off at the end (constants from the table, read
        // where they are used, so none is live across the chunk loop)
        struct Reducer {
          uint32_t mdl, magic, c16;
          int32_t c31;
          __device__ __forceinline__ explicit Reducer(int l)
              : mdl(static_cast<uint32_t>(crt_modulus(l))), magic(c_crt.magic[l]), c16(c_crt.c16[l]),
                c31(c_crt.c31[l]) {}
          __device__ __forceinline__ int32_t operator()(int32_t x) const {
            const uint32_t v = (static_cast<uint32_t>(x >> 16) + 32768u) * c16 + (static_cast<uint32_t>(x) & 0xFFFFu);
            const uint32_t q = __umulhi(v, magic);
            const int32_t r = static_cast<int32_t>(v - q * mdl) - c31;
            return r < 0 ? r + static_cast<int32_t>(mdl) : r;
          }
        };
        for (int l = l0; l < l1 && ok; ++l) {
          for (int c = 0; c < nch; ++c, ++chunk) {
            const int slot = chunk & 1;
            if (!mbar_wait(&accf_bar[slot], static_cast<uint32_t>(chunk >> 1) & 1u, wc)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < NG; ++g)
              tmem_ld8_add_i32(tmem_base + t_lane + static_cast<uint32_t>(slot * BN + col_off + g * 8), lsum[g]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if constexpr (CG >= 2)
                mbar_arrive_remote(slot ? acce_remote1 : acce_remote0);
              else
                mbar_arrive(&acce_bar[slot]);
            }
            if (((c + 1) % SEG_CHUNKS) == 0 && c + 1 < nch) {
              const Reducer reduce(l);
#pragma unroll
              for (int g = 0; g < NG; ++g)
#pragma unroll
                for (int v = 0; v < 8; ++v) lsum[g][v] = reduce(lsum[g][v]);
            }
          }
          if (!ok) break;
          if (row_ok) {
            const Reducer reduce(l);
            uint8_t* const rp = rbase + static_cast<int64_t>(l) * P.rplane;
#pragma unroll
            for (int g = 0; g < NG; ++g) {
              uint32_t lo = 0u, hi = 0u;
#pragma unroll
              for (int b = 0; b < 4; ++b) {
                lo |= static_cast<uint32_t>(reduce(lsum[g][b])) << (8 * b);
                hi |= static_cast<uint32_t>(reduce(lsum[g][4 + b])) << (8 * b);
              }
              if (col0 + 8 * g < n) *reinterpret_cast<uint2*>(rp + g * P.ldr) = make_uint2(lo, hi);
            }
          }
#pragma unroll
          for (int g = 0; g < NG; ++g)
#pragma unroll
            for (int v = 0; v < 8; ++v) lsum[g][v] = 0;
          // the previous tile's rebuild, its share for this modulus end, while
          // the tensor cores run this modulus's first chunks (the sums start
          // again from zero here, so none of them is live across it)
          const int upto = (G4 * (l + 1) + N - 1) / N;
          while (pend_t >= 0 && pend_g < upto) crt_step();
        }
        if (ok) {
          // the previous tile's rebuild, what is left of it, then this tile's
          while (pend_t >= 0) crt_step();
          pend_t = args.crt_defer ? -1 : t;
          pend_g = 0;
        }
      } else if constexpr (C_::REG_SUMS) {
        // wide tiles: TMEM holds just the two accumulator slots. Each thread
        // keeps int32 level sums of its columns in registers (one TMEM load
        // per element per chunk) and folds them into the int64 total, kept in
        // C's storage, at the end of each level.
        int64_t* const xrow = reinterpret_cast<int64_t*>(P.C) + row * P.ldc;
        const int s = job.s;
        const int nkb = P.nkb;
        const int fix_shift = job.fix;
        constexpr int NG = C_::COLS_PER_THREAD / 8;
        int32_t lsum[NG][8];
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int v = 0; v < 8; ++v) lsum[g][v] = 0;
        // Folds run from a copy of the sums parked in local memory, 16 columns
        // (one 128-byte line of the total) per group. The fold of a level is
        // spread over the following chunks, one group per chunk, so its loads
        // of the total overlap the tensor cores' next chunks; it completes
        // before the next fold and before the tile's last one, which converts
        // the total to doubles at once.
        constexpr int NQ = C_::COLS_PER_THREAD / 16;
        int32_t sums[C_::COLS_PER_THREAD];
        asm volatile("" ::"l"(sums) : "memory");
        int64_t* const xp = xrow + col0;
        const bool full = (n - col0 >= C_::COLS_PER_THREAD) && ((reinterpret_cast<uintptr_t>(xp) & 15u) == 0);
        const int ebase = Ei - 8 * (s + 1) + fix_shift;
        const bool nan_row = (Ei == EXP_NONFINITE);
        // fold groups [q0, q1) of the parked sums with the given level parameters
        auto fold_groups = [&](int q0, int q1, int lsh, bool first, bool rnd, bool last) {
          auto fold1 = [&](int i, int64_t old, int32_t Fj) -> int64_t {
            int64_t X = old + (static_cast<int64_t>(sums[i]) << lsh);
            if (rnd) X = (X + (1ll << (fix_shift - 1))) >> fix_shift;
            if (last) {
              const double o = (nan_row || Fj == EXP_NONFINITE) ? __longlong_as_double(0x7FF8000000000000ll)
                                                               : scale_pow2(__ll2double_rn(X), ebase + Fj);
              X = __double_as_longlong(o);
            }
            return X;
          };
#pragma unroll 1
          for (int q = q0; q < q1; ++q) {
            if (full) {
              // eight 16-byte loads in flight, then the stores
              longlong2 xv[8];
#pragma unroll
              for (int j = 0; j < 8; ++j)
                xv[j] = first ? make_longlong2(0, 0) : reinterpret_cast<const longlong2*>(xp)[q * 8 + j];
              int4 fv[4] = {};
              if (last) {
#pragma unroll
                for (int j = 0; j < 4; ++j) fv[j] = __ldg(reinterpret_cast<const int4*>(P.F + col0) + q * 4 + j);
              }
#pragma unroll
              for (int j = 0; j < 8; ++j) {
                const int i = q * 16 + 2 * j;
                const int4& f4 = fv[j >> 1];
                xv[j].x = fold1(i, xv[j].x, (j & 1) ? f4.z : f4.x);
                xv[j].y = fold1(i + 1, xv[j].y, (j & 1) ? f4.w : f4.y);
                reinterpret_cast<longlong2*>(xp)[q * 8 + j] = xv[j];
              }
            } else {
#pragma unroll 4
              for (int v = 0; v < 16; ++v) {
                const int i = q * 16 + v;
                if (col0 + i < n) xp[i] = fold1(i, first ? 0ll : xp[i], last ? __ldg(P.F + col0 + i) : 0);
              }
            }
          }
        };
        // Carry path, taken for s <= 7 by warps whose rows are all full
        // 16-byte aligned segments while every level fits one int32 segment
        // and the fixed point lies at or below the last level's weight (the
        // choice is warp-uniform, as the TMEM loads are warp-collective). After level d
        // the low byte of each column's running sum is final (every later
        // level adds multiples of 2^8 at this weight): it is written once to
        // the thread's own part of C and the rest, an arithmetic shift by 8,
        // carries into the next level's sum. The last sum S and the bytes b_l
        // (l = 0 .. s-2, weight 2^(8l)) give the exact total
        //   X = S 2^(8(s-1)) + sum_l b_l 2^(8l),
        // rounded once to the fixed point as the fold path rounds it; |S| stays
        // below SEG_CHUNKS 2^24 + 2^23 < 2^31. Full rows keep the bytes of each
        // 16-column group (one 16-byte word per level) in the first 16(s-1) <=
        // 96 bytes of that group's own 128-byte output. The group's 4-column
        // blocks are converted from block 3 down to block 0; block j's doubles
        // cover level words 2j and 2j+1, so before block 2 is written the
        // lower blocks' parts of words 4 and 5 are kept in registers, and
        // before block 1 is written block 0's parts of words 2 and 3.
        bool carry = false;
        // level words a group keeps: s - 1 <= 4 (s <= 5) or <= 6 (s = 6, 7)
        constexpr int LV = (MODE == SLICE_FP64EMU_CARRY7) ? 6 : 4;
        if constexpr (MODE == SLICE_FP64EMU_CARRY || MODE == SLICE_FP64EMU_CARRY7) {
          const int kc_top = chunk_blocks(s + 1);
          carry = s <= LV + 1 && ((nkb + kc_top - 1) / kc_top <= SEG_CHUNKS) && (fix_shift <= 8 * (s - 1)) &&
                  __all_sync(0xffffffffu, full);
        }
        if (carry) {
          if constexpr (MODE == SLICE_FP64EMU_CARRY || MODE == SLICE_FP64EMU_CARRY7) {
          uint8_t* const xb = reinterpret_cast<uint8_t*>(xp);
          const int W = 8 * (s - 1);
          auto total = [&](int32_t S, uint64_t R, int32_t Fj) -> double {
            int64_t X;
            if (fix_shift == 0)
              X = (static_cast<int64_t>(S) << W) + static_cast<int64_t>(R);
            else
              X = (static_cast<int64_t>(S) << (W - fix_shift)) +
                  static_cast<int64_t>((R + (1ull << (fix_shift - 1))) >> fix_shift);
            if (nan_row || Fj == EXP_NONFINITE) return __longlong_as_double(0x7FF8000000000000ll);
            return scale_pow2(__ll2double_rn(X), ebase + Fj);
          };
          for (int d = s + 1; d >= 2 && ok; --d) {
            const int kc = chunk_blocks(d);
            const int nch = (nkb + kc - 1) / kc;
            for (int c = 0; c < nch; ++c, ++chunk) {
              const int slot = chunk & 1;
              if (!mbar_wait(&accf_bar[slot], static_cast<uint32_t>(chunk >> 1) & 1u, wc)) { ok = false; break; }
              tc_fence_after();
#pragma unroll
              for (int g = 0; g < NG; ++g)
                tmem_ld8_add_i32(tmem_base + t_lane + static_cast<uint32_t>(slot * BN + col_off + g * 8), lsum[g]);
              tc_fence_before();
              __syncwarp();
              if (lane == 0) {
                if constexpr (CG >= 2)
                  mbar_arrive_remote(slot ? acce_remote1 : acce_remote0);
                else
                  mbar_arrive(&acce_bar[slot]);
              }
            }
            if (!ok || !row_ok) continue;
            const int l = s + 1 - d;
            if (d > 2) {
              // emit this level's low bytes, carry the rest
              {
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                  uint32_t w[4];
#pragma unroll
                  for (int j = 0; j < 4; ++j) {
                    uint32_t x = 0u;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                      int32_t& v = lsum[(q * 16 + j * 4 + b) >> 3][(q * 16 + j * 4 + b) & 7];
                      x |= (static_cast<uint32_t>(v) & 255u) << (8 * b);
                      v >>= 8;
                    }
                    w[j] = x;
                  }
                  *reinterpret_cast<uint4*>(xb + q * 128 + 16 * l) = make_uint4(w[0], w[1], w[2], w[3]);
                }
              }
            } else {
              // the last level: assemble, round, convert
              // word ll's bytes of 4-column block j of group q (0 past the levels)
              auto ldw = [&](int q, int j, int ll) -> uint32_t {
                return (ll < LV && ll < s - 1) ? *reinterpret_cast<const uint32_t*>(xb + q * 128 + 16 * ll + 4 * j) : 0u;
              };
              auto convert_block = [&](int q, int j, const uint32_t (&bw)[6]) {
                const int4 f4 = __ldg(reinterpret_cast<const int4*>(P.F + col0) + q * 4 + j);
                double o[4];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                  uint64_t R = 0;
#pragma unroll
                  for (int ll = 0; ll < LV; ++ll) R |= static_cast<uint64_t>((bw[ll] >> (8 * b)) & 255u) << (8 * ll);
                  const int32_t Fj = b == 0 ? f4.x : b == 1 ? f4.y : b == 2 ? f4.z : f4.w;
                  o[b] = total(lsum[(q * 16 + j * 4 + b) >> 3][(q * 16 + j * 4 + b) & 7], R, Fj);
                }
                double2* const op = reinterpret_cast<double2*>(xp) + q * 8 + j * 2;
                op[0] = make_double2(o[0], o[1]);
                op[1] = make_double2(o[2], o[3]);
              };
#pragma unroll
              for (int q = 0; q < NQ; ++q) {
                {
                  const uint32_t b3[6] = {ldw(q, 3, 0), ldw(q, 3, 1), ldw(q, 3, 2), ldw(q, 3, 3), ldw(q, 3, 4), ldw(q, 3, 5)};
                  convert_block(q, 3, b3);
                }
                const uint32_t w14 = ldw(q, 1, 4), w15 = ldw(q, 1, 5), w04 = ldw(q, 0, 4), w05 = ldw(q, 0, 5);
                {
                  const uint32_t b2[6] = {ldw(q, 2, 0), ldw(q, 2, 1), ldw(q, 2, 2), ldw(q, 2, 3), ldw(q, 2, 4), ldw(q, 2, 5)};
                  convert_block(q, 2, b2);
                }
                const uint32_t w02 = ldw(q, 0, 2), w03 = ldw(q, 0, 3);
                {
                  const uint32_t b1[6] = {ldw(q, 1, 0), ldw(q, 1, 1), ldw(q, 1, 2), ldw(q, 1, 3), w14, w15};
                  convert_block(q, 1, b1);
                }
                const uint32_t b0[6] = {ldw(q, 0, 0), ldw(q, 0, 1), w02, w03, w04, w05};
                convert_block(q, 0, b0);
              }
            }
          }
          }
        } else {
        int pend_q = NQ, pend_lsh = 0;   // the deferred fold: next group, level parameters
        bool pend_first = false, pend_rnd = false;
        bool first_fold = true;
        for (int d = s + 1; d >= 2 && ok; --d) {
          const int kc = chunk_blocks(d);
          const int nch = (nkb + kc - 1) / kc;
          const int w = 8 * (s + 1 - d);
          const bool raw = w < fix_shift;   // summed exactly, rounded after the last such level
          const int lsh = (MODE == SLICE_LEVELS) ? 0 : (raw ? w : w - fix_shift);
          const bool round_at_end = (MODE != SLICE_LEVELS) && raw && (d == 2 || w + 8 >= fix_shift);
          for (int c = 0; c < nch; ++c, ++chunk) {
            const int slot = chunk & 1;
            const bool level_end = (c == nch - 1);
            const bool seg_end = ((c + 1) % SEG_CHUNKS) == 0;
            if (!mbar_wait(&accf_bar[slot], static_cast<uint32_t>(chunk >> 1) & 1u, wc)) { ok = false; break; }
            tc_fence_after();
#pragma unroll
            for (int g = 0; g < NG; ++g)
              tmem_ld8_add_i32(tmem_base + t_lane + static_cast<uint32_t>(slot * BN + col_off + g * 8), lsum[g]);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
              if constexpr (CG >= 2)
                mbar_arrive_remote(slot ? acce_remote1 : acce_remote0);
              else
                mbar_arrive(&acce_bar[slot]);
            }
            if constexpr (MODE != SLICE_LEVELS) {
              if (pend_q < NQ && row_ok) {
                // one group of the deferred fold; the next group's line towards L2
                if (!pend_first && pend_q + 1 < NQ && col0 + (pend_q + 1) * 16 < n) prefetch_l2(xp + (pend_q + 1) * 16);
                fold_groups(pend_q, pend_q + 1, pend_lsh, pend_first, pend_rnd, false);
                ++pend_q;
              }
            }
            if (!(level_end || seg_end)) continue;
            const bool last = level_end && (d == 2);
            const bool rnd = level_end && round_at_end;
            if (row_ok) {
              if constexpr (MODE == SLICE_LEVELS) {
                int64_t* const lp = P.levels + (static_cast<int64_t>(d - 2) * P.m + row) * n + col0;
#pragma unroll
                for (int g = 0; g < NG; ++g)
#pragma unroll
                  for (int v = 0; v < 8; ++v) {
                    const int i = g * 8 + v;
                    if (col0 + i < n) lp[i] += static_cast<int64_t>(lsum[g][v]);
                    lsum[g][v] = 0;
                  }
              } else {
                // finish the previous fold, then park these sums (and reset them
                // here, inside the branch: rows past m keep stale sums that are
                // never stored; resetting outside makes the compiler spill the
                // sums in the chunk loop)
                if (pend_q < NQ) fold_groups(pend_q, NQ, pend_lsh, pend_first, pend_rnd, false);
#pragma unroll
                for (int g = 0; g < NG; ++g)
#pragma unroll
                  for (int v = 0; v < 8; ++v) { sums[g * 8 + v] = lsum[g][v]; lsum[g][v] = 0; }
                asm volatile("" ::"l"(sums) : "memory");
                if (last) {
                  fold_groups(0, NQ, lsh, first_fold, rnd, true);
                  pend_q = NQ;
                } else {
                  if (!first_fold) prefetch_l2(xp);
                  pend_q = 0;
                  pend_lsh = lsh;
                  pend_first = first_fold;
                  pend_rnd = rnd;
                }
              }
            }
            first_fold = false;
          }
        }
        }
      } else {
        double* const crow = P.C + row * P.ldc;
        const int s = job.s;
        const int nkb = P.nkb;
        const int fix_shift = job.fix;
        const uint32_t txlo = tmem_base + t_lane + static_cast<uint32_t>(C_::XLO_COL + col_off);
        const uint32_t txhi = tmem_base + t_lane + static_cast<uint32_t>(C_::XHI_COL + col_off);
        bool fresh = true;   // X holds nothing yet (reads as zero)
        for (int d = s + 1; d >= 2 && ok; --d) {
          const int kc = chunk_blocks(d);
          const int nch = (nkb + kc - 1) / kc;
          // weight of level d in the total (level output: unweighted)
          const int w = 8 * (s + 1 - d);
          const bool raw = w < fix_shift;
          const int lsh = (MODE == SLICE_LEVELS) ? 0 : (raw ? w : w - fix_shift);
          const bool round_at_end = (MODE != SLICE_LEVELS) && raw && (d == 2 || w + 8 >= fix_shift);
          if (MODE == SLICE_LEVELS) fresh = true;
          for (int c = 0; c < nch; ++c, ++chunk) {
            const int slot = chunk & 1;
            const bool level_end = (c == nch - 1);
            const bool out = (MODE == SLICE_LEVELS) ? level_end : (level_end && d == 2);
            const bool rnd = level_end && round_at_end;
            if (!mbar_wait(&accf_bar[slot], static_cast<uint32_t>(chunk >> 1) & 1u, wc)) { ok = false; break; }
            tc_fence_after();
#pragma unroll 1
            for (int cg = 0; cg < C_::COLS_PER_THREAD / 16; ++cg) {
              uint32_t r[16], lo[16], hi[16];
              const uint32_t tacc = tmem_base + t_lane + static_cast<uint32_t>(slot * BN + col_off + cg * 16);
              if (!fresh) {
                tmem_ld16x3_sync(tacc, txlo + cg * 16, txhi + cg * 16, r, lo, hi);
              } else {
                tmem_ld16_sync(tacc, r);
#pragma unroll
                for (int v = 0; v < 16; ++v) lo[v] = hi[v] = 0u;
              }
#pragma unroll
              for (int v = 0; v < 16; ++v) {
                const int64_t a = static_cast<int64_t>(__float2int_rz(__uint_as_float(r[v])));
                int64_t X = static_cast<int64_t>((static_cast<uint64_t>(hi[v]) << 32) | lo[v]) + (a << lsh);
                if (rnd) X = (X + (1ll << (fix_shift - 1))) >> fix_shift;
                lo[v] = static_cast<uint32_t>(static_cast<uint64_t>(X));
                hi[v] = static_cast<uint32_t>(static_cast<uint64_t>(X) >> 32);
              }
              if (!out) {
                tmem_st16(txlo + cg * 16, lo);
                tmem_st16(txhi + cg * 16, hi);
              } else if (row_ok) {
                // fully unrolled: lo and hi stay in registers (a partial unroll
                // would index them at run time and move them to local memory)
#pragma unroll
                for (int v = 0; v < 16; ++v) {
                  const int64_t col = col0 + cg * 16 + v;
                  if (col < n) {
                    const int64_t X = static_cast<int64_t>((static_cast<uint64_t>(hi[v]) << 32) | lo[v]);
                    if (MODE == SLICE_LEVELS) {
                      P.levels[(static_cast<int64_t>(d - 2) * P.m + row) * n + col] = X;
                    } else {
                      const int32_t Fj = __ldg(P.F + col);
                      double o;
                      if (Ei == EXP_NONFINITE || Fj == EXP_NONFINITE)
                        o = __longlong_as_double(0x7FF8000000000000ll);
                      else
                        o = scale_pow2(__ll2double_rn(X), Ei + Fj - 8 * (s + 1) + fix_shift);
                      crow[col] = o;
                    }
                  }
                }
              }
            }
            if (!out) tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
          if constexpr (CG >= 2)
            mbar_arrive_remote(slot ? acce_remote1 : acce_remote0);
          else
            mbar_arrive(&acce_bar[slot]);
        }
            fresh = false;
          }
        }
      }
    }
    if constexpr (MODE == SLICE_CRT) {
      // the last tile's rebuild
      if (ok)
        while (pend_t >= 0) crt_step();
    }
  }

  tc_fence_before();
  if constexpr (CG >= 2)
    cluster_sync_all();   // the leader's MMAs into this CTA's TMEM and all remote arrivals are done
  else
    __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    if constexpr (CG >= 2)
      tmem_dealloc_pair(tmem_base, C_::TMEM_COLS);
    else
      tmem_dealloc(tmem_base, C_::TMEM_COLS);
  }
}

template <int BN, int MODE, int CG>
static cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(slice_gemm_kernel<BN, MODE, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              Cfg<BN, MODE, CG>::SMEM_BYTES);
}

template <int BN, int MODE, int CG>
static cudaError_t launch_t(const CUtensorMap* tmA, const CUtensorMap* tmB, const SliceGemmArgs& a, int grid,
                            cudaStream_t st) {
  using C_ = Cfg<BN, MODE, CG>;
  if (CG == 1) {
    slice_gemm_kernel<BN, MODE, 1><<<grid, C_::NUM_THREADS, C_::SMEM_BYTES, st>>>(*tmA, *tmB, a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(grid));
  cfg.blockDim = dim3(C_::NUM_THREADS);
  cfg.dynamicSmemBytes = C_::SMEM_BYTES;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CG;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, slice_gemm_kernel<BN, MODE, CG>, *tmA, *tmB, a);
}

// Largest number of co-resident clusters of CG CTAs (CG = 2: CTA pairs; 4:
// clusters of two pairs) of the kernel for (BN, MODE).
template <int BN, int MODE, int CG = 2>
static int max_pairs_t() {
  using C_ = Cfg<BN, MODE, CG>;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CG);
  cfg.blockDim = dim3(C_::NUM_THREADS);
  cfg.dynamicSmemBytes = C_::SMEM_BYTES;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CG;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, slice_gemm_kernel<BN, MODE, CG>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// Per-translation-unit entry points (slice_gemm_fold.cu, slice_gemm_carry.cu).
cudaError_t slice_launch_fold(int mode, int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB,
                              const SliceGemmArgs& a, int grid, cudaStream_t st);
cudaError_t slice_prepare_fold();
int slice_max_pairs_fold(int mode);
cudaError_t slice_launch_carry(int mode, int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB,
                               const SliceGemmArgs& a, int grid, cudaStream_t st);
cudaError_t slice_prepare_carry();
int slice_max_clusters4_carry();
cudaError_t slice_launch_crt(int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB, const SliceGemmArgs& a,
                             int grid, cudaStream_t st);
cudaError_t slice_prepare_crt();
int slice_max_pairs_crt();

}  // namespace mmdev
