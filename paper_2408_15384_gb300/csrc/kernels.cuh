// kernels.cuh -- launchers shared between the kernel files and the C ABI.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

// Scale exponent marking a row/column that holds Inf or NaN.
#define EXP_NONFINITE (-1000000)

static inline uint64_t splitmix_mix_host(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ------------------------------------------------- automatic slice count
// FP64-accuracy slice count from the operands' spread. For each row i of A
// (column j of B) the scan forms alpha_i = mean_k |a_ik| / 2^E_i (beta_j
// likewise). One term a_ik b_kj of the emulated product carries an error of
// standard deviation at most SLICE_KAPPA * 2^(E_i + F_j - 8s): the rounding of
// the entries to their digit grids and the dropped level s+2 (s-1 digit pairs
// below 2^-16 of the level above) with digits independent and uniform. Over k
// terms it grows like sqrt(k), and the largest of up to 2^30 outputs stays
// within SLICE_ZMAX standard deviations; the componentwise bound is about
// 4k 2^-53 * k alpha_i beta_j 2^(E_i+F_j). The count is the smallest s in
// 3..7 with
//   SLICE_KAPPA * SLICE_ZMAX * 2^(53-8s) <= SLICE_THETA * 4 * k * sqrt(k) * alpha_min * beta_min,
// so the error stays within SLICE_THETA of the bound; SLICE_S_PLAIN (8) when
// none qualifies: the product then runs through the plain FP64 kernel.
constexpr int SLICE_S_MIN = 3, SLICE_S_MAX = 7, SLICE_S_PLAIN = 8;
#define SLICE_KAPPA 0.3
#define SLICE_ZMAX 6.5
#define SLICE_THETA 0.5

// The decision record of one product in device memory. The smallest alpha of
// A's rows and beta of B's columns are kept as their distance below +inf,
// 0x7F800000 minus the float bits (merged with atomicMax; zero, the initial
// value, means no row or column constrains the count); s is the slice count,
// written by the splitting kernels and read by the slice GEMM and the
// plain-FP64 fallback.
// With the modular form allowed, s is SLICE_CRT_BASE + N for a product that
// takes it (N moduli) and bits its bit count b.
struct SliceDecision {
  uint32_t amin_room;
  uint32_t bmin_room;
  int32_t s;
  int32_t bits;
};

__host__ __device__ inline float spread_from_room(uint32_t room) {
  union { uint32_t u; float f; } v;
  v.u = room >= 0x7F800000u ? 0u : 0x7F800000u - room;
  return v.f;
}

// The slice count for inner dimension k and the smallest spreads (double
// arithmetic, k * sqrt(k) with the correctly rounded square root).
__host__ __device__ inline int slice_count_rule(int64_t k, float amin, float bmin) {
  const double rhs = SLICE_THETA * 4.0 * static_cast<double>(k) * sqrt(static_cast<double>(k)) *
                     static_cast<double>(amin) * static_cast<double>(bmin);
  double pw = 536870912.0;   // 2^(53 - 8*3)
  for (int s = SLICE_S_MIN; s <= SLICE_S_MAX; ++s, pw *= 0.00390625) {
    if (SLICE_KAPPA * SLICE_ZMAX * pw <= rhs) return s;
  }
  return SLICE_S_PLAIN;
}

// The smallest count the rule can give for inner dimension k (the largest
// spread any row or column can have is below 1/2).
inline int slice_count_floor(int64_t k) { return slice_count_rule(k, 0.5f, 0.5f); }

// ------------------------------------------- modular (CRT) FP64-accuracy form
// Ozaki scheme II (Ozaki, Uchino, Imamura 2025) on bfloat16 tensor cores: the
// scaled integers R = round-half-even(a 2^(b - E_i)), |R| <= 2^(b-1) (E_i as
// for the digit form), are reduced modulo N pairwise coprime moduli m_l <= 256
// (centred residues in [-128, 127], exact in bfloat16); one residue product a
// modulus (each term at most 2^14, so the K-chunks of the digit form's level 2
// hold exact f32 sums); every product reduced modulo its own modulus; the
// integer product rebuilt by the Chinese remainder theorem, exact while
// k 2^(2b-1) < M_N = m_1 ... m_N, and rounded to double once. The moduli are
// the largest pairwise coprime integers <= 256, taken from 256 down.
constexpr int CRT_N_MAX = 14;
constexpr int CRT_B_MIN = 24, CRT_B_MAX = 53;
// decision code of a product that takes the modular form: SLICE_CRT_BASE + N
constexpr int SLICE_CRT_BASE = 16;
// rounding-only error constant: sqrt(2/12 * 1/4) = 0.204, rounded up
#define CRT_KAPPA 0.21

__host__ __device__ constexpr int crt_modulus(int l) {
  return l == 0 ? 256 : l == 1 ? 255 : l == 2 ? 253 : l == 3 ? 251 : l == 4 ? 247 : l == 5 ? 241 : l == 6 ? 239
       : l == 7 ? 233 : l == 8 ? 229 : l == 9 ? 227 : l == 10 ? 223 : l == 11 ? 217 : l == 12 ? 211 : 199;
}

// Whether k 2^(2b-1) < M_N (every k-term sum of b-bit integers lies strictly
// inside (-M_N/2, M_N/2)), in exact 128-bit integer arithmetic.
__host__ __device__ inline bool crt_fits(int64_t k, int b, int N) {
  unsigned __int128 M = 1;
  for (int l = 0; l < N; ++l) M *= static_cast<unsigned>(crt_modulus(l));
  const int sh = 2 * b - 1;
  int kbits = 0;
  for (uint64_t t = static_cast<uint64_t>(k); t; t >>= 1) ++kbits;
  if (kbits + sh > 127) return false;
  return (static_cast<unsigned __int128>(static_cast<uint64_t>(k)) << sh) < M;
}

// The modular form's parameters for inner dimension k and the smallest spreads:
// b0 = the smallest b in CRT_B_MIN..CRT_B_MAX with
//   CRT_KAPPA * SLICE_ZMAX * 2^(53-b) <= SLICE_THETA * 4 * k * sqrt(k) * amin * bmin
// (the digit form's estimate with only the rounding term), N = the fewest
// moduli that hold it, b = the most bits those moduli hold (at most
// CRT_B_MAX). Returns N (0: the modular form does not fit) and *bits = b.
__host__ __device__ inline int crt_rule(int64_t k, float amin, float bmin, int* bits) {
  const double rhs = SLICE_THETA * 4.0 * static_cast<double>(k) * sqrt(static_cast<double>(k)) *
                     static_cast<double>(amin) * static_cast<double>(bmin);
  double pw = 536870912.0;   // 2^(53 - CRT_B_MIN)
  int b0 = 0;
  for (int b = CRT_B_MIN; b <= CRT_B_MAX; ++b, pw *= 0.5) {
    if (CRT_KAPPA * SLICE_ZMAX * pw <= rhs) {
      b0 = b;
      break;
    }
  }
  if (b0 == 0) return 0;
  int N = 0;
  for (int c = 1; c <= CRT_N_MAX; ++c) {
    if (crt_fits(k, b0, c)) {
      N = c;
      break;
    }
  }
  if (N == 0) return 0;
  int b = b0;
  while (b < CRT_B_MAX && crt_fits(k, b + 1, N)) ++b;
  *bits = b;
  return N;
}

// The automatic FP64-accuracy decision: SLICE_CRT_BASE + N (modular form, *bits
// = b) when it is allowed and fits, else the digit count (SLICE_S_PLAIN: the
// plain FP64 kernel).
__host__ __device__ inline int fp64_decision(int64_t k, float amin, float bmin, bool modular, int* bits) {
  *bits = 0;
  if (modular) {
    const int N = crt_rule(k, amin, bmin, bits);
    if (N > 0) return SLICE_CRT_BASE + N;
  }
  return slice_count_rule(k, amin, bmin);
}

// FP32-accuracy slice count: three bfloat16 slices (the six products with
// p + q <= 2) below k = 512, two slices (the three with p + q <= 1) from
// there on: the left-out products are at most 3.03 * 2^-16 |a b| a term, half
// of the bound 4k 2^-24 |A||B| already at k = 388.
constexpr int64_t FP32_TWO_SLICE_K = 512;
inline int fp32_slice_count(int64_t k) { return k >= FP32_TWO_SLICE_K ? 2 : 3; }

// ---------------------------------------------------------------- split.cu
// Row maxima of |A| and column maxima of |B| (bit patterns); one fused launch
// when both operands are non-empty, else one per operand. *nlaunch, if given,
// receives the kernel launches made.
// With dec != nullptr the scan also forms the spreads: each row's alpha is
// merged into dec->amin_room; the columns' partial sums go to colpart
// (launch_absmax_parts(k) records of n columns each), and a short second
// launch sums them in a fixed order and merges each column's beta into
// dec->bmin_room. The caller zeroes *dec beforehand.
cudaError_t launch_absmax(const double* A, int64_t m, int64_t k, int64_t lda, const double* B, int64_t n,
                          int64_t ldb, uint64_t* rowmax, uint64_t* colmax, cudaStream_t st, int* nlaunch = nullptr,
                          SliceDecision* dec = nullptr, uint2* colpart = nullptr);
// Partial-sum records per column of B for inner dimension k.
int64_t launch_absmax_parts(int64_t k);
// Slices of rows [0, m) of A into planes of plane_rows rows (0: m), so a
// panel of a larger matrix can be sliced into its place. With dec != nullptr
// (FP64-accuracy) the slice count is slice_count_rule(k, amin, bmin) of the
// scan's spreads instead of s; the first block records it in dec->s, and no
// slices are written when it is SLICE_S_PLAIN.
// mode: 0 FP64-accuracy digits as bfloat16 (uint16 planes), 1 FP32-accuracy
// bfloat16 slices, 2 FP64-accuracy digits as signed bytes (int8 planes; the
// INT8 form, scale exponent one larger, automatic count from halved spreads),
// 3 automatic FP64-accuracy with the modular form allowed: the residues (N
// planes, code SLICE_CRT_BASE + N) or the digits the decision record holds,
// written beforehand by launch_decide_fp64.
cudaError_t launch_slice_rows(int mode, const double* A, int64_t m, int64_t k, int64_t lda, const uint64_t* rowmax,
                              int s, int64_t kp, void* slices, int32_t* E, uint32_t* err, cudaStream_t st,
                              int64_t plane_rows = 0, SliceDecision* dec = nullptr);
cudaError_t launch_slice_cols(int mode, const double* B, int64_t k, int64_t n, int64_t ldb, const uint64_t* colmax,
                              int s, int64_t kp, void* slices, int32_t* F, uint32_t* err, cudaStream_t st,
                              SliceDecision* dec = nullptr);
// The automatic FP64-accuracy decision of one product with the modular form
// allowed (fp64_decision on the record's spreads): dec->s and dec->bits.
cudaError_t launch_decide_fp64(SliceDecision* dec, int64_t k, cudaStream_t st);
// The residue bytes of a modular-form product ([N] planes of rplane bytes,
// blocks of 8 columns blk bytes apart, 8-byte row records) to a dense
// [N][m][n] byte array (diagnostics).
cudaError_t launch_crt_residues_out(const uint8_t* res, int64_t rplane, int64_t blk, int N, int64_t m, int64_t n,
                                   uint8_t* out, cudaStream_t st);
cudaError_t launch_fill_uniform(double* X, int64_t rows, int64_t cols, int64_t ld, uint64_t seed, uint64_t stream_id,
                                int scale_mode, uint64_t exp_stream_id, cudaStream_t st);

// Grouped splitting: per-problem record of one emulated product's operands and
// workspace.
struct GroupedSplit {
  int64_t m, n, k, lda, ldb, kp;
  const double* A;
  const double* B;
  int s;                  // slices (FP64-accuracy, when dec is null) or 3
  int crt;                // 1: the modular form allowed (splitting mode 3)
  uint64_t* rowmax;
  uint64_t* colmax;
  int32_t* E;
  int32_t* F;
  uint16_t* slA;
  uint16_t* slB;
  SliceDecision* dec;     // automatic slice count (FP64-accuracy), else null
  uint2* colpart;         // column partial sums of the spreads (with dec)
  uint32_t* perr;         // the problem's own error word (non-finite input), else null: the launch's
};
// Virtual block offsets: off[kind][p] = first block of problem p for kernel
// kind (0 row max, 1 column max, 2 slice rows, 3 slice cols, 4 column spreads);
// off[kind][count] = total. Arrays of count+1 int64 in device memory.
struct GroupedSplitArgs {
  const GroupedSplit* probs;
  const int64_t* off[5];
  const int* count_dev;
  uint32_t* err;
};
// mode01: 0 FP64-accuracy digits, 1 FP32-accuracy slices, 3 FP64-accuracy with
// the modular form allowed (automatic problems only: a decision kernel
// between the scan and the slicing records each problem's form). grid:
// persistent blocks.
cudaError_t launch_grouped_split(int mode01, const GroupedSplitArgs& a, int grid, cudaStream_t st);

// ----------------------------------------------------------- slice_gemm.cu
// Epilogue kinds of the slice GEMM.
// SLICE_FP64EMU_CARRY (s <= 5) and SLICE_FP64EMU_CARRY7 (s = 6, 7):
// FP64-accuracy with the byte-carry recombination, for products
// slice_fp64_carry_ok accepts (same results as SLICE_FP64EMU).
// SLICE_CRT: the modular form (residue products, CRT rebuild in the epilogue).
enum SliceMode {
  SLICE_FP32EMU = 0,
  SLICE_FP64EMU = 1,
  SLICE_LEVELS = 2,
  SLICE_FP64EMU_CARRY = 3,
  SLICE_FP64EMU_CARRY7 = 4,
  SLICE_CRT = 5
};

// Chunks per int32 level-sum segment (SLICE_SEG_CHUNKS * 2^24 < 2^31).
constexpr int SLICE_SEG_CHUNKS = 120;

// Whether an FP64-accuracy product of inner dimension k with s slices and
// fixed-point shift fix_shift can take the byte-carry epilogue: s <= 7, every
// level within one int32 segment (the top level d = s + 1 has the shortest
// chunks, 16 / s K blocks), and the fixed point at or below the last level's
// weight 8(s-1).
inline bool slice_fp64_carry_ok(int s, int64_t k, int fix_shift) {
  if (s < 1 || s > 7) return false;
  const int64_t nkb = (k + 63) / 64;
  const int kc = (16 / s) < 1 ? 1 : 16 / s;
  return (nkb + kc - 1) / kc <= SLICE_SEG_CHUNKS && fix_shift <= 8 * (s - 1);
}

// The slice GEMM mode of an FP64-accuracy product.
inline int slice_fp64_mode(int s, int64_t k, int fix_shift) {
  if (!slice_fp64_carry_ok(s, k, fix_shift)) return SLICE_FP64EMU;
  return s <= 5 ? SLICE_FP64EMU_CARRY : SLICE_FP64EMU_CARRY7;
}

// One product as the slice GEMM sees it (also the grouped problem record).
struct SliceProblem {
  int64_t m, n, k;
  int nkb;               // ceil(k / 64)
  int s;                 // FP64-accuracy slice count (when s_dev is null)
  int fix_shift;         // right shift of the int64 fixed-point total (FP64-accuracy)
  const int32_t* s_dev;  // automatic slice count in device memory, else null
  int8_t fix_tab[8];     // with s_dev: the fixed-point shift for each s <= 7
  int tiles_m, tiles_n;
  const int32_t* E;      // row scale exponents of A
  const int32_t* F;      // column scale exponents of B
  double* C;
  int64_t ldc;
  int64_t* levels;       // SLICE_LEVELS: [s][m][n] int64
  // SLICE_CRT: the products' residues as bytes; plane l at res + l * rplane;
  // within a plane, blocks of 8 columns ldr bytes apart, each block the rows'
  // 8-byte records in row order (res points at this problem's row 0)
  uint8_t* res;
  int64_t ldr, rplane;
};

// A tile of a grouped launch: problem index and tile coordinates.
struct TileRef {
  int32_t prob;
  int16_t tm, tn;
};

// The modular form's rebuild constants for N = 1 .. CRT_N_MAX moduli:
// W[N][l] = (M/m_l) ((M/m_l)^-1 mod m_l) mod M and M = M_N as four 32-bit
// words (least significant first), M/2 as two 64-bit words; the quotient
// estimate of a sum S < 2^12 M reads the window S >> wsh (below 2^32, wsh =
// bit length of M minus 20) and scales it by qscale = 2^wsh / M (a float).
// Per modulus m_l, the constants of the epilogue's reduction of an int32 sum:
// magic = floor(2^32 / m) + 1, c16 = 2^16 mod m, c31 = 2^31 mod m.
struct CrtTab {
  uint32_t W[CRT_N_MAX + 1][CRT_N_MAX][4];
  uint32_t M[CRT_N_MAX + 1][4];
  uint64_t H[CRT_N_MAX + 1][2];
  int32_t wsh[CRT_N_MAX + 1];
  float qscale[CRT_N_MAX + 1];
  uint32_t magic[CRT_N_MAX], c16[CRT_N_MAX];
  int32_t c31[CRT_N_MAX];
};

struct SliceGemmArgs {
  SliceProblem single;             // used when probs == nullptr
  const SliceProblem* probs;       // grouped: problem records (device)
  const CUtensorMap* tmaps;        // grouped: 2 per problem (A, B), device, 64-byte aligned
  const TileRef* tiles;            // grouped: tile list (device)
  const int* ntiles_dev;           // grouped: tile count (device)
  uint32_t* err;
  uint64_t timeout_ns;
  int s_lo, s_hi;                  // with s_dev: only tiles of problems with s in [s_lo, s_hi] (s_hi > 0)
  // SLICE_CRT, single products: 1 = store the residue bytes only (the rebuild
  // is a pass of its own, crt_rebuild) and split the last, partial round of
  // tiles by moduli among the walkers
  int crt_defer;
};

// bn: tile width (columns of C); cg: CTAs per tile (1, or 2 for a CTA pair on
// 256-row tiles), or 4 for CTA pairs in clusters of two on horizontally
// adjacent tiles (single products with an even tiles_n; A's tensor map box has
// 64 rows, each CTA loading half of its rows for both pairs). grid =
// persistent CTA count (a multiple of 2 when cg = 2, of 4 when cg = 4). With
// cg = 2 or 4, tiles_m counts 256-row tiles and B's tensor map box has bn/2 rows.
cudaError_t launch_slice_gemm(int mode, int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB,
                              const SliceGemmArgs& a, int grid, cudaStream_t st);
// Set the dynamic shared memory limits of every instantiation (once per device).
cudaError_t slice_gemm_prepare();
// Largest number of co-resident CTA pairs of the pair kernel for a mode.
int slice_gemm_max_pairs(int mode);
// Largest number of co-resident clusters of two CTA pairs (cg = 4: 256-wide
// tiles, A multicast between the pairs) for FP32-accuracy or the byte-carry modes.
int slice_gemm_max_clusters4(int mode);
// whether launch_slice_gemm has a kernel for (mode, tile width, CTAs per tile)
bool slice_gemm_tile_ok(int mode, int bn, int cg);
// The modular form's rebuild of P's outputs (C) from its residue bytes, after
// a slice GEMM of P launched with crt_defer; returns at once for a product
// whose decision record names the digit form.
cudaError_t slice_rebuild_crt(const SliceProblem& P, int sm_count, cudaStream_t st);

// ------------------------------------------------------------- int8_gemm.cu
// FP64-accuracy product from INT8-form digit planes on mma.sync m16n8k32 s8.
struct Int8GemmArgs {
  int64_t m, n, k, kp;       // kp: bytes between rows of a digit plane (a multiple of 16)
  const int8_t* A;           // A's digits [s][m][kp]
  int64_t plane_a;           // bytes between A's planes
  const int8_t* B;           // B's digits, transposed: [s][n][kp]
  int64_t plane_b;
  const int32_t* E;          // row scale exponents of A (INT8 form)
  const int32_t* F;          // column scale exponents of B
  double* C;
  int64_t ldc;
  int64_t* levels;           // level output [s][m][n] int64 (added to; zeroed by the caller), else null
  int s;                     // slice count when s_dev is null
  int fix_shift;             // fixed-point shift for s (when s_dev is null)
  const int32_t* s_dev;      // automatic slice count in device memory, else null
  int8_t fix_tab[8];         // with s_dev: the shift for each count
};
cudaError_t launch_int8_slice_gemm(const Int8GemmArgs& a, cudaStream_t st);

// ------------------------------------------------------------- fp64_gemm.cu
struct Fp64GemmArgs {
  int64_t m, n, k;
  const double* A;
  int64_t lda;
  const double* B;
  int64_t ldb;
  double* C;
  int64_t ldc;
  const int32_t* only_if_plain;   // if set: run only when it holds SLICE_S_PLAIN (emulated-mode fallback)
};
// kind: 1 = DFMA tiles, 2 = DMMA (mma.sync m8n8k4 f64) tiles.
cudaError_t launch_fp64_gemm(int kind, const Fp64GemmArgs& a, cudaStream_t st);
// Grouped: one persistent launch over a tile list of many problems (device
// arrays; the tile count is read from device memory).
// count_dev (the problem count in device memory) marks a launch of fallback
// guards: the grid returns at once unless some problem's guard is set.
cudaError_t launch_fp64_grouped(int kind, const Fp64GemmArgs* probs, const TileRef* tiles, const int* ntiles_dev,
                                int grid, cudaStream_t st, const int* count_dev = nullptr);
int fp64_tile_size();
cudaError_t fp64_gemm_prepare();
cudaError_t launch_zero_c(double* C, int64_t m, int64_t n, int64_t ldc, cudaStream_t st);
cudaError_t launch_peak_fp64(int kind, double* sink, int iters, int blocks, cudaStream_t st);
// a bounded wait on an mbarrier nothing arrives at (failure-detection check)
cudaError_t launch_wait_probe(uint32_t* err, uint64_t timeout_ns, int* gave_up, cudaStream_t st);
