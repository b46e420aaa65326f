// slice_gemm.cu -- FP32-accuracy instances of the slice GEMM and the dispatch
// over modes, tile widths and CTA groupings (the kernel itself is in
// slice_gemm_kernel.cuh; the FP64-accuracy instances are in
// slice_gemm_fold.cu and slice_gemm_carry.cu).
#include "slice_gemm_kernel.cuh"

using namespace mmdev;

cudaError_t slice_gemm_prepare() {
  cudaError_t e;
  if ((e = set_smem_attr<256, SLICE_FP32EMU, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<128, SLICE_FP32EMU, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<256, SLICE_FP32EMU, 2>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<256, SLICE_FP32EMU, 4>()) != cudaSuccess) return e;
  if ((e = slice_prepare_fold()) != cudaSuccess) return e;
  if ((e = slice_prepare_crt()) != cudaSuccess) return e;
  return slice_prepare_carry();
}

int slice_gemm_max_pairs(int mode) {
  if (mode == SLICE_FP32EMU) return max_pairs_t<256, SLICE_FP32EMU>();
  if (mode == SLICE_CRT) return slice_max_pairs_crt();
  return slice_max_pairs_fold(mode == SLICE_LEVELS ? SLICE_LEVELS : SLICE_FP64EMU);
}

int slice_gemm_max_clusters4(int mode) {
  if (mode == SLICE_FP32EMU) return max_pairs_t<256, SLICE_FP32EMU, 4>();
  return slice_max_clusters4_carry();
}

bool slice_gemm_tile_ok(int mode, int bn, int cg) {
  if (cg == 4)   // clusters of two CTA pairs: 256-wide tiles, FP32-accuracy or the byte-carry modes
    return bn == 256 && (mode == SLICE_FP32EMU || mode == SLICE_FP64EMU_CARRY || mode == SLICE_FP64EMU_CARRY7);
  if (cg != 1 && cg != 2) return false;
  if (mode == SLICE_FP32EMU) return bn == 256 || (bn == 128 && cg == 1);
  if (mode == SLICE_CRT) return bn == 128 || bn == 256;
  return bn == 128 || bn == 192 || bn == 240 || bn == 256;
}

// FP32-accuracy: bn 256 (cg 1 or 2) or 128 (cg 1). FP64-accuracy and level
// output: bn 128 keeps the int64 total in TMEM (grouped launches of small
// products); bn 192, 240, 256 keep int32 level sums in registers, with the
// int64 total in C (fold) or the byte-carry recombination (carry modes; on
// bn 128 a carry mode runs the fold kernel, same results). cg = 2: CTA pairs
// on 256-row tiles (grid = 2 x pairs).
cudaError_t launch_slice_gemm(int mode, int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB,
                              const SliceGemmArgs& a, int grid, cudaStream_t st) {
  if (grid <= 0) return cudaSuccess;
  if (!slice_gemm_tile_ok(mode, bn, cg)) return cudaErrorInvalidValue;
  if (mode == SLICE_FP32EMU) {
    if (cg == 4) return launch_t<256, SLICE_FP32EMU, 4>(tmA, tmB, a, grid, st);
    if (cg == 2) return launch_t<256, SLICE_FP32EMU, 2>(tmA, tmB, a, grid, st);
    if (bn == 256) return launch_t<256, SLICE_FP32EMU, 1>(tmA, tmB, a, grid, st);
    return launch_t<128, SLICE_FP32EMU, 1>(tmA, tmB, a, grid, st);
  }
  if (mode == SLICE_CRT) return slice_launch_crt(bn, cg, tmA, tmB, a, grid, st);
  if (mode == SLICE_FP64EMU_CARRY || mode == SLICE_FP64EMU_CARRY7) {
    if (bn != 128) return slice_launch_carry(mode, bn, cg, tmA, tmB, a, grid, st);
    mode = SLICE_FP64EMU;
  }
  if (cg == 4) return cudaErrorInvalidValue;
  return slice_launch_fold(mode, bn, cg, tmA, tmB, a, grid, st);
}
