// slice_gemm_fold.cu -- instances of the slice GEMM for FP64-accuracy with the
// int64 fold recombination (SLICE_FP64EMU) and for the level-product output
// (SLICE_LEVELS), on every tile width and CTA grouping.
#include "slice_gemm_kernel.cuh"

namespace mmdev {

namespace {

template <int BN, int CG>
cudaError_t launch_bn(int mode, const CUtensorMap* tmA, const CUtensorMap* tmB, const SliceGemmArgs& a, int grid,
                      cudaStream_t st) {
  if (mode == SLICE_FP64EMU) return launch_t<BN, SLICE_FP64EMU, CG>(tmA, tmB, a, grid, st);
  if (mode == SLICE_LEVELS) return launch_t<BN, SLICE_LEVELS, CG>(tmA, tmB, a, grid, st);
  return cudaErrorInvalidValue;
}

template <int BN>
cudaError_t prepare_bn() {
  cudaError_t e;
  if ((e = set_smem_attr<BN, SLICE_FP64EMU, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<BN, SLICE_FP64EMU, 2>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<BN, SLICE_LEVELS, 1>()) != cudaSuccess) return e;
  return set_smem_attr<BN, SLICE_LEVELS, 2>();
}

}  // namespace

cudaError_t slice_launch_fold(int mode, int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB,
                              const SliceGemmArgs& a, int grid, cudaStream_t st) {
  switch (bn * 4 + cg) {
    case 128 * 4 + 1: return launch_bn<128, 1>(mode, tmA, tmB, a, grid, st);
    case 128 * 4 + 2: return launch_bn<128, 2>(mode, tmA, tmB, a, grid, st);
    case 192 * 4 + 1: return launch_bn<192, 1>(mode, tmA, tmB, a, grid, st);
    case 192 * 4 + 2: return launch_bn<192, 2>(mode, tmA, tmB, a, grid, st);
    case 240 * 4 + 1: return launch_bn<240, 1>(mode, tmA, tmB, a, grid, st);
    case 240 * 4 + 2: return launch_bn<240, 2>(mode, tmA, tmB, a, grid, st);
    case 256 * 4 + 1: return launch_bn<256, 1>(mode, tmA, tmB, a, grid, st);
    case 256 * 4 + 2: return launch_bn<256, 2>(mode, tmA, tmB, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t slice_prepare_fold() {
  cudaError_t e;
  if ((e = prepare_bn<128>()) != cudaSuccess) return e;
  if ((e = prepare_bn<192>()) != cudaSuccess) return e;
  if ((e = prepare_bn<240>()) != cudaSuccess) return e;
  return prepare_bn<256>();
}

int slice_max_pairs_fold(int mode) {
  if (mode == SLICE_LEVELS) return max_pairs_t<256, SLICE_LEVELS>();
  return max_pairs_t<256, SLICE_FP64EMU>();
}

}  // namespace mmdev
