// slice_gemm_carry.cu -- instances of the slice GEMM for FP64-accuracy with the
// byte-carry recombination, s <= 5 (SLICE_FP64EMU_CARRY) and s = 6, 7
// (SLICE_FP64EMU_CARRY7), on tiles wider than 128 columns.
#include "slice_gemm_kernel.cuh"

namespace mmdev {

namespace {

template <int BN, int CG>
cudaError_t launch_bn(int mode, const CUtensorMap* tmA, const CUtensorMap* tmB, const SliceGemmArgs& a, int grid,
                      cudaStream_t st) {
  if (mode == SLICE_FP64EMU_CARRY) return launch_t<BN, SLICE_FP64EMU_CARRY, CG>(tmA, tmB, a, grid, st);
  if (mode == SLICE_FP64EMU_CARRY7) return launch_t<BN, SLICE_FP64EMU_CARRY7, CG>(tmA, tmB, a, grid, st);
  return cudaErrorInvalidValue;
}

template <int BN>
cudaError_t prepare_bn() {
  cudaError_t e;
  if ((e = set_smem_attr<BN, SLICE_FP64EMU_CARRY, 1>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<BN, SLICE_FP64EMU_CARRY, 2>()) != cudaSuccess) return e;
  if ((e = set_smem_attr<BN, SLICE_FP64EMU_CARRY7, 1>()) != cudaSuccess) return e;
  return set_smem_attr<BN, SLICE_FP64EMU_CARRY7, 2>();
}

// 256-wide tiles also on clusters of two CTA pairs (A multicast)
cudaError_t prepare_clusters4() {
  cudaError_t e;
  if ((e = set_smem_attr<256, SLICE_FP64EMU_CARRY, 4>()) != cudaSuccess) return e;
  return set_smem_attr<256, SLICE_FP64EMU_CARRY7, 4>();
}

}  // namespace

cudaError_t slice_launch_carry(int mode, int bn, int cg, const CUtensorMap* tmA, const CUtensorMap* tmB,
                               const SliceGemmArgs& a, int grid, cudaStream_t st) {
  switch (cg == 4 ? bn * 8 + 4 : bn * 4 + cg) {
    case 192 * 4 + 1: return launch_bn<192, 1>(mode, tmA, tmB, a, grid, st);
    case 192 * 4 + 2: return launch_bn<192, 2>(mode, tmA, tmB, a, grid, st);
    case 240 * 4 + 1: return launch_bn<240, 1>(mode, tmA, tmB, a, grid, st);
    case 240 * 4 + 2: return launch_bn<240, 2>(mode, tmA, tmB, a, grid, st);
    case 256 * 4 + 1: return launch_bn<256, 1>(mode, tmA, tmB, a, grid, st);
    case 256 * 4 + 2: return launch_bn<256, 2>(mode, tmA, tmB, a, grid, st);
    case 256 * 8 + 4: return launch_bn<256, 4>(mode, tmA, tmB, a, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t slice_prepare_carry() {
  cudaError_t e;
  if ((e = prepare_bn<192>()) != cudaSuccess) return e;
  if ((e = prepare_bn<240>()) != cudaSuccess) return e;
  if ((e = prepare_bn<256>()) != cudaSuccess) return e;
  return prepare_clusters4();
}

int slice_max_clusters4_carry() { return max_pairs_t<256, SLICE_FP64EMU_CARRY, 4>(); }

}  // namespace mmdev
