// Element kernel (Eq. 4 / Eq. 5) of the FP64-pairs mode: FP64 accuracy from
// (hi, lo) float pairs on the FP32 units; single-mesh and ragged launches.
#include "kernels_common.cuh"

namespace numa {

cudaError_t launch_volume_pairs(int N, bool affine, const VolumeArgs& a, cudaStream_t s) {
  (void)affine;  // the pairs mode has only the per-node form
  return launch_volume_p<Pairs, false>(N, a, s);
}

cudaError_t launch_volume_ragged_pairs(int N, bool affine, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s) {
  (void)affine;
  return launch_volume_ragged_p<Pairs, false>(N, d, g, s);
}

}  // namespace numa
