// Element kernels (Eq. 4 / Eq. 5) of the FP64-pairs mode: FP64 accuracy from
// (hi, lo) float pairs on the FP32 units; per-node and affine-element forms,
// single-mesh and ragged launches.
#include "kernels_common.cuh"

namespace numa {

cudaError_t launch_volume_pairs(int N, bool affine, const VolumeArgs& a, cudaStream_t s) {
  return affine ? launch_volume_p<Pairs, true>(N, a, s) : launch_volume_p<Pairs, false>(N, a, s);
}

cudaError_t launch_volume_ragged_pairs(int N, bool affine, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s) {
  return affine ? launch_volume_ragged_p<Pairs, true>(N, d, g, s) : launch_volume_ragged_p<Pairs, false>(N, d, g, s);
}

}  // namespace numa
