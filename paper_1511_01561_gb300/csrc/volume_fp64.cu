// Element kernels (Eq. 4 / Eq. 5) in FP64: the per-node, affine-element and
// rectilinear forms, single-mesh and ragged multi-member launches.
#include "kernels_common.cuh"

namespace numa {

cudaError_t launch_volume_fp64(int N, bool affine, const VolumeArgs& a, cudaStream_t s) {
  return affine ? launch_volume_p<double, true>(N, a, s) : launch_volume_p<double, false>(N, a, s);
}

cudaError_t launch_volume_ragged_fp64(int N, bool affine, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s) {
  return affine ? launch_volume_ragged_p<double, true>(N, d, g, s) : launch_volume_ragged_p<double, false>(N, d, g, s);
}

}  // namespace numa
