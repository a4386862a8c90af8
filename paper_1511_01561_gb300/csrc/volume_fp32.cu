// Element kernels (Eq. 4 / Eq. 5) in the FP32 form (line organisation, D in
// constant memory): per-node and affine-element metric forms, single-mesh
// and ragged multi-member launches; the upload of the constant D table.
#include "kernels_common.cuh"

namespace numa {

cudaError_t launch_volume_fp32(int N, bool affine, const VolumeArgs& a, cudaStream_t s) {
  return affine ? launch_volume_p<float, true>(N, a, s) : launch_volume_p<float, false>(N, a, s);
}

cudaError_t launch_volume_ragged_fp32(int N, bool affine, const MemberDesc* d, const RaggedGroup* g, cudaStream_t s) {
  return affine ? launch_volume_ragged_p<float, true>(N, d, g, s) : launch_volume_ragged_p<float, false>(N, d, g, s);
}

cudaError_t upload_d32_constant(int N, const float* D, cudaStream_t s) {
  if (N < 1 || N > 8) return cudaErrorInvalidValue;
  return cudaMemcpyToSymbolAsync(c_D32, D, sizeof(float) * (N + 1) * (N + 1), sizeof(float) * 81 * N,
                                 cudaMemcpyHostToDevice, s);
}

}  // namespace numa
