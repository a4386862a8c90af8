// Per-global-node kernels of the GB300 NUMA hot path (sm_103a):
//   prim_kernel   : the primitive fields of a state, which the element
//                   kernels build their fluxes from (FP64: the flux
//                   components themselves; FP32 and pairs: U, u, theta, p'),
//                   optionally copying the state in the same pass;
//   update_kernel : deterministic direct stiffness summation over a
//                   precomputed inverse map (fixed order, no atomics), inverse
//                   mass matrix, sources, wall condition, the SSP-RK3 stage
//                   combination and the primitive fields of the new state;
//                   on CG boxes the element nodes of each global node come
//                   from the structured numbering instead of the map;
// and the launch entry points of all kernels (the element kernels are
// compiled per precision in volume_fp64.cu, volume_fp32.cu, volume_pairs.cu).
#include "kernels_common.cuh"

namespace numa {

namespace {

__global__ void __launch_bounds__(256) prim_kernel(PrimArgs a) {
  const long long I = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= a.Ng) return;
  const long long Ng = a.Ng;
  const double q0 = a.q[I], q1 = a.q[Ng + I], q2 = a.q[2 * Ng + I], q3 = a.q[3 * Ng + I], q4 = a.q[4 * Ng + I];
  if (a.qcopy) {  // (q and qcopy may be the same array: each thread rewrites its own node)
    a.qcopy[I] = q0;
    a.qcopy[Ng + I] = q1;
    a.qcopy[2 * Ng + I] = q2;
    a.qcopy[3 * Ng + I] = q3;
    a.qcopy[4 * Ng + I] = q4;
  }
  if (a.precision == NUMA_FP32_MIXED) write_prim<true>(a, I, q0, q1, q2, q3, q4);
  else write_prim<false>(a, I, q0, q1, q2, q3, q4);
}

template <int MODE, typename RT>
void launch_update_m(const UpdateArgs& a, unsigned nb, int nt, cudaStream_t s) {
  if (a.gvec) update_kernel<MODE, true, RT><<<nb, nt, 0, s>>>(a);
  else if (a.box_N) update_kernel<MODE, false, RT, true><<<nb, nt, 0, s>>>(a);
  else update_kernel<MODE, false, RT><<<nb, nt, 0, s>>>(a);
}

}  // namespace

cudaError_t launch_prim(const PrimArgs& a, cudaStream_t s) {
  if (a.Ng == 0) return cudaSuccess;
  const int nt = 256;
  prim_kernel<<<(unsigned)((a.Ng + nt - 1) / nt), nt, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_volume(int N, int precision, const VolumeArgs& a, cudaStream_t s) {
  if (precision == NUMA_FP64_PAIRS) return launch_volume_pairs(N, a.affine != 0, a, s);
  if (precision == NUMA_FP32_MIXED) return launch_volume_fp32(N, a.affine != 0, a, s);
  return launch_volume_fp64(N, a.affine != 0, a, s);
}

cudaError_t launch_update(int precision, const UpdateArgs& a, cudaStream_t s) {
  if (a.iend <= a.ibeg) return cudaSuccess;
  if (a.ibeg % kDssBlock) return cudaErrorInvalidValue;
  const int nt = kDssBlock;  // the kernel's block size: one block per DSS-order block
  const unsigned nb = (unsigned)((a.iend - a.ibeg + nt - 1) / nt);
  const bool f32 = precision == NUMA_FP32_MIXED;
  if (a.mode == 0) {
    if (f32) launch_update_m<0, float>(a, nb, nt, s);
    else launch_update_m<0, double>(a, nb, nt, s);
  } else if (a.mode == 3) {
    if (f32) launch_update_m<3, float>(a, nb, nt, s);
    else launch_update_m<3, double>(a, nb, nt, s);
  } else if (a.mode == 4) {
    if (a.first_stage) {
      if (f32) launch_update_m<5, float>(a, nb, nt, s);
      else launch_update_m<5, double>(a, nb, nt, s);
    } else {
      if (f32) launch_update_m<4, float>(a, nb, nt, s);
      else launch_update_m<4, double>(a, nb, nt, s);
    }
  } else if (a.first_stage) {
    if (f32) launch_update_m<2, float>(a, nb, nt, s);
    else launch_update_m<2, double>(a, nb, nt, s);
  } else {
    if (f32) launch_update_m<1, float>(a, nb, nt, s);
    else launch_update_m<1, double>(a, nb, nt, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_volume_ragged(int N, int precision, bool affine, const MemberDesc* d, const RaggedGroup* g,
                                 cudaStream_t s) {
  if (precision == NUMA_FP64_PAIRS) return launch_volume_ragged_pairs(N, affine, d, g, s);
  if (precision == NUMA_FP32_MIXED) return launch_volume_ragged_fp32(N, affine, d, g, s);
  return launch_volume_ragged_fp64(N, affine, d, g, s);
}

cudaError_t launch_update_ragged(int precision, bool shell, int stage, const MemberDesc* d, const RaggedGroup* g,
                                 cudaStream_t s) {
  const int grid = 16 * sm_count();  // persistent: blocks of kDssBlock threads loop over the groups' node blocks
  const bool f32 = precision == NUMA_FP32_MIXED;
  auto go = [&](auto mode_tag) {
    constexpr int M = decltype(mode_tag)::value;
    if (shell) {
      if (f32) update_ragged<M, true, float><<<grid, kDssBlock, 0, s>>>(d, g, stage);
      else update_ragged<M, true, double><<<grid, kDssBlock, 0, s>>>(d, g, stage);
    } else {
      if (f32) update_ragged<M, false, float><<<grid, kDssBlock, 0, s>>>(d, g, stage);
      else update_ragged<M, false, double><<<grid, kDssBlock, 0, s>>>(d, g, stage);
    }
  };
  // stage 0 of SSP-RK3 is the first stage (a = 0, b = 1)
  if (stage == 0) go(std::integral_constant<int, 2>());
  else go(std::integral_constant<int, 1>());
  return cudaGetLastError();
}

}  // namespace numa
