// Kernels of the batched instances: per-instance setup and the level march, each CTA taking whole
// instances from a work queue (largest first) and running them with a one-CTA team.  A
// translation unit of its own so that the build compiles it in parallel with the other kernels;
// the device code is level_device.cuh.
#include "level_device.cuh"

namespace tsf {

__global__ void __launch_bounds__(kThreads, 2) batch_setup_kernel(BatchArgs B) {
  __shared__ Args sA;
  cta_team_init();
  for (int i = next_instance(B); i >= 0; i = next_instance(B)) {
    if (threadIdx.x == 0) {
      sA = B.inst[i];
      patch_cta_scratch(sA, B.cta[blockIdx.x]);
      team().grid = 0;
      team().abort = 0;   // the abort mirror is per instance
    }
    __syncthreads();
    const InstanceSetup &I = B.setup[i];
    instance_tables(sA, I.omega, I.gtmp, I.alpha, I.beta, I.tau, I.h, I.gamma, I.d_plus, I.d_minus);
    SetupArgs T;
    T.omega = I.omega;
    T.What = const_cast<double2 *>(sA.What);
    T.LamW = const_cast<double2 *>(sA.LamW);
    T.LamQ = const_cast<double2 *>(sA.LamQ);
    T.BhI = const_cast<double2 *>(sA.BhI);
    T.BhF = I.BhF;
    T.chirpI = const_cast<double2 *>(sA.chirpI);
    T.twL = const_cast<double2 *>(sA.twL);
    T.precond = sA.precond;
    const Smem S = smem_view(lp_max_of(sA), tw_max_of(sA));
    setup_body(sA, T, S);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kThreads, 2) batch_level_kernel(BatchArgs B, int j0, int j1) {
  __shared__ Args sA;
  cta_team_init();
  for (int i = next_instance(B); i >= 0; i = next_instance(B)) {
    if (threadIdx.x == 0) {
      sA = B.inst[i];
      patch_cta_scratch(sA, B.cta[blockIdx.x]);
      team().abort = 0;   // the abort mirror is per instance
    }
    __syncthreads();
    const Smem S = smem_view(lp_max_of(sA), tw_max_of(sA));
    march_body(sA, S, j0, j1);
    __syncthreads();
  }
}

const void *batch_level_kernel_ptr() { return (const void *)batch_level_kernel; }
const void *batch_setup_kernel_ptr() { return (const void *)batch_setup_kernel; }

int launch_batch(const BatchArgs &B, int grid, size_t smem, cudaStream_t st, int setup, int j0, int j1) {
  if (setup)
    batch_setup_kernel<<<grid, kThreads, smem, st>>>(B);
  else
    batch_level_kernel<<<grid, kThreads, smem, st>>>(B, j0, j1);
  return cudaGetLastError() == cudaSuccess ? kOK : kECuda;
}

}  // namespace tsf
