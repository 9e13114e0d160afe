// The whole-grid level march with 512 threads per CTA (FFT half-lengths >= 2^19) and the one-CTA
// march of small instances.  They sit in a translation unit of their own so that the build
// compiles them in parallel with the other kernels; the device code is level_device.cuh.
#include "level_device.cuh"

namespace tsf {

// Small instances: the same march by one CTA with block barriers only (no grid barrier cost).
// With A.resident the level's working arrays live in shared memory after the line buffers
// (resident_patch), so that a phase touches global memory only for the history ring, u and the
// tables; the region is cleared first (the vectors' zero tails are read as zeros).
__global__ void __launch_bounds__(kThreads, 1) level_kernel_cta(Args Ap, int j0, int j1) {
  __shared__ Args A;
  extern __shared__ double2 dsm[];
  if (threadIdx.x == 0) A = Ap;
  __syncthreads();
  if (A.resident) {
    char *base = reinterpret_cast<char *>(dsm) + smem_lines_bytes(A);
    Args probe = A;
    const size_t bytes = resident_patch(probe, nullptr);
    double2 *z = reinterpret_cast<double2 *>(base);
    for (size_t i = threadIdx.x; i < bytes / 16; i += blockDim.x) z[i] = make_double2(0.0, 0.0);
    __syncthreads();
    if (threadIdx.x == 0) resident_patch(A, base);
    __syncthreads();
  }
  const Smem S = smem_view(lp_max_of(A), tw_max_of(A));
  cta_team_init();
  march_body(A, S, j0, j1);
}

const void *level_kernel_wide_ptr() { return (const void *)level_kernel<kWideThreads>; }
const void *level_kernel_cta_ptr() { return (const void *)level_kernel_cta; }

int launch_levels_wide(const Args &A, int grid, size_t smem, cudaStream_t st, int j0, int j1) {
  Args a = A;
  void *args[] = {&a, &j0, &j1};
  return coop_launch_n((const void *)level_kernel<kWideThreads>, grid, kWideThreads, smem, st, args);
}

int launch_levels_cta(const Args &A, size_t smem, cudaStream_t st, int j0, int j1) {
  Args a = A;
  level_kernel_cta<<<1, kThreads, smem, st>>>(a, j0, j1);
  return cudaGetLastError() == cudaSuccess ? kOK : kECuda;
}

}  // namespace tsf
