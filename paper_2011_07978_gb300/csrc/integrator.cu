// Launch side of the batched Rosenbrock integrator: the kernel itself is in
// integrator_impl.cuh and is compiled once per team size (one, two or four
// warps per cell) in integrator_w1.cu, integrator_w2.cu, integrator_w4.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "integrator_impl.cuh"

namespace dlb {

// Diagnostic: the integrator's exp and reciprocal next to CUDA's exp and
// IEEE division, for the accuracy test of the two replacements.
__global__ void check_math_kernel(int64_t n, const double* __restrict__ x, const double* __restrict__ tab,
                                  double* __restrict__ out) {
  const int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (i >= n) return;
  out[4 * i + 0] = exp_tab(x[i], tab);
  out[4 * i + 1] = exp(x[i]);
  out[4 * i + 2] = rcp_nr(x[i]);
  out[4 * i + 3] = 1.0 / x[i];
}

cudaError_t launch_check_math(int64_t n, const double* x, const double* tab, double* out, cudaStream_t s) {
  check_math_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, x, tab, out);
  return cudaGetLastError();
}

cudaError_t launch_rosenbrock(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a) {
  if (wpc == 1) return launch_rosenbrock_w1(grid, threads, smem, s, a);
  if (wpc == 2) return launch_rosenbrock_w2(grid, threads, smem, s, a);
  return launch_rosenbrock_w4(grid, threads, smem, s, a);
}

cudaError_t launch_gate(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const GateArgs& a) {
  if (wpc == 1) return launch_gate_w1(grid, threads, smem, s, a);
  if (wpc == 2) return launch_gate_w2(grid, threads, smem, s, a);
  return launch_gate_w4(grid, threads, smem, s, a);
}

const void* gate_kernel_ptr(int wpc) {
  return wpc == 1 ? gate_kernel_ptr_w1() : (wpc == 2 ? gate_kernel_ptr_w2() : gate_kernel_ptr_w4());
}

const void* rosenbrock_kernel_ptr(int wpc) {
  return wpc == 1 ? rosenbrock_kernel_ptr_w1() : (wpc == 2 ? rosenbrock_kernel_ptr_w2() : rosenbrock_kernel_ptr_w4());
}

}  // namespace dlb
