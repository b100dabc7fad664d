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

// FP64 FMA throughput probe: eight independent chains per thread, bounded
// values (a <- a m + c with |m| < 1), one result per thread kept live.
__global__ void __launch_bounds__(256) fp64_fma_probe_kernel(int64_t iters, double* __restrict__ out) {
  const int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  double a0 = 1e-3 * threadIdx.x, a1 = a0 + 1.0, a2 = a0 + 2.0, a3 = a0 + 3.0;
  double a4 = a0 + 4.0, a5 = a0 + 5.0, a6 = a0 + 6.0, a7 = a0 + 7.0;
  const double m = 0.9999999, c = 1e-7 * (1 + (blockIdx.x & 7));
  for (int64_t i = 0; i < iters; ++i) {
    a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    a4 = fma(a4, m, c); a5 = fma(a5, m, c); a6 = fma(a6, m, c); a7 = fma(a7, m, c);
  }
  out[t] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
}

cudaError_t launch_fp64_fma_probe(int64_t iters, double* out, int64_t nout, cudaStream_t s) {
  fp64_fma_probe_kernel<<<unsigned(nout / 256), 256, 0, s>>>(iters, out);
  return cudaGetLastError();
}

cudaError_t launch_check_math(int64_t n, const double* x, const double* tab, double* out, cudaStream_t s) {
  check_math_kernel<<<unsigned((n + 255) / 256), 256, 0, s>>>(n, x, tab, out);
  return cudaGetLastError();
}

cudaError_t launch_rosenbrock(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a) {
  if (general_kernel(a.m)) {
    if (wpc == 1) return launch_rosenbrock_w1p(grid, threads, smem, s, a);
    if (wpc == 2) return launch_rosenbrock_w2p(grid, threads, smem, s, a);
    return launch_rosenbrock_w4p(grid, threads, smem, s, a);
  }
  if (wpc == 1) return launch_rosenbrock_w1(grid, threads, smem, s, a);
  if (wpc == 2) return launch_rosenbrock_w2(grid, threads, smem, s, a);
  return launch_rosenbrock_w4(grid, threads, smem, s, a);
}

cudaError_t launch_gate(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const GateArgs& a) {
  if (wpc == 1) return launch_gate_w1(grid, threads, smem, s, a);
  if (wpc == 2) return launch_gate_w2(grid, threads, smem, s, a);
  return launch_gate_w4(grid, threads, smem, s, a);
}

cudaError_t launch_rhs(int wpc, unsigned grid, int threads, int smem, cudaStream_t s, const RhsArgs& a) {
  if (wpc == 1) return launch_rhs_w1(grid, threads, smem, s, a);
  if (wpc == 2) return launch_rhs_w2(grid, threads, smem, s, a);
  return launch_rhs_w4(grid, threads, smem, s, a);
}

const void* rhs_kernel_ptr(int wpc) {
  return wpc == 1 ? rhs_kernel_ptr_w1() : (wpc == 2 ? rhs_kernel_ptr_w2() : rhs_kernel_ptr_w4());
}

const void* gate_kernel_ptr(int wpc) {
  return wpc == 1 ? gate_kernel_ptr_w1() : (wpc == 2 ? gate_kernel_ptr_w2() : gate_kernel_ptr_w4());
}

const void* rosenbrock_kernel_ptr(int wpc, bool plog) {
  if (plog) return wpc == 1 ? rosenbrock_kernel_ptr_w1p() : (wpc == 2 ? rosenbrock_kernel_ptr_w2p() : rosenbrock_kernel_ptr_w4p());
  return wpc == 1 ? rosenbrock_kernel_ptr_w1() : (wpc == 2 ? rosenbrock_kernel_ptr_w2() : rosenbrock_kernel_ptr_w4());
}

}  // namespace dlb
