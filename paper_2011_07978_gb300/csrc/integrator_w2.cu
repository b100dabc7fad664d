// The batched Rosenbrock integrator with 2 warps per cell (see integrator_impl.cuh).
#include "integrator_impl.cuh"

namespace dlb {

cudaError_t launch_rosenbrock_w2(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a) {
  rosenbrock_kernel<2, false><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

const void* rosenbrock_kernel_ptr_w2() { return reinterpret_cast<const void*>(&rosenbrock_kernel<2, false>); }

const void* gate_kernel_ptr_w2() { return reinterpret_cast<const void*>(&gate_kernel<2>); }

cudaError_t launch_gate_w2(unsigned grid, int threads, int smem, cudaStream_t s, const GateArgs& a) {
  gate_kernel<2><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rhs_w2(unsigned grid, int threads, int smem, cudaStream_t s, const RhsArgs& a) {
  rhs_kernel<2><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

const void* rhs_kernel_ptr_w2() { return reinterpret_cast<const void*>(&rhs_kernel<2>); }

}  // namespace dlb
