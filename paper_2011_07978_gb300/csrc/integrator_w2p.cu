// The batched Rosenbrock integrator with 2 warps per cell for mechanisms with PLOG
// reactions or NASA-7 thermo (see integrator_impl.cuh).
#include "integrator_impl.cuh"

namespace dlb {

cudaError_t launch_rosenbrock_w2p(unsigned grid, int threads, int smem, cudaStream_t s, const KernelArgs& a) {
  rosenbrock_kernel<2, true><<<grid, threads, smem, s>>>(a);
  return cudaGetLastError();
}

const void* rosenbrock_kernel_ptr_w2p() { return reinterpret_cast<const void*>(&rosenbrock_kernel<2, true>); }

}  // namespace dlb
