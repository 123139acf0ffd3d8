// kern_fwd32_n56.cu -- instantiations of the FP32 forward kernel for 5 and 6
// angle nodes (see kern_forward32.cuh).
#include "kern_forward32.cuh"

namespace hr2 {

cudaError_t launch_forward32_n5(const FwdArgs& a, int grid, bool cached, bool linear, bool para, int max_k,
                                int kt, int stages, cudaStream_t s) {
  return launch_nmu<5>(a, grid, cached, linear, para, max_k, kt, stages, s);
}

cudaError_t launch_forward32_n6(const FwdArgs& a, int grid, bool cached, bool linear, bool para, int max_k,
                                int kt, int stages, cudaStream_t s) {
  return launch_nmu<6>(a, grid, cached, linear, para, max_k, kt, stages, s);
}

}  // namespace hr2
