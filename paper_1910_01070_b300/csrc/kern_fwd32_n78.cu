// kern_fwd32_n78.cu -- instantiations of the FP32 forward kernel for 7 and 8
// angle nodes (see kern_forward32.cuh).
#include "kern_forward32.cuh"

namespace hr2 {

cudaError_t launch_forward32_n7(const FwdArgs& a, int grid, bool cached, bool linear, bool para, int max_k,
                                int kt, int stages, cudaStream_t s) {
  return launch_nmu<7>(a, grid, cached, linear, para, max_k, kt, stages, s);
}

cudaError_t launch_forward32_n8(const FwdArgs& a, int grid, bool cached, bool linear, bool para, int max_k,
                                int kt, int stages, cudaStream_t s) {
  return launch_nmu<8>(a, grid, cached, linear, para, max_k, kt, stages, s);
}

}  // namespace hr2
