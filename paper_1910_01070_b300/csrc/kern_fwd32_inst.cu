// kern_fwd32_inst.cu -- instantiations of the FP32 forward kernel for one
// angle-node count, HR2_FWD32_NMU (1..8); the build compiles this file once
// per count so that the instantiations compile in parallel.
#include "kern_forward32.cuh"

#ifndef HR2_FWD32_NMU
#error "HR2_FWD32_NMU (the angle-node count) must be defined"
#endif
#define HR2_CAT_(a, b) a##b
#define HR2_CAT(a, b) HR2_CAT_(a, b)

namespace hr2 {

cudaError_t HR2_CAT(launch_forward32_n, HR2_FWD32_NMU)(const FwdArgs& a, int grid, bool cached, bool linear,
                                                      bool para, int max_k, int kt, int stages, cudaStream_t s) {
  return launch_nmu<HR2_FWD32_NMU>(a, grid, cached, linear, para, max_k, kt, stages, s);
}

}  // namespace hr2
