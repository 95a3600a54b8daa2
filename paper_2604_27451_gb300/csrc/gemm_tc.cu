// tcgen05 tensor-core complex GEMM (placeholder until the kernel lands).
#include "common.cuh"
#include "kernels.cuh"

namespace cvs {

bool tc_available() { return false; }

size_t tc_workspace_bytes(int, int, int) { return 0; }

void zgemm_tc(cudaStream_t, int, int, int, double, View, View, double, View,
              void*, size_t) {
  throw Error{-1, "tensor-core GEMM not available"};
}

}  // namespace cvs
