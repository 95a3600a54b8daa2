// Allocation-free variant of the library's FP64 complex GEMM for small
// outputs (cvsadc_zgemm_small_noalloc in include/cvsadc.h).
//
// Some callers cannot let a library call cudaMalloc: a process whose device
// memory is already reserved by another allocator (a framework's caching
// allocator or a pre-sized memory pool), where an extra runtime allocation
// fails or fragments that pool; and latency-sensitive loops, where the
// implicit device synchronisation of cudaMalloc / cudaFree is not
// acceptable.  This entry point therefore takes the split-K partial
// products of the small-output GEMM from a fixed device array that is part
// of the loaded library image instead of allocating them.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds it until the process exits, and every call on a device
// shares it, so calls that overlap on the GPU (different streams or
// threads) race on it.  Each call writes every partial slot it later reads,
// so nothing in the array has to start at zero and the previous call's
// contents are irrelevant.
#include <map>
#include <mutex>

#include "../../include/cvsadc.h"
#include "common.cuh"
#include "kernels.cuh"

namespace cvs {
namespace {

// 2^19 complex doubles = 8 MiB of device memory per GPU
constexpr size_t NOALLOC_SCRATCH_ELEMS = (size_t)1 << 19;
static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_SCRATCH_ELEMS];

std::mutex g_na_mu;
std::map<int, cplx*> g_na_addr;  // device -> address of the array there

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, once per device, with that device current.  This
// set-up runs inside the first call on each device, which should therefore
// come before any stream capture begins.
cplx* noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> l(g_na_mu);
  auto it = g_na_addr.find(dev);
  if (it != g_na_addr.end()) return it->second;
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    (void)cudaGetLastError();
    throw Error{CVSADC_ECUDA,
                std::string("cudaGetSymbolAddress of the scratch array failed: ") +
                    cudaGetErrorString(e)};
  }
  init_gemm_attributes();
  g_na_addr[dev] = (cplx*)p;
  return (cplx*)p;
}

}  // namespace
}  // namespace cvs

using namespace cvs;

extern "C" int cvsadc_zgemm_small_noalloc(void* cuda_stream, int32_t M,
                                          int32_t N, int32_t K, const void* A,
                                          int64_t lda, const void* B,
                                          int64_t ldb, void* C, int64_t ldc) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1) return CVSADC_EINVAL;
  if ((int64_t)M * N > CVSADC_NOALLOC_MAX_MN || M + N > CVSADC_NOALLOC_MAX_M_PLUS_N)
    return CVSADC_EINVAL;
  if (lda < K || ldb < N || ldc < N) return CVSADC_EINVAL;
  try {
    int dev = 0;
    CVS_CUDA(cudaGetDevice(&dev));
    cplx* scratch = noalloc_scratch(dev);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // M N <= 4096 and K >= 4096 take the small-output kernel, whose
    // launcher splits K into at most NOALLOC_SCRATCH_ELEMS / (M N) >= 128
    // slices, so every partial fits the array; shorter K runs the tile
    // kernel without split-K partials
    zgemm_f64(s, M, N, K, 1.0, view(A, lda, 1), view(B, ldb, 1), 0.0,
              view(C, ldc, 1), 1, scratch, NOALLOC_SCRATCH_ELEMS);
    CVS_CUDA(cudaStreamSynchronize(s));
    return CVSADC_OK;
  } catch (const Error& e) {
    return e.code;
  } catch (...) {
    return CVSADC_ECUDA;
  }
}
