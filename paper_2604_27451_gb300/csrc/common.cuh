// Shared definitions for the libcvsadc CUDA sources (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>

namespace cvs {

// ---------------------------------------------------------------- status
struct Status {
  int code = 0;
  std::string msg;
};

// Internal error carrier: host code throws, the C-ABI layer catches and
// converts to a status code; nothing is thrown across the ABI.
struct Error {
  int code;
  std::string msg;
};

#define CVS_CUDA(call)                                                        \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      char b_[512];                                                           \
      snprintf(b_, sizeof b_, "%s failed: %s (%s:%d)", #call,                 \
               cudaGetErrorString(e_), __FILE__, __LINE__);                   \
      throw ::cvs::Error{e_ == cudaErrorMemoryAllocation ? -3 : -4, b_};      \
    }                                                                         \
  } while (0)

// every kernel launch of the library goes through CVS_CHECK_LAUNCH, which
// also counts it
extern unsigned long long g_launch_count;
#define CVS_CHECK_LAUNCH()                                 \
  do {                                                     \
    __atomic_fetch_add(&::cvs::g_launch_count, 1ull, __ATOMIC_RELAXED); \
    CVS_CUDA(cudaGetLastError());                          \
  } while (0)

#define CVS_REQUIRE(cond, code, text)                                         \
  do {                                                                        \
    if (!(cond)) throw ::cvs::Error{code, text};                              \
  } while (0)

// ----------------------------------------------------------- complex ops
typedef double2 cplx;

__host__ __device__ __forceinline__ cplx cmake(double r, double i) {
  return make_double2(r, i);
}
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) {
  return make_double2(a.x - b.x, a.y - b.y);
}
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) {
  return make_double2(a.x, -a.y);
}
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) {
  return make_double2(a.x * s, a.y * s);
}
// conj(a) * b
__host__ __device__ __forceinline__ cplx cdotc(cplx a, cplx b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------- matrix views
// A complex matrix whose row and column indices each split into two
// modes: r -> (r / r_lo, r % r_lo) with strides (rs_hi, rs_lo), same for
// columns.  One-mode dimensions use r_lo = INT32_MAX.  Strides are in
// complex elements.  `conj` conjugates every element on read.
struct View {
  cplx* p;
  int64_t rs_hi, rs_lo;
  int32_t r_lo;
  int64_t cs_hi, cs_lo;
  int32_t c_lo;
  int64_t batch;  // batch stride
  int32_t conj;
  int64_t ext;  // elements addressable from p (-1: not checked)
};

static inline View view(const void* p, int64_t rs, int64_t cs,
                        int64_t ext = -1) {
  View v;
  v.ext = ext;
  v.p = (cplx*)p;
  v.rs_hi = 0;
  v.rs_lo = rs;
  v.r_lo = INT32_MAX;
  v.cs_hi = 0;
  v.cs_lo = cs;
  v.c_lo = INT32_MAX;
  v.batch = 0;
  v.conj = 0;
  return v;
}
static inline View rows2(View v, int64_t hi, int64_t lo, int32_t lo_extent) {
  v.rs_hi = hi;
  v.rs_lo = lo;
  v.r_lo = lo_extent;
  return v;
}
static inline View cols2(View v, int64_t hi, int64_t lo, int32_t lo_extent) {
  v.cs_hi = hi;
  v.cs_lo = lo;
  v.c_lo = lo_extent;
  return v;
}
static inline View conj_of(View v) {
  v.conj ^= 1;
  return v;
}
static inline View batched(View v, int64_t stride) {
  v.batch = stride;
  return v;
}
static inline View extent(View v, int64_t ext) {
  v.ext = ext;
  return v;
}
// Largest element offset a view reaches over rows x cols (x batch).
static inline int64_t view_max_offset(const View& v, int64_t rows,
                                      int64_t cols, int64_t batch) {
  auto span = [](int64_t cnt, int64_t hi, int64_t lo, int32_t lo_ext) {
    if (cnt <= 0) return (int64_t)0;
    if (lo_ext == INT32_MAX || cnt <= lo_ext) return (cnt - 1) * lo;
    return ((cnt - 1) / lo_ext) * hi + (int64_t)(lo_ext - 1) * lo;
  };
  return span(rows, v.rs_hi, v.rs_lo, v.r_lo) +
         span(cols, v.cs_hi, v.cs_lo, v.c_lo) + (batch - 1) * v.batch;
}
// Throws unless every element a rows x cols (x batch) access touches lies
// inside the view's declared extent.
static inline void check_view(const View& v, int64_t rows, int64_t cols,
                              int64_t batch, const char* what) {
  if (v.rs_hi < 0 || v.rs_lo < 0 || v.cs_hi < 0 || v.cs_lo < 0 || v.batch < 0)
    throw Error{-1, std::string("negative stride in view ") + what};
  if (v.ext < 0) return;
  int64_t m = view_max_offset(v, rows, cols, batch);
  if (rows > 0 && cols > 0 && m >= v.ext) {
    char b[200];
    snprintf(b, sizeof b, "view %s out of range: max offset %lld >= extent %lld",
             what, (long long)m, (long long)v.ext);
    throw Error{-1, b};
  }
}

// Transposed view: rows <-> columns.
static inline View trans(View v) {
  View t = v;
  t.rs_hi = v.cs_hi;
  t.rs_lo = v.cs_lo;
  t.r_lo = v.c_lo;
  t.cs_hi = v.rs_hi;
  t.cs_lo = v.rs_lo;
  t.c_lo = v.r_lo;
  return t;
}

__device__ __forceinline__ int64_t vrow(const View& v, int64_t r) {
  if (v.r_lo == INT32_MAX) return r * v.rs_lo;
  int64_t h = r / v.r_lo;
  return h * v.rs_hi + (r - h * v.r_lo) * v.rs_lo;
}
__device__ __forceinline__ int64_t vcol(const View& v, int64_t c) {
  if (v.c_lo == INT32_MAX) return c * v.cs_lo;
  int64_t h = c / v.c_lo;
  return h * v.cs_hi + (c - h * v.c_lo) * v.cs_lo;
}

// ------------------------------------------------------ kernel timing
// When enabled, the GEMM drivers bracket each launch of their main kernel
// with CUDA events on the launching stream and record its algorithmic
// flops; kstats_collect() turns finished pairs into per-kernel totals.
enum KernelId { K_TC_BF16X3 = 0, K_TC_SLICE = 1, K_F64_GEMM = 2, K_NKERNELS = 3 };
bool kstats_enabled();
void kstats_set(bool on);
// returns an opaque token to pass to kstats_end (or -1 when disabled)
int kstats_begin(cudaStream_t s, int kernel, double flops);
void kstats_end(cudaStream_t s, int token);
void kstats_collect(int kernel, int64_t* count, double* ms, double* flops);
void kstats_reset();

// ------------------------------------------------------------- launching
static inline unsigned grid1d(int64_t n, int block, int64_t cap = 152 * 32) {
  int64_t g = (n + block - 1) / block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

}  // namespace cvs
