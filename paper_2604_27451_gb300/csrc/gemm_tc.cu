// Complex GEMM on the 5th-generation tensor cores (tcgen05, sm_103a).
//
//   C = alpha * A * B + beta * C, A: M x K, B: K x N complex (two-mode
//   views), C complex128.
//
// Precision: every real value x is split into bfloat16 parts x = x_h + x_l
// (x_h = bf16(x), x_l = bf16(x - x_h)); a real product keeps x_h y_h +
// x_h y_l + x_l y_h (~2^-16 relative), accumulated in FP32 in tensor
// memory.  The tensor-memory accumulation rounds each MMA step, so its
// error grows linearly with K (measured: ~1e-5 relative at K' ~ 10^4); the
// exact-slice kernel further down removes that limit.
//
// Layout: one real GEMM computes the complex product.  For every product
// term p = (pa, pb) the K dimension carries two segments of length Kp:
//   A row m       : [ re_pa(a) , im_pa(a) ]
//   B' row 2n     : [ re_pb(b) , -im_pb(b) ]   -> column 2n   = Re(a b)
//   B' row 2n + 1 : [ im_pb(b) ,  re_pb(b) ]   -> column 2n+1 = Im(a b)
// so K' = 2 * (number of product terms) * Kp and N' = 2 N, with real and
// imaginary parts of one output
// element in adjacent accumulator columns.  Packing (split + transpose into
// K-major rows, zero padding to the tile grid) is a bandwidth kernel; the
// GEMM itself is TMA -> shared memory (128B swizzle) -> tcgen05.mma with
// the accumulator in tensor memory -> tcgen05.ld -> complex128 epilogue.
//
// CTA: 128 threads.  Thread 0 issues the TMA loads, thread 32 issues the
// MMAs, all four warps drain TMEM (warp w owns TMEM lanes 32w..32w+31).
// Every mbarrier wait is bounded by a globaltimer deadline; on expiry the
// kernel records an error code, releases its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace cvs {

namespace {

constexpr int BM = 128;   // UMMA M
constexpr int BN = 256;   // UMMA N (real columns = 128 complex columns)
constexpr int BK = 64;    // bf16 elements per 128-byte swizzle row
constexpr int STAGES = 4;
constexpr int A_TILE = BM * BK * 2;
constexpr int B_TILE = BN * BK * 2;
constexpr int STAGE_BYTES = A_TILE + B_TILE;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr uint64_t WAIT_NS = 4000000000ull;  // 4 s bound on any wait

// product tables: (part of A, part of B), part 0 = hi, 1 = mid/lo, 2 = lo
template <int NP>
struct Split;
template <>
struct Split<3> {
  static constexpr int parts = 2;
  __device__ static int pa(int p) { return p == 2 ? 1 : 0; }
  __device__ static int pb(int p) { return p == 1 ? 1 : 0; }
};
template <>
struct Split<6> {
  static constexpr int parts = 3;
  // (0,0) (0,1) (1,0) (0,2) (1,1) (2,0)
  __device__ static int pa(int p) {
    return p == 2 ? 1 : p == 4 ? 1 : p == 5 ? 2 : 0;
  }
  __device__ static int pb(int p) {
    return p == 1 ? 1 : p == 3 ? 2 : p == 4 ? 1 : 0;
  }
};

// CTA rasterisation: consecutive CTAs walk groups of RASTER M-tiles
// column by column, so the CTAs resident at one time share A and B panels
// in L2 instead of streaming the whole B operand once per M-tile row.
constexpr int RASTER = 8;
__device__ __forceinline__ void tile_coords(int& mt, int& nt) {
  const int num_n = gridDim.x, num_m = gridDim.y;
  const int pid = blockIdx.y * num_n + blockIdx.x;
  const int per_group = RASTER * num_n;
  const int first_m = (pid / per_group) * RASTER;
  const int gsz = min(num_m - first_m, RASTER);
  const int local = pid - (first_m / RASTER) * per_group;
  mt = first_m + local % gsz;
  nt = local / gsz;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtime() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait on the phase with the given parity: try_wait suspends the
// thread in hardware for a while before it reports "not yet", so the loop
// polls without sleeping and reads the clock only every 64 tries
// true once the phase completes; false after limit_ns of the global timer
__device__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = gtime();
  for (uint32_t n = 1;; ++n) {
    if (mbar_try(bar, parity)) return true;
    if ((n & 63) == 0 && gtime() - t0 > limit_ns) return false;
  }
}
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  return mbar_wait_for(bar, parity, WAIT_NS);
}

// The error path of the bounded waits, on demand: one thread waits, with
// limit_ns, on an mbarrier that nothing arrives on.  The wait gives up, the
// kernel records code 5 in *err (as a GEMM's expired wait records its
// code) and returns.
__global__ void wait_probe_kernel(uint64_t limit_ns, int* err) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait_for(&bar, 0, limit_ns)) atomicExch(err, 5);
  }
}
__device__ __forceinline__ void tma_load(const CUtensorMap* map, uint64_t* bar,
                                         void* dst, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// shared-memory matrix descriptor: K-major, 128B swizzle, 8-row atoms of
// 1024 bytes stacked along M/N (stride 1024 B)
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)1 << 16;            // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;            // descriptor version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}
// instruction descriptor, kind::f16: D f32, A/B bf16, both K-major
__device__ __forceinline__ uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void umma(uint32_t dtm, uint64_t a, uint64_t b,
                                     uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtm),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
      "[%0];" ::"r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]),
        "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]),
        "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                   const __grid_constant__ CUtensorMap tmB, int nkt, int zkt,
                   int M, int N, double alpha, double beta, View C,
                   cplx* part, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + STAGES * A_TILE;
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tslot = (uint32_t*)(done + 1);
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mt, nt;
  tile_coords(mt, nt);
  const int m0 = mt * BM, n0 = nt * BN;
  const int z = blockIdx.z;
  const int ktb = z * zkt, kte = min(nkt, ktb + zkt);  // non-empty by launch

  if (threadIdx.x == 0) {
    fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(tslot)),
        "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (threadIdx.x == 0) {
    // TMA producer
    for (int i = 0; i < kte - ktb; ++i) {
      const int kt = ktb + i;
      const int s = i % STAGES;
      const uint32_t ph = (i / STAGES) & 1;
      if (i >= STAGES && !mbar_wait(&empty[s], ph ^ 1)) {
        fail = 1;
        break;
      }
      if (fail) break;
      mbar_expect_tx(&full[s], STAGE_BYTES);
      tma_load(&tmA, &full[s], sA + s * A_TILE, kt * BK, m0);
      tma_load(&tmB, &full[s], sB + s * B_TILE, kt * BK, n0);
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer
    const uint32_t id = idesc_bf16(BM, BN);
    for (int i = 0; i < kte - ktb; ++i) {
      const int s = i % STAGES;
      const uint32_t ph = (i / STAGES) & 1;
      if (!mbar_wait(&full[s], ph)) {
        fail = 2;
        break;
      }
      fence_after();
      const uint64_t ad = sdesc(smem_u32(sA + s * A_TILE));
      const uint64_t bd = sdesc(smem_u32(sB + s * B_TILE));
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        umma(tmem, ad + 2 * kk, bd + 2 * kk, id, (i | kk) ? 1u : 0u);
      umma_commit(&empty[s]);
    }
    umma_commit(done);
  }
  __syncwarp();
  const bool ok = mbar_wait(done, 0);
  __syncwarp();
  fence_after();
  if (ok && !fail) {
    const int m = m0 + warp * 32 + lane;
    const int64_t ro = (m < M && !part) ? vrow(C, m) : 0;
#pragma unroll 1
    for (int c = 0; c < BN; c += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + c, v);
      if (m < M) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int n = (n0 + c) / 2 + q;
          if (n < N) {
            cplx o = cmake(alpha * (double)v[2 * q], alpha * (double)v[2 * q + 1]);
            if (part) {
              part[((int64_t)z * M + m) * N + n] = o;
              continue;
            }
            cplx* d = C.p + ro + vcol(C, n);
            if (beta != 0.0) {
              cplx old = *d;
              o.x += beta * old.x;
              o.y += beta * old.y;
            }
            *d = o;
          }
        }
      }
    }
  } else if (lane == 0) {
    atomicExch(err, fail ? fail : 3);
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(BN));
}

// ------------------------------------------------------------ packing
template <int PARTS>
__device__ __forceinline__ void split(double x, __nv_bfloat16* p) {
  double r = x;
#pragma unroll
  for (int q = 0; q < PARTS; ++q) {
    __nv_bfloat16 h = __double2bfloat16(r);
    p[q] = h;
    r -= (double)__bfloat162float(h);
  }
}

// A' [Mp][2 NP Kp]: row m, segment 2p + {0: re, 1: im} of part pa(p)
template <int NP>
__global__ void pack_a_kernel(View A, int M, int K, int k0, int Mp, int Kp,
                              __nv_bfloat16* out) {
  constexpr int PARTS = Split<NP>::parts;
  const int64_t ld = (int64_t)2 * NP * Kp;
  const int64_t total = (int64_t)Mp * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int m = idx / Kp, k = idx % Kp;
    cplx a = cmake(0, 0);
    if (m < M && k < K) {
      a = A.p[vrow(A, m) + vcol(A, k0 + k)];
      if (A.conj) a.y = -a.y;
    }
    __nv_bfloat16 re[PARTS], im[PARTS];
    split<PARTS>(a.x, re);
    split<PARTS>(a.y, im);
    __nv_bfloat16* o = out + (int64_t)m * ld + k;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      o[(2 * p) * (int64_t)Kp] = re[Split<NP>::pa(p)];
      o[(2 * p + 1) * (int64_t)Kp] = im[Split<NP>::pa(p)];
    }
  }
}

// B' [Np2][2 NP Kp]: rows 2n (real part column) and 2n+1 (imaginary)
template <int NP>
__global__ void pack_b_kernel(View B, int K, int k0, int N, int Np2, int Kp,
                              __nv_bfloat16* out) {
  constexpr int PARTS = Split<NP>::parts;
  const int64_t ld = (int64_t)2 * NP * Kp;
  const int64_t total = (int64_t)(Np2 / 2) * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int n = idx / Kp, k = idx % Kp;
    cplx b = cmake(0, 0);
    if (n < N && k < K) {
      b = B.p[vrow(B, k0 + k) + vcol(B, n)];
      if (B.conj) b.y = -b.y;
    }
    __nv_bfloat16 re[PARTS], im[PARTS];
    split<PARTS>(b.x, re);
    split<PARTS>(b.y, im);
    __nv_bfloat16* o0 = out + (int64_t)(2 * n) * ld + k;
    __nv_bfloat16* o1 = o0 + ld;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
      const int q = Split<NP>::pb(p);
      o0[(2 * p) * (int64_t)Kp] = re[q];
      o0[(2 * p + 1) * (int64_t)Kp] = __hneg(im[q]);
      o1[(2 * p) * (int64_t)Kp] = im[q];
      o1[(2 * p + 1) * (int64_t)Kp] = re[q];
    }
  }
}

// ------------------------------------------------------- host helpers
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t,
                                  void*, const cuuint64_t*, const cuuint64_t*,
                                  const cuuint32_t*, const cuuint32_t*,
                                  CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      (void)cudaGetLastError();
  });
  return fn;
}

CUtensorMap make_map(const void* base, int64_t rows, int64_t cols_bf16,
                     int box_rows) {
  EncodeTiledFn fn = encode_fn();
  CVS_REQUIRE(fn, -4, "cuTensorMapEncodeTiled unavailable");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)cols_bf16, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols_bf16 * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
                  dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CVS_REQUIRE(r == CUDA_SUCCESS, -4, "cuTensorMapEncodeTiled failed");
  return m;
}

struct Dims {
  int Mp, Np2, Kp, nseg;
  size_t a_bytes, b_bytes;
};
Dims dims_of(int M, int N, int K, int nprod) {
  Dims d;
  d.Mp = (M + BM - 1) / BM * BM;
  d.Np2 = (2 * N + BN - 1) / BN * BN;
  d.Kp = (K + BK - 1) / BK * BK;
  d.nseg = 2 * nprod;
  d.a_bytes = (size_t)d.Mp * d.nseg * d.Kp * 2;
  d.b_bytes = (size_t)d.Np2 * d.nseg * d.Kp * 2;
  return d;
}

}  // namespace

bool tc_available() {
  static int avail = -1;
  static std::once_flag once;
  std::call_once(once, [] {
    int dev = 0, major = 0, minor = 0;
    avail = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) ==
            cudaSuccess &&
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) ==
            cudaSuccess)
      avail = (major == 10 && minor == 3 && encode_fn() != nullptr) ? 1 : 0;
    (void)cudaGetLastError();
    if (avail)
      cudaFuncSetAttribute(tc_gemm_kernel,
                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                           SMEM_BYTES);
  });
  return avail == 1;
}

// packed-operand budget per K chunk
constexpr size_t PACK_BUDGET = (size_t)3 << 30;

int chunk_k(int Mp, int Np2, int K, int nseg) {
  // complex K per chunk so that both packed operands fit the budget
  const size_t per_k = (size_t)(Mp + Np2) * nseg * 2;
  int64_t kc = (int64_t)(PACK_BUDGET / per_k) / BK * BK;
  kc = std::max<int64_t>(kc, BK);
  return (int)std::min<int64_t>(kc, ((int64_t)K + BK - 1) / BK * BK);
}

size_t tc_workspace_bytes(int M, int N, int K, int nprod) {
  Dims d = dims_of(M, N, K, nprod);
  const int kc = chunk_k(d.Mp, d.Np2, K, d.nseg);
  return (size_t)(d.Mp + d.Np2) * d.nseg * kc * 2 + 256;
}

// number of K splits for an output of `tiles` CTA tiles over `kt` k-tiles
int tc_splits(int64_t tiles, int kt, int min_kt) {
  if (tiles >= 152) return 1;
  int64_t s = (2 * 152 + tiles - 1) / tiles;
  s = std::min<int64_t>(s, std::max(1, kt / min_kt));
  return (int)std::max<int64_t>(1, s);
}

void zgemm_tc(cudaStream_t s, int nprod, int M, int N, int K, double alpha,
              View A, View B, double beta, View C, void* work,
              size_t work_bytes, cplx* part, size_t part_elems, int* err) {
  if (M <= 0 || N <= 0) return;
  CVS_REQUIRE(nprod == 3 || nprod == 6, -1, "zgemm_tc: nprod must be 3 or 6");
  Dims d = dims_of(M, N, K, nprod);
  const int kc = chunk_k(d.Mp, d.Np2, K, d.nseg);
  CVS_REQUIRE(work_bytes >= (size_t)(d.Mp + d.Np2) * d.nseg * kc * 2, -1,
              "zgemm_tc: workspace too small");
  __nv_bfloat16* ap = (__nv_bfloat16*)work;
  __nv_bfloat16* bp = ap + (size_t)d.Mp * d.nseg * kc;
  const int64_t tiles = (int64_t)(d.Np2 / BN) * (d.Mp / BM);
  for (int k0 = 0; k0 < K; k0 += kc) {
    const int Kc = std::min(kc, K - k0);
    const int Kp = (Kc + BK - 1) / BK * BK;
    const unsigned ga = grid1d((int64_t)d.Mp * Kp, 256);
    const unsigned gb = grid1d((int64_t)(d.Np2 / 2) * Kp, 256);
    if (nprod == 3) {
      pack_a_kernel<3><<<ga, 256, 0, s>>>(A, M, Kc, k0, d.Mp, Kp, ap);
      CVS_CHECK_LAUNCH();
      pack_b_kernel<3><<<gb, 256, 0, s>>>(B, Kc, k0, N, d.Np2, Kp, bp);
    } else {
      pack_a_kernel<6><<<ga, 256, 0, s>>>(A, M, Kc, k0, d.Mp, Kp, ap);
      CVS_CHECK_LAUNCH();
      pack_b_kernel<6><<<gb, 256, 0, s>>>(B, Kc, k0, N, d.Np2, Kp, bp);
    }
    CVS_CHECK_LAUNCH();
    CUtensorMap ma = make_map(ap, d.Mp, (int64_t)d.nseg * Kp, BM);
    CUtensorMap mb = make_map(bp, d.Np2, (int64_t)d.nseg * Kp, BN);
    const int nkt = d.nseg * Kp / BK;
    int sp = tc_splits(tiles, nkt, 8);
    if (part == nullptr || (size_t)sp * M * N > part_elems) sp = 1;
    const int zkt = (nkt + sp - 1) / sp;
    const int nz = (nkt + zkt - 1) / zkt;
    const double beta_c = (k0 == 0) ? beta : 1.0;
    dim3 grid(d.Np2 / BN, d.Mp / BM, nz);
    const int tok = kstats_begin(s, K_TC_BF16X3, 8.0 * M * N * (double)Kc);
    tc_gemm_kernel<<<grid, 128, SMEM_BYTES, s>>>(ma, mb, nkt, zkt, M, N, alpha,
                                                 beta_c, C, nz > 1 ? part : nullptr,
                                                 err);
    CVS_CHECK_LAUNCH();
    kstats_end(s, tok);
    if (nz > 1) splitk_reduce(s, M, N, nz, part, beta_c, C);
  }
}

// ===========================================================================
// Exact-accumulation slice GEMM (an error-free splitting in the manner of
// Ozaki et al., Numer. Algorithms 59 (2012), mapped onto tcgen05).
//
// Every row m of A' and every output column n of B' gets a power-of-two
// scale 2^e with max |entry| < 2^e.  A scaled value a in (-1, 1) is cut into
// integer slices q_i in [-128, 128] with a = sum_i q_i 2^{-7(i+1)} + r,
// |r| <= 2^{-7 s - 1}; each slice is exactly a bf16.  A product of slices is
// an integer with |q q'| <= 2^14, so a run of up to 1024 products sums
// exactly in the FP32 tensor-memory accumulator (< 2^24).  Slice products
// (i, j) with i + j <= s - 1 are kept and grouped so that a run never mixes
// two (i, j) pairs; each finished run is drained from tensor memory (two
// accumulator buffers, so draining overlaps the next run) and added, times
// 2^{-7(i+j+2)}, to float-float accumulators (about 48 bits) in registers.
// The epilogue applies 2^{e_m + f_n}, alpha and beta in FP64.
//
// CTA: 576 threads.  Warp 0 lane 0: TMA producer; warp 1 lane 0: MMA
// issuer; warps 2..17: drain (warp w reads TMEM lanes 32 (w % 4) .. +31 and
// the 32 columns [32 c, 32 c + 32), c = (w - 2) / 4, of a 128 x 128 tile).
// ===========================================================================
namespace {

constexpr int SBN = 128;          // N' per CTA (64 complex columns)
constexpr int SSTAGES = 7;
constexpr int S_A_TILE = BM * BK * 2;
constexpr int S_B_TILE = SBN * BK * 2;
constexpr int S_STAGE = S_A_TILE + S_B_TILE;
constexpr int S_SMEM = SSTAGES * S_STAGE + 1024 + 512;
constexpr int RUN_KT = 16;         // k-tiles per exact run: 16 * 64 = 1024 terms
constexpr int SLICE_BITS = 7;
constexpr int MAX_PAIRS = 36;

// Slice pairs (i, j) ordered by order o = i + j, then by i.  With this
// order the pairs of a 4-slice product (orders 0..3, 10 pairs) are the first
// 10 of the 7-slice table (orders 0..6, 28 pairs), so one table, fixed at
// compile time, serves both and no launch ever rewrites constant memory
// under a kernel running on another stream.
// slice of A for pair p
__constant__ int c_si[MAX_PAIRS] = {0, 0, 1, 0, 1, 2, 0, 1, 2, 3,
                                    0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 5,
                                    0, 1, 2, 3, 4, 5, 6};
// slice of B for pair p
__constant__ int c_sj[MAX_PAIRS] = {0, 1, 0, 2, 1, 0, 3, 2, 1, 0,
                                    4, 3, 2, 1, 0, 5, 4, 3, 2, 1, 0,
                                    6, 5, 4, 3, 2, 1, 0};

__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
  // TwoSum without contraction
  float s = __fadd_rn(hi, x);
  float bp = __fsub_rn(s, hi);
  float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
  hi = s;
  lo = __fadd_rn(lo, e);
}

__global__ void __launch_bounds__(576, 1)
    tc_slice_kernel(const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB, int npairs,
                    int ktpp, int kpb, int kb_off, int zl, int M, int N,
                    const int* __restrict__ eA,
                    const int* __restrict__ eB, double alpha, double beta,
                    View C, cplx* part, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = smem + SSTAGES * S_A_TILE;
  uint64_t* full = (uint64_t*)(smem + SSTAGES * S_STAGE);
  uint64_t* empty = full + SSTAGES;
  uint64_t* afull = empty + SSTAGES;  // [2]
  uint64_t* aempty = afull + 2;       // [2]
  uint32_t* tslot = (uint32_t*)(aempty + 2);
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mt, nt;
  tile_coords(mt, nt);
  const int m0 = mt * BM, n0 = nt * SBN;
  const int z = blockIdx.z;
  // this CTA's k-tiles of every pair: [zb, ze) relative to the pair start
  const int zb = z * zl, ze = min(ktpp, zb + zl);
  const int zlen = max(0, ze - zb);
  const int runs_pp = (zlen + RUN_KT - 1) / RUN_KT;
  const int nruns = npairs * runs_pp;

  if (threadIdx.x == 0) {
    fail = 0;
    for (int s = 0; s < SSTAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 1);
      mbar_init(&aempty[b], 16);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(tslot)),
        "r"(2 * SBN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (threadIdx.x == 0) {
    // TMA producer over this CTA's k-tiles of every pair
    const int nkt = npairs * zlen;
    for (int i = 0; i < nkt; ++i) {
      const int p = i / zlen, t = zb + i % zlen;  // pair, k-tile within it
      const int kt = p * ktpp + t;
      // B: segment 2 p + (re / im half), K block kb_off + (t mod Kp / BK)
      const int hk = ktpp >> 1;
      const int xb = (2 * p + t / hk) * kpb + (kb_off + t % hk) * BK;
      const int s = i % SSTAGES;
      const uint32_t ph = (i / SSTAGES) & 1;
      if (i >= SSTAGES && !mbar_wait(&empty[s], ph ^ 1)) {
        fail = 1;
        break;
      }
      if (fail) break;
      mbar_expect_tx(&full[s], S_STAGE);
      tma_load(&tmA, &full[s], sA + s * S_A_TILE, kt * BK, m0);
      tma_load(&tmB, &full[s], sB + s * S_B_TILE, xb, n0);
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer: one exact run per (pair, run) into alternating buffers
    const uint32_t id = idesc_bf16(BM, SBN);
    int i = 0;  // position in the producer's sequence
    for (int r = 0; r < nruns && !fail; ++r) {
      const int rr = r % runs_pp;
      const int i0 = i, i1 = i + min(RUN_KT, zlen - rr * RUN_KT);
      const int b = r & 1;
      if (r >= 2 && !mbar_wait(&aempty[b], ((r >> 1) + 1) & 1)) {
        fail = 4;
        break;
      }
      fence_after();
      const uint32_t dt = tmem + (uint32_t)(b * SBN);
      for (i = i0; i < i1; ++i) {
        const int s = i % SSTAGES;
        const uint32_t ph = (i / SSTAGES) & 1;
        if (!mbar_wait(&full[s], ph)) {
          fail = 2;
          break;
        }
        fence_after();
        const uint64_t ad = sdesc(smem_u32(sA + s * S_A_TILE));
        const uint64_t bd = sdesc(smem_u32(sB + s * S_B_TILE));
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk)
          umma(dt, ad + 2 * kk, bd + 2 * kk, id, (i != i0 || kk) ? 1u : 0u);
        umma_commit(&empty[s]);
      }
      umma_commit(&afull[b]);
    }
  } else if (warp >= 2) {
    // drain warps
    const int q = warp & 3;            // TMEM lane quarter
    const int cq = (warp - 2) >> 2;     // 32-column quarter of the tile
    float hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) hi[i] = lo[i] = 0.f;
    bool ok = true;
    for (int r = 0; r < nruns; ++r) {
      const int p = r / runs_pp;
      const int b = r & 1;
      if (!mbar_wait(&afull[b], (r >> 1) & 1)) {
        ok = false;
        break;
      }
      fence_after();
      const float sc = exp2f(-(float)(SLICE_BITS * (c_si[p] + c_sj[p] + 2)));
      const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) +
                            (uint32_t)(b * SBN + cq * 32);
#pragma unroll
      for (int c2 = 0; c2 < 2; ++c2) {
        float v[16];
        tmem_ld16(base + 16 * c2, v);
#pragma unroll
        for (int i = 0; i < 16; ++i)
          ff_add(hi[16 * c2 + i], lo[16 * c2 + i], v[i] * sc);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                         smem_u32(&aempty[b]))
                     : "memory");
      }
    }
    if (!ok || fail) {
      if (lane == 0) atomicExch(err, fail ? fail : 3);
    } else {
      const int m = m0 + q * 32 + lane;
      if (m < M) {
        const int64_t ro = part ? 0 : vrow(C, m);
        const double em = ldexp(1.0, eA[m]);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int n = (n0 + cq * 32) / 2 + i;
          if (n < N) {
            const double s = alpha * em * ldexp(1.0, eB[n]);
            cplx o = cmake(s * ((double)hi[2 * i] + (double)lo[2 * i]),
                           s * ((double)hi[2 * i + 1] + (double)lo[2 * i + 1]));
            if (part) {
              part[((int64_t)z * M + m) * N + n] = o;
              continue;
            }
            cplx* d = C.p + ro + vcol(C, n);
            if (beta != 0.0) {
              cplx old = *d;
              o.x += beta * old.x;
              o.y += beta * old.y;
            }
            *d = o;
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(
                     tmem),
                 "r"(2 * SBN));
}

// Exponents and slices work on the IEEE bits with integer arithmetic (this
// GPU runs FP64 at a small fraction of its integer and FP32 rates).  For a
// normal double the biased exponent field E gives |x| < 2^(E - 1022); zeros
// and subnormals count as 0.

__device__ __forceinline__ int exp_field(double x) {
  return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// column offset of a view for an int column index (32-bit index math)
__device__ __forceinline__ int64_t vcol32(const View& v, int c) {
  if (v.c_lo == INT32_MAX) return (int64_t)c * v.cs_lo;
  const int h = c / v.c_lo;
  return (int64_t)h * v.cs_hi + (int64_t)(c - h * v.c_lo) * v.cs_lo;
}

// Exponents over [k0, k0 + K): e with max |re|, |im| < 2^e for every
// element of a row of A (row_exp) or a column of B (col_exp); an all-zero
// line gets -1022.  A warp takes one (line, K segment of EXP_SEG) task and
// folds its maximum into e[] with atomicMax, so an operand with few lines
// and a K in the millions still spreads over every SM; the caller presets
// e[] below -1022 (bytes 0x80).
constexpr int EXP_SEG = 4096;
__global__ void row_exp_kernel(View A, int M, int K, int k0, int* e) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nsg = (K + EXP_SEG - 1) / EXP_SEG;
  const int64_t ntask = (int64_t)M * nsg;
  for (int64_t t = warp; t < ntask; t += nwarp) {
    const int m = (int)(t / nsg), k1 = (int)(t % nsg) * EXP_SEG;
    const int k2 = min(K, k1 + EXP_SEG);
    const int64_t ro = vrow(A, m);
    int mx = 0;
    for (int k = k1 + lane; k < k2; k += 32) {
      const cplx a = A.p[ro + vcol32(A, k0 + k)];
      mx = max(mx, max(exp_field(a.x), exp_field(a.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) atomicMax(e + m, mx - 1022);
  }
}

__global__ void col_exp_kernel(View B, int K, int k0, int N, int* e) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nsg = (K + EXP_SEG - 1) / EXP_SEG;
  const int64_t ntask = (int64_t)N * nsg;
  for (int64_t t = warp; t < ntask; t += nwarp) {
    const int n = (int)(t / nsg), k1 = (int)(t % nsg) * EXP_SEG;
    const int k2 = min(K, k1 + EXP_SEG);
    const int64_t co = vcol(B, n);
    int mx = 0;
    for (int k = k1 + lane; k < k2; k += 32) {
      const cplx b = B.p[vrow(B, k0 + k) + co];
      mx = max(mx, max(exp_field(b.x), exp_field(b.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) atomicMax(e + n, mx - 1022);
  }
}

unsigned warp_tasks_grid(int64_t lines, int K, int seg) {
  const int64_t ntask = lines * ((K + seg - 1) / seg);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>((ntask + 7) / 8, 152 * 32));
}

// S balanced 7-bit slices of t = x 2^-e (|t| < 1): T = round(t 2^(7S))
// in integer arithmetic, then digits q_{S-1} .. q_1 in [-64, 63] from the
// bottom and q_0 = the rest, in [-128, 128], so that
// t = sum_i q_i 2^(-7(i+1)) + r with |r| <= 2^(-7S-1); each q_i is exact
// in bf16.
template <int S>
__device__ __forceinline__ void slices(double x, int e, __nv_bfloat16* q) {
  const long long bits = __double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long T = 0;
  if (E != 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = E - 1075 - e + SLICE_BITS * S;
    if (sh >= 0)
      T = m << sh;
    else if (sh > -63)
      T = (m + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) T = -T;
  }
#pragma unroll
  for (int i = S - 1; i > 0; --i) {
    const long long d = ((T + 64) & 127) - 64;
    q[i] = __float2bfloat16_rn((float)d);
    T = (T - d) >> SLICE_BITS;
  }
  q[0] = __float2bfloat16_rn((float)T);
}

// A' [Mp][2 npairs Kp]: row m, segment 2p + {0: re, 1: im} of slice c_si[p].
// A warp takes one (row, K segment of PACK_SEG) task; a lane packs two
// adjacent k into bf16 pairs (4-byte stores).
constexpr int PACK_SEG = 2048;
__device__ __forceinline__ void ld_pair(const View& A, int64_t ro, bool live, int K,
                                        int k0, int k, cplx& a0, cplx& a1) {
  a0 = a1 = cmake(0, 0);
  if (!live) return;
  if (k < K) a0 = A.p[ro + vcol32(A, k0 + k)];
  if (k + 1 < K) a1 = A.p[ro + vcol32(A, k0 + k + 1)];
  if (A.conj) {
    a0.y = -a0.y;
    a1.y = -a1.y;
  }
}

template <int S>
__global__ void slice_pack_a(View A, int M, int K, int k0, int Mp, int Kp,
                             int npairs, const int* __restrict__ eA,
                             __nv_bfloat16* out) {
  const int64_t ld = (int64_t)2 * npairs * Kp;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nsg = (Kp + PACK_SEG - 1) / PACK_SEG;
  const int64_t ntask = (int64_t)Mp * nsg;
  for (int64_t t = warp; t < ntask; t += nwarp) {
    const int m = (int)(t / nsg), k1 = (int)(t % nsg) * PACK_SEG;
    const int k2 = min(Kp, k1 + PACK_SEG);
    const bool live = m < M;
    const int64_t ro = live ? vrow(A, m) : 0;
    const int e = live ? eA[m] : 0;
    __nv_bfloat16* o = out + (int64_t)m * ld;
    for (int k = k1 + 2 * lane; k < k2; k += 64) {
      cplx a0, a1;
      ld_pair(A, ro, live, K, k0, k, a0, a1);
      __nv_bfloat16 r0[S], i0[S], r1[S], i1[S];
      slices<S>(a0.x, e, r0);
      slices<S>(a0.y, e, i0);
      slices<S>(a1.x, e, r1);
      slices<S>(a1.y, e, i1);
      for (int p = 0; p < npairs; ++p) {
        const int q = c_si[p];
        *(__nv_bfloat162*)(o + (2 * p) * (int64_t)Kp + k) = __halves2bfloat162(r0[q], r1[q]);
        *(__nv_bfloat162*)(o + (2 * p + 1) * (int64_t)Kp + k) =
            __halves2bfloat162(i0[q], i1[q]);
      }
    }
  }
}

template <int S>
__global__ void slice_pack_b(View B, int K, int k0, int N, int Np2, int Kp,
                             int npairs, const int* __restrict__ eB,
                             __nv_bfloat16* out) {
  const int64_t ld = (int64_t)2 * npairs * Kp;
  const int64_t total = (int64_t)(Np2 / 2) * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int n = idx / Kp, k = idx % Kp;
    cplx b = cmake(0, 0);
    int e = 0;
    if (n < N) {
      e = eB[n];
      if (k < K) {
        b = B.p[vrow(B, k0 + k) + vcol(B, n)];
        if (B.conj) b.y = -b.y;
      }
    }
    __nv_bfloat16 re[S], im[S];
    slices<S>(b.x, e, re);
    slices<S>(b.y, e, im);
    __nv_bfloat16* o0 = out + (int64_t)(2 * n) * ld + k;
    __nv_bfloat16* o1 = o0 + ld;
    for (int p = 0; p < npairs; ++p) {
      const int j = c_sj[p];
      o0[(2 * p) * (int64_t)Kp] = re[j];
      o0[(2 * p + 1) * (int64_t)Kp] = __hneg(im[j]);
      o1[(2 * p) * (int64_t)Kp] = im[j];
      o1[(2 * p + 1) * (int64_t)Kp] = re[j];
    }
  }
}

// ---------------------------------------------------------------------------
// SLICE4 with slice reuse.  The packed operands hold each slice once: A''
// row m = 8 segments (slice i, re / im) of Kp values; B'' rows 2n (the real
// output column) and 2n+1 (the imaginary one) = 8 segments (slice j,
// re-part / im-part: [re b, -im b] for row 2n and [im b, re b] for row
// 2n+1).  One pipeline stage is one K block of 64 in one part c (re or im):
// the four A tiles A_{i,c} (128 x 64) and four B tiles B_{j,c} (64 x 64),
// 96 KB, from which all ten slice pairs are issued.  Pairs of one order
// o = i + j share the scale 2^{-7(o+2)} and one tensor-memory accumulator;
// a run is 2 K blocks x 2 parts: at most 4 pairs x 256 products of
// |q q'| <= 2^13 (2^14 for order 0, one pair) per element, so every run
// sums exactly in FP32.  TMEM: 2 buffers x 4 orders x 64 columns = 512.
// The B tiles of a stage lie back to back (one 256-row K-major operand) and
// the orders of a buffer side by side, so the pairs (i, 0..3-i) are one MMA
// of A_i with B_0..B_{3-i} (N = 64 (4 - i)) into orders i..3: four MMAs
// per K step instead of ten, and each A tile is read from shared memory
// once.  The drain adds each order, times its scale, to float-float
// accumulators.
//
// CTA: 576 threads, tile 128 x 64 (N' = 64: 32 complex columns).  Warp 0
// lane 0: TMA producer; warp 1 lane 0: MMA issuer; warps 2..17: drain (warp
// w reads TMEM lanes 32 (w % 4) .. +31 and the 16 columns [16 c, 16 c + 16),
// c = (w - 2) / 4, of every order).
// ---------------------------------------------------------------------------
constexpr int RBN = 64;                  // N' per CTA
constexpr int R_A_TILE = BM * BK * 2;    // 16 KB
constexpr int R_B_TILE = RBN * BK * 2;   // 8 KB
constexpr int R_STAGE = 4 * R_A_TILE + 4 * R_B_TILE;  // 96 KB
constexpr int R_STAGES = 2;
constexpr int R_SMEM = R_STAGES * R_STAGE + 1024 + 512;
constexpr int R_RUN = 4;                 // units (K block, part) per exact run

__global__ void __launch_bounds__(576, 1)
    tc_slice4r_kernel(const __grid_constant__ CUtensorMap tmA,
                      const __grid_constant__ CUtensorMap tmB, int kpa, int ka_off,
                      int kpb, int kb_off, int nkb, int zl, int M, int N,
                      const int* __restrict__ eA,
                      const int* __restrict__ eB, double alpha, double beta,
                      View C, cplx* part, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + R_STAGES * R_STAGE);
  uint64_t* empty = full + R_STAGES;
  uint64_t* afull = empty + R_STAGES;  // [2]
  uint64_t* aempty = afull + 2;        // [2]
  uint32_t* tslot = (uint32_t*)(aempty + 2);
  __shared__ int fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int mt, nt;
  tile_coords(mt, nt);
  const int m0 = mt * BM, n0 = nt * RBN;
  const int z = blockIdx.z;
  // this CTA's K blocks [kb0, kb1); units u = 2 (kb - kb0) + c
  const int kb0 = z * zl, kb1 = min(nkb, kb0 + zl);
  const int nunits = 2 * max(0, kb1 - kb0);
  const int nruns = (nunits + R_RUN - 1) / R_RUN;

  if (threadIdx.x == 0) {
    fail = 0;
    for (int s = 0; s < R_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&afull[b], 1);
      mbar_init(&aempty[b], 16);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
            smem_u32(tslot)),
        "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tslot;

  if (threadIdx.x == 0) {
    // TMA producer: unit u -> K block kb0 + u / 2, part c = u % 2
    for (int u = 0; u < nunits; ++u) {
      const int s = u % R_STAGES;
      const uint32_t ph = (u / R_STAGES) & 1;
      if (u >= R_STAGES && !mbar_wait(&empty[s], ph ^ 1)) {
        fail = 1;
        break;
      }
      if (fail) break;
      const int kb = kb0 + u / 2, c = u & 1;
      uint8_t* st = smem + s * R_STAGE;
      mbar_expect_tx(&full[s], R_STAGE);
#pragma unroll
      for (int i = 0; i < 4; ++i)
        tma_load(&tmA, &full[s], st + i * R_A_TILE, (2 * i + c) * kpa + (ka_off + kb) * BK,
                 m0);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        tma_load(&tmB, &full[s], st + 4 * R_A_TILE + j * R_B_TILE,
                 (2 * j + c) * kpb + (kb_off + kb) * BK, n0);
    }
  } else if (threadIdx.x == 32) {
    // MMA issuer: for each unit, the ten pairs into their order's
    // accumulator of the run's buffer
    // N = 64 (4 - i) for the MMA of A_i
    uint32_t idn[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) idn[i] = idesc_bf16(BM, RBN * (4 - i));
    for (int r = 0; r < nruns && !fail; ++r) {
      const int b = r & 1;
      if (r >= 2 && !mbar_wait(&aempty[b], ((r >> 1) + 1) & 1)) {
        fail = 4;
        break;
      }
      fence_after();
      const int u0 = r * R_RUN, u1 = min(nunits, u0 + R_RUN);
      for (int u = u0; u < u1; ++u) {
        const int s = u % R_STAGES;
        const uint32_t ph = (u / R_STAGES) & 1;
        if (!mbar_wait(&full[s], ph)) {
          fail = 2;
          break;
        }
        fence_after();
        const uint32_t st = smem_u32(smem + s * R_STAGE);
        const uint64_t bd = sdesc(st + 4 * R_A_TILE);  // B_0 .. B_3
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          // pairs (i, 0 .. 3 - i) into orders i .. 3; the first MMA of a
          // run (i = 0 covers every order) starts the accumulators
          const uint32_t dt = tmem + (uint32_t)((b * 4 + i) * RBN);
          const uint64_t ad = sdesc(st + i * R_A_TILE);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            umma(dt, ad + 2 * kk, bd + 2 * kk, idn[i],
                 (u != u0 || i != 0 || kk != 0) ? 1u : 0u);
        }
        umma_commit(&empty[s]);
      }
      umma_commit(&afull[b]);
    }
  } else if (warp >= 2) {
    // drain warps
    const int q = warp & 3;          // TMEM lane quarter
    const int cq = (warp - 2) >> 2;  // 16-column chunk of the 64
    float hi[16], lo[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) hi[i] = lo[i] = 0.f;
    bool ok = true;
    for (int r = 0; r < nruns; ++r) {
      const int b = r & 1;
      if (!mbar_wait(&afull[b], (r >> 1) & 1)) {
        ok = false;
        break;
      }
      fence_after();
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        const float sc = exp2f(-(float)(SLICE_BITS * (o + 2)));
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((b * 4 + o) * RBN + cq * 16), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) ff_add(hi[i], lo[i], v[i] * sc);
      }
      fence_before();
      __syncwarp();
      if (lane == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&aempty[b]))
                     : "memory");
      }
    }
    if (!ok || fail) {
      if (lane == 0) atomicExch(err, fail ? fail : 3);
    } else {
      const int m = m0 + q * 32 + lane;
      if (m < M) {
        const int64_t ro = part ? 0 : vrow(C, m);
        const double em = ldexp(1.0, eA[m]);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int n = (n0 + cq * 16) / 2 + i;
          if (n < N) {
            const double sc = alpha * em * ldexp(1.0, eB[n]);
            cplx o = cmake(sc * ((double)hi[2 * i] + (double)lo[2 * i]),
                           sc * ((double)hi[2 * i + 1] + (double)lo[2 * i + 1]));
            if (part) {
              part[((int64_t)z * M + m) * N + n] = o;
              continue;
            }
            cplx* d = C.p + ro + vcol(C, n);
            if (beta != 0.0) {
              const cplx old = *d;
              o.x += beta * old.x;
              o.y += beta * old.y;
            }
            *d = o;
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// A'' [Mp][8 Kp]: segment 2 i + {0: re, 1: im} holds slice i; tasks as in
// slice_pack_a
__global__ void slice4r_pack_a(View A, int M, int K, int k0, int Mp, int Kp,
                               const int* __restrict__ eA, __nv_bfloat16* out) {
  const int64_t ld = (int64_t)8 * Kp;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nsg = (Kp + PACK_SEG - 1) / PACK_SEG;
  const int64_t ntask = (int64_t)Mp * nsg;
  for (int64_t t = warp; t < ntask; t += nwarp) {
    const int m = (int)(t / nsg), k1 = (int)(t % nsg) * PACK_SEG;
    const int k2 = min(Kp, k1 + PACK_SEG);
    const bool live = m < M;
    const int64_t ro = live ? vrow(A, m) : 0;
    const int e = live ? eA[m] : 0;
    __nv_bfloat16* o = out + (int64_t)m * ld;
    for (int k = k1 + 2 * lane; k < k2; k += 64) {
      cplx a0, a1;
      ld_pair(A, ro, live, K, k0, k, a0, a1);
      __nv_bfloat16 r0[4], i0[4], r1[4], i1[4];
      slices<4>(a0.x, e, r0);
      slices<4>(a0.y, e, i0);
      slices<4>(a1.x, e, r1);
      slices<4>(a1.y, e, i1);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        *(__nv_bfloat162*)(o + (2 * i) * (int64_t)Kp + k) = __halves2bfloat162(r0[i], r1[i]);
        *(__nv_bfloat162*)(o + (2 * i + 1) * (int64_t)Kp + k) = __halves2bfloat162(i0[i], i1[i]);
      }
    }
  }
}

// B'' [Np2][8 Kp]: rows 2n and 2n + 1, segment 2 j + {0, 1} of slice j
__global__ void slice4r_pack_b(View B, int K, int k0, int N, int Np2, int Kp,
                               const int* __restrict__ eB, __nv_bfloat16* out) {
  const int64_t ld = (int64_t)8 * Kp;
  const int64_t total = (int64_t)(Np2 / 2) * Kp;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(idx / Kp), k = (int)(idx % Kp);
    cplx b = cmake(0, 0);
    int e = 0;
    if (n < N) {
      e = eB[n];
      if (k < K) {
        b = B.p[vrow(B, k0 + k) + vcol(B, n)];
        if (B.conj) b.y = -b.y;
      }
    }
    __nv_bfloat16 re[4], im[4];
    slices<4>(b.x, e, re);
    slices<4>(b.y, e, im);
    __nv_bfloat16* o0 = out + (int64_t)(2 * n) * ld + k;
    __nv_bfloat16* o1 = o0 + ld;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      o0[(2 * j) * (int64_t)Kp] = re[j];
      o0[(2 * j + 1) * (int64_t)Kp] = __hneg(im[j]);
      o1[(2 * j) * (int64_t)Kp] = im[j];
      o1[(2 * j + 1) * (int64_t)Kp] = re[j];
    }
  }
}

// packed geometry: SLICE4 packs each slice once (8 segments, N' tiles of
// 64, the slice-reuse kernel); SLICE7 packs one segment pair per slice pair
// (56 segments, N' tiles of 128).  K runs in chunks of kc so that the packs
// of a chunk stay within PACK_BUDGET; a B operand held in a cache is packed
// once over its whole K (KpF) and only A's pack counts against the budget.
struct SDims {
  int Mp, Np2, npairs, nseg, kc, KpF;
  size_t a_bytes, b_bytes, e_bytes;
};
SDims sdims_of(int M, int N, int K, int nslices, bool b_cached, bool a_cached = false) {
  SDims d;
  const int tn = nslices == 4 ? RBN : SBN;
  d.Mp = (M + BM - 1) / BM * BM;
  d.Np2 = (2 * N + tn - 1) / tn * tn;
  d.npairs = nslices * (nslices + 1) / 2;
  d.nseg = nslices == 4 ? 8 : 2 * d.npairs;
  d.KpF = (int)(((int64_t)K + BK - 1) / BK * BK);
  const size_t per_k = (size_t)((a_cached ? 0 : d.Mp) + (b_cached ? 0 : d.Np2)) * d.nseg * 2;
  int64_t kc = per_k ? (int64_t)(PACK_BUDGET / per_k) / BK * BK : (int64_t)d.KpF;
  kc = std::max<int64_t>(kc, BK);
  d.kc = (int)std::min<int64_t>(kc, d.KpF);
  d.a_bytes = a_cached ? 0 : (size_t)d.Mp * d.nseg * d.kc * 2;
  d.b_bytes = b_cached ? 0 : (size_t)d.Np2 * d.nseg * d.kc * 2;
  d.e_bytes = ((size_t)d.Mp + d.Np2 / 2 + 64) * sizeof(int);
  return d;
}

}  // namespace

void wait_probe(cudaStream_t s, int64_t limit_ns, int* err) {
  const uint64_t lim = (uint64_t)std::min<int64_t>(std::max<int64_t>(limit_ns, 1000000),
                                                   (int64_t)WAIT_NS);
  wait_probe_kernel<<<1, 32, 0, s>>>(lim, err);
  CVS_CHECK_LAUNCH();
}

size_t slice_workspace_bytes(int M, int N, int K, int nslices, bool b_cached, bool a_cached) {
  SDims d = sdims_of(M, N, K, nslices, b_cached, a_cached);
  return d.a_bytes + d.b_bytes + d.e_bytes + 256;
}

size_t slice_acache_bytes(int M, int K, int nslices) {
  SDims d = sdims_of(M, 1, K, nslices, true, true);
  return (size_t)d.Mp * d.nseg * d.KpF * 2 + (size_t)d.Mp * sizeof(int) + 256;
}

size_t slice_bcache_bytes(int N, int K, int nslices) {
  SDims d = sdims_of(1, N, K, nslices, true);
  return (size_t)d.Np2 * d.nseg * d.KpF * 2 + ((size_t)d.Np2 / 2 + 64) * sizeof(int) + 256;
}

int64_t slice_row_slab(int M, int N, int K, int nslices) {
  SDims d = sdims_of(M, N, K, nslices, false);
  if (d.kc >= d.KpF) return M;  // K is whole already
  const size_t per_row = (size_t)d.nseg * d.KpF * 2;
  const size_t bfull = (size_t)d.Np2 * d.nseg * d.KpF * 2;
  if (bfull >= PACK_BUDGET / 2) return M;
  const int64_t rows = (int64_t)((PACK_BUDGET - bfull) / per_row) / BM * BM;
  return rows >= 16 * BM ? rows : M;
}

void zgemm_slice(cudaStream_t s, int nslices, int M, int N, int K,
                 double alpha, View A, View B, double beta, View C, void* work,
                 size_t work_bytes, cplx* part, size_t part_elems, int* err,
                 SliceBCache* bc, SliceBCache* ac) {
  if (M <= 0 || N <= 0) return;
  CVS_REQUIRE(nslices == 4 || nslices == 7, -1, "zgemm_slice: 4 or 7 slices");
  CVS_REQUIRE(!ac || nslices == 4, -1, "zgemm_slice: cached A needs 4 slices");
  SDims d = sdims_of(M, N, K, nslices, bc != nullptr, ac != nullptr);
  CVS_REQUIRE(work_bytes >= d.a_bytes + d.b_bytes + d.e_bytes, -1,
              "zgemm_slice: workspace too small");
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(tc_slice_kernel,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, S_SMEM);
    cudaFuncSetAttribute(tc_slice4r_kernel,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, R_SMEM);
  });
  __nv_bfloat16* ap = (__nv_bfloat16*)work;
  __nv_bfloat16* bp = (__nv_bfloat16*)((char*)work + d.a_bytes);
  int* eA = (int*)((char*)work + d.a_bytes + d.b_bytes);
  int* eB = eA + d.Mp;
  const bool reuse = nslices == 4;
  const int64_t tiles = (int64_t)(d.Np2 / (reuse ? RBN : SBN)) * (d.Mp / BM);
  const size_t eb_n = (size_t)d.Np2 / 2 + 64;
  const size_t bfull = (size_t)d.Np2 * d.nseg * d.KpF * 2;
  if (bc) {
    // the cached B: packed once over the whole K, with whole-column exponents
    CVS_REQUIRE(bc->bytes >= bfull + eb_n * sizeof(int), -1, "zgemm_slice: B cache too small");
    if (!bc->filled) {
      int* ec = (int*)((char*)bc->base + bfull);
      __nv_bfloat16* bq = (__nv_bfloat16*)bc->base;
      CVS_CUDA(cudaMemsetAsync(ec, 0x80, eb_n * sizeof(int), s));
      col_exp_kernel<<<warp_tasks_grid(N, K, EXP_SEG), 256, 0, s>>>(B, K, 0, N, ec);
      CVS_CHECK_LAUNCH();
      const unsigned gb = grid1d((int64_t)(d.Np2 / 2) * d.KpF, 256);
      if (reuse)
        slice4r_pack_b<<<gb, 256, 0, s>>>(B, K, 0, N, d.Np2, d.KpF, ec, bq);
      else
        slice_pack_b<7><<<gb, 256, 0, s>>>(B, K, 0, N, d.Np2, d.KpF, d.npairs, ec, bq);
      CVS_CHECK_LAUNCH();
      bc->filled = true;
    }
  }
  // the cached A: packed once over the whole K, with whole-row exponents
  const size_t afull = (size_t)d.Mp * d.nseg * d.KpF * 2;
  if (ac) {
    CVS_REQUIRE(ac->bytes >= afull + (size_t)d.Mp * sizeof(int), -1,
                "zgemm_slice: A cache too small");
    if (!ac->filled) {
      int* ea = (int*)((char*)ac->base + afull);
      CVS_CUDA(cudaMemsetAsync(ea, 0x80, (size_t)d.Mp * sizeof(int), s));
      row_exp_kernel<<<warp_tasks_grid(M, K, EXP_SEG), 256, 0, s>>>(A, M, K, 0, ea);
      CVS_CHECK_LAUNCH();
      slice4r_pack_a<<<warp_tasks_grid(d.Mp, d.KpF, PACK_SEG), 256, 0, s>>>(
          A, M, K, 0, d.Mp, d.KpF, ea, (__nv_bfloat16*)ac->base);
      CVS_CHECK_LAUNCH();
      ac->filled = true;
    }
  }
  for (int k0 = 0; k0 < K; k0 += d.kc) {
    const int Kc = std::min(d.kc, K - k0);
    const int Kp = (Kc + BK - 1) / BK * BK;
    // B's packed slices and exponents: the cache (whole K; this chunk starts
    // at K block k0 / BK of each segment of KpF) or this chunk's packs in
    // the workspace
    const __nv_bfloat16* bpc = bc ? (const __nv_bfloat16*)bc->base : bp;
    const int* eBc = bc ? (const int*)((const char*)bc->base + bfull) : eB;
    const int kpb = bc ? d.KpF : Kp, kb_off = bc ? k0 / BK : 0;
    // A's packed slices and exponents: the cache (whole K) or this chunk's
    const __nv_bfloat16* apc = ac ? (const __nv_bfloat16*)ac->base : ap;
    const int* eAc = ac ? (const int*)((const char*)ac->base + afull) : eA;
    const int kpa = ac ? d.KpF : Kp, ka_off = ac ? k0 / BK : 0;
    if (!ac) {
      CVS_CUDA(cudaMemsetAsync(eA, 0x80, (size_t)d.Mp * sizeof(int), s));
      row_exp_kernel<<<warp_tasks_grid(M, Kc, EXP_SEG), 256, 0, s>>>(A, M, Kc, k0, eA);
      CVS_CHECK_LAUNCH();
    }
    if (!bc) {
      CVS_CUDA(cudaMemsetAsync(eB, 0x80, eb_n * sizeof(int), s));
      col_exp_kernel<<<warp_tasks_grid(N, Kc, EXP_SEG), 256, 0, s>>>(B, Kc, k0, N, eB);
      CVS_CHECK_LAUNCH();
    }
    const unsigned ga = warp_tasks_grid(d.Mp, Kp, PACK_SEG);
    const unsigned gb = grid1d((int64_t)(d.Np2 / 2) * Kp, 256);
    if (reuse) {
      if (!ac) {
        slice4r_pack_a<<<ga, 256, 0, s>>>(A, M, Kc, k0, d.Mp, Kp, eA, ap);
        CVS_CHECK_LAUNCH();
      }
      if (!bc) {
        slice4r_pack_b<<<gb, 256, 0, s>>>(B, Kc, k0, N, d.Np2, Kp, eB, bp);
        CVS_CHECK_LAUNCH();
      }
    } else {
      slice_pack_a<7><<<ga, 256, 0, s>>>(A, M, Kc, k0, d.Mp, Kp, d.npairs, eA, ap);
      CVS_CHECK_LAUNCH();
      if (!bc) {
        slice_pack_b<7><<<gb, 256, 0, s>>>(B, Kc, k0, N, d.Np2, Kp, d.npairs, eB, bp);
        CVS_CHECK_LAUNCH();
      }
    }
    const int64_t kcols = (int64_t)d.nseg * Kp, kcols_b = (int64_t)d.nseg * kpb;
    const double beta_c = (k0 == 0) ? beta : 1.0;
    if (reuse) {
      CUtensorMap ma = make_map(apc, d.Mp, (int64_t)d.nseg * kpa, BM);
      CUtensorMap mb = make_map(bpc, d.Np2, kcols_b, RBN);
      const int nkb = Kp / BK;  // K blocks; a run spans two
      int sp = tc_splits(tiles, nkb, 2 * (R_RUN / 2));
      if (part == nullptr || (size_t)sp * M * N > part_elems) sp = 1;
      const int zl = (nkb + sp - 1) / sp;
      const int nz = (nkb + zl - 1) / zl;
      dim3 grid(d.Np2 / RBN, d.Mp / BM, nz);
      const int tok = kstats_begin(s, K_TC_SLICE, 8.0 * M * N * (double)Kc);
      tc_slice4r_kernel<<<grid, 576, R_SMEM, s>>>(ma, mb, kpa, ka_off, kpb, kb_off, nkb, zl,
                                                  M, N, eAc, eBc, alpha, beta_c, C,
                                                  nz > 1 ? part : nullptr, err);
      CVS_CHECK_LAUNCH();
      kstats_end(s, tok);
      if (nz > 1) splitk_reduce(s, M, N, nz, part, beta_c, C);
      continue;
    }
    CUtensorMap ma = make_map(ap, d.Mp, kcols, BM);
    CUtensorMap mb = make_map(bpc, d.Np2, kcols_b, SBN);
    const int ktpp = 2 * Kp / BK;
    int sp = tc_splits(tiles, ktpp, RUN_KT);
    if (part == nullptr || (size_t)sp * M * N > part_elems) sp = 1;
    const int zl = (ktpp + sp - 1) / sp;
    const int nz = (ktpp + zl - 1) / zl;
    dim3 grid(d.Np2 / SBN, d.Mp / BM, nz);
    const int tok = kstats_begin(s, K_TC_SLICE, 8.0 * M * N * (double)Kc);
    tc_slice_kernel<<<grid, 576, S_SMEM, s>>>(ma, mb, d.npairs, ktpp, kpb, kb_off, zl, M, N,
                                              eA, eBc, alpha, beta_c, C,
                                              nz > 1 ? part : nullptr, err);
    CVS_CHECK_LAUNCH();
    kstats_end(s, tok);
    if (nz > 1) splitk_reduce(s, M, N, nz, part, beta_c, C);
  }
}

}  // namespace cvs
