// Complex FP64 GEMM on the CUDA cores (FP64 FMA), C = alpha*A*B + beta*C,
// for matrices given as two-mode strided views (common.cuh).  This is the
// arithmetic of the FP64 path: every contraction of t2, M11 and the sigma
// vector goes through it when precision = CVSADC_FP64.
//
// Tile 64x64x8, 256 threads, 4x4 complex outputs per thread, register
// prefetch of the next K tile.  Loads are mapped so that consecutive
// threads follow whichever mode of the operand has unit stride.
#include "common.cuh"
#include "kernels.cuh"

namespace cvs {

namespace {
constexpr int BM = 64, BN = 64, BK = 8;

__device__ __forceinline__ cplx ldv(const cplx* p, int conj) {
  cplx v = __ldg(p);
  if (conj) v.y = -v.y;
  return v;
}

__global__ void __launch_bounds__(256)
    zgemm_f64_kernel(int M, int N, int K, double alpha, View A, View B,
                     double beta, View C, int a_kfast, int b_kfast) {
  __shared__ cplx As[BK][BM];
  __shared__ cplx Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int64_t z = blockIdx.z;
  const cplx* Ap = A.p + z * A.batch;
  const cplx* Bp = B.p + z * B.batch;
  cplx* Cp = C.p + z * C.batch;

  // load assignment: 2 elements of each tile per thread
  int am[2], ak[2], bk[2], bn[2];
  int64_t aro[2], bco[2];
  bool aok[2], bok[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    int idx = tid + e * 256;
    if (a_kfast) {
      am[e] = idx / BK;
      ak[e] = idx % BK;
    } else {
      am[e] = idx % BM;
      ak[e] = idx / BM;
    }
    if (b_kfast) {
      bn[e] = idx / BK;
      bk[e] = idx % BK;
    } else {
      bn[e] = idx % BN;
      bk[e] = idx / BN;
    }
    aok[e] = (m0 + am[e]) < M;
    bok[e] = (n0 + bn[e]) < N;
    aro[e] = aok[e] ? vrow(A, m0 + am[e]) : 0;
    bco[e] = bok[e] ? vcol(B, n0 + bn[e]) : 0;
  }

  cplx ra[2], rb[2];
  auto load = [&](int k0) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      int ka = k0 + ak[e];
      ra[e] = (aok[e] && ka < K) ? ldv(Ap + aro[e] + vcol(A, ka), A.conj)
                                 : cmake(0, 0);
      int kb = k0 + bk[e];
      rb[e] = (bok[e] && kb < K) ? ldv(Bp + vrow(B, kb) + bco[e], B.conj)
                                 : cmake(0, 0);
    }
  };
  auto store = [&]() {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      As[ak[e]][am[e]] = ra[e];
      Bs[bk[e]][bn[e]] = rb[e];
    }
  };

  double accr[4][4], acci[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accr[i][j] = acci[i][j] = 0.0;

  const int ntiles = (K + BK - 1) / BK;
  load(0);
  store();
  __syncthreads();
  for (int t = 0; t < ntiles; ++t) {
    if (t + 1 < ntiles) load((t + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      cplx a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          accr[i][j] = fma(a[i].x, b[j].x, accr[i][j]);
          accr[i][j] = fma(-a[i].y, b[j].y, accr[i][j]);
          acci[i][j] = fma(a[i].x, b[j].y, acci[i][j]);
          acci[i][j] = fma(a[i].y, b[j].x, acci[i][j]);
        }
    }
    __syncthreads();
    if (t + 1 < ntiles) {
      store();
      __syncthreads();
    }
  }

#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int r = m0 + ty + 16 * i;
    if (r >= M) continue;
    int64_t ro = vrow(C, r);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = n0 + tx + 16 * j;
      if (c >= N) continue;
      cplx* dst = Cp + ro + vcol(C, c);
      cplx v = cmake(alpha * accr[i][j], alpha * acci[i][j]);
      if (beta != 0.0) {
        cplx o = *dst;
        v.x += beta * o.x;
        v.y += beta * o.y;
      }
      *dst = v;
    }
  }
}
}  // namespace

void zgemm_f64(cudaStream_t s, int M, int N, int K, double alpha, View A,
               View B, double beta, View C, int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // C = beta * C
    scale_view(s, M, N, beta, C, batch);
    return;
  }
  int a_kfast = (A.cs_lo == 1) ? 1 : 0;
  int b_kfast = (B.rs_lo == 1) ? 1 : 0;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  zgemm_f64_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, B, beta, C,
                                        a_kfast, b_kfast);
  CVS_CHECK_LAUNCH();
}

}  // namespace cvs
