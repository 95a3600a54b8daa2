// Complex FP64 GEMM on the CUDA cores (FP64 FMA), C = alpha*A*B + beta*C,
// for matrices given as two-mode strided views (common.cuh).  This is the
// arithmetic of the FP64 path: every contraction of t2, M11 and the sigma
// vector goes through it when precision = CVSADC_FP64, and the small
// contractions of every precision do.
//
// Tile kernel: 64x64x8 tiles, 256 threads, 4x4 complex outputs per thread,
// register prefetch of the next K tile; loads follow whichever mode of the
// operand has unit stride.  Outputs with few tiles and a long K are split
// along K (each z-slice writes alpha * partial product to a dense buffer,
// a reduction adds them and beta * C).
//
// Small-output kernel: for M*N <= 4096 and a long K (e.g. the ncore x ncore
// and ncore x nvirt intermediates, K up to 10^6-10^7) every block takes a K
// chunk, stages A and B slices in shared memory and accumulates all M*N
// dot products; the partials are reduced the same way.
#include <algorithm>

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

// part == nullptr: z is the batch index (operand batch strides), full K.
// part != nullptr: z is a K slice [z*kchunk, (z+1)*kchunk); alpha * the
// partial product goes to part[z][M][N].
__global__ void __launch_bounds__(256)
    zgemm_f64_kernel(int M, int N, int K, double alpha, View A, View B,
                     double beta, View C, int a_kfast, int b_kfast,
                     int kchunk, cplx* part) {
  __shared__ cplx As[BK][BM];
  __shared__ cplx Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int64_t z = blockIdx.z;
  const cplx* Ap = A.p;
  const cplx* Bp = B.p;
  cplx* Cp = C.p;
  int kb = 0, ke = K;
  if (part) {
    kb = (int)(z * kchunk);
    ke = min(K, kb + kchunk);
  } else {
    Ap += z * A.batch;
    Bp += z * B.batch;
    Cp += z * C.batch;
  }

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
      ra[e] = (aok[e] && ka < ke) ? ldv(Ap + aro[e] + vcol(A, ka), A.conj)
                                  : cmake(0, 0);
      int kb2 = k0 + bk[e];
      rb[e] = (bok[e] && kb2 < ke) ? ldv(Bp + vrow(B, kb2) + bco[e], B.conj)
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

  const int ntiles = (ke - kb + BK - 1) / BK;
  if (ntiles > 0) {
    load(kb);
    store();
  }
  __syncthreads();
  for (int t = 0; t < ntiles; ++t) {
    if (t + 1 < ntiles) load(kb + (t + 1) * BK);
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
    int64_t ro = part ? 0 : vrow(C, r);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int c = n0 + tx + 16 * j;
      if (c >= N) continue;
      cplx v = cmake(alpha * accr[i][j], alpha * acci[i][j]);
      if (part) {
        part[(z * M + r) * (int64_t)N + c] = v;
        continue;
      }
      cplx* dst = Cp + ro + vcol(C, c);
      if (beta != 0.0) {
        cplx o = *dst;
        v.x += beta * o.x;
        v.y += beta * o.y;
      }
      *dst = v;
    }
  }
}

// all M*N (<= 4096) dot products over a K chunk per block
constexpr int STK = 16;
__global__ void __launch_bounds__(256)
    zgemm_smallmn_kernel(int M, int N, int K, double alpha, View A, View B,
                         int kchunk, cplx* part) {
  extern __shared__ cplx sh[];
  cplx* sa = sh;            // [M][STK]
  cplx* sb = sh + M * STK;  // [N][STK]
  const int npairs = M * N;
  const int per = (npairs + blockDim.x - 1) / blockDim.x;  // <= 16
  double ar[16], ai[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) ar[q] = ai[q] = 0.0;
  const int kb = blockIdx.x * kchunk, ke = min(K, kb + kchunk);
  for (int k0 = kb; k0 < ke; k0 += STK) {
    __syncthreads();
    for (int e = threadIdx.x; e < (M + N) * STK; e += blockDim.x) {
      int row = e / STK, kk = e % STK, k = k0 + kk;
      cplx v = cmake(0, 0);
      if (k < ke) {
        if (row < M) {
          v = A.p[vrow(A, row) + vcol(A, k)];
          if (A.conj) v.y = -v.y;
        } else {
          v = B.p[vrow(B, k) + vcol(B, row - M)];
          if (B.conj) v.y = -v.y;
        }
      }
      sh[e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (q >= per) break;
      int pr = threadIdx.x + q * blockDim.x;
      if (pr >= npairs) break;
      const cplx* x = sa + (pr / N) * STK;
      const cplx* y = sb + (pr % N) * STK;
      double sr = 0, si = 0;
#pragma unroll
      for (int kk = 0; kk < STK; ++kk) {
        sr = fma(x[kk].x, y[kk].x, sr);
        sr = fma(-x[kk].y, y[kk].y, sr);
        si = fma(x[kk].x, y[kk].y, si);
        si = fma(x[kk].y, y[kk].x, si);
      }
      ar[q] += sr;
      ai[q] += si;
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    if (q >= per) break;
    int pr = threadIdx.x + q * blockDim.x;
    if (pr >= npairs) break;
    part[(int64_t)blockIdx.x * npairs + pr] = cmake(alpha * ar[q], alpha * ai[q]);
  }
}

// C(m, n) = sum_z part[z][m][n] + beta * C(m, n)
__global__ void splitk_reduce_kernel(int M, int N, int nz, const cplx* part,
                                     double beta, View C) {
  const int64_t MN = (int64_t)M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < MN;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double sr = 0, si = 0;
    for (int z = 0; z < nz; ++z) {
      cplx v = part[z * MN + idx];
      sr += v.x;
      si += v.y;
    }
    int r = idx / N, c = idx % N;
    cplx* d = C.p + vrow(C, r) + vcol(C, c);
    if (beta != 0.0) {
      cplx o = *d;
      sr += beta * o.x;
      si += beta * o.y;
    }
    *d = cmake(sr, si);
  }
}
// C = alpha A B + beta C for a few columns (N <= GEMV_MAXN) when A's rows
// are contiguous along k: a warp per row of A, lanes along k, the N sums in
// registers; B's N columns are re-read from L2 by every row.
constexpr int GEMV_MAXN = 8;
__global__ void __launch_bounds__(256)
    zgemv_rows_kernel(int M, int N, int K, double alpha, View A, View B, double beta,
                      View C) {
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t m = warp; m < M; m += nwarp) {
    const cplx* a = A.p + vrow(A, m);
    double re[GEMV_MAXN], im[GEMV_MAXN];
#pragma unroll
    for (int q = 0; q < GEMV_MAXN; ++q) re[q] = im[q] = 0.0;
    for (int k = lane; k < K; k += 32) {
      cplx x = a[k];
      if (A.conj) x.y = -x.y;
      const int64_t bo = vrow(B, k);
#pragma unroll
      for (int q = 0; q < GEMV_MAXN; ++q) {
        if (q < N) {
          cplx y = B.p[bo + vcol(B, q)];
          if (B.conj) y.y = -y.y;
          re[q] = fma(x.x, y.x, fma(-x.y, y.y, re[q]));
          im[q] = fma(x.x, y.y, fma(x.y, y.x, im[q]));
        }
      }
    }
#pragma unroll
    for (int q = 0; q < GEMV_MAXN; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        re[q] += __shfl_xor_sync(0xffffffffu, re[q], o);
        im[q] += __shfl_xor_sync(0xffffffffu, im[q], o);
      }
    }
    if (lane < N) {
      double r = 0.0, i = 0.0;
#pragma unroll
      for (int q = 0; q < GEMV_MAXN; ++q)
        if (q == lane) {
          r = re[q];
          i = im[q];
        }
      cplx* d = C.p + vrow(C, m) + vcol(C, lane);
      cplx o = cmake(alpha * r, alpha * i);
      if (beta != 0.0) {
        const cplx old = *d;
        o.x += beta * old.x;
        o.y += beta * old.y;
      }
      *d = o;
    }
  }
}

}  // namespace

void splitk_reduce(cudaStream_t s, int M, int N, int nz, const cplx* part,
                   double beta, View C) {
  splitk_reduce_kernel<<<grid1d((int64_t)M * N, 256), 256, 0, s>>>(M, N, nz,
                                                                   part, beta, C);
  CVS_CHECK_LAUNCH();
}

int f64_splits(int M, int N, int K) {
  const int64_t tiles = (int64_t)((M + BM - 1) / BM) * ((N + BN - 1) / BN);
  if (tiles >= 2 * 152 || K < 4096) return 1;
  int64_t s = (4 * 152 + tiles - 1) / tiles;
  s = std::min<int64_t>(s, K / 2048);
  return (int)std::max<int64_t>(1, std::min<int64_t>(s, 1024));
}

bool smallmn_ok(int M, int N, int K) {
  return (int64_t)M * N <= 4096 && M + N <= 384 && K >= 4096;
}
int smallmn_blocks(int M, int N, int K) {
  (void)M;
  (void)N;
  int64_t b = std::min<int64_t>(4 * 152, (K + 1023) / 1024);
  return (int)std::max<int64_t>(1, b);
}

void zgemm_f64(cudaStream_t s, int M, int N, int K, double alpha, View A,
               View B, double beta, View C, int batch, cplx* part,
               size_t part_elems) {
  if (M <= 0 || N <= 0 || batch <= 0) return;
  if (K <= 0) {
    // C = beta * C
    scale_view(s, M, N, beta, C, batch);
    return;
  }
  if (batch == 1 && N <= GEMV_MAXN && A.cs_lo == 1 && A.c_lo == INT32_MAX &&
      (int64_t)M * K >= (1 << 20) && M >= 8 * 152) {
    const int tok = kstats_begin(s, K_F64_GEMM, 8.0 * M * N * (double)K);
    zgemv_rows_kernel<<<grid1d((int64_t)M * 32, 256), 256, 0, s>>>(M, N, K, alpha, A, B,
                                                                   beta, C);
    CVS_CHECK_LAUNCH();
    kstats_end(s, tok);
    return;
  }
  if (batch == 1 && part && smallmn_ok(M, N, K)) {
    // as many K slices as the partial-product scratch holds (a caller with
    // a small fixed scratch gets fewer, longer slices, never the one-CTA
    // tile path)
    const int nb = (int)std::min<int64_t>(smallmn_blocks(M, N, K),
                                          (int64_t)(part_elems / ((size_t)M * N)));
    if (nb >= 1) {
      const int kchunk = (K + nb - 1) / nb;
      size_t sh = (size_t)(M + N) * STK * sizeof(cplx);
      zgemm_smallmn_kernel<<<nb, 256, sh, s>>>(M, N, K, alpha, A, B, kchunk,
                                               part);
      CVS_CHECK_LAUNCH();
      splitk_reduce(s, M, N, nb, part, beta, C);
      return;
    }
  }
  int a_kfast = (A.cs_lo == 1) ? 1 : 0;
  int b_kfast = (B.rs_lo == 1) ? 1 : 0;
  const int sp = (batch == 1 && part) ? f64_splits(M, N, K) : 1;
  if (sp > 1 && (size_t)sp * M * N <= part_elems) {
    const int kchunk = ((K + sp - 1) / sp + BK - 1) / BK * BK;
    const int nz = (K + kchunk - 1) / kchunk;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, nz);
    const int tok = kstats_begin(s, K_F64_GEMM, 8.0 * M * N * (double)K);
    zgemm_f64_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, B, beta, C,
                                          a_kfast, b_kfast, kchunk, part);
    CVS_CHECK_LAUNCH();
    kstats_end(s, tok);
    splitk_reduce(s, M, N, nz, part, beta, C);
    return;
  }
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
  const int tok = kstats_begin(s, K_F64_GEMM, 8.0 * M * N * (double)K * batch);
  zgemm_f64_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, B, beta, C, a_kfast,
                                        b_kfast, 0, nullptr);
  CVS_CHECK_LAUNCH();
  kstats_end(s, tok);
}

void init_gemm_attributes() {
  CVS_CUDA(cudaFuncSetAttribute(zgemm_smallmn_kernel,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (384 * STK) * (int)sizeof(cplx)));
}

}  // namespace cvs
