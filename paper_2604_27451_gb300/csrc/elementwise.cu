// Bandwidth-bound kernels of the CVS-ADC(2) path: Hermiticity check, the
// t2 epilogue with the MP2 energy, M11 assembly, the CVS pack/unpack with
// the on-the-fly M22, and the Davidson vector kernels.
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>
#include <mutex>
#include <vector>

namespace cvs {

namespace {

__device__ __forceinline__ int64_t pair_index(int a, int b, int v) {
  // a < b; pair(a,b) = a(2v-a-1)/2 + (b-a-1)
  return (int64_t)a * (2 * v - a - 1) / 2 + (b - a - 1);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double, result valid in thread 0
__device__ double block_sum(double v) {
  __shared__ double red[32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  v = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) v = warp_sum(v);
  return v;
}

__global__ void scale_view_kernel(int M, int N, double beta, View C) {
  int64_t total = (int64_t)M * N;
  cplx* p = C.p + (int64_t)blockIdx.y * C.batch;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int r = idx / N, c = idx % N;
    cplx* d = p + vrow(C, r) + vcol(C, c);
    *d = beta == 0.0 ? cmake(0, 0) : cscale(*d, beta);
  }
}

__global__ void herm_kernel(const cplx* B, int n, int64_t nmat, double* out) {
  int64_t total = nmat * n * (int64_t)n;
  double dev = 0.0, mx = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t P = idx / ((int64_t)n * n);
    int64_t rem = idx - P * n * (int64_t)n;
    int p = rem / n, q = rem % n;
    cplx a = B[idx];
    cplx b = B[P * n * (int64_t)n + (int64_t)q * n + p];
    double d = hypot(a.x - b.x, a.y + b.y);
    dev = fmax(dev, d);
    mx = fmax(mx, hypot(a.x, a.y));
  }
  // block max via shared memory
  __shared__ double s0[256], s1[256];
  s0[threadIdx.x] = dev;
  s1[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s0[threadIdx.x] = fmax(s0[threadIdx.x], s0[threadIdx.x + o]);
      s1[threadIdx.x] = fmax(s1[threadIdx.x], s1[threadIdx.x + o]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long*)&out[0], __double_as_longlong(s0[0]));
    atomicMax((unsigned long long*)&out[1], __double_as_longlong(s1[0]));
  }
}

__global__ void t2_band_kernel(const cplx* __restrict__ V, int a0, int na,
                               int o, int v, const double* __restrict__ eps,
                               cplx* __restrict__ t2, cplx* __restrict__ g2,
                               double* part) {
  const int64_t ldV = (int64_t)v * o;
  const int64_t total = (int64_t)na * o * o * v;
  double acc = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int b = idx % v;
    int64_t r = idx / v;
    int j = r % o;
    r /= o;
    int i = r % o;
    int al = r / o;
    int a = a0 + al;
    cplx v1 = V[((int64_t)al * o + i) * ldV + (int64_t)b * o + j];
    cplx v2 = V[((int64_t)al * o + j) * ldV + (int64_t)b * o + i];
    cplx g = csub(v1, v2);
    double den = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    int64_t dst = (((int64_t)i * o + j) * v + a) * v + b;
    g2[dst] = g;
    t2[dst] = cscale(g, 1.0 / den);
    acc += 0.25 * (g.x * g.x + g.y * g.y) / den;
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) part[blockIdx.x] += s;
}

// In-place band transform.  X holds a band [al][i][b][j] = (a i | b j)
// (a = a0 + al, i, j occupied, b virtual).  Each CTA takes one (al, b) and
// one pair of 32 x 32 tiles (i-tile ti <= j-tile tj) together with its
// mirror, stages both in shared memory (coalesced rows) and writes
//   X[al][i][b][j] <- <ab||ij> = (a i|b j) - (a j|b i)
//   T[al][i][b][j]  = <ab||ij> / (e_i + e_j - e_a - e_b)
// for both tiles, so each (i, j), (j, i) pair is read and written by one
// CTA only.  part[block] = the block's share of E_MP2 = 1/4 sum |g|^2 / den.
constexpr int TB2 = 32;
__global__ void t2_band_ip_kernel(cplx* __restrict__ X, cplx* __restrict__ T,
                                  int a0, int o, int v,
                                  const double* __restrict__ eps, int ntile,
                                  double* __restrict__ part) {
  __shared__ cplx sa[TB2][TB2 + 1], sb[TB2][TB2 + 1];
  const int npt = ntile * (ntile + 1) / 2;
  const int64_t blk = blockIdx.x;
  const int tp = (int)(blk % npt);
  const int64_t ab = blk / npt;
  const int b = (int)(ab % v);
  const int al = (int)(ab / v);
  int ti = 0, rem = tp;
  while (rem >= ntile - ti) {
    rem -= ntile - ti;
    ++ti;
  }
  const int tj = ti + rem;
  const int i0 = ti * TB2, j0 = tj * TB2;
  const bool dg = ti == tj;
  const int64_t vo = (int64_t)v * o;
  cplx* Xa = X + (int64_t)al * o * vo + (int64_t)b * o;  // (i, j) -> i vo + j
  cplx* Ta = T + (int64_t)al * o * vo + (int64_t)b * o;
  for (int e = threadIdx.x; e < TB2 * TB2; e += blockDim.x) {
    const int r = e / TB2, cc = e % TB2;
    const int i = i0 + r, j = j0 + cc;
    sa[r][cc] = (i < o && j < o) ? Xa[(int64_t)i * vo + j] : cmake(0, 0);
    if (!dg) {
      const int jj = j0 + r, ii = i0 + cc;
      sb[r][cc] = (jj < o && ii < o) ? Xa[(int64_t)jj * vo + ii] : cmake(0, 0);
    }
  }
  __syncthreads();
  const double eab = eps[o + a0 + al] + eps[o + b];
  double acc = 0.0;
  for (int e = threadIdx.x; e < TB2 * TB2; e += blockDim.x) {
    const int r = e / TB2, cc = e % TB2;
    {
      const int i = i0 + r, j = j0 + cc;
      if (i < o && j < o) {
        const cplx xji = dg ? sa[cc][r] : sb[cc][r];
        const cplx g = csub(sa[r][cc], xji);
        const double den = eps[i] + eps[j] - eab;
        Xa[(int64_t)i * vo + j] = g;
        Ta[(int64_t)i * vo + j] = cscale(g, 1.0 / den);
        acc += (dg ? 0.25 : 0.5) * (g.x * g.x + g.y * g.y) / den;
      }
    }
    if (!dg) {
      const int jj = j0 + r, ii = i0 + cc;
      if (jj < o && ii < o) {
        const cplx g = csub(sb[r][cc], sa[cc][r]);
        const double den = eps[ii] + eps[jj] - eab;
        Xa[(int64_t)jj * vo + ii] = g;
        Ta[(int64_t)jj * vo + ii] = cscale(g, 1.0 / den);
      }
    }
  }
  const double sum = block_sum(acc);
  if (threadIdx.x == 0) part[blk] = sum;
}

// *out += sum of in[0..n)
__global__ void reduce_sum_add_kernel(const double* in, int64_t n, double* out) {
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += in[i];
  double s = block_sum(acc);
  if (threadIdx.x == 0) *out += s;
}

__global__ void reduce_sum_kernel(const double* in, int n, double* out) {
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += in[i];
  double s = block_sum(acc);
  if (threadIdx.x == 0) *out = s;
}

__global__ void m11_kernel(int nc, int nv, int o, const double* eps,
                           const cplx* C1, const cplx* C2, const cplx* X,
                           const cplx* Y, const cplx* Z, int second,
                           cplx* M11) {
  const int64_t N1 = (int64_t)nc * nv;
  const int64_t total = N1 * N1;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t row = idx / N1, col = idx % N1;
    int I = row / nv, a = row % nv, J = col / nv, b = col % nv;
    cplx val = cmake(0, 0);
    if (I == J && a == b) val.x = eps[o + a] - eps[I];
    // <aJ||bI> = (ab|JI) - (aI|Jb)
    cplx c1 = C1[((int64_t)a * nv + b) * (nc * nc) + J * nc + I];
    cplx c2 = C2[row * N1 + col];
    val = csub(val, csub(c1, c2));
    if (second) {
      if (I == J) {
        cplx x = cadd(X[(int64_t)a * nv + b], cconj(X[(int64_t)b * nv + a]));
        val = csub(val, cscale(x, 0.25));
      }
      if (a == b) {
        cplx y = cadd(Y[I * nc + J], cconj(Y[J * nc + I]));
        val = csub(val, cscale(y, 0.25));
      }
      cplx z = cadd(Z[row * N1 + col], cconj(Z[col * N1 + row]));
      val = cadd(val, cscale(z, 0.5));
    }
    M11[idx] = val;
  }
}

__global__ void unpack_kernel(const cplx* __restrict__ x2, int nc, int nw,
                              int nv, cplx* __restrict__ Yt) {
  const int64_t npair = (int64_t)nv * (nv - 1) / 2;
  const int64_t total = (int64_t)nc * nv * nw * nv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int b = idx % nv;
    int64_t r = idx / nv;
    int j = r % nw;
    r /= nw;
    int a = r % nv;
    int I = r / nv;
    int64_t base = ((int64_t)I * nw + j) * npair;
    cplx val;
    if (a < b)
      val = x2[base + pair_index(a, b, nv)];
    else if (a > b) {
      val = x2[base + pair_index(b, a, nv)];
      val.x = -val.x;
      val.y = -val.y;
    } else
      val = cmake(0, 0);
    Yt[idx] = val;
  }
}

// F[I][j][a][b] = -(A[a][b] - A[b][a]) + T[a][b], A and T as [I][j][a][b]
__global__ void pack_moment_kernel(const cplx* __restrict__ A,
                                   const cplx* __restrict__ T, int nc, int nw,
                                   int nv, cplx* __restrict__ out) {
  const int64_t npair = (int64_t)nv * (nv - 1) / 2;
  const int64_t nrows = (int64_t)nc * nw * nv;
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    int a = row % nv;
    int64_t r = row / nv;
    int j = r % nw;
    int I = r / nw;
    int64_t base = ((int64_t)I * nw + j) * npair + pair_index(a, a + 1, nv) - (a + 1);
    int64_t blk = ((int64_t)I * nw + j) * nv * (int64_t)nv;
    for (int b = a + 1 + threadIdx.x; b < nv; b += blockDim.x) {
      cplx ab = A[blk + (int64_t)a * nv + b];
      cplx ba = A[blk + (int64_t)b * nv + a];
      cplx t = T[blk + (int64_t)a * nv + b];
      out[base + b] = cadd(csub(ba, ab), t);
    }
  }
}

__global__ void diag_kernel(const cplx* M11, const double* eps, int nc,
                            int nw, int nv, double* diag) {
  const int64_t N1 = (int64_t)nc * nv;
  const int64_t npair = (int64_t)nv * (nv - 1) / 2;
  const int o = nc + nw;
  const int64_t nrows = (int64_t)nc * nw * nv;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N1;
       s += (int64_t)gridDim.x * blockDim.x)
    diag[s] = M11[s * N1 + s].x;
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    int a = row % nv;
    int64_t r = row / nv;
    int j = r % nw;
    int I = r / nw;
    int64_t base = N1 + ((int64_t)I * nw + j) * npair + pair_index(a, a + 1, nv) - (a + 1);
    double e0 = eps[o + a] - eps[I] - eps[nc + j];
    for (int b = a + 1 + threadIdx.x; b < nv; b += blockDim.x)
      diag[base + b] = e0 + eps[o + b];
  }
}

// ---------------------------------------------------- tall-skinny kernels
// ---- double-float arithmetic for the Davidson vector algebra
// FP64 runs at a small fraction of the FP32 rate on this GPU, so the dot
// products and linear combinations over N-long vectors use pairs of floats
// (hi + lo, ~48-bit significand): each FP64 operand is split once as it is
// loaded, a product keeps the exact rounding error of hi*hi (an FMA) plus
// the cross terms, and the accumulator adds with TwoSum (no contraction).
struct dfc {  // complex double-float: re = (rh, rl), im = (ih, il)
  float rh, rl, ih, il;
};

__device__ __forceinline__ dfc to_dfc(cplx x) {
  dfc d;
  d.rh = __double2float_rn(x.x);
  d.rl = __double2float_rn(x.x - (double)d.rh);
  d.ih = __double2float_rn(x.y);
  d.il = __double2float_rn(x.y - (double)d.ih);
  return d;
}

// (sh, sl) += (ah + al)(bh + bl), sign s = +-1 applied to the product
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al,
                                       float bh, float bl, float sg) {
  const float p = __fmul_rn(sg * ah, bh);
  float e = __fmaf_rn(sg * ah, bh, -p);
  e = __fmaf_rn(sg * ah, bl, e);
  e = __fmaf_rn(sg * al, bh, e);
  const float t = __fadd_rn(sh, p);
  const float bb = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// acc += conj(a) * b  (acc as two (hi, lo) pairs)
__device__ __forceinline__ void dfc_conj_mac(float* acc, const dfc& a, const dfc& b) {
  // re += ar br + ai bi ; im += ar bi - ai br
  df_mac(acc[0], acc[1], a.rh, a.rl, b.rh, b.rl, 1.0f);
  df_mac(acc[0], acc[1], a.ih, a.il, b.ih, b.il, 1.0f);
  df_mac(acc[2], acc[3], a.rh, a.rl, b.ih, b.il, 1.0f);
  df_mac(acc[2], acc[3], a.ih, a.il, b.rh, b.rl, -1.0f);
}

// acc += a * b
__device__ __forceinline__ void dfc_mac(float* acc, const dfc& a, const dfc& b) {
  df_mac(acc[0], acc[1], a.rh, a.rl, b.rh, b.rl, 1.0f);
  df_mac(acc[0], acc[1], a.ih, a.il, b.ih, b.il, -1.0f);
  df_mac(acc[2], acc[3], a.rh, a.rl, b.ih, b.il, 1.0f);
  df_mac(acc[2], acc[3], a.ih, a.il, b.rh, b.rl, 1.0f);
}

__device__ __forceinline__ cplx dfc_value(const float* acc) {
  return cmake((double)acc[0] + (double)acc[1], (double)acc[2] + (double)acc[3]);
}

// Arithmetic policies of the tall-skinny kernels: ArDF is the double-float
// arithmetic above (mixed precisions), Ar64 plain FP64 (FP64-class
// precisions).  E is the element type staged in shared memory, Acc an
// accumulator of one complex sum.
struct ArDF {
  typedef dfc E;
  struct Acc {
    float v[4];
  };
  __device__ static E load(cplx x) { return to_dfc(x); }
  __device__ static void zero(Acc& a) { a.v[0] = a.v[1] = a.v[2] = a.v[3] = 0.f; }
  __device__ static void cmac(Acc& a, const E& x, const E& y) { dfc_conj_mac(a.v, x, y); }
  __device__ static void mac(Acc& a, const E& x, const E& y) { dfc_mac(a.v, x, y); }
  __device__ static cplx value(const Acc& a) { return dfc_value(a.v); }
};
struct Ar64 {
  typedef cplx E;
  struct Acc {
    double re, im;
  };
  __device__ static E load(cplx x) { return x; }
  __device__ static void zero(Acc& a) { a.re = a.im = 0.0; }
  __device__ static void cmac(Acc& a, const E& x, const E& y) {
    a.re = fma(x.x, y.x, fma(x.y, y.y, a.re));
    a.im = fma(x.x, y.y, fma(-x.y, y.x, a.im));
  }
  __device__ static void mac(Acc& a, const E& x, const E& y) {
    a.re = fma(x.x, y.x, fma(-x.y, y.y, a.re));
    a.im = fma(x.x, y.y, fma(x.y, y.x, a.im));
  }
  __device__ static cplx value(const Acc& a) { return cmake(a.re, a.im); }
};
static_assert(sizeof(ArDF::E) == sizeof(cplx) && sizeof(Ar64::E) == sizeof(cplx),
              "staged elements are 16 bytes under both policies");

// sigma2 = -(G_{Ia,jb} - G_{Ib,ja}) + sum_K (x_Ka h_KbIj - x_Kb h_KaIj)
// + M22 x2, packed over a < b (x2 may be NULL: no M22 term; h may be NULL:
// no h term); h[K][b][I][j] = <Kb||Ij>, x1 the singles [K][a].  Tiled: one
// CTA per (I, j) and pair of 32 x 32
// tiles (a-tile ta <= b-tile tb).  G[I][a][j][b] and G[I][b][j][a] of the
// two tiles are staged in shared memory with coalesced row reads, so the
// transposed element is read from shared memory; x1[K][a], x1[K][b] and
// h[K][.][I][j] of the tile's a and b are staged too.  Writes follow the
// packed pair order (contiguous in b for each a).  The <Kb||Ij> terms take
// 24 complex products per element: P = ArDF runs them in double-float on
// the FP32 pipes (this GPU's FP64 rate is a small fraction of its FP32
// rate), P = Ar64 in FP64.
constexpr int ST = 32;
constexpr int ST_MAXC = 16;  // ncore staged per tile (larger ncore: rows loop)
template <class P>
__global__ void __launch_bounds__(256)
    sigma2_tiled_kernel(const cplx* __restrict__ G, const cplx* __restrict__ x2,
                        const cplx* __restrict__ x1, const cplx* __restrict__ h,
                        const double* __restrict__ eps, int nc, int nw, int nv,
                        int ntile, cplx* __restrict__ s2) {
  typedef typename P::E E;
  __shared__ cplx ga[ST][ST + 1], gb[ST][ST + 1];
  __shared__ E xa[ST_MAXC][ST], xb[ST_MAXC][ST], ha[ST_MAXC][ST], hb[ST_MAXC][ST];
  const int npt = ntile * (ntile + 1) / 2;
  const int64_t blk = blockIdx.x;
  const int tp = (int)(blk % npt);
  const int64_t ij = blk / npt;  // I * nw + j
  const int j = (int)(ij % nw), I = (int)(ij / nw);
  int ta = 0, rem = tp;
  while (rem >= ntile - ta) {
    rem -= ntile - ta;
    ++ta;
  }
  const int tb = ta + rem;
  const int a0 = ta * ST, b0 = tb * ST;
  const int64_t ldG = (int64_t)nw * nv;  // stride between a rows of one (I, j)
  const cplx* Gij = G + ((int64_t)I * nv * nw + j) * nv;  // (a, b) -> a ldG + b
  for (int e = threadIdx.x; e < ST * ST; e += blockDim.x) {
    const int r = e / ST, c = e % ST;
    const int a = a0 + r, b = b0 + c;
    ga[r][c] = (a < nv && b < nv) ? Gij[(int64_t)a * ldG + b] : cmake(0, 0);
    const int bb = b0 + r, aa = a0 + c;
    gb[r][c] = (bb < nv && aa < nv) ? Gij[(int64_t)bb * ldG + aa] : cmake(0, 0);
  }
  const int o = nc + nw;
  const int64_t npair = (int64_t)nv * (nv - 1) / 2;
  const int64_t dbase = ij * npair;
  const int64_t hs = (int64_t)nv * nc * nw;  // stride of K in h
  const int64_t hij = (int64_t)I * nw + j;
  // sum_K x1[K][a] h[K][b] and sum_K x1[K][b] h[K][a] per element
  typename P::Acc acc_p[4], acc_m[4];
  for (int q = 0; q < 4; ++q) {
    P::zero(acc_p[q]);
    P::zero(acc_m[q]);
  }
  // the <Kb||Ij> terms, sum_K x1[K][a] h[K][b] - x1[K][b] h[K][a], in
  // groups of ST_MAXC cores
  for (int K0 = 0; h && K0 < nc; K0 += ST_MAXC) {
    const int kc = min(ST_MAXC, nc - K0);
    __syncthreads();
    for (int e = threadIdx.x; e < kc * ST; e += blockDim.x) {
      const int K = e / ST, t = e % ST;
      const int a = a0 + t, b = b0 + t;
      xa[K][t] = P::load(a < nv ? x1[(int64_t)(K0 + K) * nv + a] : cmake(0, 0));
      xb[K][t] = P::load(b < nv ? x1[(int64_t)(K0 + K) * nv + b] : cmake(0, 0));
      ha[K][t] = P::load(a < nv ? h[(K0 + K) * hs + (int64_t)a * nc * nw + hij] : cmake(0, 0));
      hb[K][t] = P::load(b < nv ? h[(K0 + K) * hs + (int64_t)b * nc * nw + hij] : cmake(0, 0));
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int e = threadIdx.x + q * blockDim.x;
      const int r = e / ST, c = e % ST;
      for (int K = 0; K < kc; ++K) {
        P::mac(acc_p[q], xa[K][r], hb[K][c]);
        P::mac(acc_m[q], xb[K][c], ha[K][r]);
      }
    }
  }
  __syncthreads();
  for (int q = 0; q < 4; ++q) {
    const int e = threadIdx.x + q * blockDim.x;
    const int r = e / ST, c = e % ST;
    const int a = a0 + r, b = b0 + c;
    if (a >= nv || b >= nv || a >= b) continue;
    const int64_t d = dbase + pair_index(a, b, nv);
    cplx out = csub(gb[c][r], ga[r][c]);
    if (h) out = cadd(out, csub(P::value(acc_p[q]), P::value(acc_m[q])));
    if (x2) {
      const cplx x = x2[d];
      const double m22 = eps[o + a] + eps[o + b] - eps[I] - eps[nc + j];
      out.x += m22 * x.x;
      out.y += m22 * x.y;
    }
    s2[d] = out;
  }
}


constexpr int TSN = 16;  // n-tile of ts_dot

template <class P>
__global__ void ts_dot_kernel(const cplx* __restrict__ A, int ma,
                              const cplx* __restrict__ B, int mb, int64_t N,
                              cplx* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char ts_sm[];
  typedef typename P::E E;
  E* shd = (E*)ts_sm;
  E* sa = shd;             // [ma][TSN]
  E* sb = shd + ma * TSN;  // [mb][TSN]
  const int npairs = ma * mb;
  const int per = (npairs + blockDim.x - 1) / blockDim.x;  // <= 16
  double ar[16], ai[16];
  for (int q = 0; q < 16; ++q) ar[q] = ai[q] = 0.0;
  int64_t chunk = (N + gridDim.x - 1) / gridDim.x;
  int64_t n0 = blockIdx.x * chunk, n1 = min(N, n0 + chunk);
  for (int64_t t0 = n0; t0 < n1; t0 += TSN) {
    __syncthreads();
    for (int e = threadIdx.x; e < (ma + mb) * TSN; e += blockDim.x) {
      int vec = e / TSN, k = e % TSN;
      int64_t n = t0 + k;
      cplx val = cmake(0, 0);
      if (n < n1) val = vec < ma ? A[(int64_t)vec * N + n] : B[(int64_t)(vec - ma) * N + n];
      shd[e] = P::load(val);
    }
    __syncthreads();
    for (int q = 0; q < per; ++q) {
      int pr = threadIdx.x + q * blockDim.x;
      if (pr >= npairs) break;
      int i = pr / mb, j = pr % mb;
      const E* x = sa + i * TSN;
      const E* y = sb + j * TSN;
      typename P::Acc acc;
      P::zero(acc);
#pragma unroll
      for (int k = 0; k < TSN; ++k) P::cmac(acc, x[k], y[k]);
      const cplx v = P::value(acc);
      ar[q] += v.x;
      ai[q] += v.y;
    }
  }
  for (int q = 0; q < per; ++q) {
    int pr = threadIdx.x + q * blockDim.x;
    if (pr >= npairs) break;
    part[(int64_t)pr * gridDim.x + blockIdx.x] = cmake(ar[q], ai[q]);
  }
}

__global__ void ts_dot_reduce(const cplx* part, int npairs, int mb,
                              int chunks, cplx* out, int ldo) {
  int pr = blockIdx.x;
  if (pr >= npairs) return;
  double sr = 0, si = 0;
  for (int c = threadIdx.x; c < chunks; c += blockDim.x) {
    cplx v = part[(int64_t)pr * chunks + c];
    sr += v.x;
    si += v.y;
  }
  sr = block_sum(sr);
  si = block_sum(si);
  if (threadIdx.x == 0) out[(pr / mb) * ldo + (pr % mb)] = cmake(sr, si);
}

// out[r][n] = sum_i W[i][n] cw[i*ldc+r] + V[i][n] cv[i*ldc+r]
template <class P>
__global__ void ts_combine_kernel(const cplx* __restrict__ V,
                                  const cplx* __restrict__ cv,
                                  const cplx* __restrict__ W,
                                  const cplx* __restrict__ cw, int m, int ldc,
                                  int k, int64_t N, cplx* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char ts_sm[];
  typedef typename P::E E;
  E* coefd = (E*)ts_sm;  // [2][m][k]
  for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
    int i = e / k, r = e % k;
    coefd[e] = P::load(cv ? cv[i * ldc + r] : cmake(0, 0));
    coefd[m * k + e] = P::load(cw ? cw[i * ldc + r] : cmake(0, 0));
  }
  __syncthreads();
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    for (int r0 = 0; r0 < k; r0 += 8) {
      typename P::Acc acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) P::zero(acc[q]);
      for (int i = 0; i < m; ++i) {
        const E vv = P::load(V ? V[(int64_t)i * N + n] : cmake(0, 0));
        const E ww = P::load(W ? W[(int64_t)i * N + n] : cmake(0, 0));
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          int r = r0 + q;
          if (r < k) {
            if (V) P::mac(acc[q], vv, coefd[i * k + r]);
            if (W) P::mac(acc[q], ww, coefd[m * k + i * k + r]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int r = r0 + q;
        if (r < k) out[(int64_t)r * N + n] = P::value(acc[q]);
      }
    }
  }
}

template <class P>
__global__ void ts_subtract_kernel(const cplx* __restrict__ V, int m,
                                   const cplx* __restrict__ c, int ldc, int k,
                                   int64_t N, cplx* __restrict__ y) {
  extern __shared__ __align__(16) unsigned char ts_sm[];
  typedef typename P::E E;
  E* coefd = (E*)ts_sm;  // [k][m]
  for (int e = threadIdx.x; e < m * k; e += blockDim.x) {
    int r = e / m, i = e % m;
    coefd[e] = P::load(c[i * ldc + r]);
  }
  __syncthreads();
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    for (int r0 = 0; r0 < k; r0 += 8) {
      typename P::Acc acc[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) P::zero(acc[q]);
      for (int i = 0; i < m; ++i) {
        const E vv = P::load(V[(int64_t)i * N + n]);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          int r = r0 + q;
          if (r < k) P::mac(acc[q], vv, coefd[r * m + i]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        int r = r0 + q;
        if (r < k) {
          cplx* d = y + (int64_t)r * N + n;
          const cplx o = *d, a = P::value(acc[q]);
          *d = cmake(o.x - a.x, o.y - a.y);
        }
      }
    }
  }
}

__global__ void resid_kernel(const cplx* __restrict__ AX,
                             const cplx* __restrict__ X,
                             const double* __restrict__ theta,
                             const double* __restrict__ diag, int64_t N,
                             cplx* __restrict__ t, double* part) {
  const int r = blockIdx.y;
  const double th = theta[r];
  double acc = 0.0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    cplx ax = AX[(int64_t)r * N + n];
    cplx x = X[(int64_t)r * N + n];
    cplx res = cmake(ax.x - th * x.x, ax.y - th * x.y);
    acc += res.x * res.x + res.y * res.y;
    if (!diag) {  // the raw residual, for a preconditioner applied later
      t[(int64_t)r * N + n] = res;
      continue;
    }
    double den = th - diag[n];
    if (fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
    t[(int64_t)r * N + n] = cscale(res, 1.0 / den);
  }
  double s = block_sum(acc);
  if (threadIdx.x == 0) part[r * gridDim.x + blockIdx.x] = s;
}

__global__ void reduce_rows_kernel(const double* part, int chunks,
                                   double* out) {
  double acc = 0.0;
  for (int c = threadIdx.x; c < chunks; c += blockDim.x)
    acc += part[blockIdx.x * chunks + c];
  double s = block_sum(acc);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

__global__ void scale_vectors_kernel(cplx* x, const double* scale,
                                     int64_t N) {
  const int r = blockIdx.y;
  const double sc = scale[r];
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x)
    x[(int64_t)r * N + n] = cscale(x[(int64_t)r * N + n], sc);
}


__global__ void copy_view_kernel(int M, int N, double alpha, View src,
                                 View dst) {
  int64_t total = (int64_t)M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    int r = idx / N, c = idx % N;
    cplx v = src.p[vrow(src, r) + vcol(src, c)];
    if (src.conj) v.y = -v.y;
    dst.p[vrow(dst, r) + vcol(dst, c)] = cscale(v, alpha);
  }
}

// one pass of an argmin over d[N] skipping the indices already chosen
__global__ void argmin_kernel(const double* d, int64_t N, const int64_t* taken,
                              int ntaken, double* pv, int64_t* pi) {
  double best = 1e300;
  int64_t bi = -1;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    double x = d[n];
    if (x < best || (x == best && n < bi)) {
      bool skip = false;
      for (int q = 0; q < ntaken; ++q) skip |= (taken[q] == n);
      if (!skip) {
        best = x;
        bi = n;
      }
    }
  }
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v2 = sv[threadIdx.x + o];
      int64_t i2 = si[threadIdx.x + o];
      if (i2 >= 0 && (si[threadIdx.x] < 0 || v2 < sv[threadIdx.x] ||
                      (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x]))) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}

__global__ void argmin_final(const double* pv, const int64_t* pi, int nb,
                             int64_t* taken, int slot) {
  if (threadIdx.x != 0) return;
  double best = 1e300;
  int64_t bi = -1;
  for (int b = 0; b < nb; ++b)
    if (pi[b] >= 0 && (bi < 0 || pv[b] < best || (pv[b] == best && pi[b] < bi))) {
      best = pv[b];
      bi = pi[b];
    }
  taken[slot] = bi;
}

// per vector: block partial argmax of |x|
__global__ void absmax_kernel(const cplx* x, int64_t N, double* pv,
                              int64_t* pi) {
  const int r = blockIdx.y;
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    cplx v = x[(int64_t)r * N + n];
    double m = v.x * v.x + v.y * v.y;
    if (m > best) {
      best = m;
      bi = n;
    }
  }
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      double v2 = sv[threadIdx.x + o];
      int64_t i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[r * gridDim.x + blockIdx.x] = sv[0];
    pi[r * gridDim.x + blockIdx.x] = si[0];
  }
}

// per vector: the unit phase that makes its largest-modulus entry real and
// positive, from the block partials of absmax_kernel.  It runs as its own
// launch, before any entry is rotated: a phase computed inside the rotating
// kernel would read a pivot that another block may already have rotated.
__global__ void phase_pick_kernel(const cplx* x, int64_t N, const double* pv,
                                  const int64_t* pi, int nb, cplx* ph) {
  const int r = blockIdx.x;
  if (threadIdx.x != 0) return;
  double best = -1.0;
  int64_t bi = 0;
  for (int b = 0; b < nb; ++b) {
    double v = pv[r * nb + b];
    int64_t i = pi[r * nb + b];
    if (v > best || (v == best && i < bi)) {
      best = v;
      bi = i;
    }
  }
  cplx v = x[(int64_t)r * N + bi];
  double m = hypot(v.x, v.y);
  ph[r] = m > 0 ? cmake(v.x / m, -v.y / m) : cmake(1, 0);
}

__global__ void phase_apply_kernel(cplx* x, int64_t N, const cplx* ph) {
  const int r = blockIdx.y;
  const cplx p = ph[r];
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x)
    x[(int64_t)r * N + n] = cmul(x[(int64_t)r * N + n], p);
}


// A[i][j] = (h(i,j) + conj(h(j,i))) / 2 where h(i,j) = H[i][j] if that
// entry was computed (column j >= jdone, or row i < jdone), else
// conj(H[j][i]); H has leading dimension ldh
__global__ void hermitize_kernel(const cplx* H, int ldh, int m, int jdone,
                                 cplx* A) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       e < (int64_t)m * m; e += (int64_t)gridDim.x * blockDim.x) {
    int i = e / m, j = e % m;
    bool vij = (j >= jdone) || (i < jdone);
    bool vji = (i >= jdone) || (j < jdone);
    cplx hij = H[(int64_t)i * ldh + j], hji = H[(int64_t)j * ldh + i];
    cplx a = vij ? hij : cconj(hji);
    cplx b = vji ? hji : cconj(hij);
    A[e] = cmake(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
}

// Orthonormalising transform of a block of cnt vectors from their Gram
// matrix G (cnt x cnt, leading dimension ldg): Gram-Schmidt in coefficient
// space with the G inner product, two projection passes per column; a
// column is dropped when its remaining norm is below tol * norm0[j].
// X[j][q] (leading dimension cnt) holds kept column q; *kept = their count.
__global__ void block_orth_kernel(const cplx* G, int ldg, int cnt,
                                  const double* norm0, double tol, cplx* X,
                                  int* kept, int* src) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int nk = 0;
  cplx u[64], gu[64];
  for (int j = 0; j < cnt; ++j) {
    for (int a = 0; a < cnt; ++a) u[a] = cmake(a == j ? 1.0 : 0.0, 0.0);
    for (int pass = 0; pass < 2; ++pass) {
      // gu = G u
      for (int a = 0; a < cnt; ++a) {
        cplx acc = cmake(0, 0);
        for (int b = 0; b < cnt; ++b) acc = cadd(acc, cmul(G[a * ldg + b], u[b]));
        gu[a] = acc;
      }
      for (int q = 0; q < nk; ++q) {
        // c = x_q^H G u
        cplx c = cmake(0, 0);
        for (int a = 0; a < cnt; ++a) c = cadd(c, cdotc(X[a * cnt + q], gu[a]));
        for (int a = 0; a < cnt; ++a) u[a] = csub(u[a], cmul(c, X[a * cnt + q]));
      }
    }
    for (int a = 0; a < cnt; ++a) {
      cplx acc = cmake(0, 0);
      for (int b = 0; b < cnt; ++b) acc = cadd(acc, cmul(G[a * ldg + b], u[b]));
      gu[a] = acc;
    }
    double nrm2 = 0;
    for (int a = 0; a < cnt; ++a) nrm2 += cdotc(u[a], gu[a]).x;
    double nrm = sqrt(fmax(nrm2, 0.0));
    if (nrm > tol * norm0[j] && nrm > 1e-300) {
      for (int a = 0; a < cnt; ++a) X[a * cnt + nk] = cscale(u[a], 1.0 / nrm);
      if (src) src[nk] = j;
      ++nk;
    }
  }
  *kept = nk;
}

// H[i][j] = conj(H[j][i]) for i in [i0, i1), j < i0 (the block of new rows
// against old columns, known from Hermiticity once the new columns exist)
__global__ void herm_fill_kernel(cplx* H, int ldh, int i0, int i1) {
  const int64_t total = (int64_t)(i1 - i0) * i0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int i = i0 + (int)(e / i0), j = (int)(e % i0);
    H[(int64_t)i * ldh + j] = cconj(H[(int64_t)j * ldh + i]);
  }
}

__global__ void gram_diag_sqrt_kernel(const cplx* G, int ldg, int cnt,
                                      double* out) {
  int j = threadIdx.x;
  if (j < cnt) out[j] = sqrt(fmax(G[j * ldg + j].x, 0.0));
}

// X[r][c] *= s[r]
__global__ void scale_rows_kernel(cplx* X, int rows, int cols, int ld,
                                  const double* sc) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       e < (int64_t)rows * cols; e += (int64_t)gridDim.x * blockDim.x) {
    int r = e / cols, c = e % cols;
    X[(int64_t)r * ld + c] = cscale(X[(int64_t)r * ld + c], sc[r]);
  }
}

}  // namespace

void scale_view(cudaStream_t s, int M, int N, double beta, View C, int batch) {
  dim3 grid(grid1d((int64_t)M * N, 256), batch);
  scale_view_kernel<<<grid, 256, 0, s>>>(M, N, beta, C);
  CVS_CHECK_LAUNCH();
}

void hermiticity(cudaStream_t s, const cplx* B, int n, int64_t nmat,
                 double* out_dev) {
  CVS_CUDA(cudaMemsetAsync(out_dev, 0, 2 * sizeof(double), s));
  herm_kernel<<<grid1d(nmat * n * (int64_t)n, 256), 256, 0, s>>>(B, n, nmat,
                                                                out_dev);
  CVS_CHECK_LAUNCH();
}

void t2_band(cudaStream_t s, const cplx* V, int a0, int na, int o, int v,
             const double* eps, cplx* t2, cplx* g2, double* part, int nblk) {
  t2_band_kernel<<<nblk, 256, 0, s>>>(V, a0, na, o, v, eps, t2, g2, part);
  CVS_CHECK_LAUNCH();
}

int64_t t2_band_ip_blocks(int nb, int o, int v) {
  const int nt = (o + TB2 - 1) / TB2;
  return (int64_t)nt * (nt + 1) / 2 * nb * v;
}

void t2_band_inplace(cudaStream_t s, cplx* X, cplx* T, int a0, int nb, int o,
                     int v, const double* eps, double* part, double* emp2) {
  const int nt = (o + TB2 - 1) / TB2;
  const int64_t nblk = t2_band_ip_blocks(nb, o, v);
  CVS_REQUIRE(nblk < (1LL << 31), -1, "t2_band_inplace: band too large");
  t2_band_ip_kernel<<<(unsigned)nblk, 256, 0, s>>>(X, T, a0, o, v, eps, nt, part);
  CVS_CHECK_LAUNCH();
  reduce_sum_add_kernel<<<1, 256, 0, s>>>(part, nblk, emp2);
  CVS_CHECK_LAUNCH();
}

// I(E_g) = sum_n f_n (h / pi) / ((E_g - E_n)^2 + h^2), E_g = e0 + g de,
// E_n = omega_n * ev_per_eh + shift, h = fwhm / 2; one grid point per thread
__global__ void lorentz_kernel(const double* __restrict__ omega,
                               const double* __restrict__ f, int nroots, double e0,
                               double de, int npts, double h, double shift,
                               double ev_per_eh, double* __restrict__ out) {
  const double inv_pi = 0.318309886183790671537767526745;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < npts; g += gridDim.x * blockDim.x) {
    const double E = e0 + g * de;
    double acc = 0.0;
    for (int r = 0; r < nroots; ++r) {
      const double x = E - (omega[r] * ev_per_eh + shift);
      acc += f[r] * h / (x * x + h * h);
    }
    out[g] = acc * inv_pi;
  }
}

void lorentz_spectrum(cudaStream_t s, const double* omega, const double* f, int nroots,
                      double e0, double de, int npts, double fwhm, double shift,
                      double ev_per_eh, double* out) {
  lorentz_kernel<<<grid1d(npts, 256), 256, 0, s>>>(omega, f, nroots, e0, de, npts,
                                                   0.5 * fwhm, shift, ev_per_eh, out);
  CVS_CHECK_LAUNCH();
}

void reduce_sum(cudaStream_t s, const double* in, int n, double* out) {
  reduce_sum_kernel<<<1, 256, 0, s>>>(in, n, out);
  CVS_CHECK_LAUNCH();
}

void m11_assemble(cudaStream_t s, int ncore, int nvirt, int o,
                  const double* eps, const cplx* C1, const cplx* C2,
                  const cplx* X, const cplx* Y, const cplx* Z, int second,
                  cplx* M11) {
  int64_t N1 = (int64_t)ncore * nvirt;
  m11_kernel<<<grid1d(N1 * N1, 256), 256, 0, s>>>(ncore, nvirt, o, eps, C1,
                                                   C2, X, Y, Z, second, M11);
  CVS_CHECK_LAUNCH();
}

void unpack_doubles(cudaStream_t s, const cplx* x2, int ncore, int nval,
                    int nvirt, cplx* Yt) {
  int64_t total = (int64_t)ncore * nvirt * nval * nvirt;
  unpack_kernel<<<grid1d(total, 256), 256, 0, s>>>(x2, ncore, nval, nvirt,
                                                    Yt);
  CVS_CHECK_LAUNCH();
}

namespace {
// hT[((I nw + j) nv + b) nc + K] = conj(h[K][b][I][j])
__global__ void h_conj_t_kernel(const cplx* __restrict__ h, int nc, int nw,
                                int nv, cplx* __restrict__ hT) {
  const int64_t total = (int64_t)nc * nw * nv * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int K = e % nc;
    int64_t r = e / nc;
    const int b = r % nv;
    r /= nv;
    const int j = r % nw, I = r / nw;
    hT[e] = cconj(h[(((int64_t)K * nv + b) * nc + I) * nw + j]);
  }
}
}  // namespace

void h_conj_transpose(cudaStream_t s, const cplx* h, int nc, int nw, int nv,
                      cplx* hT) {
  h_conj_t_kernel<<<grid1d((int64_t)nc * nw * nv * nc, 256), 256, 0, s>>>(
      h, nc, nw, nv, hT);
  CVS_CHECK_LAUNCH();
}

void sigma2_finish(cudaStream_t s, const cplx* G, const cplx* x2,
                   const cplx* x1, const cplx* h, const double* eps, int ncore,
                   int nval, int nvirt, cplx* s2, bool fp64) {
  const int nt = (nvirt + ST - 1) / ST;
  const int64_t nblk = (int64_t)ncore * nval * (nt * (nt + 1) / 2);
  CVS_REQUIRE(nblk < (1LL << 31), -1, "sigma2_finish: too many tiles");
  if (fp64)
    sigma2_tiled_kernel<Ar64><<<(unsigned)nblk, 256, 0, s>>>(G, x2, x1, h, eps, ncore, nval,
                                                             nvirt, nt, s2);
  else
    sigma2_tiled_kernel<ArDF><<<(unsigned)nblk, 256, 0, s>>>(G, x2, x1, h, eps, ncore, nval,
                                                             nvirt, nt, s2);
  CVS_CHECK_LAUNCH();
}

void pack_moment_doubles(cudaStream_t s, const cplx* A, const cplx* T,
                         int ncore, int nval, int nvirt, cplx* out) {
  int64_t rows = (int64_t)ncore * nval * nvirt;
  unsigned g = rows > 65535 * 8 ? 65535 * 8 : (unsigned)rows;
  pack_moment_kernel<<<g, 128, 0, s>>>(A, T, ncore, nval, nvirt, out);
  CVS_CHECK_LAUNCH();
}

void build_diag(cudaStream_t s, const cplx* M11, const double* eps,
                int ncore, int nval, int nvirt, double* diag) {
  int64_t rows = (int64_t)ncore * nval * nvirt;
  unsigned g = rows > 65535 * 8 ? 65535 * 8 : (unsigned)rows;
  diag_kernel<<<g, 128, 0, s>>>(M11, eps, ncore, nval, nvirt, diag);
  CVS_CHECK_LAUNCH();
}

void ts_dot(cudaStream_t s, const cplx* A, int ma, const cplx* B, int mb,
            int64_t N, cplx* part, cplx* out, int ldo, bool fp64) {
  if (ma > 96) {
    for (int i0 = 0; i0 < ma; i0 += 96)
      ts_dot(s, A + (int64_t)i0 * N, std::min(96, ma - i0), B, mb, N, part,
             out + (int64_t)i0 * ldo, ldo, fp64);
    return;
  }
  if (ma * mb > 16 * 256 || ma + mb > 192) {
    int g = std::max(1, std::min(192 - ma, 4096 / ma));
    for (int j0 = 0; j0 < mb; j0 += g)
      ts_dot(s, A, ma, B + (int64_t)j0 * N, std::min(g, mb - j0), N, part,
             out + j0, ldo, fp64);
    return;
  }
  int chunks = TS_CHUNKS;
  size_t sh = (size_t)(ma + mb) * TSN * sizeof(cplx);
  if (fp64)
    ts_dot_kernel<Ar64><<<chunks, 256, sh, s>>>(A, ma, B, mb, N, part);
  else
    ts_dot_kernel<ArDF><<<chunks, 256, sh, s>>>(A, ma, B, mb, N, part);
  CVS_CHECK_LAUNCH();
  ts_dot_reduce<<<ma * mb, 256, 0, s>>>(part, ma * mb, mb, chunks, out, ldo);
  CVS_CHECK_LAUNCH();
}

void ts_combine(cudaStream_t s, const cplx* V, const cplx* cv, const cplx* W,
                const cplx* cw, int m, int ldc, int k, int64_t N,
                cplx* out, bool fp64) {
  if (2 * (size_t)m * k * sizeof(cplx) > 96 * 1024) {
    int g = std::max(1, (int)(96 * 1024 / (2 * (size_t)m * sizeof(cplx))));
    CVS_REQUIRE(2 * (size_t)m * sizeof(cplx) <= 96 * 1024, -1, "ts_combine: m too large");
    for (int r0 = 0; r0 < k; r0 += g)
      ts_combine(s, V, cv ? cv + r0 : nullptr, W, cw ? cw + r0 : nullptr, m,
                 ldc, std::min(g, k - r0), N, out + (int64_t)r0 * N, fp64);
    return;
  }
  size_t sh = 2 * (size_t)m * k * sizeof(cplx);
  if (fp64)
    ts_combine_kernel<Ar64><<<grid1d(N, 256), 256, sh, s>>>(V, cv, W, cw, m, ldc, k,
                                                            N, out);
  else
    ts_combine_kernel<ArDF><<<grid1d(N, 256), 256, sh, s>>>(V, cv, W, cw, m, ldc, k,
                                                            N, out);
  CVS_CHECK_LAUNCH();
}

void ts_subtract(cudaStream_t s, const cplx* V, int m, const cplx* c, int ldc,
                 int k, int64_t N, cplx* y, bool fp64) {
  if ((size_t)m * k * sizeof(cplx) > 96 * 1024) {
    int g = std::max(1, (int)(96 * 1024 / ((size_t)m * sizeof(cplx))));
    for (int r0 = 0; r0 < k; r0 += g)
      ts_subtract(s, V, m, c + r0, ldc, std::min(g, k - r0), N,
                  y + (int64_t)r0 * N, fp64);
    return;
  }
  size_t sh = (size_t)m * k * sizeof(cplx);
  if (fp64)
    ts_subtract_kernel<Ar64><<<grid1d(N, 256), 256, sh, s>>>(V, m, c, ldc, k, N, y);
  else
    ts_subtract_kernel<ArDF><<<grid1d(N, 256), 256, sh, s>>>(V, m, c, ldc, k, N, y);
  CVS_CHECK_LAUNCH();
}

void residual_precond(cudaStream_t s, const cplx* AX, const cplx* X,
                      const double* theta, const double* diag, int k,
                      int64_t N, cplx* t, double* part, double* rnorm2) {
  const int chunks = 304;
  dim3 grid(chunks, k);
  resid_kernel<<<grid, 256, 0, s>>>(AX, X, theta, diag, N, t, part);
  CVS_CHECK_LAUNCH();
  reduce_rows_kernel<<<k, 256, 0, s>>>(part, chunks, rnorm2);
  CVS_CHECK_LAUNCH();
}

void scale_vectors(cudaStream_t s, cplx* x, const double* scale, int k,
                   int64_t N) {
  dim3 grid(grid1d(N, 256, 1216), k);
  scale_vectors_kernel<<<grid, 256, 0, s>>>(x, scale, N);
  CVS_CHECK_LAUNCH();
}


__global__ void gather_columns_kernel(const cplx* __restrict__ src, int rows, int64_t lds,
                                      const int* __restrict__ idx, int ncols,
                                      cplx* __restrict__ dst, int64_t ldd) {
  const int64_t total = (int64_t)rows * ncols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ncols), q = (int)(e % ncols);
    dst[(int64_t)r * ldd + q] = src[(int64_t)r * lds + idx[q]];
  }
}

void gather_columns(cudaStream_t s, const cplx* src, int rows, int64_t lds, const int* idx,
                    int ncols, cplx* dst, int64_t ldd) {
  if (rows <= 0 || ncols <= 0) return;
  gather_columns_kernel<<<grid1d((int64_t)rows * ncols, 256), 256, 0, s>>>(
      src, rows, lds, idx, ncols, dst, ldd);
  CVS_CHECK_LAUNCH();
}

void copy_view(cudaStream_t s, int M, int N, double alpha, View src,
               View dst) {
  copy_view_kernel<<<grid1d((int64_t)M * N, 256), 256, 0, s>>>(M, N, alpha,
                                                              src, dst);
  CVS_CHECK_LAUNCH();
}

void k_smallest(cudaStream_t s, const double* d, int64_t N, int k,
                int64_t* idx_dev, double* work) {
  CVS_REQUIRE(k >= 1 && k <= 64 && k <= N, -1, "k_smallest: bad k");
  const int nb = 304;
  double* pv = work;
  int64_t* pi = (int64_t*)(work + nb);
  for (int q = 0; q < k; ++q) {
    argmin_kernel<<<nb, 256, 0, s>>>(d, N, idx_dev, q, pv, pi);
    CVS_CHECK_LAUNCH();
    argmin_final<<<1, 32, 0, s>>>(pv, pi, nb, idx_dev, q);
    CVS_CHECK_LAUNCH();
  }
}

void phase_fix(cudaStream_t s, cplx* x, int k, int64_t N, double* work) {
  const int nb = 152;
  double* pv = work;
  int64_t* pi = (int64_t*)(work + (size_t)nb * k);
  cplx* ph = (cplx*)(pi + (size_t)nb * k);
  dim3 grid(nb, k);
  absmax_kernel<<<grid, 256, 0, s>>>(x, N, pv, pi);
  CVS_CHECK_LAUNCH();
  phase_pick_kernel<<<k, 32, 0, s>>>(x, N, pv, pi, nb, ph);
  CVS_CHECK_LAUNCH();
  phase_apply_kernel<<<grid, 256, 0, s>>>(x, N, ph);
  CVS_CHECK_LAUNCH();
}

void init_kernel_attributes() {
  CVS_CUDA(cudaFuncSetAttribute(ts_combine_kernel<ArDF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024));
  CVS_CUDA(cudaFuncSetAttribute(ts_subtract_kernel<ArDF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024));
  CVS_CUDA(cudaFuncSetAttribute(ts_dot_kernel<ArDF>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024));
  CVS_CUDA(cudaFuncSetAttribute(ts_combine_kernel<Ar64>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024));
  CVS_CUDA(cudaFuncSetAttribute(ts_subtract_kernel<Ar64>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024));
  CVS_CUDA(cudaFuncSetAttribute(ts_dot_kernel<Ar64>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                96 * 1024));
}


void hermitize(cudaStream_t s, const cplx* H, int ldh, int m, cplx* A,
               int jdone) {
  hermitize_kernel<<<grid1d((int64_t)m * m, 256), 256, 0, s>>>(H, ldh, m,
                                                               jdone, A);
  CVS_CHECK_LAUNCH();
}

void herm_fill(cudaStream_t s, cplx* H, int ldh, int i0, int i1) {
  if (i0 <= 0 || i1 <= i0) return;
  herm_fill_kernel<<<grid1d((int64_t)(i1 - i0) * i0, 256), 256, 0, s>>>(H, ldh,
                                                                       i0, i1);
  CVS_CHECK_LAUNCH();
}

void block_orth(cudaStream_t s, const cplx* G, int ldg, int cnt,
                const double* norm0, double tol, cplx* X, int* kept, int* src) {
  CVS_REQUIRE(cnt >= 1 && cnt <= 64, -1, "block_orth: at most 64 vectors");
  CVS_REQUIRE(cnt >= 1 && cnt <= 64, -1, "block_orth: block of 1..64 vectors");
  block_orth_kernel<<<1, 32, 0, s>>>(G, ldg, cnt, norm0, tol, X, kept, src);
  CVS_CHECK_LAUNCH();
}

void gram_diag_sqrt(cudaStream_t s, const cplx* G, int ldg, int cnt,
                    double* out) {
  gram_diag_sqrt_kernel<<<1, 64, 0, s>>>(G, ldg, cnt, out);
  CVS_CHECK_LAUNCH();
}

void scale_rows(cudaStream_t s, cplx* X, int rows, int cols, int ld,
                const double* sc) {
  scale_rows_kernel<<<grid1d((int64_t)rows * cols, 256), 256, 0, s>>>(
      X, rows, cols, ld, sc);
  CVS_CHECK_LAUNCH();
}


// ------------------------------------------------------ kernel timing
namespace {
struct KPair {
  cudaEvent_t a, b;
  int kernel;
  double flops;
};
std::mutex g_ks_mu;
std::vector<KPair> g_ks_pending;
bool g_ks_on = false;
int64_t g_ks_count[K_NKERNELS];
double g_ks_ms[K_NKERNELS], g_ks_flops[K_NKERNELS];
}  // namespace

bool kstats_enabled() { return g_ks_on; }
void kstats_set(bool on) { g_ks_on = on; }

int kstats_begin(cudaStream_t s, int kernel, double flops) {
  if (!g_ks_on) return -1;
  std::lock_guard<std::mutex> l(g_ks_mu);
  KPair p;
  CVS_CUDA(cudaEventCreate(&p.a));
  CVS_CUDA(cudaEventCreate(&p.b));
  p.kernel = kernel;
  p.flops = flops;
  CVS_CUDA(cudaEventRecord(p.a, s));
  g_ks_pending.push_back(p);
  return (int)g_ks_pending.size() - 1;
}

void kstats_end(cudaStream_t s, int token) {
  if (token < 0) return;
  std::lock_guard<std::mutex> l(g_ks_mu);
  CVS_CUDA(cudaEventRecord(g_ks_pending[token].b, s));
}

static void kstats_drain() {
  for (auto& p : g_ks_pending) {
    CVS_CUDA(cudaEventSynchronize(p.b));
    float ms = 0;
    CVS_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
    g_ks_count[p.kernel] += 1;
    g_ks_ms[p.kernel] += ms;
    g_ks_flops[p.kernel] += p.flops;
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  g_ks_pending.clear();
}

void kstats_collect(int kernel, int64_t* count, double* ms, double* flops) {
  std::lock_guard<std::mutex> l(g_ks_mu);
  kstats_drain();
  *count = g_ks_count[kernel];
  *ms = g_ks_ms[kernel];
  *flops = g_ks_flops[kernel];
}

void kstats_reset() {
  std::lock_guard<std::mutex> l(g_ks_mu);
  kstats_drain();
  for (int k = 0; k < K_NKERNELS; ++k) {
    g_ks_count[k] = 0;
    g_ks_ms[k] = 0;
    g_ks_flops[k] = 0;
  }
}

}  // namespace cvs
