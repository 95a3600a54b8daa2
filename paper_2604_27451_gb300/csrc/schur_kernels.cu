// Kernels of the Schur-complement preconditioner of the Davidson solver.
//
// M22 is diagonal, so for a trial energy theta the doubles can be folded
// into the singles block exactly:
//   S(theta) = M11 + M12 (theta - M22)^-1 M21,
// and an eigenvalue of M below the lowest M22 entry is an eigenvalue of
// S(theta) at theta = that eigenvalue.  With A_{Ijab,Kc} the M21 element
// (-d_IK <ab||cj> + d_ac <Kb||Ij> - d_bc <Ka||Ij>, antisymmetric in ab) and
// w_{Ijab} = 1 / (theta - e_a - e_b + e_I + e_j), the self-energy splits
// into five pieces (K, K' core; c, c' virtual; sums over all a, b):
//   (11) d_KK' 1/2 sum_{jab} w_Kjab conj(<ab||cj>) <ab||c'j>
//   (12) -sum_{jb} w_{K j c' b} conj(<c'b||cj>) <K'b||Kj>
//   (21) the conjugate transpose of (12)
//   (22) d_cc' sum_{Ijb} w_{Ijcb} conj(<Kb||Ij>) <K'b||Ij>
//   (23) -sum_{Ij} w_{Ijcc'} conj(<Kc'||Ij>) <K'c||Ij>
// Term (11) is a weighted Gram matrix per core index and runs as a GEMM;
// (12) as a batched GEMM; (22) and (23) involve only the small <Kb||Ij>
// tensor and are summed here while S is assembled.
//
// Also here: a Jacobi eigensolver for Hermitian matrices too large for one
// CTA (the same cyclic round-robin rotations as jacobi.cu, each step split
// into three grid-wide launches), and the elementwise steps of applying
// the preconditioner.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace cvs {

namespace {

// sum of v over the block, valid in thread 0; safe to call repeatedly
__device__ double sum_block(double v) {
  __shared__ double lanes[32];
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) lanes[threadIdx.x >> 5] = v;
  __syncthreads();
  const int nwarp = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nwarp ? lanes[threadIdx.x] : 0.0;
  if (threadIdx.x < 32)
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ double wgt(const double* eps, int nc, int o,
                                      double theta, int I, int j, int a,
                                      int b) {
  return 1.0 / (theta - (eps[o + a] + eps[o + b] - eps[I] - eps[nc + j]));
}

// h[K][b][I][j] = (KI|bj) - (Kj|bI) from hc1[(K,I)][(b,j)] and
// hc2[(K,j)][(b,I)]
__global__ void h_assemble_kernel(const cplx* __restrict__ hc1,
                                  const cplx* __restrict__ hc2, int nc, int nw,
                                  int nv, cplx* __restrict__ h) {
  const int64_t total = (int64_t)nc * nv * nc * nw;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = e % nw;
    int64_t r = e / nw;
    const int I = r % nc;
    r /= nc;
    const int b = r % nv;
    const int K = r / nv;
    const cplx x = hc1[((int64_t)K * nc + I) * ((int64_t)nv * nw) + (int64_t)b * nw + j];
    const cplx y = hc2[((int64_t)K * nw + j) * ((int64_t)nv * nc) + (int64_t)b * nc + I];
    h[e] = csub(x, y);
  }
}

// G[jl][a][b][c] = <ab||c j> = X1[(a,c)][(jl,b)] - X2[(jl,a)][(b,c)]
__global__ void g_assemble_kernel(const cplx* __restrict__ X1,
                                  const cplx* __restrict__ X2, int jc, int nv,
                                  cplx* __restrict__ G) {
  const int64_t v = nv, total = (int64_t)jc * v * v * v;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = e % v;
    int64_t r = e / v;
    const int b = r % v;
    r /= v;
    const int a = r % v;
    const int jl = r / v;
    const cplx x1 = X1[((int64_t)a * v + c) * (jc * v) + (int64_t)jl * v + b];
    // (aj|bc) = (bc|aj): without X2 it is the permuted element of X1
    const cplx x2 = X2 ? X2[((int64_t)jl * v + a) * (v * v) + (int64_t)b * v + c]
                       : X1[((int64_t)b * v + c) * (jc * v) + (int64_t)jl * v + a];
    G[e] = csub(x1, x2);
  }
}

// Gw[K][jl][a][b][c] = 1/2 w_{K, j0+jl, a, b} G[jl][a][b][c] for every core K
__global__ void g_weight_kernel(const cplx* __restrict__ G, int jc, int j0,
                                int nc, int nw, int nv,
                                const double* __restrict__ eps, double theta,
                                cplx* __restrict__ Gw) {
  const int o = nc + nw;
  const int64_t v = nv, per = (int64_t)jc * v * v * v, total = per * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int K = e / per;
    const int64_t g = e % per;
    int64_t r = g / v;
    const int b = r % v;
    r /= v;
    const int a = r % v;
    const int jl = r / v;
    Gw[e] = cscale(G[g], 0.5 * wgt(eps, nc, o, theta, K, j0 + jl, a, b));
  }
}

// S22[c][K][K'] = sum_{Ijb} w_{Ijcb} conj(<Kb||Ij>) <K'b||Ij>: one block per
// c, each thread a slice of (I, j, b) for all (K, K'), then a block sum
__global__ void __launch_bounds__(128) s22_kernel(
    const cplx* __restrict__ h, int nc, int nw, int nv,
    const double* __restrict__ eps, double theta, cplx* __restrict__ S22) {
  const int c = blockIdx.x;
  const int o = nc + nw;
  const int64_t cnt = (int64_t)nc * nw * nv;
  constexpr int MAXC = 16;  // ncore <= 16 on this path
  for (int K = 0; K < nc; ++K)
    for (int Kp = 0; Kp < nc; ++Kp) {
      double sr = 0.0, si = 0.0;
      for (int64_t q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int b = q % nv;
        const int64_t ij = q / nv;
        const int j = ij % nw, I = ij / nw;
        const double w = wgt(eps, nc, o, theta, I, j, c, b);
        const cplx hk = h[(((int64_t)K * nv + b) * nc + I) * nw + j];
        const cplx hq = h[(((int64_t)Kp * nv + b) * nc + I) * nw + j];
        sr += w * (hk.x * hq.x + hk.y * hq.y);
        si += w * (hk.x * hq.y - hk.y * hq.x);
      }
      sr = sum_block(sr);
      si = sum_block(si);
      if (threadIdx.x == 0)
        S22[((int64_t)c * nc + K) * nc + Kp] = cmake(sr, si);
    }
  (void)MAXC;
}

// Hw[c'][b][K][K'] = w_{K j c' b} h[K'][b][K][j]
__global__ void h_weight_kernel(const cplx* __restrict__ h, int j, int nc,
                                int nw, int nv, const double* __restrict__ eps,
                                double theta, cplx* __restrict__ Hw) {
  const int o = nc + nw;
  const int64_t total = (int64_t)nv * nv * nc * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int Kp = e % nc;
    int64_t r = e / nc;
    const int K = r % nc;
    r /= nc;
    const int b = r % nv;
    const int cp = r / nv;
    const cplx x = h[(((int64_t)Kp * nv + b) * nc + K) * nw + j];
    Hw[e] = cscale(x, wgt(eps, nc, o, theta, K, j, cp, b));
  }
}

// Hw[b][(K,K')] = wbar^p h[K'][b][K][j] with the weight taken at the mean
// virtual energy ebar in place of e_c' (p = 1, 2): the large-singles-space
// preconditioner's cross term (12), w(e_c') = wbar + (e_c' - ebar) wbar^2
// + O((e_c' - ebar)^2 wbar^3)
__global__ void h_weight_mean_kernel(const cplx* __restrict__ h, int j, int nc, int nw,
                                     int nv, const double* __restrict__ eps, double theta,
                                     double ebar, int power, cplx* __restrict__ Hw) {
  const int o = nc + nw;
  const int64_t total = (int64_t)nv * nc * nc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int Kp = e % nc;
    int64_t r = e / nc;
    const int K = r % nc;
    const int b = r / nc;
    const double w = 1.0 / (theta - (ebar + eps[o + b] - eps[K] - eps[nc + j]));
    const cplx x = h[(((int64_t)Kp * nv + b) * nc + K) * nw + j];
    Hw[e] = cscale(x, power == 2 ? w * w : w);
  }
}

// C[(c', c)][q] += (e_c' - ebar) P[(c', c)][q] over q < nq
__global__ void add_row_scaled_kernel(cplx* __restrict__ C, const cplx* __restrict__ P,
                                      int nv, int nq, const double* __restrict__ eps,
                                      int o, double ebar) {
  const int64_t total = (int64_t)nv * nv * nq;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int cp = (int)(e / ((int64_t)nv * nq));
    C[e] = cadd(C[e], cscale(P[e], eps[o + cp] - ebar));
  }
}

// Partial eigensystem preconditioner: Y[i][r] (i < p, U_p^H r~) becomes
// Y (1/den_i(r) - 1/(theta_r - lam_c)) with den_i = theta_r - lam_i +
// (theta_r - theta0) d_i, so that U_p Y + r~ / (theta_r - lam_c) applies
// (S - theta)^-1 on the computed eigenvectors and a scalar on the rest.
__global__ void eig_shift_partial_kernel(cplx* Y, int p, int k,
                                         const double* __restrict__ lam,
                                         const double* __restrict__ d, double theta0,
                                         const double* __restrict__ theta, double lam_c) {
  const int64_t total = (int64_t)p * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = e % k;
    const int64_t i = e / k;
    double den = theta[r] - lam[i] + (theta[r] - theta0) * d[i];
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    double dc = theta[r] - lam_c;
    if (fabs(dc) < 1e-8) dc = dc < 0 ? -1e-8 : 1e-8;
    Y[e] = cscale(Y[e], 1.0 / den - 1.0 / dc);
  }
}

// S[(K,c)][(K',c')] = M11 + (11) + (12) + (21) + (22) + (23); C11 is
// [K][c][c'] and C12 is [c'][c][K][K'] holding sum_{jb} conj(<c'b||cj>)
// w <K'b||Kj> (the sign of (12) is applied here).
__global__ void schur_assemble_kernel(const cplx* __restrict__ M11,
                                      const cplx* __restrict__ C11,
                                      const cplx* __restrict__ C12,
                                      const cplx* __restrict__ S22,
                                      const cplx* __restrict__ h, int nc,
                                      int nw, int nv,
                                      const double* __restrict__ eps,
                                      double theta, cplx* __restrict__ S) {
  const int o = nc + nw;
  const int64_t N1 = (int64_t)nc * nv, total = N1 * N1;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = e / N1, col = e % N1;
    const int K = row / nv, c = row % nv, Kp = col / nv, cp = col % nv;
    cplx val = M11[e];
    if (K == Kp) val = cadd(val, C11[((int64_t)K * nv + c) * nv + cp]);
    const cplx x12 = C12[(((int64_t)cp * nv + c) * nc + K) * nc + Kp];
    const cplx x21 = C12[(((int64_t)c * nv + cp) * nc + Kp) * nc + K];
    val = csub(val, cadd(x12, cconj(x21)));
    if (c == cp) val = cadd(val, S22[((int64_t)c * nc + K) * nc + Kp]);
    double sr = 0.0, si = 0.0;
    for (int I = 0; I < nc; ++I)
      for (int j = 0; j < nw; ++j) {
        // (23): -w conj(h_{K c' I j}) h_{K' c I j}
        const double w = wgt(eps, nc, o, theta, I, j, c, cp);
        const cplx hk = h[(((int64_t)K * nv + cp) * nc + I) * nw + j];
        const cplx hq = h[(((int64_t)Kp * nv + c) * nc + I) * nw + j];
        sr -= w * (hk.x * hq.x + hk.y * hq.y);
        si -= w * (hk.x * hq.y - hk.y * hq.x);
      }
    val.x += sr;
    val.y += si;
    S[e] = val;
  }
}

// ------------------------------------------------------ parallel Jacobi
// Pairs of step s of the round-robin tournament over np (even) positions:
// position 0 stays, the others rotate by one per step.
__device__ __forceinline__ void rr_pair(int k, int np, int s, int& p, int& q) {
  auto pos = [&](int kk) {
    return kk == 0 ? 0 : 1 + ((kk - 1 - s) % (np - 1) + (np - 1)) % (np - 1);
  };
  p = pos(k);
  q = pos(np - 1 - k);
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

__global__ void pj_identity_kernel(cplx* V, int n) {
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    V[e] = cmake(e / n == e % n ? 1.0 : 0.0, 0.0);
}

__global__ void pj_params_kernel(const cplx* __restrict__ A, int n, int np,
                                 int s, double* __restrict__ cc,
                                 cplx* __restrict__ se) {
  const int half = np / 2;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < half;
       k += gridDim.x * blockDim.x) {
    int p, q;
    rr_pair(k, np, s, p, q);
    double c = 1.0;
    cplx sv = cmake(0, 0);
    if (q < n) {
      const cplx apq = A[(int64_t)p * n + q];
      const double r = hypot(apq.x, apq.y);
      const double app = A[(int64_t)p * n + p].x, aqq = A[(int64_t)q * n + q].x;
      if (r > 1e-300 && r > 1e-18 * sqrt(fabs(app * aqq))) {
        const double tau = (aqq - app) / (2.0 * r);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        c = 1.0 / sqrt(1.0 + t * t);
        const double sn = t * c;
        sv = cmake(sn * apq.x / r, sn * apq.y / r);
      }
    }
    cc[k] = c;
    se[k] = sv;
  }
}

// rows p, q of A: A <- J^H A
__global__ void pj_rows_kernel(cplx* A, int n, int np, int s,
                               const double* __restrict__ cc,
                               const cplx* __restrict__ se) {
  const int half = np / 2;
  const int64_t total = (int64_t)half * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = e / n, col = e % n;
    int p, q;
    rr_pair(k, np, s, p, q);
    if (q >= n) continue;
    const cplx sv = se[k];
    if (sv.x == 0.0 && sv.y == 0.0) continue;
    const double c = cc[k];
    const cplx ap = A[(int64_t)p * n + col], aq = A[(int64_t)q * n + col];
    A[(int64_t)p * n + col] = csub(cscale(ap, c), cmul(sv, aq));
    A[(int64_t)q * n + col] = cadd(cmul(cconj(sv), ap), cscale(aq, c));
  }
}

// columns p, q of A and V: A <- A J, V <- V J
__global__ void pj_cols_kernel(cplx* A, cplx* V, int n, int np, int s,
                               const double* __restrict__ cc,
                               const cplx* __restrict__ se) {
  const int half = np / 2;
  const int64_t total = (int64_t)half * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = e / n, row = e % n;
    int p, q;
    rr_pair(k, np, s, p, q);
    if (q >= n) continue;
    const cplx sv = se[k];
    if (sv.x == 0.0 && sv.y == 0.0) continue;
    const double c = cc[k];
    const cplx ap = A[(int64_t)row * n + p], aq = A[(int64_t)row * n + q];
    A[(int64_t)row * n + p] = csub(cscale(ap, c), cmul(cconj(sv), aq));
    A[(int64_t)row * n + q] = cadd(cmul(sv, ap), cscale(aq, c));
    const cplx vp = V[(int64_t)row * n + p], vq = V[(int64_t)row * n + q];
    V[(int64_t)row * n + p] = csub(cscale(vp, c), cmul(cconj(sv), vq));
    V[(int64_t)row * n + q] = cadd(cmul(sv, vp), cscale(vq, c));
  }
}

// per-block partial sums of the off-diagonal and total squared modulus
__global__ void pj_offnorm_kernel(const cplx* __restrict__ A, int n,
                                  double* __restrict__ part) {
  double off = 0.0, tot = 0.0;
  const int64_t total = (int64_t)n * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const cplx a = A[e];
    const double m2 = a.x * a.x + a.y * a.y;
    tot += m2;
    if (e / n != e % n) off += m2;
  }
  off = sum_block(off);
  tot = sum_block(tot);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = off;
    part[2 * blockIdx.x + 1] = tot;
  }
}

// ascending eigenvalues w and the matching columns of V into U
__global__ void pj_sort_kernel(const cplx* __restrict__ A,
                               const cplx* __restrict__ V, int n,
                               double* __restrict__ w, cplx* __restrict__ U) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += gridDim.x * blockDim.x) {
    const double wi = A[(int64_t)i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double wj = A[(int64_t)j * n + j].x;
      rank += (wj < wi) || (wj == wi && j < i);
    }
    w[rank] = wi;
    for (int r = 0; r < n; ++r) U[(int64_t)r * n + rank] = V[(int64_t)r * n + i];
  }
}

// ------------------------------------------------ preconditioner steps
// out[r][d] = (R[r][d] + U2[r][d]) / (theta_r - M22_d) over the doubles of
// k vectors (R and U2 may be NULL); the singles part of out is set to zero
// when zero_singles, else left alone.  One block row per (I, j, a), the
// threads over b > a (the packed pair order).
__global__ void fold_doubles_kernel(const cplx* __restrict__ R,
                                    const cplx* __restrict__ U2,
                                    const double* __restrict__ theta,
                                    int64_t N, int64_t N1, int nc, int nw,
                                    int nv, const double* __restrict__ eps,
                                    int zero_singles, cplx* __restrict__ out) {
  const int r = blockIdx.y;
  const int o = nc + nw;
  const int64_t npair = (int64_t)nv * (nv - 1) / 2;
  const int64_t nrows = (int64_t)nc * nw * nv;
  const double th = theta[r];
  cplx* outr = out + (int64_t)r * N;
  if (zero_singles)
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N1;
         s += (int64_t)gridDim.x * blockDim.x)
      outr[s] = cmake(0, 0);
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int a = row % nv;
    const int64_t ij = row / nv;
    const int j = ij % nw, I = ij / nw;
    const int64_t base = N1 + ij * npair + (int64_t)a * (2 * nv - a - 1) / 2 - (a + 1);
    const double e0 = eps[o + a] - eps[I] - eps[nc + j];
    for (int b = a + 1 + threadIdx.x; b < nv; b += blockDim.x) {
      const int64_t e = (int64_t)r * N + base + b;
      cplx x = R ? R[e] : cmake(0, 0);
      if (U2) x = cadd(x, U2[e]);
      double den = th - (e0 + eps[o + b]);
      if (fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
      outr[base + b] = cscale(x, 1.0 / den);
    }
  }
}

// part[blk] = this block's share of sum_d |u_d|^2 / (theta - M22_d)^2
__global__ void fold_norm_kernel(const cplx* __restrict__ u, int64_t N1,
                                 int nc, int nw, int nv,
                                 const double* __restrict__ eps, double theta,
                                 double* __restrict__ part) {
  const int o = nc + nw;
  const int64_t npair = (int64_t)nv * (nv - 1) / 2;
  const int64_t nrows = (int64_t)nc * nw * nv;
  double acc = 0.0;
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int a = row % nv;
    const int64_t ij = row / nv;
    const int j = ij % nw, I = ij / nw;
    const int64_t base = N1 + ij * npair + (int64_t)a * (2 * nv - a - 1) / 2 - (a + 1);
    const double e0 = eps[o + a] - eps[I] - eps[nc + j];
    for (int b = a + 1 + threadIdx.x; b < nv; b += blockDim.x) {
      const double den = theta - (e0 + eps[o + b]);
      const cplx x = u[base + b];
      acc += (x.x * x.x + x.y * x.y) / (den * den);
    }
  }
  acc = sum_block(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// out[n] = r[n] / (theta - diag[n]) (the diagonal preconditioner), one vector
__global__ void diag_precond_kernel(const cplx* __restrict__ r, double theta,
                                    const double* __restrict__ diag, int64_t N,
                                    cplx* __restrict__ out) {
  for (int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; n < N;
       n += (int64_t)gridDim.x * blockDim.x) {
    double den = theta - diag[n];
    if (fabs(den) < 1e-4) den = den < 0 ? -1e-4 : 1e-4;
    out[n] = cscale(r[n], 1.0 / den);
  }
}

// Y[i][r] /= (theta_r - lam_i), Y is [n1][k]
__global__ void eig_shift_kernel(cplx* Y, int64_t n1, int k,
                                 const double* __restrict__ lam,
                                 const double* __restrict__ theta) {
  const int64_t total = n1 * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = e % k;
    const int64_t i = e / k;
    double den = theta[r] - lam[i];
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    Y[e] = cscale(Y[e], 1.0 / den);
  }
}

// Y[i][r] /= (theta_r - lam_i(theta_r)) with the eigenvalues of S(theta)
// taken to first order about theta0: lam_i(theta) ~ lam_i - (theta -
// theta0) d_i, d_i = u_i^H M12 W(theta0)^2 M21 u_i (Y is [n1][k])
__global__ void eig_shift_d_kernel(cplx* Y, int64_t n1, int k,
                                   const double* __restrict__ lam,
                                   const double* __restrict__ d, double theta0,
                                   const double* __restrict__ theta) {
  const int64_t total = n1 * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = e % k;
    const int64_t i = e / k;
    double den = theta[r] - lam[i] + (theta[r] - theta0) * d[i];
    if (fabs(den) < 1e-8) den = den < 0 ? -1e-8 : 1e-8;
    Y[e] = cscale(Y[e], 1.0 / den);
  }
}

// out[r][s] = a[r][s] + b[r][s] over the first n1 entries of k vectors of
// length N
__global__ void add_singles_kernel(const cplx* __restrict__ a,
                                   const cplx* __restrict__ b, int64_t N,
                                   int64_t n1, int k, cplx* __restrict__ out) {
  const int64_t total = n1 * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = e / n1;
    const int64_t s = e % n1;
    out[r * N + s] = cadd(a[r * N + s], b[r * N + s]);
  }
}

// Projected matrices of the folded solver's lifted basis z_j = (v_j,
// W_j M21 v_j), W_j = (theta_j - M22)^-1, from singles-space products:
//   E = V^H R (R_j = M12 W_j M21 v_j), VD = V^H D (D_j = M12 W_j^2 M21 v_j),
//   A = V^H M11 V, VV = V^H V  (all m x m, leading dimension ld).
// Doubles overlap Q_ij = (W_i M21 v_i)^H (W_j M21 v_j):
//   |theta_i - theta_j| > delta: partial fractions,
//     Q_ij = (E_ij - conj(E_ji)) / (theta_i - theta_j);
//   otherwise the midpoint (W_i W_j = (W_i^2 + W_j^2)/2 + O(dtheta^2)),
//     Q_ij = (VD_ij + conj(VD_ji)) / 2.
// Then H = A + E + Q diag(theta) and O = VV + Q, both Hermitised.
__global__ void lift_assemble_kernel(const cplx* __restrict__ E,
                                     const cplx* __restrict__ VD,
                                     const cplx* __restrict__ A,
                                     const cplx* __restrict__ VV,
                                     const double* __restrict__ th, int m, int ld,
                                     double delta, cplx* __restrict__ Q,
                                     cplx* __restrict__ H, cplx* __restrict__ O) {
  const int total = m * m;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / m, j = e % m;
    auto q = [&](int a, int b) {
      const double dt = th[a] - th[b];
      if (fabs(dt) > delta)
        return cscale(csub(E[a * ld + b], cconj(E[b * ld + a])), 1.0 / dt);
      return cscale(cadd(VD[a * ld + b], cconj(VD[b * ld + a])), 0.5);
    };
    // Hermitian by construction up to rounding: average (i,j) and (j,i)
    const cplx qij = cscale(cadd(q(i, j), cconj(q(j, i))), 0.5);
    const cplx hij = cadd(cadd(A[i * ld + j], E[i * ld + j]), cscale(q(i, j), th[j]));
    const cplx hji = cadd(cadd(A[j * ld + i], E[j * ld + i]), cscale(q(j, i), th[i]));
    Q[i * ld + j] = qij;
    H[i * ld + j] = cscale(cadd(hij, cconj(hji)), 0.5);
    O[i * ld + j] = cadd(cscale(cadd(VV[i * ld + j], cconj(VV[j * ld + i])), 0.5), qij);
  }
}

// Cp[j][q] = C[j][q] (w[q] - th[j]), j < m, q < k (leading dimensions ldc)
__global__ void lift_coef_kernel(const cplx* __restrict__ C, int m, int k, int ldc,
                                 const double* __restrict__ w,
                                 const double* __restrict__ th, cplx* __restrict__ Cp) {
  const int total = m * k;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int j = e / k, q = e % k;
    Cp[j * ldc + q] = cscale(C[j * ldc + q], w[q] - th[j]);
  }
}

// Y[q][s] = X[q][s] - w[q] Z[q][s] for k rows of n
__global__ void row_axpy_kernel(const cplx* __restrict__ X, const cplx* __restrict__ Z,
                                const double* __restrict__ w, int k, int64_t n,
                                cplx* __restrict__ Y) {
  const int q = blockIdx.y;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = (int64_t)q * n + s;
    const cplx z = Z[e];
    Y[e] = cmake(X[e].x - w[q] * z.x, X[e].y - w[q] * z.y);
  }
}

// out[q] = sum_s |X[q][s]|^2 (FP64), one block per row
__global__ void row_norm2_kernel(const cplx* __restrict__ X, int64_t n,
                                 double* __restrict__ out) {
  const int q = blockIdx.x;
  double acc = 0.0;
  for (int64_t s = threadIdx.x; s < n; s += blockDim.x) {
    const cplx x = X[(int64_t)q * n + s];
    acc += x.x * x.x + x.y * x.y;
  }
  acc = sum_block(acc);
  if (threadIdx.x == 0) out[q] = acc;
}

// Oi[i][c] = U[i][off + c] / sqrt(w[off + c]), i < m, c < kept (ld ldu)
__global__ void inv_sqrt_cols_kernel(const cplx* __restrict__ U, const double* __restrict__ w,
                                     int m, int off, int kept, int ldu,
                                     cplx* __restrict__ Oi) {
  const int total = m * kept;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int i = e / kept, cc = e % kept;
    Oi[i * ldu + cc] = cscale(U[i * ldu + off + cc], 1.0 / sqrt(w[off + cc]));
  }
}

}  // namespace

void lift_assemble(cudaStream_t s, const cplx* E, const cplx* VD, const cplx* A,
                   const cplx* VV, const double* th, int m, int ld, double delta,
                   cplx* Q, cplx* H, cplx* O) {
  lift_assemble_kernel<<<grid1d((int64_t)m * m, 128), 128, 0, s>>>(E, VD, A, VV, th, m, ld,
                                                                    delta, Q, H, O);
  CVS_CHECK_LAUNCH();
}

void lift_coef(cudaStream_t s, const cplx* C, int m, int k, int ldc, const double* w,
               const double* th, cplx* Cp) {
  lift_coef_kernel<<<grid1d((int64_t)m * k, 128), 128, 0, s>>>(C, m, k, ldc, w, th, Cp);
  CVS_CHECK_LAUNCH();
}

void row_axpy(cudaStream_t s, const cplx* X, const cplx* Z, const double* w, int k,
              int64_t n, cplx* Y) {
  dim3 grid(grid1d(n, 256, 304), k);
  row_axpy_kernel<<<grid, 256, 0, s>>>(X, Z, w, k, n, Y);
  CVS_CHECK_LAUNCH();
}

void row_norm2(cudaStream_t s, const cplx* X, int k, int64_t n, double* out) {
  row_norm2_kernel<<<k, 256, 0, s>>>(X, n, out);
  CVS_CHECK_LAUNCH();
}

void inv_sqrt_cols(cudaStream_t s, const cplx* U, const double* w, int m, int off, int kept,
                   int ldu, cplx* Oi) {
  inv_sqrt_cols_kernel<<<grid1d((int64_t)m * kept, 128), 128, 0, s>>>(U, w, m, off, kept,
                                                                        ldu, Oi);
  CVS_CHECK_LAUNCH();
}

void h_assemble(cudaStream_t s, const cplx* hc1, const cplx* hc2, int nc,
                int nw, int nv, cplx* h) {
  h_assemble_kernel<<<grid1d((int64_t)nc * nv * nc * nw, 256), 256, 0, s>>>(
      hc1, hc2, nc, nw, nv, h);
  CVS_CHECK_LAUNCH();
}

void g_assemble(cudaStream_t s, const cplx* X1, const cplx* X2, int jc, int nv,
                cplx* G) {
  g_assemble_kernel<<<grid1d((int64_t)jc * nv * nv * nv, 256), 256, 0, s>>>(
      X1, X2, jc, nv, G);
  CVS_CHECK_LAUNCH();
}

void g_weight(cudaStream_t s, const cplx* G, int jc, int j0, int nc, int nw,
              int nv, const double* eps, double theta, cplx* Gw) {
  g_weight_kernel<<<grid1d((int64_t)nc * jc * nv * nv * nv, 256), 256, 0, s>>>(
      G, jc, j0, nc, nw, nv, eps, theta, Gw);
  CVS_CHECK_LAUNCH();
}

void h_weight(cudaStream_t s, const cplx* h, int j, int nc, int nw, int nv,
              const double* eps, double theta, cplx* Hw) {
  h_weight_kernel<<<grid1d((int64_t)nv * nv * nc * nc, 256), 256, 0, s>>>(
      h, j, nc, nw, nv, eps, theta, Hw);
  CVS_CHECK_LAUNCH();
}

void schur_assemble(cudaStream_t s, const cplx* M11, const cplx* C11,
                    const cplx* C12, const cplx* h, int nc, int nw, int nv,
                    const double* eps, double theta, cplx* S22, cplx* S) {
  const int64_t N1 = (int64_t)nc * nv;
  s22_kernel<<<nv, 128, 0, s>>>(h, nc, nw, nv, eps, theta, S22);
  CVS_CHECK_LAUNCH();
  schur_assemble_kernel<<<grid1d(N1 * N1, 128), 128, 0, s>>>(
      M11, C11, C12, S22, h, nc, nw, nv, eps, theta, S);
  CVS_CHECK_LAUNCH();
}

// Eigen-decomposition A = U diag(w) U^H of a Hermitian n x n matrix (A is
// overwritten; V is an n x n work matrix; part holds 2 * 304 doubles; cc,
// se hold n/2 + 1 entries).  Sweeps until the off-diagonal norm falls below
// 1e-13 of the total (at most max_sweeps); returns the sweeps done.
int jacobi_eigh_parallel(cudaStream_t s, cplx* A, int n, double* w, cplx* U,
                         cplx* V, double* part, double* cc, cplx* se,
                         int max_sweeps) {
  CVS_REQUIRE(n >= 1 && n <= 16384, -1, "jacobi_eigh_parallel: n out of range");
  const int np = (n + 1) & ~1;
  const int half = np / 2;
  pj_identity_kernel<<<grid1d((int64_t)n * n, 256), 256, 0, s>>>(V, n);
  CVS_CHECK_LAUNCH();
  const unsigned gp = (unsigned)std::max(1, (half + 127) / 128);
  const unsigned gr = grid1d((int64_t)half * n, 256);
  int sweep = 0;
  double prev = 1e300;
  std::vector<double> hp(2 * 304);
  for (; sweep < max_sweeps; ++sweep) {
    pj_offnorm_kernel<<<304, 256, 0, s>>>(A, n, part);
    CVS_CHECK_LAUNCH();
    CVS_CUDA(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaStreamSynchronize(s));
    double off = 0.0, tot = 0.0;
    for (int b = 0; b < 304; ++b) {
      off += hp[2 * b];
      tot += hp[2 * b + 1];
    }
    const double ratio = tot > 0.0 ? std::sqrt(off / tot) : 0.0;
    // converged, or stalled at the rounding level of the largest entries
    if (ratio < 1e-10 || (ratio < 1e-7 && ratio > 0.5 * prev)) break;
    prev = ratio;
    for (int st = 0; st < np - 1; ++st) {
      pj_params_kernel<<<gp, 128, 0, s>>>(A, n, np, st, cc, se);
      CVS_CHECK_LAUNCH();
      pj_rows_kernel<<<gr, 256, 0, s>>>(A, n, np, st, cc, se);
      CVS_CHECK_LAUNCH();
      pj_cols_kernel<<<gr, 256, 0, s>>>(A, V, n, np, st, cc, se);
      CVS_CHECK_LAUNCH();
    }
  }
  pj_sort_kernel<<<grid1d(n, 128), 128, 0, s>>>(A, V, n, w, U);
  CVS_CHECK_LAUNCH();
  return sweep;
}

void fold_doubles(cudaStream_t s, const cplx* R, const cplx* U2,
                  const double* theta, int k, int64_t N, int64_t N1, int nc,
                  int nw, int nv, const double* eps, bool zero_singles,
                  cplx* out) {
  const int64_t rows = (int64_t)nc * nw * nv;
  dim3 grid((unsigned)std::min<int64_t>(std::max<int64_t>(rows, 1), 152 * 16), k);
  fold_doubles_kernel<<<grid, 128, 0, s>>>(R, U2, theta, N, N1, nc, nw, nv, eps,
                                           zero_singles ? 1 : 0, out);
  CVS_CHECK_LAUNCH();
}

double fold_norm(cudaStream_t s, const cplx* u, int64_t N, int64_t N1, int nc,
                 int nw, int nv, const double* eps, double theta,
                 double* part) {
  (void)N;
  fold_norm_kernel<<<304, 128, 0, s>>>(u, N1, nc, nw, nv, eps, theta, part);
  CVS_CHECK_LAUNCH();
  std::vector<double> hp(304);
  CVS_CUDA(cudaMemcpyAsync(hp.data(), part, 304 * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  CVS_CUDA(cudaStreamSynchronize(s));
  double t = 0.0;
  for (double x : hp) t += x;
  return t;
}

void diag_precond(cudaStream_t s, const cplx* r, double theta,
                  const double* diag, int64_t N, cplx* out) {
  diag_precond_kernel<<<grid1d(N, 256), 256, 0, s>>>(r, theta, diag, N, out);
  CVS_CHECK_LAUNCH();
}

void eig_shift(cudaStream_t s, cplx* Y, int64_t n1, int k, const double* lam,
               const double* theta) {
  eig_shift_kernel<<<grid1d(n1 * k, 256), 256, 0, s>>>(Y, n1, k, lam, theta);
  CVS_CHECK_LAUNCH();
}

void h_weight_mean(cudaStream_t s, const cplx* h, int j, int nc, int nw, int nv,
                   const double* eps, double theta, double ebar, int power, cplx* Hw) {
  h_weight_mean_kernel<<<grid1d((int64_t)nv * nc * nc, 256), 256, 0, s>>>(
      h, j, nc, nw, nv, eps, theta, ebar, power, Hw);
  CVS_CHECK_LAUNCH();
}

void add_row_scaled(cudaStream_t s, cplx* C, const cplx* P, int nv, int nq,
                    const double* eps, int o, double ebar) {
  add_row_scaled_kernel<<<grid1d((int64_t)nv * nv * nq, 256), 256, 0, s>>>(C, P, nv, nq, eps,
                                                                          o, ebar);
  CVS_CHECK_LAUNCH();
}

void eig_shift_partial(cudaStream_t s, cplx* Y, int p, int k, const double* lam,
                       const double* d, double theta0, const double* theta, double lam_c) {
  eig_shift_partial_kernel<<<grid1d((int64_t)p * k, 256), 256, 0, s>>>(Y, p, k, lam, d, theta0,
                                                                       theta, lam_c);
  CVS_CHECK_LAUNCH();
}

void eig_shift_d(cudaStream_t s, cplx* Y, int64_t n1, int k, const double* lam,
                 const double* d, double theta0, const double* theta) {
  eig_shift_d_kernel<<<grid1d(n1 * k, 256), 256, 0, s>>>(Y, n1, k, lam, d, theta0, theta);
  CVS_CHECK_LAUNCH();
}

void add_singles(cudaStream_t s, const cplx* a, const cplx* b, int64_t N,
                 int64_t n1, int k, cplx* out) {
  add_singles_kernel<<<grid1d(n1 * k, 256), 256, 0, s>>>(a, b, N, n1, k, out);
  CVS_CHECK_LAUNCH();
}

}  // namespace cvs
