// Elementwise kernels of the adjoint (gradient) pass: the backward of the
// M11 assembly, of the t2 epilogue (with the energy denominators), of the
// on-the-fly M22, and the Hermitian projection of the B^P gradient.
//
// Convention: for a real objective f and a complex variable z the gradient
// is g_z = df/dRe z + i df/dIm z, so df = Re sum conj(g_z) dz.
#include "common.cuh"
#include "kernels.cuh"

namespace cvs {

namespace {

__device__ __forceinline__ void atomic_add_d(double* p, double v) {
  atomicAdd(p, v);
}

// gM = conj(rho): M11 = d d (e_a - e_I) - (C1 - C2) - 1/4 d_IJ (X + X^H)
//                 - 1/4 d_ab (Y + Y^H) + 1/2 (Z + Z^H)
__global__ void m11_back_kernel(const cplx* __restrict__ rho, int nc, int nv,
                                int o, cplx* gC1, cplx* gC2, cplx* gZ,
                                double* gE) {
  const int64_t N1 = (int64_t)nc * nv;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < N1 * N1; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / N1, col = idx % N1;
    const int I = row / nv, a = row % nv, J = col / nv, b = col % nv;
    const cplx g = cconj(rho[idx]);
    const cplx gT = cconj(cconj(rho[col * N1 + row]));  // conj(gM[col][row])
    gC1[((int64_t)a * nv + b) * (nc * nc) + J * nc + I] = cscale(g, -1.0);
    gC2[idx] = g;
    gZ[idx] = cscale(cadd(g, gT), 0.5);
    if (row == col) {
      const double d = rho[idx].x;
      atomic_add_d(&gE[o + a], d);
      atomic_add_d(&gE[I], -d);
    }
  }
}

// gX[a][b] = -1/4 sum_I (gM[Ia,Ib] + conj(gM[Ib,Ia])), gY likewise over a
__global__ void m11_back_small_kernel(const cplx* __restrict__ rho, int nc,
                                      int nv, cplx* gX, cplx* gY) {
  const int64_t N1 = (int64_t)nc * nv;
  const int64_t nx = (int64_t)nv * nv, ny = (int64_t)nc * nc;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < nx + ny; idx += (int64_t)gridDim.x * blockDim.x) {
    cplx acc = cmake(0, 0);
    if (idx < nx) {
      const int a = idx / nv, b = idx % nv;
      for (int I = 0; I < nc; ++I) {
        const cplx g1 = cconj(rho[((int64_t)I * nv + a) * N1 + I * nv + b]);
        const cplx g2 = rho[((int64_t)I * nv + b) * N1 + I * nv + a];
        acc = cadd(acc, cadd(g1, g2));
      }
      gX[idx] = cscale(acc, -0.25);
    } else {
      const int64_t e = idx - nx;
      const int I = e / nc, J = e % nc;
      for (int a = 0; a < nv; ++a) {
        const cplx g1 = cconj(rho[((int64_t)I * nv + a) * N1 + J * nv + a]);
        const cplx g2 = rho[((int64_t)J * nv + a) * N1 + I * nv + a];
        acc = cadd(acc, cadd(g1, g2));
      }
      gY[e] = cscale(acc, -0.25);
    }
  }
}

// t2 = g2/D, g2 = (ai|bj) - (aj|bi):  gR = g_t2 / D + g_g2 (in place over
// g_g2), and the denominators' share of gE.
__global__ void t2_back_kernel(const cplx* __restrict__ gt2, cplx* gg2,
                               const cplx* __restrict__ g2, int o, int v,
                               const double* __restrict__ eps, double* gE) {
  const int64_t total = (int64_t)o * o * v * v;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = idx % v;
    int64_t r = idx / v;
    const int a = r % v;
    r /= v;
    const int j = r % o, i = r / o;
    const double D = eps[i] + eps[j] - eps[o + a] - eps[o + b];
    const cplx gt = gt2[idx];
    const cplx gg = gg2[idx];
    const cplx g = g2[idx];
    gg2[idx] = cadd(gg, cscale(gt, 1.0 / D));
    // d t / d D = -g / D^2;  df = Re conj(gt) (-g/D^2) dD
    const double dD = -(gt.x * g.x + gt.y * g.y) / (D * D);
    if (dD != 0.0) {
      atomic_add_d(&gE[i], dD);
      atomic_add_d(&gE[j], dD);
      atomic_add_d(&gE[o + a], -dD);
      atomic_add_d(&gE[o + b], -dD);
    }
  }
}

// gQband[(al,i),(b,j)] = gR[i][j][a][b] - gR[j][i][a][b] for a = a0 + al
__global__ void q_back_band_kernel(const cplx* __restrict__ gR, int a0, int na,
                                   int o, int v, cplx* gQ) {
  const int64_t ldQ = (int64_t)v * o;
  const int64_t total = (int64_t)na * o * ldQ;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = idx / ldQ, col = idx % ldQ;
    const int al = row / o, i = row % o;
    const int b = col / o, j = col % o;
    const int a = a0 + al;
    const cplx x = gR[(((int64_t)i * o + j) * v + a) * v + b];
    const cplx y = gR[(((int64_t)j * o + i) * v + a) * v + b];
    gQ[idx] = csub(x, y);
  }
}

// M22 = e_a + e_b - e_I - e_j on packed doubles: gE from |x2|^2
__global__ void m22_back_kernel(const cplx* __restrict__ X, int k, int64_t N,
                                int64_t N1, int nc, int nw, int nv,
                                double* gE) {
  const int64_t npair = (int64_t)nv * (nv - 1) / 2;
  const int o = nc + nw;
  const int64_t nrows = (int64_t)nc * nw * nv;
  for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
    const int a = row % nv;
    int64_t r = row / nv;
    const int j = r % nw, I = r / nw;
    const int64_t base = ((int64_t)I * nw + j) * npair +
                         ((int64_t)a * (2 * nv - a - 1) / 2) - (a + 1);
    double sa = 0.0;
    for (int b = a + 1 + threadIdx.x; b < nv; b += blockDim.x) {
      double w = 0.0;
      for (int q = 0; q < k; ++q) {
        const cplx x = X[q * N + N1 + base + b];
        w += x.x * x.x + x.y * x.y;
      }
      sa += w;
      if (w != 0.0) atomic_add_d(&gE[o + b], w);
    }
    // block sum for the a, I, j shares
    __shared__ double red[128];
    red[threadIdx.x] = sa;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0 && red[0] != 0.0) {
      atomic_add_d(&gE[o + a], red[0]);
      atomic_add_d(&gE[I], -red[0]);
      atomic_add_d(&gE[nc + j], -red[0]);
    }
    __syncthreads();
  }
}

// G^P <- (G^P + G^P^H) / 2 in place, every P
__global__ void herm_project_kernel(cplx* G, int n, int64_t nmat) {
  const int64_t per = (int64_t)n * (n + 1) / 2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
       idx < nmat * per; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t P = idx / per;
    int64_t e = idx % per;
    // e -> (p <= q) in row-major upper triangle
    int p = 0;
    while (e >= n - p) {
      e -= n - p;
      ++p;
    }
    const int q = p + (int)e;
    cplx* A = G + P * n * (int64_t)n;
    const cplx x = A[(int64_t)p * n + q], y = A[(int64_t)q * n + p];
    const cplx h = cscale(cadd(x, cconj(y)), 0.5);
    A[(int64_t)p * n + q] = h;
    A[(int64_t)q * n + p] = cconj(h);
  }
}

}  // namespace

void m11_backward(cudaStream_t s, const cplx* rho, int nc, int nv, int o,
                  cplx* gC1, cplx* gC2, cplx* gX, cplx* gY, cplx* gZ,
                  double* gE) {
  const int64_t N1 = (int64_t)nc * nv;
  m11_back_kernel<<<grid1d(N1 * N1, 256), 256, 0, s>>>(rho, nc, nv, o, gC1, gC2,
                                                       gZ, gE);
  CVS_CHECK_LAUNCH();
  m11_back_small_kernel<<<grid1d((int64_t)nv * nv + nc * nc, 128), 128, 0, s>>>(
      rho, nc, nv, gX, gY);
  CVS_CHECK_LAUNCH();
}

void t2_backward(cudaStream_t s, const cplx* gt2, cplx* gg2, const cplx* g2,
                 int o, int v, const double* eps, double* gE) {
  t2_back_kernel<<<grid1d((int64_t)o * o * v * v, 256), 256, 0, s>>>(
      gt2, gg2, g2, o, v, eps, gE);
  CVS_CHECK_LAUNCH();
}

void q_backward_band(cudaStream_t s, const cplx* gR, int a0, int na, int o,
                     int v, cplx* gQ) {
  q_back_band_kernel<<<grid1d((int64_t)na * o * v * o, 256), 256, 0, s>>>(
      gR, a0, na, o, v, gQ);
  CVS_CHECK_LAUNCH();
}

void m22_backward(cudaStream_t s, const cplx* X, int k, int64_t N, int64_t N1,
                  int nc, int nw, int nv, double* gE) {
  const int64_t rows = (int64_t)nc * nw * nv;
  const unsigned g = rows > 65535 * 8 ? 65535 * 8 : (unsigned)rows;
  m22_back_kernel<<<g, 128, 0, s>>>(X, k, N, N1, nc, nw, nv, gE);
  CVS_CHECK_LAUNCH();
}

void herm_project(cudaStream_t s, cplx* G, int n, int64_t nmat) {
  herm_project_kernel<<<grid1d(nmat * n * (int64_t)(n + 1) / 2, 256), 256, 0,
                        s>>>(G, n, nmat);
  CVS_CHECK_LAUNCH();
}

}  // namespace cvs
