// FP64 complex Hermitian eigensolver: cyclic Jacobi with the round-robin
// (Brent-Luk) pair ordering, so that the n/2 rotations of one step act on
// disjoint index pairs and are applied in parallel by one CTA.  Used for
// the Davidson subspace matrix and for the MP2 vv density and the
// truncated Fock block of the frozen-natural-spinor step (Eqs. 17 and 19).
//
// Each rotation zeroes a_pq with the unitary J = [[c, s e], [-s conj(e), c]]
// (e = a_pq/|a_pq|, t = tan(theta) = sgn(tau)/(|tau| + sqrt(1+tau^2)),
// tau = (a_qq - a_pp)/(2|a_pq|)): A <- J^H A J, V <- V J.
#include "common.cuh"
#include "kernels.cuh"

namespace cvs {

namespace {

__global__ void __launch_bounds__(1024)
    jacobi_kernel(cplx* A, int n, double* w, cplx* V, int max_sweeps,
                  double* info) {
  extern __shared__ char smem[];
  const int np = (n + 1) & ~1;
  const int half = np / 2;
  cplx* se = (cplx*)smem;                 // [half] s * e per pair
  double* cc = (double*)(se + half);      // [half] c per pair
  int* arr = (int*)(cc + half);           // [np] tournament positions
  __shared__ double red[32];
  __shared__ int stop;
  const int tid = threadIdx.x, nt = blockDim.x;

  for (int64_t e = tid; e < (int64_t)n * n; e += nt) {
    int r = e / n, c = e % n;
    V[e] = cmake(r == c ? 1.0 : 0.0, 0.0);
  }
  for (int k = tid; k < np; k += nt) arr[k] = k;
  __syncthreads();

  int sweep = 0;
  double ratio = 0.0;
  for (; sweep <= max_sweeps; ++sweep) {
    // convergence: off-diagonal norm against the full norm
    double off = 0.0, tot = 0.0;
    for (int64_t e = tid; e < (int64_t)n * n; e += nt) {
      int r = e / n, c = e % n;
      cplx a = A[e];
      double m2 = a.x * a.x + a.y * a.y;
      tot += m2;
      if (r != c) off += m2;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_down_sync(0xffffffffu, off, o);
      tot += __shfl_down_sync(0xffffffffu, tot, o);
    }
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int q = 0; q < (nt + 31) / 32; ++q) s += red[q];
      red[0] = s;
    }
    __syncthreads();
    double offs = red[0];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = tot;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int q = 0; q < (nt + 31) / 32; ++q) s += red[q];
      ratio = s > 0 ? sqrt(offs / s) : 0.0;
      stop = (ratio < 1e-15) || (sweep == max_sweeps);
      red[1] = ratio;
    }
    __syncthreads();
    ratio = red[1];
    if (stop) break;

    for (int step = 0; step < np - 1; ++step) {
      // rotation parameters from the current matrix
      for (int k = tid; k < half; k += nt) {
        int p = arr[k], q = arr[np - 1 - k];
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        double c = 1.0;
        cplx sv = cmake(0, 0);
        if (q < n) {
          cplx apq = A[(int64_t)p * n + q];
          double r = hypot(apq.x, apq.y);
          double app = A[(int64_t)p * n + p].x, aqq = A[(int64_t)q * n + q].x;
          if (r > 1e-300 && r > 1e-18 * sqrt(fabs(app * aqq))) {
            double tau = (aqq - app) / (2.0 * r);
            double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            double s = t * c;
            sv = cmake(s * apq.x / r, s * apq.y / r);  // s * e
          }
        }
        cc[k] = c;
        se[k] = sv;
      }
      __syncthreads();
      // rows: A <- J^H A
      for (int64_t e = tid; e < (int64_t)half * n; e += nt) {
        int k = e / n, col = e % n;
        int p = arr[k], q = arr[np - 1 - k];
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        if (q >= n) continue;
        double c = cc[k];
        cplx sv = se[k];
        if (sv.x == 0.0 && sv.y == 0.0) continue;
        cplx ap = A[(int64_t)p * n + col], aq = A[(int64_t)q * n + col];
        // row p: c a_p - (s e) a_q ; row q: conj(s e) a_p + c a_q
        A[(int64_t)p * n + col] = csub(cscale(ap, c), cmul(sv, aq));
        A[(int64_t)q * n + col] = cadd(cmul(cconj(sv), ap), cscale(aq, c));
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int64_t e = tid; e < (int64_t)half * n; e += nt) {
        int k = e / n, row = e % n;
        int p = arr[k], q = arr[np - 1 - k];
        if (p > q) {
          int t = p;
          p = q;
          q = t;
        }
        if (q >= n) continue;
        double c = cc[k];
        cplx sv = se[k];
        if (sv.x == 0.0 && sv.y == 0.0) continue;
        // col p: c a_p - conj(s e) a_q ; col q: (s e) a_p + c a_q
        cplx ap = A[(int64_t)row * n + p], aq = A[(int64_t)row * n + q];
        A[(int64_t)row * n + p] = csub(cscale(ap, c), cmul(cconj(sv), aq));
        A[(int64_t)row * n + q] = cadd(cmul(sv, ap), cscale(aq, c));
        cplx vp = V[(int64_t)row * n + p], vq = V[(int64_t)row * n + q];
        V[(int64_t)row * n + p] = csub(cscale(vp, c), cmul(cconj(sv), vq));
        V[(int64_t)row * n + q] = cadd(cmul(sv, vp), cscale(vq, c));
      }
      __syncthreads();
      // advance the tournament: position 0 fixed, the rest rotate
      if (tid == 0) {
        int last = arr[np - 1];
        for (int k = np - 1; k > 1; --k) arr[k] = arr[k - 1];
        arr[1] = last;
      }
      __syncthreads();
    }
  }

  // ascending eigenvalues: rank sort, permuted copy of V through A
  for (int i = tid; i < n; i += nt) {
    double wi = A[(int64_t)i * n + i].x;
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      double wj = A[(int64_t)j * n + j].x;
      rank += (wj < wi) || (wj == wi && j < i);
    }
    arr[i] = rank;
  }
  __syncthreads();
  for (int i = tid; i < n; i += nt) w[arr[i]] = A[(int64_t)i * n + i].x;
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)n * n; e += nt) {
    int r = e / n, c = e % n;
    A[(int64_t)r * n + arr[c]] = V[e];
  }
  __syncthreads();
  for (int64_t e = tid; e < (int64_t)n * n; e += nt) V[e] = A[e];
  if (tid == 0 && info) {
    info[0] = sweep;
    info[1] = ratio;
  }
}

}  // namespace

void jacobi_eigh(cudaStream_t s, cplx* A, int n, double* w, cplx* Vec,
                 int max_sweeps, double* info_dev) {
  CVS_REQUIRE(n >= 1 && n <= 4096, -1, "jacobi_eigh: n out of range");
  int np = (n + 1) & ~1;
  int half = np / 2;
  size_t sh = (size_t)(np + 2) * sizeof(int) + (size_t)(half + 2) * sizeof(double) +
              (size_t)half * sizeof(cplx) + 64;
  jacobi_kernel<<<1, 1024, sh, s>>>(A, n, w, Vec, max_sweeps, info_dev);
  CVS_CHECK_LAUNCH();
}

}  // namespace cvs
