// Host-side launchers of the libcvsadc device kernels.
#pragma once

#include "common.cuh"

namespace cvs {

// ------------------------------------------------------------- GEMMs
// C = alpha * A * B + beta * C, complex, two-mode views, batch over z.
// `part` (part_elems complex) is scratch for split-K partial products; with
// part == nullptr the kernel runs without splitting.
void zgemm_f64(cudaStream_t s, int M, int N, int K, double alpha, View A,
               View B, double beta, View C, int batch = 1,
               cplx* part = nullptr, size_t part_elems = 0);
// C(m, n) = sum_z part[z][m][n] + beta * C(m, n), part dense [nz][M][N]
void splitk_reduce(cudaStream_t s, int M, int N, int nz, const cplx* part,
                   double beta, View C);
void init_gemm_attributes();

// Same contract on the tcgen05 tensor cores: A and B are split into bf16
// parts, nprod = 3 (hi/lo, BF16x3) or 6 (hi/mid/lo, BF16x6) products per
// real product, FP32 accumulation.  `work` must hold
// tc_workspace_bytes(M, N, K, nprod) bytes; a bounded wait that expires
// writes a non-zero code to *err (device int, never cleared here).
size_t tc_workspace_bytes(int M, int N, int K, int nprod);
void zgemm_tc(cudaStream_t s, int nprod, int M, int N, int K, double alpha,
              View A, View B, double beta, View C, void* work,
              size_t work_bytes, cplx* part, size_t part_elems, int* err);
bool tc_available();
// Exact-accumulation slice GEMM on the tensor cores (see gemm_tc.cu):
// nslices = 4 (10 slice products, ~2^-28 of row max x column max) or 7
// (28 products, FP64 class).
// one bounded wait that expires after limit_ns (clamped to [1 ms, 4 s]) and
// records its code in *err
void wait_probe(cudaStream_t s, int64_t limit_ns, int* err);
// workspace of one call (b_cached / a_cached: B / A comes from a SliceBCache)
size_t slice_workspace_bytes(int M, int N, int K, int nslices, bool b_cached = false,
                             bool a_cached = false);
// Packed slices (and column or row exponents) of a B (or A) operand that
// does not change between calls, over its whole K; filled by the first call
// that gets it.
struct SliceBCache {
  void* base = nullptr;
  size_t bytes = 0;
  bool filled = false;
};
// bytes such a cache needs for a K x N operand (independent of M)
size_t slice_bcache_bytes(int N, int K, int nslices);
// the same for an M x K A operand (4 slices only: packed rows and row
// exponents over the whole K)
size_t slice_acache_bytes(int M, int K, int nslices);
// rows per slab when a tall product is better split over M with K whole
// (its A packs dominate and K would otherwise run in chunks); M when not
int64_t slice_row_slab(int M, int N, int K, int nslices);
void zgemm_slice(cudaStream_t s, int nslices, int M, int N, int K,
                 double alpha, View A, View B, double beta, View C, void* work,
                 size_t work_bytes, cplx* part, size_t part_elems, int* err, SliceBCache* bc = nullptr,
                 SliceBCache* ac = nullptr);

// C = beta * C over a view
void scale_view(cudaStream_t s, int M, int N, double beta, View C, int batch);

// --------------------------------------------------------- utilities
// max |B_pq - conj(B_qp)| and max |B_pq| over nmat n x n matrices;
// out[0], out[1] (device doubles, zeroed by the launcher).
void hermiticity(cudaStream_t s, const cplx* B, int n, int64_t nmat,
                 double* out_dev);

// ------------------------------------------------------------ MP2 / t2
// From V[(al, i), (b, j)] = (a i | b j) for a = a0 + al, write
// g2[i][j][a][b] = <ab||ij> = V[(al,i),(b,j)] - V[(al,j),(b,i)] and
// t2 = g2 / (e_i + e_j - e_a - e_b) for a in [a0, a0+na); accumulate
// 1/4 |g2|^2 / den into per-block partials part[nblk].
void t2_band(cudaStream_t s, const cplx* V, int a0, int na, int o, int v,
             const double* eps, cplx* t2, cplx* g2, double* part, int nblk);
// Band transform in place: X [al][i][b][j] = (a i|b j) for a = a0 + al
// becomes <ab||ij>, T (same layout) = t^{ab}_{ij}; *emp2 (device) += the
// band's share of E_MP2.  part must hold t2_band_ip_blocks(nb, o, v)
// doubles.
int64_t t2_band_ip_blocks(int nb, int o, int v);
void t2_band_inplace(cudaStream_t s, cplx* X, cplx* T, int a0, int nb, int o,
                     int v, const double* eps, double* part, double* emp2);
// Lorentzian-broadened spectrum on a uniform grid (see cvsadc_spectrum)
void lorentz_spectrum(cudaStream_t s, const double* omega, const double* f, int nroots,
                      double e0, double de, int npts, double fwhm, double shift,
                      double ev_per_eh, double* out);
// Deterministic sum of n doubles into *out (device).
void reduce_sum(cudaStream_t s, const double* in, int n, double* out);

// ----------------------------------------------------------------- M11
// M11 assembly from the pieces (see solver.cu).
void m11_assemble(cudaStream_t s, int ncore, int nvirt, int o,
                  const double* eps, const cplx* C1, const cplx* C2,
                  const cplx* X, const cplx* Y, const cplx* Z, int second,
                  cplx* M11);

// --------------------------------------------------------------- sigma
// Yt[I][a][j][b] = antisymmetric unpack of packed doubles x2.
void unpack_doubles(cudaStream_t s, const cplx* x2, int ncore, int nval,
                    int nvirt, cplx* Yt);
// sigma2[d] = -(G[I,a,j,b] - G[I,b,j,a]) + (e_a+e_b-e_I-e_j) x2[d] plus the
// <Kb||Ij> terms of x1 (h != NULL): in FP64 (fp64) or double-float
void sigma2_finish(cudaStream_t s, const cplx* G, const cplx* x2,
                   const cplx* x1, const cplx* h, const double* eps, int ncore,
                   int nval, int nvirt, cplx* s2, bool fp64);
void h_conj_transpose(cudaStream_t s, const cplx* h, int nc, int nw, int nv,
                      cplx* hT);
// pack an antisymmetric-by-construction full tensor F[I][j][a][b] with
// F = -(A[a][b] - A[b][a]) + T[a][b] into packed doubles (a < b).
void pack_moment_doubles(cudaStream_t s, const cplx* A, const cplx* T,
                         int ncore, int nval, int nvirt, cplx* out);
// diagonal of M: dM11 (from M11) and M22 on the fly, into diag[N] (real)
void build_diag(cudaStream_t s, const cplx* M11, const double* eps,
                int ncore, int nval, int nvirt, double* diag);

// ------------------------------------------------------------ Davidson
// Arithmetic of ts_dot / ts_combine / ts_subtract: fp64 = true runs plain
// FP64 FMAs (the FP64-class precisions); fp64 = false runs double-float
// (float hi/lo pairs, ~48-bit significand, float exponent range) on the
// FP32 pipes (the mixed precisions).  Both stage 16-element tiles and sum
// the tile results in FP64.
// out[i*ldo + j] = sum_n conj(A[i][n]) B[j][n], i < ma, j < mb
// part must hold ma*mb*TS_CHUNKS complex.
constexpr int TS_CHUNKS = 304;
void ts_dot(cudaStream_t s, const cplx* A, int ma, const cplx* B, int mb,
            int64_t N, cplx* part, cplx* out, int ldo, bool fp64 = false);
// out[r][n] = sum_i W[i][n] cw[i*ldc + r] + V[i][n] cv[i*ldc + r], r < k
// (either input may be NULL); out may not alias inputs.
void ts_combine(cudaStream_t s, const cplx* V, const cplx* cv,
                const cplx* W, const cplx* cw, int m, int ldc, int k,
                int64_t N, cplx* out, bool fp64 = false);
// t[r] = (AX[r] - theta[r] X[r]) / (theta[r] - diag), |denominator|
// clamped to >= 1e-4; rnorm2[r] = ||AX[r] - theta[r] X[r]||^2.
void residual_precond(cudaStream_t s, const cplx* AX, const cplx* X,
                      const double* theta, const double* diag, int k,
                      int64_t N, cplx* t, double* part, double* rnorm2);
// y[r] -= sum_i V[i] c[i*ldc+r] for r < k (classical Gram-Schmidt step;
// c laid out as ts_dot writes it)
void ts_subtract(cudaStream_t s, const cplx* V, int m, const cplx* c,
                 int ldc, int k, int64_t N, cplx* y, bool fp64 = false);
// x[r] *= scale[r]
void scale_vectors(cudaStream_t s, cplx* x, const double* scale, int k,
                   int64_t N);
// generic strided copy dst(r, c) = alpha * src(r, c)
// dst[r][q] = src[r][idx[q]] (row-major, leading dimensions lds / ldd;
// idx a device array of ncols column indices)
void gather_columns(cudaStream_t s, const cplx* src, int rows, int64_t lds, const int* idx,
                    int ncols, cplx* dst, int64_t ldd);
void copy_view(cudaStream_t s, int M, int N, double alpha, View src, View dst);
// indices of the k smallest entries of d[N] (ascending), k <= 64
void k_smallest(cudaStream_t s, const double* d, int64_t N, int k,
                int64_t* idx_dev, double* work);
// make the largest-modulus entry of each of k vectors real positive
void phase_fix(cudaStream_t s, cplx* x, int k, int64_t N, double* work);
// A = (H + H^H)/2 for an m x m block of H (leading dimension ldh); entries
// H[i][j] with j < jdone <= i were not computed and are taken from the
// Hermitian partner (jdone = m when every entry is present)
void hermitize(cudaStream_t s, const cplx* H, int ldh, int m, cplx* A,
               int jdone);
// H[i][j] = conj(H[j][i]) for i0 <= i < i1, j < i0
void herm_fill(cudaStream_t s, cplx* H, int ldh, int i0, int i1);
// transform X (cnt x kept) making the block with Gram matrix G orthonormal
// (Gram-Schmidt in coefficient space, cnt <= 64); src[q] (optional) = the
// input vector kept column q was started from
void block_orth(cudaStream_t s, const cplx* G, int ldg, int cnt,
                const double* norm0, double tol, cplx* X, int* kept,
                int* src = nullptr);
void gram_diag_sqrt(cudaStream_t s, const cplx* G, int ldg, int cnt,
                    double* out);
// X[r][c] *= sc[r] (device scale vector)
void scale_rows(cudaStream_t s, cplx* X, int rows, int cols, int ld,
                const double* sc);
// one-time kernel attribute setup for the current device
void init_kernel_attributes();

// ------------------------------------------------------------ adjoint
// backward of the M11 assembly from rho[s][t] = sum_n conj(x_s) x_t
void m11_backward(cudaStream_t s, const cplx* rho, int nc, int nv, int o,
                  cplx* gC1, cplx* gC2, cplx* gX, cplx* gY, cplx* gZ,
                  double* gE);
// gg2 <- gg2 + gt2 / D (in place) and the denominators' share of gE
void t2_backward(cudaStream_t s, const cplx* gt2, cplx* gg2, const cplx* g2,
                 int o, int v, const double* eps, double* gE);
// gQ band [(al,i),(b,j)] from gR [i][j][a][b]
void q_backward_band(cudaStream_t s, const cplx* gR, int a0, int na, int o,
                     int v, cplx* gQ);
// M22's share of gE from k packed vectors X [k][N]
void m22_backward(cudaStream_t s, const cplx* X, int k, int64_t N, int64_t N1,
                  int nc, int nw, int nv, double* gE);
// G^P <- (G^P + G^P^H)/2 for nmat n x n matrices
void herm_project(cudaStream_t s, cplx* G, int n, int64_t nmat);

// ---------------------------------------------------- Jacobi (FP64)
// Hermitian eigensolver: A [n][n] row-major (destroyed), eigenvalues w
// ascending, eigenvectors as columns of Vec [n][n].  One CTA, cyclic
// round-robin (Brent-Luk) ordering; at most max_sweeps sweeps.
// info_dev[0] = sweeps used (as double), [1] = final off-norm ratio.
void jacobi_eigh(cudaStream_t s, cplx* A, int n, double* w, cplx* Vec,
                 int max_sweeps, double* info_dev);

// Schur-complement preconditioner (schur_kernels.cu)
void h_assemble(cudaStream_t s, const cplx* hc1, const cplx* hc2, int nc,
                int nw, int nv, cplx* h);
// G[jl][a][b][c] = <ab||cj> from X1 = (ac|bj) and X2 = (aj|bc); with X2 ==
// NULL the second comes from X1 as (bc|aj)
void g_assemble(cudaStream_t s, const cplx* X1, const cplx* X2, int jc, int nv,
                cplx* G);
void g_weight(cudaStream_t s, const cplx* G, int jc, int j0, int nc, int nw,
              int nv, const double* eps, double theta, cplx* Gw);
void h_weight(cudaStream_t s, const cplx* h, int j, int nc, int nw, int nv,
              const double* eps, double theta, cplx* Hw);
void schur_assemble(cudaStream_t s, const cplx* M11, const cplx* C11,
                    const cplx* C12, const cplx* h, int nc, int nw, int nv,
                    const double* eps, double theta, cplx* S22, cplx* S);
int jacobi_eigh_parallel(cudaStream_t s, cplx* A, int n, double* w, cplx* U,
                         cplx* V, double* part, double* cc, cplx* se,
                         int max_sweeps);
void fold_doubles(cudaStream_t s, const cplx* R, const cplx* U2,
                  const double* theta, int k, int64_t N, int64_t N1, int nc,
                  int nw, int nv, const double* eps, bool zero_singles,
                  cplx* out);
double fold_norm(cudaStream_t s, const cplx* u, int64_t N, int64_t N1, int nc,
                 int nw, int nv, const double* eps, double theta,
                 double* part);
void eig_shift(cudaStream_t s, cplx* Y, int64_t n1, int k, const double* lam,
               const double* theta);
void diag_precond(cudaStream_t s, const cplx* r, double theta,
                  const double* diag, int64_t N, cplx* out);
// folded solver (see lift_assemble_kernel in schur_kernels.cu)
void lift_assemble(cudaStream_t s, const cplx* E, const cplx* VD, const cplx* A,
                   const cplx* VV, const double* th, int m, int ld, double delta,
                   cplx* Q, cplx* H, cplx* O);
void lift_coef(cudaStream_t s, const cplx* C, int m, int k, int ldc, const double* w,
               const double* th, cplx* Cp);
void row_axpy(cudaStream_t s, const cplx* X, const cplx* Z, const double* w, int k,
              int64_t n, cplx* Y);
void row_norm2(cudaStream_t s, const cplx* X, int k, int64_t n, double* out);
void inv_sqrt_cols(cudaStream_t s, const cplx* U, const double* w, int m, int off, int kept,
                   int ldu, cplx* Oi);
void h_weight_mean(cudaStream_t s, const cplx* h, int j, int nc, int nw, int nv,
                   const double* eps, double theta, double ebar, int power, cplx* Hw);
void add_row_scaled(cudaStream_t s, cplx* C, const cplx* P, int nv, int nq,
                    const double* eps, int o, double ebar);
void eig_shift_partial(cudaStream_t s, cplx* Y, int p, int k, const double* lam,
                       const double* d, double theta0, const double* theta, double lam_c);
void eig_shift_d(cudaStream_t s, cplx* Y, int64_t n1, int k, const double* lam,
                 const double* d, double theta0, const double* theta);
void add_singles(cudaStream_t s, const cplx* a, const cplx* b, int64_t N,
                 int64_t n1, int k, cplx* out);

}  // namespace cvs
