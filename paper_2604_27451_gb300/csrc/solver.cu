// libcvsadc host orchestration and C ABI.
//
// Stages (section "Implementation and Computational Details"):
//   ingest      copy inputs to the device, check B^P and dipoles Hermitian
//   fns         (tau > 0) MP2 vv density (Eq. 15), natural spinors (Eq. 17),
//               truncation, semicanonicalisation (Eqs. 18-20), rotation of B^P
//   mp2         t2 and E_MP2 from (ai|bj) = sum_P B^P_ai B^P_bj
//   m11         core-singles block through second order
//   moments     modified transition moments through first order
//   davidson    block Davidson on sigma = M x, FP64 subspace algebra
//   refine      (mixed precision) FP64 sigma on the converged vectors
//
// The element formulas (negative-denominator t2, CVS basis operators
// a_a^+ a_I and a_a^+ a_b^+ a_I a_j):
//   M11_{Ia,Jb} = d_IJ d_ab (e_a - e_I) - <aJ||bI> - 1/4 d_IJ Ivv_ab
//                 - 1/4 d_ab Joo_IJ + 1/2 K_{Ia,Jb}
//   M21_{(Ijab),(Kc)} = -d_IK <ab||cj> + d_ac <Kb||Ij> - d_bc <Ka||Ij>
//   M22 = diag(e_a + e_b - e_I - e_j)
// Through B^P the couplings read
//   sigma2_{Ijab} = -(G_{Ia,jb} - G_{Ib,ja}) + M22 x2,
//   G_{Ia,jb} = sum_P (Y - W)^P_{aI} B^P_{bj} - B^P_{aI} V^P_{bj},
//   Y^P_{aI} = sum_c B^P_ac x_Ic, W^P_{aI} = sum_K B^P_KI x_Ka,
//   V^P_{bj} = sum_K B^P_Kj x_Kb,
//   sigma1_{Kc} = M11 x1 - sum_{P,a} B^P_ca S^P_{aK} + sum_{P,I} B^P_IK S^P_{cI}
//                 - sum_{P,j} B^P_jK R^P_{cj},
//   S^P_{aI} = sum_{jb} y_{Ijab} B^P_jb, R^P_{cj} = sum_{Ib} y_{Ijcb} B^P_Ib,
// with y the antisymmetric unpacking of x2; <pq||rs> is never formed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <mutex>
#include <array>
#include <complex>
#include <condition_variable>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/cvsadc.h"
#include "common.cuh"
#include "kernels.cuh"

namespace cvs {
unsigned long long g_launch_count = 0;
}
using namespace cvs;

namespace {

// ------------------------------------------------------- allocation registry
// Every live device buffer, so that a view built on a pointer into one can
// be bounds-checked on the host before any kernel reads through it.
std::mutex g_reg_mu;
std::map<uintptr_t, size_t> g_reg;

void reg_add(const void* p, size_t b) {
  std::lock_guard<std::mutex> l(g_reg_mu);
  g_reg[(uintptr_t)p] = b;
}
void reg_del(const void* p) {
  std::lock_guard<std::mutex> l(g_reg_mu);
  g_reg.erase((uintptr_t)p);
}
// complex elements from p to the end of its registered buffer, or -1
int64_t ext_from(const void* p) {
  std::lock_guard<std::mutex> l(g_reg_mu);
  uintptr_t a = (uintptr_t)p;
  auto it = g_reg.upper_bound(a);
  if (it == g_reg.begin()) return -1;
  --it;
  if (a >= it->first + it->second) return -1;
  return (int64_t)((it->first + it->second - a) / sizeof(cplx));
}
struct RegGuard {  // registers a caller buffer for the duration of a call
  const void* p;
  RegGuard(const void* p_, size_t b) : p(p_) { reg_add(p, b); }
  ~RegGuard() { reg_del(p); }
};

View checked(View v) {
  if (v.ext < 0) v.ext = ext_from(v.p);
  return v;
}

// ------------------------------------------------------------ device buffer
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) {
      reg_del(p);
      cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
  }
  void ensure(size_t b) {
    if (b <= bytes && p) return;
    release();
    if (b == 0) return;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      p = nullptr;
      char msg[160];
      snprintf(msg, sizeof msg, "cudaMalloc of %.3f GB failed", b / 1e9);
      throw Error{CVSADC_ENOMEM, msg};
    }
    bytes = b;
    reg_add(p, b);
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
  cplx* c() const { return (cplx*)p; }
  double* d() const { return (double*)p; }
};

bool verbose() {
  static int v = -1;
  if (v < 0) {
    const char* e = getenv("CVSADC_VERBOSE");
    v = (e && *e && *e != '0') ? 1 : 0;
  }
  return v == 1;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

}  // namespace

struct cvsadc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;

  // prepared problem
  bool prepared = false;
  int ncore = 0, nval = 0, nvirt = 0, nvirt_in = 0, naux = 0, o = 0, n = 0;
  int64_t N1 = 0, npair = 0, N2 = 0, N = 0;
  bool has_dip = false, has_fns = false;
  double emp2 = 0.0;
  int prep_prec = 0;  // precision the prepared problem was built with
  // t2, g2: t2 and <ab||ij> whole, [i][j][a][b]; held only when asked for
  DBuf eps, B, dip, t2, g2, M11, diag, F, fns_occ, fns_U;
  // <Kb||Ij> as h[K][b][I][j], and conj(h) as hT[(I,j,b)][K]
  DBuf h1, hT;

  // scratch
  DBuf s_big1, s_big2, s_S, s_R, s_Y, s_V, s_part, s_small, s_tc;
  DBuf dv_V, dv_W, dv_X, dv_AX, dv_T, dv_H, dv_A, dv_U, dv_w, dv_misc;
  DBuf err;  // device int: non-zero after a bounded device wait expired
  DBuf s_kpart;  // split-K partial products

  // folded solver: fold work vectors [2g][N] x 2, singles-space basis and
  // its folds [msub][N1], small projected matrices
  DBuf fd_A, fd_B, fd_th, fv_V, fv_B, fv_R, fv_D, fv_MV, fv_T, fv_T2, fv_small;

  // Schur-complement preconditioner of the prepared problem
  DBuf sch_W, sch_g, sch_S, sch_U, sch_V, sch_lam, sch_C11, sch_C12, sch_work,
      sch_tmp, sch_th;
  bool sch_on = false;
  // eigenvectors held in sch_U ([N1][sch_p] columns): all N1, or the lowest
  // SCHUR_PL for large singles spaces (the folded solver only)
  int sch_p = 0;
  // first-order drift of the Schur eigenvalues with theta (folded solver)
  DBuf sch_d;
  bool sch_d_on = false;
  double sch_theta = 0.0, sch_ms = 0.0, sch_pole = 0.0;
  int sch_builds = 0, sch_couplings = 0;

  // packed slices of static B^P operands (key: view geometry, sizes,
  // slice count, K chunk), valid for the prepared problem
  struct BEntry {
    DBuf buf;
    SliceBCache sc;
  };
  std::map<std::array<int64_t, 12>, std::unique_ptr<BEntry>> bcache;
  size_t bcache_bytes = 0;
  void clear_bcache() {
    bcache.clear();
    bcache_bytes = 0;
  }

  // worker contexts of cvsadc_solve_batched (own streams), kept for reuse
  std::vector<cvsadc_ctx*> lanes;

  void sync() { CVS_CUDA(cudaStreamSynchronize(stream)); }
  std::vector<DBuf*> problem_buffers() {
    return {&eps,   &B,     &dip,   &t2,   &g2,     &M11,  &diag, &F, &h1, &hT,
            &fns_occ, &fns_U, &s_big1, &s_big2, &s_S, &s_R, &s_Y, &s_V,
            &s_part, &s_small, &s_tc, &dv_V, &dv_W, &dv_X, &dv_AX, &dv_T,
            &dv_H,  &dv_A,  &dv_U,  &dv_w, &dv_misc, &sch_W, &sch_g,
            &sch_S, &sch_U, &sch_V, &sch_lam, &sch_C11, &sch_C12, &sch_work,
            &sch_tmp, &sch_th, &fd_A, &fd_B, &fd_th, &fv_V, &fv_B, &fv_R, &fv_D,
            &fv_MV, &fv_T, &fv_T2, &fv_small};
  }
  // give back every problem-sized buffer (the context stays usable)
  void trim() {
    prepared = false;
    for (DBuf* b : problem_buffers()) b->release();
    sch_on = false;
    clear_bcache();
  }
  size_t held_bytes() {
    size_t t = s_kpart.bytes + err.bytes + bcache_bytes;
    for (DBuf* b : problem_buffers()) t += b->bytes;
    return t;
  }
};

namespace {

bool valid_precision(int p) {
  return p == CVSADC_FP64 || p == CVSADC_MIXED_BF16X3 ||
         p == CVSADC_MIXED_SLICE4 || p == CVSADC_FP64_SLICE7;
}
// precisions whose results need the FP64 residual correction
bool needs_refine(int p) {
  return p == CVSADC_MIXED_BF16X3 || p == CVSADC_MIXED_SLICE4;
}

// --------------------------------------------------------------- GEMM hub
// A cache slot for the packed slices of a GEMM operand (whole K) when the
// caller asks for one (a product repeated on every sigma), the operand is a
// view of the prepared B^P (it does not change between calls) and the
// caches stay within min(35 % of free memory, 64 GB); else NULL.  side 0:
// the B operand (K x N, any slice count); side 1: the A operand (M x K, 4
// slices).
constexpr double BCACHE_MAX = 64e9;
SliceBCache* op_cache(cvsadc_ctx* c, int side, int ns, int MN, int K, const View& X) {
  if (!c->B.p) return nullptr;
  const cplx* b0 = c->B.c();
  const size_t nb = c->B.bytes / sizeof(cplx);
  if (!b0 || X.p < b0 || X.p >= b0 + nb) return nullptr;
  const size_t bytes = side ? slice_acache_bytes(MN, K, ns) : slice_bcache_bytes(MN, K, ns);
  const std::array<int64_t, 12> key = {side, (int64_t)(X.p - b0), X.rs_hi, X.rs_lo, X.r_lo,
                                       X.cs_hi, X.cs_lo, X.c_lo, X.conj, MN, K, ns};
  auto it = c->bcache.find(key);
  if (it != c->bcache.end()) return &it->second->sc;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  if ((double)(c->bcache_bytes + bytes) > std::min(0.35 * (double)free_b, BCACHE_MAX))
    return nullptr;
  auto e = std::make_unique<cvsadc_ctx::BEntry>();
  e->buf.ensure(bytes);
  e->sc.base = e->buf.p;
  e->sc.bytes = bytes;
  e->sc.filled = false;
  c->bcache_bytes += bytes;
  SliceBCache* r = &e->sc;
  c->bcache[key] = std::move(e);
  return r;
}


// the view from row m0 on (m0 a multiple of its inner row extent when the
// rows are two-level)
View rows_from(View v, int64_t m0) {
  const int64_t off = v.r_lo == INT32_MAX
                          ? m0 * v.rs_lo
                          : (m0 / v.r_lo) * v.rs_hi + (m0 % v.r_lo) * v.rs_lo;
  v.p += off;
  if (v.ext >= 0) v.ext -= off;
  return v;
}

// cache_b / cache_a: B / A is the same view of B^P on every call (the sigma
// products), so its packed slices may be kept
void gemm(cvsadc_ctx* c, int prec, int M, int N, int K, double alpha, View A,
          View B, double beta, View C, int batch = 1, bool cache_b = false,
          bool cache_a = false) {
  A = checked(A);
  B = checked(B);
  C = checked(C);
  check_view(A, M, K, batch, "A");
  check_view(B, K, N, batch, "B");
  check_view(C, M, N, batch, "C");
  // the tensor-core path pays a packing pass per operand: keep it for
  // contractions with enough work per packed element
  // small outputs with a long K: all dot products at once, FP64
  const bool small = (int64_t)M * N <= 4096 && M + N <= 384 && K >= 4096;
  const bool tc = !small && prec != CVSADC_FP64 && M >= 32 && K >= 64 &&
                  (double)M * N * K >= 1e7;
  if (tc) {
    CVS_REQUIRE(tc_available(), CVSADC_EINVAL,
                "tensor-core precisions need an sm_103 GPU with tcgen05");
    const int ns = prec == CVSADC_MIXED_SLICE4 ? 4 : prec == CVSADC_FP64_SLICE7 ? 7 : 0;
    SliceBCache* bc = (ns && batch == 1 && cache_b) ? op_cache(c, 0, ns, N, K, B) : nullptr;
    SliceBCache* ac =
        (ns == 4 && batch == 1 && cache_a) ? op_cache(c, 1, ns, M, K, A) : nullptr;
    if (ns && batch == 1 && !bc && !ac) {
      // a tall product whose A packs dominate: slabs of rows with K whole
      // (slab boundaries on the inner row extents of A and C)
      int64_t slab = slice_row_slab(M, N, K, ns);
      int64_t q = 1;
      if (A.r_lo < M) q = A.r_lo;
      if (C.r_lo < M) q = std::lcm(q, (int64_t)C.r_lo);
      slab = slab / q * q;
      if (slab > 0 && slab < M) {
        const size_t need = slice_workspace_bytes((int)slab, N, K, ns);
        c->s_tc.ensure(need);
        for (int64_t m0 = 0; m0 < M; m0 += slab) {
          const int Mi = (int)std::min<int64_t>(slab, M - m0);
          zgemm_slice(c->stream, ns, Mi, N, K, alpha, rows_from(A, m0), B, beta,
                      rows_from(C, m0), c->s_tc.p, need, c->s_kpart.c(),
                      c->s_kpart.bytes / sizeof(cplx), c->err.as<int>(), nullptr);
        }
        return;
      }
    }
    size_t need = ns ? slice_workspace_bytes(M, N, K, ns, bc != nullptr, ac != nullptr)
                     : tc_workspace_bytes(M, N, K, 3);
    c->s_tc.ensure(need);
    for (int z = 0; z < batch; ++z) {
      View a = A, b = B, cc = C;
      a.p += z * A.batch;
      b.p += z * B.batch;
      cc.p += z * C.batch;
      if (a.ext >= 0) a.ext -= z * A.batch;
      if (b.ext >= 0) b.ext -= z * B.batch;
      if (cc.ext >= 0) cc.ext -= z * C.batch;
      if (ns)
        zgemm_slice(c->stream, ns, M, N, K, alpha, a, b, beta, cc, c->s_tc.p,
                    need, c->s_kpart.c(), c->s_kpart.bytes / sizeof(cplx),
                    c->err.as<int>(), bc, ac);
      else
        zgemm_tc(c->stream, 3, M, N, K, alpha, a, b, beta, cc, c->s_tc.p, need,
                 c->s_kpart.c(), c->s_kpart.bytes / sizeof(cplx),
                 c->err.as<int>());
    }
    return;
  }
  zgemm_f64(c->stream, M, N, K, alpha, A, B, beta, C, batch, c->s_kpart.c(),
            c->s_kpart.bytes / sizeof(cplx));
}

void gemm64(cvsadc_ctx* c, int M, int N, int K, double alpha, View A,
            View B, double beta, View C, int batch = 1) {
  A = checked(A);
  B = checked(B);
  C = checked(C);
  check_view(A, M, K, batch, "A");
  check_view(B, K, N, batch, "B");
  check_view(C, M, N, batch, "C");
  zgemm_f64(c->stream, M, N, K, alpha, A, B, beta, C, batch, c->s_kpart.c(),
            c->s_kpart.bytes / sizeof(cplx));
}

void copyv(cvsadc_ctx* c, int M, int N, double alpha, View src, View dst) {
  src = checked(src);
  dst = checked(dst);
  check_view(src, M, N, 1, "copy src");
  check_view(dst, M, N, 1, "copy dst");
  copy_view(c->stream, M, N, alpha, src, dst);
}

void upload(cvsadc_ctx* c, DBuf& dst, const void* src, size_t bytes,
            bool device_ptrs) {
  dst.ensure(bytes);
  CVS_CUDA(cudaMemcpyAsync(dst.p, src, bytes,
                           device_ptrs ? cudaMemcpyDeviceToDevice
                                       : cudaMemcpyHostToDevice,
                           c->stream));
}

void download(cvsadc_ctx* c, void* dst, const void* src, size_t bytes,
              bool device_ptrs) {
  CVS_CUDA(cudaMemcpyAsync(dst, src, bytes,
                           device_ptrs ? cudaMemcpyDeviceToDevice
                                       : cudaMemcpyDeviceToHost,
                           c->stream));
}

void check_hermitian(cvsadc_ctx* c, const cplx* M, int n, int64_t nmat,
                     const char* what) {
  c->s_small.ensure(4096);
  hermiticity(c->stream, M, n, nmat, c->s_small.d());
  double h[2];
  CVS_CUDA(cudaMemcpyAsync(h, c->s_small.p, sizeof h, cudaMemcpyDeviceToHost,
                           c->stream));
  c->sync();
  if (h[0] > 1e-12 * std::max(h[1], 1e-300)) {
    char msg[200];
    snprintf(msg, sizeof msg, "%s is not Hermitian: max|M-M^H| = %.3e, max|M| = %.3e",
             what, h[0], h[1]);
    throw Error{CVSADC_ENONHERM, msg};
  }
}

// ------------------------------------------------------------------ t2
// t2[i][j][a][b], g2 = <ab||ij>, E_MP2; B is [L][n][n] with o occupied.
void build_t2(cvsadc_ctx* c, int prec, const cplx* B, const double* eps,
              int o, int v, int L, DBuf& t2, DBuf& g2, double* emp2) {
  const int n = o + v;
  const int64_t nn = (int64_t)n * n;
  const int64_t vo = (int64_t)v * o;
  const size_t tsz = (size_t)o * o * v * v * sizeof(cplx);
  t2.ensure(tsz);
  g2.ensure(tsz);
  // band over a so that the (ai|bj) band stays within ~4 GB
  int64_t per_a = (int64_t)o * vo * sizeof(cplx);
  int na = (int)std::max<int64_t>(1, std::min<int64_t>(v, (4LL << 30) / per_a));
  c->s_big1.ensure((size_t)na * per_a);
  const int nblk = 608;
  c->s_part.ensure(nblk * sizeof(double) + 64);
  CVS_CUDA(cudaMemsetAsync(c->s_part.p, 0, nblk * sizeof(double), c->stream));
  for (int a0 = 0; a0 < v; a0 += na) {
    int nb = std::min(na, v - a0);
    // V[(al,i),(b,j)] = sum_P B^P_{o+a0+al, i} B^P_{o+b, j}
    View A = rows2(view(B + (int64_t)(o + a0) * n, 0, nn), n, 1, o);
    View Bv = cols2(view(B + (int64_t)o * n, nn, 0), n, 1, o);
    View C = view(c->s_big1.p, vo, 1);
    gemm(c, prec, nb * o, (int)vo, L, 1.0, A, Bv, 0.0, C);
    t2_band(c->stream, c->s_big1.c(), a0, nb, o, v, eps, t2.c(), g2.c(),
            c->s_part.d(), nblk);
  }
  double* dE = (double*)((char*)c->s_part.p + nblk * sizeof(double));
  reduce_sum(c->stream, c->s_part.d(), nblk, dE);
  CVS_CUDA(cudaMemcpyAsync(emp2, dE, sizeof(double), cudaMemcpyDeviceToHost,
                           c->stream));
  c->sync();
}

// ------------------------------------------------------------ t2 in bands
// t2 and <ab||ij> are never stored whole: every consumer (M11's Ivv, Joo and
// K pieces, E_MP2, the transition moments, the Eq. 15 density) is a sum over
// the first virtual index of the amplitudes, so it is accumulated band by
// band.  A band of the first virtual index a in [a0, a0 + nb) is the GEMM
//   X[(al, i)][(b, j)] = (a i | b j) = sum_P B^P_ai B^P_bj   (a = a0 + al),
// laid out [al][i][b][j], which t2_band_inplace turns into
//   G[al][i][b][j] = <ab||ij>   (in place)   and   T[al][i][b][j] = t^{ab}_{ij}.
// Contractions over a virtual index c of t^{.c} or t^{c.} take c as the band
// index through antisymmetry (t^{ac} = -t^{ca}).

// band rows (values of the first virtual index) per band: the in-place
// (ai|bj) block and the t2 block of each row within ~16 GB
int band_rows(int o, int v) {
  const double row = 2.0 * o * o * (double)v * sizeof(cplx);
  return (int)std::max(1.0, std::min((double)v, std::floor(16e9 / row)));
}

struct Band {
  int a0, nb;
  const cplx* T;  // [nb][o][v][o] t^{ab}_{ij}
  const cplx* G;  // [nb][o][v][o] <ab||ij>
};

// Runs `use` on every band of t2 built from B (o occupied and v virtual
// spinors, L Cholesky vectors) and energies eps; returns E_MP2.
template <class F>
double t2_bands(cvsadc_ctx* c, int prec, const cplx* B, const double* eps, int o,
                int v, int L, F&& use) {
  const int n = o + v;
  const int64_t nn = (int64_t)n * n, vo = (int64_t)v * o;
  const int na = band_rows(o, v);
  const int64_t nblk = t2_band_ip_blocks(na, o, v);
  DBuf X, T, part;
  X.ensure((size_t)na * o * vo * sizeof(cplx));
  T.ensure((size_t)na * o * vo * sizeof(cplx));
  part.ensure((size_t)(nblk + 1) * sizeof(double));
  double* dE = part.d() + nblk;
  CVS_CUDA(cudaMemsetAsync(dE, 0, sizeof(double), c->stream));
  for (int a0 = 0; a0 < v; a0 += na) {
    const int nb = std::min(na, v - a0);
    View A = rows2(view(B + (int64_t)(o + a0) * n, 0, nn), n, 1, o);
    View Bv = cols2(view(B + (int64_t)o * n, nn, 0), n, 1, o);
    gemm(c, prec, nb * o, (int)vo, L, 1.0, A, Bv, 0.0, view(X.p, vo, 1));
    t2_band_inplace(c->stream, X.c(), T.c(), a0, nb, o, v, eps, part.d(), dE);
    use(Band{a0, nb, T.c(), X.c()});
  }
  double e = 0.0;
  CVS_CUDA(cudaMemcpyAsync(&e, dE, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  return e;
}

// ------------------------------------------------------------------ M11
// M11 (and, with dipoles, the transition moments through first order) of
// the current basis, and E_MP2, from one pass over the t2 bands.
void build_m11(cvsadc_ctx* c, int prec) {
  const int nc = c->ncore, nw = c->nval, v = c->nvirt, o = c->o, n = c->n, L = c->naux;
  const int64_t nn = (int64_t)n * n, N1 = c->N1, N = c->N;
  const int64_t vo = (int64_t)v * o, ovo = (int64_t)o * vo, vv = (int64_t)v * v;
  const cplx* B = c->B.c();
  c->M11.ensure(N1 * N1 * sizeof(cplx));
  size_t need = ((size_t)v * v * nc * nc + 2 * N1 * N1 + (size_t)v * v + nc * nc) *
                sizeof(cplx);
  c->s_big2.ensure(need);
  cplx* C1 = c->s_big2.c();
  cplx* C2 = C1 + (size_t)v * v * nc * nc;
  cplx* Z = C2 + N1 * N1;
  cplx* X = Z + N1 * N1;
  cplx* Y = X + (size_t)v * v;
  // C1[(a,b),(J,I)] = (ab|JI)
  gemm(c, prec, v * v, nc * nc, L, 1.0,
       rows2(view(B + (int64_t)o * n + o, 0, nn), n, 1, v),
       cols2(view(B, nn, 0), n, 1, nc), 0.0, view(C1, nc * nc, 1));
  // C2[(I,a),(J,b)] = (aI|Jb)
  gemm(c, prec, (int)N1, (int)N1, L, 1.0,
       rows2(view(B + (int64_t)o * n, 0, nn), 1, n, v),
       cols2(view(B + o, nn, 0), n, 1, v), 0.0, view(C2, N1, 1));
  // transition moments: F_S starts as d_aI; the doubles pieces
  //   A[I][j][a][b] = sum_c d_ac t^{cb}_{Ij}  and
  //   R[I][j][a][b] = sum_k d_kI t^{ab}_{kj} - sum_k d_kj t^{ab}_{kI}
  // accumulate over the bands, three Cartesian components at once
  const bool mom = c->has_dip;
  const int64_t blk = (int64_t)nc * nw * vv;
  DBuf macc;
  if (mom) {
    c->F.ensure(3 * N * sizeof(cplx));
    macc.ensure((size_t)6 * blk * sizeof(cplx));
    for (int x = 0; x < 3; ++x)
      copyv(c, nc, v, 1.0, view(c->dip.c() + (int64_t)x * nn + (int64_t)o * n, 1, n),
            view(c->F.c() + (int64_t)x * N, v, 1));
  }
  c->emp2 = t2_bands(c, prec, B, c->eps.d(), o, v, L, [&](const Band& b) {
    const double beta = b.a0 == 0 ? 0.0 : 1.0;
    // X_ab += sum_{(c,k),l} t^{ca}_{kl} conj(<cb||kl>)   (the Ivv piece)
    gemm(c, prec, v, v, b.nb * o * o, 1.0, cols2(view(b.T, o, 0), vo, 1, o),
         conj_of(rows2(view(b.G, 0, o), vo, 1, o)), beta, view(X, v, 1));
    // Y_IJ += sum_{c,(d,k)} t^{cd}_{Ik} conj(<cd||Jk>)   (the Joo piece)
    gemm(c, prec, nc, nc, b.nb * (int)vo, 1.0, cols2(view(b.T, vo, 0), ovo, 1, (int)vo),
         conj_of(rows2(view(b.G, 0, vo), ovo, 1, (int)vo)), beta, view(Y, nc, 1));
    // Z_{Ia,Jb} += sum_{c,k} t^{ca}_{Ik} conj(<cb||Jk>)   (the K piece)
    const View Tia = cols2(rows2(view(b.T, 0, 0), vo, o, v), ovo, 1, o);
    gemm(c, prec, (int)N1, (int)N1, b.nb * o, 1.0, Tia,
         conj_of(cols2(rows2(view(b.G, 0, 0), ovo, 1, o), vo, o, v)), beta,
         view(Z, N1, 1));
    if (!mom) return;
    for (int x = 0; x < 3; ++x) {
      const cplx* d = c->dip.c() + (int64_t)x * nn;
      cplx* Ax = macc.c() + (int64_t)(2 * x) * blk;
      cplx* Rx = Ax + blk;
      // F_S[I][a] += sum_{kc} t^{ac}_{Ik} d_kc = -sum_{c,k} t^{ca}_{Ik} d_kc
      gemm(c, prec, (int)N1, 1, b.nb * o, -1.0, Tia,
           rows2(view(d + o + b.a0, 0, 0), 1, n, o), 1.0,
           view(c->F.c() + (int64_t)x * N, 1, 1));
      // A[I][j][a][b] += sum_{c in band} d_ac t^{cb}_{Ij}   (batched over I)
      gemm(c, prec, v, nw * v, b.nb, 1.0, view(d + (int64_t)o * n + o + b.a0, n, 1),
           batched(cols2(view(b.T + nc, ovo, 0), 1, o, v), vo), beta,
           batched(cols2(view(Ax, v, 0), vv, 1, v), (int64_t)nw * vv), nc);
      // R[I][j][a][b] for a in the band (batched over a):
      //   sum_k d_kI t^{ab}_{kj} - sum_k d_kj t^{ab}_{kI}
      gemm(c, prec, nc, nw * v, o, 1.0, view(d, 1, n),
           batched(cols2(view(b.T + nc, vo, 0), 1, o, v), ovo), 0.0,
           batched(cols2(view(Rx + (int64_t)b.a0 * v, (int64_t)nw * vv, 0), vv, 1, v), v),
           b.nb);
      gemm(c, prec, nw, nc * v, o, -1.0, view(d + nc, 1, n),
           batched(cols2(view(b.T, vo, 0), 1, o, v), ovo), 1.0,
           batched(cols2(view(Rx + (int64_t)b.a0 * v, vv, 0), (int64_t)nw * vv, 1, v), v),
           b.nb);
    }
  });
  m11_assemble(c->stream, nc, v, o, c->eps.d(), C1, C2, X, Y, Z, 1, c->M11.c());
  if (mom)
    for (int x = 0; x < 3; ++x) {
      const cplx* Ax = macc.c() + (int64_t)(2 * x) * blk;
      pack_moment_doubles(c->stream, Ax, Ax + blk, nc, nw, v,
                          c->F.c() + (int64_t)x * N + N1);
    }
}

// ------------------------------------------------- <Kb||Ij> (1-external)
// h[K][b][I][j] = <Kb||Ij> = (KI|bj) - (Kj|bI), and its conjugate laid out
// as hT[(I,j,b)][K].  Small (ncore^2 nval nvirt) and kept with the
// prepared problem: the couplings' terms with one virtual index go through
// it, the ones with three (<ab||cj>) through B^P.
void build_h(cvsadc_ctx* c, int prec) {
  const int nc = c->ncore, nw = c->nval, v = c->nvirt, o = c->o, n = c->n,
            L = c->naux;
  const int64_t nn = (int64_t)n * n;
  cudaStream_t s = c->stream;
  c->h1.ensure((size_t)nc * v * nc * nw * sizeof(cplx));
  c->hT.ensure((size_t)nc * v * nc * nw * sizeof(cplx));
  DBuf hc1, hc2;
  hc1.ensure((size_t)nc * nc * v * nw * sizeof(cplx));
  hc2.ensure((size_t)nc * nw * v * nc * sizeof(cplx));
  const cplx* B = c->B.c();
  // hc1[(K,I)][(b,j)] = sum_P B^P_KI B^P_bj
  gemm(c, prec, nc * nc, v * nw, L, 1.0, rows2(view(B, 0, nn), n, 1, nc),
       cols2(view(B + (int64_t)o * n + nc, nn, 0), n, 1, nw), 0.0,
       view(hc1.p, (int64_t)v * nw, 1));
  // hc2[(K,j)][(b,I)] = sum_P B^P_Kj B^P_bI
  gemm(c, prec, nc * nw, v * nc, L, 1.0, rows2(view(B + nc, 0, nn), n, 1, nw),
       cols2(view(B + (int64_t)o * n, nn, 0), n, 1, nc), 0.0,
       view(hc2.p, (int64_t)v * nc, 1));
  h_assemble(s, hc1.c(), hc2.c(), nc, nw, v, c->h1.c());
  h_conj_transpose(s, c->h1.c(), nc, nw, v, c->hT.c());
  c->sync();
}

// ----------------------------------------------------------------- sigma
// sigma for a group of g vectors at once: every contraction runs over the
// whole group, so the ncore-sized dimensions become g * ncore and operands
// built from B^P are packed once per group.
// mode SIG_FULL: sigma = M x.  SIG_FWD: only the doubles part, sigma2 =
// M21 x1 (no M22 term, singles part untouched).  SIG_ADJ: only the singles
// part, sigma1 = M12 x2 (no M11 term, doubles part untouched).
enum { SIG_FULL = 0, SIG_FWD = 1, SIG_ADJ = 2 };
// bytes of sigma intermediates (unpacked doubles, G, S, Y) one group holds
constexpr double SIGMA_BUDGET = 48e9;
void sigma_group(cvsadc_ctx* c, int prec, const cplx* x, cplx* sig, int g,
                 int mode = SIG_FULL) {
  const int nc = c->ncore, nw = c->nval, v = c->nvirt, o = c->o, n = c->n,
            L = c->naux;
  const int64_t nn = (int64_t)n * n, N1 = c->N1, N = c->N;
  const int64_t wv = (int64_t)nw * v, vL = (int64_t)v * L;
  const int64_t N1L = N1 * L, N1wv = N1 * wv;
  const cplx* B = c->B.c();
  c->s_big1.ensure((size_t)g * N1wv * sizeof(cplx));
  c->s_big2.ensure((size_t)g * N1wv * sizeof(cplx));
  c->s_S.ensure((size_t)g * N1L * sizeof(cplx));
  c->s_Y.ensure((size_t)g * N1L * sizeof(cplx));
  cplx* Yt = c->s_big1.c();  // [q][I][a][j][b]
  cplx* G = c->s_big2.c();   // [q][(I,a)][(j,b)]
  cplx* S = c->s_S.c();      // [(q,I)][P][a]
  cplx* Y = c->s_Y.c();      // [(q,I,a)][P]
  if (mode != SIG_FWD) {
    for (int q = 0; q < g; ++q)
      unpack_doubles(c->stream, x + q * N + N1, nc, nw, v, Yt + q * N1wv);
    // S[(q,I,a)][P] = sum_{jb} y_{Ijab} B^P_{jb}, stored as [(q,I)][P][a]
    // (the tile epilogue's lanes, consecutive a, write consecutive elements)
    gemm(c, prec, (int)(g * N1), L, (int)wv, 1.0, view(Yt, wv, 1),
         rows2(view(B + (int64_t)nc * n + o, 0, nn), n, 1, v), 0.0,
         rows2(view(S, 0, v), vL, 1, v), 1, true);
    // sigma1 (M12 x2), the <ab||cj> part, transposed so that the long side
    // (c) is the row dimension: sigma1^T[c][(q, K)] = -sum_{(P,a)} B^P_ca
    // S[(q,K)][P][a]; the contraction index (P, a) runs contiguously through
    // both B^P_c. and S
    const View s1rows = rows2(view(sig, 0, 1), N, v, nc);
    gemm(c, prec, v, g * nc, (int)vL, -1.0,
         cols2(view(B + (int64_t)o * n + o, n, 0), nn, 1, v), view(S, 1, vL),
         0.0, trans(s1rows), 1, false, true);
    // the <Kb||Ij> part: sigma1[K][c] += sum_{Ijb} y_{Ijcb} conj(h[K][b][I][j]),
    // rows (q, c), columns K
    const View s1t = rows2(view(sig, 0, v), N, 1, v);  // ((q,c), K)
    gemm(c, prec, g * v, nc, (int)(nc * wv), 1.0,
         cols2(rows2(view(Yt, 0, 0), N1wv, wv, v), wv * v, 1, (int)wv),
         view(c->hT.c(), nc, 1), 1.0, s1t);
  }
  if (mode == SIG_ADJ) return;
  // Y[(q,I,a)][P] = sum_c x_Ic B^P_ac, as its transpose
  // Y^T[(a,P)][(q,I)] = sum_c B^P_ac x_Ic (the long side (a, P) as rows)
  gemm(c, prec, (int)vL, g * nc, v, 1.0,
       rows2(view(B + (int64_t)o * n + o, 0, 1), n, nn, L),
       trans(rows2(view(x, 0, 1), N, v, nc)), 0.0, trans(view(Y, vL, 1)), 1, false, true);
  // G[q][(I,a)][(j,b)] = sum_P Y B^P_{bj} (the <ab||cj> part of M21 x1; the
  // <Kb||Ij> part is added while packing)
  gemm(c, prec, (int)(g * N1), (int)wv, L, 1.0, view(Y, L, 1),
       cols2(view(B + (int64_t)o * n + nc, nn, 0), 1, n, v), 0.0,
       view(G, wv, 1), 1, true);
  for (int q = 0; q < g; ++q)
    sigma2_finish(c->stream, G + q * N1wv,
                  mode == SIG_FWD ? nullptr : x + q * N + N1, x + q * N,
                  c->h1.c(), c->eps.d(), nc, nw, v, sig + q * N + N1,
                  prec == CVSADC_FP64);
  if (mode == SIG_FWD) return;
  // sigma1 += M11 x1 (dense product, FP64 for the small block)
  gemm64(c, (int)N1, g, (int)N1, 1.0, view(c->M11.c(), N1, 1), view(x, 1, N),
         1.0, view(sig, 1, N));
}

void sigma_impl(cvsadc_ctx* c, int prec, const cplx* x, cplx* sig, int nvec,
                int mode = SIG_FULL) {
  const int64_t N1 = c->N1, wv = (int64_t)c->nval * c->nvirt, L = c->naux;
  const double per_vec = (2.0 * N1 * wv + 2.0 * N1 * L + 2.0 * wv * L) * sizeof(cplx);
  int g = (int)std::max(1.0, std::min((double)nvec, SIGMA_BUDGET / per_vec));
  for (int q0 = 0; q0 < nvec; q0 += g) {
    const int gg = std::min(g, nvec - q0);
    sigma_group(c, prec, x + q0 * c->N, sig + q0 * c->N, gg, mode);
  }
}

// --------------------------------------------------------------- FNS
void build_fns(cvsadc_ctx* c, int prec, double tau) {
  const int nc = c->ncore, nw = c->nval, v = c->nvirt_in, o = c->o,
            L = c->naux;
  const int n = o + v;
  (void)nc;
  (void)nw;
  // D_ab = 1/2 sum_{cij} t^{ac}_{ij} conj(t^{bc}_{ij})
  //      = 1/2 sum_{c,(i,j)} t^{ca}_{ij} conj(t^{cb}_{ij})  over the bands of
  // the canonical amplitudes
  DBuf D;
  D.ensure((size_t)v * v * sizeof(cplx));
  const int64_t vv = (int64_t)v * v, vo = (int64_t)v * o;
  t2_bands(c, prec, c->B.c(), c->eps.d(), o, v, L, [&](const Band& b) {
    gemm(c, prec, v, v, b.nb * o * o, 0.5, cols2(view(b.T, o, 0), vo, 1, o),
         conj_of(rows2(view(b.T, 0, o), vo, 1, o)), b.a0 == 0 ? 0.0 : 1.0,
         view(D.p, v, 1));
  });
  // Hermitian part for the eigensolver
  DBuf A, Vec, w;
  A.ensure(vv * sizeof(cplx));
  Vec.ensure(vv * sizeof(cplx));
  w.ensure(v * sizeof(double) + 64);
  hermitize(c->stream, D.c(), v, v, A.c(), v);
  c->s_small.ensure(4096);
  jacobi_eigh(c->stream, A.c(), v, w.d(), Vec.c(), 40, c->s_small.d());
  std::vector<double> occ_asc(v);
  CVS_CUDA(cudaMemcpyAsync(occ_asc.data(), w.p, v * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
  c->sync();
  // descending occupations; keep n >= tau (degenerate pairs kept together)
  std::vector<int> keep;
  for (int k = v - 1; k >= 0; --k)
    if (occ_asc[k] >= tau * (1.0 - 1e-10)) keep.push_back(k);
  int vk = (int)keep.size();
  CVS_REQUIRE(vk >= 2, CVSADC_EINVAL, "FNS threshold keeps fewer than 2 virtuals");
  std::vector<double> occ_desc(v);
  for (int k = 0; k < v; ++k) occ_desc[k] = occ_asc[v - 1 - k];
  c->fns_occ.ensure(v * sizeof(double));
  CVS_CUDA(cudaMemcpyAsync(c->fns_occ.p, occ_desc.data(), v * sizeof(double),
                           cudaMemcpyHostToDevice, c->stream));
  // V~ columns (descending occupation order) gathered into Vt [v][vk]
  DBuf Vt, kidx;
  Vt.ensure((size_t)v * vk * sizeof(cplx));
  kidx.ensure((size_t)vk * sizeof(int));
  CVS_CUDA(cudaMemcpyAsync(kidx.p, keep.data(), (size_t)vk * sizeof(int),
                           cudaMemcpyHostToDevice, c->stream));
  gather_columns(c->stream, Vec.c(), v, v, (const int*)kidx.p, vk, Vt.c(), vk);
  // F^NS = V~^H diag(eps_v) V~ (Eq. 18): scale rows of V~ by eps_v, GEMM
  DBuf EV, Fns, Fh, Z, et;
  EV.ensure((size_t)v * vk * sizeof(cplx));
  Fns.ensure((size_t)vk * vk * sizeof(cplx));
  CVS_CUDA(cudaMemcpyAsync(EV.p, Vt.p, (size_t)v * vk * sizeof(cplx),
                           cudaMemcpyDeviceToDevice, c->stream));
  scale_rows(c->stream, EV.c(), v, vk, vk, c->eps.d() + o);
  gemm64(c, vk, vk, v, 1.0, conj_of(trans(view(Vt.p, vk, 1))),
            view(EV.p, vk, 1), 0.0, view(Fns.p, vk, 1));
  // Hermitise and diagonalise (Eq. 19)
  Fh.ensure((size_t)vk * vk * sizeof(cplx));
  Z.ensure((size_t)vk * vk * sizeof(cplx));
  et.ensure(vk * sizeof(double) + 64);
  hermitize(c->stream, Fns.c(), vk, vk, Fh.c(), vk);
  jacobi_eigh(c->stream, Fh.c(), vk, et.d(), Z.c(), 40, c->s_small.d());
  // U = V~ Z~ (Eq. 20)
  c->fns_U.ensure((size_t)v * vk * sizeof(cplx));
  gemm64(c, v, vk, vk, 1.0, view(Vt.p, vk, 1), view(Z.p, vk, 1),
            0.0, view(c->fns_U.p, vk, 1));
  // rotate B^P (and dipoles): occupied rows/cols unchanged, virtual with U
  const int n2 = o + vk;
  const int64_t nn = (int64_t)n * n, nn2 = (int64_t)n2 * n2;
  auto rotate = [&](const cplx* src, int64_t nmat, DBuf& dst) {
    dst.ensure((size_t)nmat * nn2 * sizeof(cplx));
    DBuf tmp;
    tmp.ensure((size_t)nmat * n * vk * sizeof(cplx));
    const cplx* U = c->fns_U.c();
    // oo block copy, rows (P, i) of all matrices at once
    copyv(c, (int)(nmat * o), o, 1.0, rows2(view(src, 0, 1), nn, n, o),
          rows2(view(dst.c(), 0, 1), nn2, n2, o));
    // tmp[P][p][b'] = sum_b src[P][p][o+b] U[b][b']   (all rows p)
    gemm(c, CVSADC_FP64, n, vk, v, 1.0,
         batched(view(src + o, n, 1), nn), view(U, vk, 1), 0.0,
         batched(view(tmp.p, vk, 1), (int64_t)n * vk), (int)nmat);
    // ov block: rows i < o of every matrix
    copyv(c, (int)(nmat * o), vk, 1.0, rows2(view(tmp.c(), 0, 1), (int64_t)n * vk, vk, o),
          rows2(view(dst.c() + o, 0, 1), nn2, n2, o));
    // vv block: U^H tmp[P][o:][:]
    gemm(c, CVSADC_FP64, vk, vk, v, 1.0,
         conj_of(trans(view(U, vk, 1))),
         batched(view(tmp.c() + (int64_t)o * vk, vk, 1), (int64_t)n * vk), 0.0,
         batched(view(dst.c() + (int64_t)o * n2 + o, n2, 1), nn2), (int)nmat);
    // vo block: U^H src[P][o:][:o]
    gemm(c, CVSADC_FP64, vk, o, v, 1.0, conj_of(trans(view(U, vk, 1))),
         batched(view(src + (int64_t)o * n, n, 1), nn), 0.0,
         batched(view(dst.c() + (int64_t)o * n2, n2, 1), nn2), (int)nmat);
  };
  DBuf Bn;
  rotate(c->B.c(), L, Bn);
  std::swap(c->B.p, Bn.p);
  std::swap(c->B.bytes, Bn.bytes);
  if (c->has_dip) {
    DBuf dn;
    rotate(c->dip.c(), 3, dn);
    std::swap(c->dip.p, dn.p);
    std::swap(c->dip.bytes, dn.bytes);
  }
  // new energies: occupied unchanged, virtual = eps~
  DBuf en;
  en.ensure((size_t)n2 * sizeof(double));
  CVS_CUDA(cudaMemcpyAsync(en.p, c->eps.p, o * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->stream));
  CVS_CUDA(cudaMemcpyAsync(en.d() + o, et.p, vk * sizeof(double),
                           cudaMemcpyDeviceToDevice, c->stream));
  c->sync();
  std::swap(c->eps.p, en.p);
  std::swap(c->eps.bytes, en.bytes);
  c->nvirt = vk;
}

void set_sizes(cvsadc_ctx* c) {
  c->o = c->ncore + c->nval;
  c->n = c->o + c->nvirt;
  c->N1 = (int64_t)c->ncore * c->nvirt;
  c->npair = (int64_t)c->nvirt * (c->nvirt - 1) / 2;
  c->N2 = (int64_t)c->ncore * c->nval * c->npair;
  c->N = c->N1 + c->N2;
}

void validate(const cvsadc_params* p) {
  CVS_REQUIRE(p != nullptr, CVSADC_EINVAL, "params is NULL");
  CVS_REQUIRE(p->ncore >= 1 && p->nval >= 1 && p->nvirt >= 2 && p->naux >= 1,
              CVSADC_EINVAL, "partition sizes must be ncore>=1, nval>=1, nvirt>=2, naux>=1");
  CVS_REQUIRE(valid_precision(p->precision), CVSADC_EINVAL, "unknown precision");
  int64_t n = (int64_t)p->ncore + p->nval + p->nvirt;
  int64_t o = (int64_t)p->ncore + p->nval;
  CVS_REQUIRE(n <= 20000 && (int64_t)p->naux * n * n < (1LL << 40), CVSADC_EINVAL,
              "problem too large");
  CVS_REQUIRE(o * p->nvirt * (int64_t)p->nvirt * p->nval < (1LL << 31) * 64LL,
              CVSADC_EINVAL, "problem too large");
}

// keep_t2: also store t2 and <ab||ij> whole (o^2 v^2 each; the gradient's
// reverse pass reads them)
void prepare_impl(cvsadc_ctx* c, const cvsadc_params* p, const double* eps,
                  const void* B, const void* dip, cvsadc_info* info,
                  bool keep_t2 = false) {
  validate(p);
  CVS_REQUIRE(eps && B, CVSADC_EINVAL, "eps and B are required");
  double t0 = now_ms();
  bool dev = (p->flags & CVSADC_FLAG_DEVICE_PTRS) != 0;
  c->prepared = false;
  c->sch_on = false;
  c->sch_g.release();
  c->clear_bcache();
  c->ncore = p->ncore;
  c->nval = p->nval;
  c->nvirt_in = c->nvirt = p->nvirt;
  c->naux = p->naux;
  set_sizes(c);
  const int n = c->n;
  upload(c, c->eps, eps, n * sizeof(double), dev);
  upload(c, c->B, B, (size_t)c->naux * n * n * sizeof(cplx), dev);
  c->has_dip = dip != nullptr;
  if (c->has_dip) upload(c, c->dip, dip, (size_t)3 * n * n * sizeof(cplx), dev);
  check_hermitian(c, c->B.c(), n, c->naux, "B");
  if (c->has_dip) check_hermitian(c, c->dip.c(), n, 3, "dip");
  c->has_fns = p->fns_threshold > 0;
  // the problem (FNS, t2, M11, couplings, moments) is built at the requested
  // precision, except for BF16X3, whose accumulation-limited products
  // (~1e-5 relative) would leave M itself ~1e-4 Eh off: its problem is built
  // with the FP64-class 7-slice product and BF16X3 runs the Davidson sigma
  int prec = p->precision;
  if (prec == CVSADC_MIXED_BF16X3)
    prec = tc_available() ? CVSADC_FP64_SLICE7 : CVSADC_FP64;
  if (c->has_fns) {
    build_fns(c, prec, p->fns_threshold);
    set_sizes(c);
    c->clear_bcache();  // B^P was rotated
  }
  auto stage = [&](const char* what, double t) {
    if (verbose()) {
      c->sync();
      fprintf(stderr, "[cvsadc] %-8s %10.2f ms\n", what, now_ms() - t);
    }
  };
  c->prep_prec = prec;
  c->t2.release();
  c->g2.release();
  double ts = now_ms();
  build_m11(c, prec);  // with E_MP2 and, with dipoles, the moments
  stage("t2+m11", ts);
  ts = now_ms();
  build_h(c, prec);
  if (keep_t2) {
    double e = 0.0;
    build_t2(c, prec, c->B.c(), c->eps.d(), c->o, c->nvirt, c->naux, c->t2, c->g2, &e);
  }
  stage("h", ts);
  c->diag.ensure(c->N * sizeof(double));
  build_diag(c->stream, c->M11.c(), c->eps.d(), c->ncore, c->nval, c->nvirt,
             c->diag.d());
  c->sync();
  c->prepared = true;
  if (info) {
    info->emp2 = c->emp2;
    info->nvirt_kept = c->nvirt;
    info->t_prepare_ms = now_ms() - t0;
  }
}

// ------------------------------------------- Schur-complement preconditioner
// Because M22 is diagonal, the doubles fold into the singles exactly:
// S(theta) = M11 + M12 (theta - M22)^-1 M21 (schur_kernels.cu gives the five
// pieces of the second term).  The Davidson solver takes the eigen-
// decomposition S(theta0) = U diag(lam) U^H at a trial energy theta0 near
// the lowest root and uses it twice: its lowest eigenvectors, with their
// folded doubles (theta0 - M22)^-1 M21 u, are the initial guesses, and a
// residual (r1, r2) of a root with Ritz value theta is corrected by block
// elimination with S(theta0) in place of S(theta):
//   t1 = U (theta - lam)^-1 U^H [r1 + M12 (theta - M22)^-1 r2]
//   t2 = (theta - M22)^-1 (r2 + M21 t1).
// This is a preconditioner only: its arithmetic (the tensor-core precision
// where available) leaves the converged roots unchanged.

// eigenvectors of S(theta) kept for the projected theta0 search
constexpr int SCHUR_P = 16;

// the preconditioner's GEMM precision
int schur_precision() {
  return tc_available() ? CVSADC_MIXED_SLICE4 : CVSADC_FP64;
}

// <ab||cj> for j in [j0, j0 + jc) into G[jl][a][b][c]; X1 holds jc v^3
// complex.  One GEMM: (aj|bc) = (bc|aj) is an element of the same product.
void build_g_chunk(cvsadc_ctx* c, int prec, int j0, int jc, cplx* X1, cplx* G) {
  const int nc = c->ncore, v = c->nvirt, o = c->o, n = c->n, L = c->naux;
  const int64_t nn = (int64_t)n * n;
  const cplx* B = c->B.c();
  // X1[(a,c)][(jl,b)] = sum_P B^P_ac B^P_bj
  gemm(c, prec, v * v, jc * v, L, 1.0,
       rows2(view(B + (int64_t)o * n + o, 0, nn), n, 1, v),
       cols2(view(B + (int64_t)o * n + nc + j0, nn, 0), 1, n, v), 0.0,
       view(X1, (int64_t)jc * v, 1));
  g_assemble(c->stream, X1, nullptr, jc, v, G);
}

// j per chunk so that the chunk buffers (X1, G and ncore weighted copies)
// stay within ~6 GB
int schur_jchunk(cvsadc_ctx* c) {
  const double per_j = (2.0 + c->ncore) * std::pow((double)c->nvirt, 3) * sizeof(cplx);
  return (int)std::max(1.0, std::min((double)c->nval, 6e9 / per_j));
}

// singles spaces above this size take the large-space preconditioner: the
// lowest SCHUR_PL eigenpairs of S(theta0) from a block Davidson instead of
// a full decomposition, and the cross term (12) with the weight expanded
// to first order about the mean virtual energy
constexpr int64_t SCHUR_FULL_MAX = 4096;
constexpr int SCHUR_PL = 64;

// S(theta) into sch_S (schur_eigh decomposes it).  approx12: the (12)
// cross term with the weight w(e_c') expanded to first order about the mean
// virtual energy, as two GEMMs per valence spinor (preconditioner use for
// large singles spaces; the exact term is a batched product per c')
void build_schur(cvsadc_ctx* c, int prec, double theta, bool cached, bool approx12 = false) {
  const int nc = c->ncore, nw = c->nval, v = c->nvirt, o = c->o;
  const int64_t v3 = (int64_t)v * v * v;
  cudaStream_t s = c->stream;
  const int jc = schur_jchunk(c);
  CVS_CUDA(cudaMemsetAsync(c->sch_C11.p, 0, (size_t)nc * v * v * sizeof(cplx), s));
  CVS_CUDA(cudaMemsetAsync(c->sch_C12.p, 0,
                           (size_t)v * v * nc * nc * sizeof(cplx), s));
  double ebar = 0.0;
  if (approx12) {
    std::vector<double> ev(v);
    CVS_CUDA(cudaMemcpyAsync(ev.data(), c->eps.d() + o, v * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    c->sync();
    for (double x : ev) ebar += x / v;
  }
  // chunk buffers: [X1 | G | Gw (ncore copies)] (X1, G unused when cached)
  cplx* X1 = c->sch_work.c();
  cplx* Gt = X1 + (int64_t)jc * v3;
  cplx* Gw = Gt + (int64_t)jc * v3;
  cplx* Hw = c->sch_tmp.c();
  const bool vb = verbose();
  double tv = vb ? (c->sync(), now_ms()) : 0.0, t11 = 0.0, t12 = 0.0;
  for (int j0 = 0; j0 < nw; j0 += jc) {
    const int jn = std::min(jc, nw - j0);
    cplx* G = Gt;
    if (cached)
      G = c->sch_g.c() + (int64_t)j0 * v3;
    else
      build_g_chunk(c, prec, j0, jn, X1, Gt);
    // (11): C11[(K,c)][c'] += sum_{jab} 1/2 w_Kjab conj(g_abc) g_abc', all K
    // in one GEMM (rows (K, c) of the weighted copies)
    g_weight(s, G, jn, j0, nc, nw, v, c->eps.d(), theta, Gw);
    gemm(c, prec, nc * v, v, jn * v * v, 1.0,
         conj_of(rows2(view(Gw, 0, v), (int64_t)jn * v3, 1, v)), view(G, v, 1),
         1.0, view(c->sch_C11.c(), v, 1));
    if (vb) {
      c->sync();
      t11 += now_ms() - tv;
      tv = now_ms();
    }
    // (12): C12[c'][c][K][K'] += sum_b conj(<c'b||cj>) w_{Kjc'b} <K'b||Kj>
    for (int jl = 0; jl < jn; ++jl) {
      if (approx12) {
        // w = wbar + (e_c' - ebar) wbar^2: rows (c', c), columns (K, K')
        const View Gc = conj_of(rows2(view(G + (int64_t)jl * v3, 0, v), (int64_t)v * v, 1, v));
        h_weight_mean(s, c->h1.c(), j0 + jl, nc, nw, v, c->eps.d(), theta, ebar, 1, Hw);
        gemm(c, prec, v * v, nc * nc, v, 1.0, Gc, view(Hw, nc * nc, 1), 1.0,
             view(c->sch_C12.c(), nc * nc, 1));
        h_weight_mean(s, c->h1.c(), j0 + jl, nc, nw, v, c->eps.d(), theta, ebar, 2, Hw);
        gemm(c, prec, v * v, nc * nc, v, 1.0, Gc, view(Hw, nc * nc, 1), 0.0,
             view(c->sch_V.c(), nc * nc, 1));
        add_row_scaled(s, c->sch_C12.c(), c->sch_V.c(), v, nc * nc, c->eps.d(), o, ebar);
        continue;
      }
      h_weight(s, c->h1.c(), j0 + jl, nc, nw, v, c->eps.d(), theta, Hw);
      gemm(c, CVSADC_FP64, v, nc * nc, v, 1.0,
           batched(conj_of(view(G + (int64_t)jl * v3, 1, v)), (int64_t)v * v),
           batched(view(Hw, nc * nc, 1), (int64_t)v * nc * nc), 1.0,
           batched(view(c->sch_C12.c(), nc * nc, 1), (int64_t)v * nc * nc), v);
    }
    if (vb) {
      c->sync();
      t12 += now_ms() - tv;
      tv = now_ms();
    }
  }
  schur_assemble(s, c->M11.c(), c->sch_C11.c(), c->sch_C12.c(), c->h1.c(), nc,
                 nw, v, c->eps.d(), theta, c->sch_V.c(), c->sch_S.c());
  if (vb) {
    c->sync();
    fprintf(stderr, "[cvsadc] schur build: (11) %.1f ms  (12) %.1f ms  assemble %.1f ms\n",
            t11, t12, now_ms() - tv);
  }
}

// scratch of sch_th (doubles): [0,128) per-root theta, [128, 736) partial
// sums, then the rotation cosines and (16-byte aligned) the sines
size_t schur_th_doubles(int64_t N1) {
  const size_t cc_n = (size_t)(N1 / 2 + 2);
  return 736 + ((cc_n + 1) & ~(size_t)1) + 2 * cc_n;
}

// Lowest p eigenpairs of the dense Hermitian sch_S (N1 x N1) into sch_U
// ([N1][p], columns) and sch_lam, by block Davidson with S products as FP64
// GEMMs, the diagonal preconditioner, FP64 subspace algebra and the Jacobi
// kernel for the small projected matrices.  Residuals to 1e-6 of the
// spectral scale: this is the preconditioner's eigensystem.
__global__ void diag_real_kernel(const cplx* __restrict__ S, int64_t n, double* __restrict__ d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    d[i] = S[i * n + i].x;
}

void schur_eigh_partial(cvsadc_ctx* c, int p) {
  const double t0 = verbose() ? (c->sync(), now_ms()) : 0.0;
  const int64_t n = c->N1;
  cudaStream_t s = c->stream;
  const int ms = std::min<int64_t>(3 * p, n);
  DBuf Xb, AXb, Tb, U, AU, sm, dS, rpart;
  rpart.ensure((size_t)(304 * p + 64) * sizeof(double));
  Xb.ensure((size_t)ms * n * sizeof(cplx));
  AXb.ensure((size_t)ms * n * sizeof(cplx));
  Tb.ensure((size_t)p * n * sizeof(cplx));
  U.ensure((size_t)p * n * sizeof(cplx));
  AU.ensure((size_t)p * n * sizeof(cplx));
  const size_t TSP = (size_t)96 * 192 * TS_CHUNKS;
  sm.ensure(((size_t)4 * ms * ms + 64 * 64 * 2 + TSP) * sizeof(cplx) +
            (size_t)(4 * ms + 4096) * sizeof(double));
  dS.ensure((size_t)n * sizeof(double));
  cplx* H = sm.c();
  cplx* A = H + (size_t)ms * ms;
  cplx* Y = A + (size_t)ms * ms;
  cplx* Cp = Y + (size_t)ms * ms;
  cplx* G0 = Cp + (size_t)ms * ms;
  cplx* Xo = G0 + 64 * 64;
  cplx* tsp = Xo + 64 * 64;
  double* w = (double*)(tsp + TSP);
  double* rn = w + ms;
  double* dw = rn + ms;
  double* nrm0 = dw + 2 * ms;
  int* kept_d = (int*)(nrm0 + 256);
  diag_real_kernel<<<grid1d(n, 256), 256, 0, s>>>(c->sch_S.c(), n, dS.d());
  CVS_CHECK_LAUNCH();
  cplx* X = Xb.c();
  cplx* AX = AXb.c();
  int m = 0;
  auto append = [&](cplx* T, int cnt) {
    int added = 0;
    for (int q0 = 0; q0 < cnt && m < ms; q0 += 64) {
      const int cn = std::min(64, cnt - q0);
      cplx* Tq = T + (int64_t)q0 * n;
      ts_dot(s, Tq, cn, Tq, cn, n, tsp, G0, cn, true);
      gram_diag_sqrt(s, G0, cn, cn, nrm0);
      for (int pass = 0; pass < 2 && m > 0; ++pass) {
        ts_dot(s, X, m, Tq, cn, n, tsp, Cp, cn, true);
        ts_subtract(s, X, m, Cp, cn, cn, n, Tq, true);
      }
      ts_dot(s, Tq, cn, Tq, cn, n, tsp, G0, cn, true);
      block_orth(s, G0, cn, cn, nrm0, 1e-10, Xo, kept_d);
      int kept = 0;
      CVS_CUDA(cudaMemcpyAsync(&kept, kept_d, sizeof(int), cudaMemcpyDeviceToHost, s));
      c->sync();
      kept = std::min(kept, ms - m);
      if (kept <= 0) continue;
      ts_combine(s, Tq, Xo, nullptr, nullptr, cn, cn, kept, n, X + (int64_t)m * n, true);
      // S x for the new rows: (S x)^T = x^T S^T
      gemm64(c, kept, (int)n, (int)n, 1.0, view(X + (int64_t)m * n, n, 1),
             trans(view(c->sch_S.c(), n, 1)), 0.0, view(AX + (int64_t)m * n, n, 1));
      m += kept;
      added += kept;
    }
    return added;
  };
  // start: unit vectors at the p smallest diagonal entries
  {
    int64_t* idx = (int64_t*)(dw);
    DBuf kw;
    kw.ensure(4096 * sizeof(double));
    const int kk = std::min(p, 64);
    k_smallest(s, dS.d(), n, kk, (int64_t*)(nrm0 + 512), kw.d());
    std::vector<int64_t> hi(kk);
    CVS_CUDA(cudaMemcpyAsync(hi.data(), nrm0 + 512, kk * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemsetAsync(Tb.p, 0, (size_t)kk * n * sizeof(cplx), s));
    c->sync();
    const cplx one = cmake(1, 0);
    for (int q = 0; q < kk; ++q)
      CVS_CUDA(cudaMemcpyAsync(Tb.c() + q * n + hi[q], &one, sizeof(cplx), cudaMemcpyHostToDevice, s));
    (void)idx;
    append(Tb.c(), kk);
  }
  double scale = 1.0;
  int it = 0;
  std::vector<double> hw(ms), hr(p);
  for (; it < 300; ++it) {
    ts_dot(s, X, m, AX, m, n, tsp, H, m, true);
    hermitize(s, H, m, m, A, m);
    jacobi_eigh(s, A, m, w, Y, 60, dw);
    const int kk = std::min(p, m);
    // Ritz vectors U = Y[:, :kk]^T X, AU = Y^T AX
    ts_combine(s, X, Y, nullptr, nullptr, m, m, kk, n, U.c(), true);
    ts_combine(s, nullptr, nullptr, AX, Y, m, m, kk, n, AU.c(), true);
    residual_precond(s, AU.c(), U.c(), w, dS.d(), kk, n, Tb.c(), rpart.d(), rn);
    CVS_CUDA(cudaMemcpyAsync(hw.data(), w, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemcpyAsync(hr.data(), rn, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
    c->sync();
    scale = std::max(std::fabs(hw[0]), std::fabs(hw[m - 1]));
    std::vector<int> todo;
    for (int q = 0; q < kk; ++q)
      if (std::sqrt(std::max(hr[q], 0.0)) > 1e-6 * scale) todo.push_back(q);
    if (todo.empty() || kk < p) {
      if (todo.empty()) break;
    }
    if (m + (int)todo.size() > ms) {
      CVS_CUDA(cudaMemcpyAsync(X, U.p, (size_t)kk * n * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
      CVS_CUDA(cudaMemcpyAsync(AX, AU.p, (size_t)kk * n * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
      m = kk;
    }
    for (size_t q = 0; q < todo.size(); ++q)
      if (todo[q] != (int)q)
        CVS_CUDA(cudaMemcpyAsync(Tb.c() + q * n, Tb.c() + (int64_t)todo[q] * n,
                                 n * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    if (append(Tb.c(), (int)todo.size()) == 0) break;
  }
  // sch_U columns = U rows; eigenvalues ascending
  copyv(c, p, (int)n, 1.0, view(U.p, n, 1), view(c->sch_U.p, 1, p));
  CVS_CUDA(cudaMemcpyAsync(c->sch_lam.p, w, p * sizeof(double), cudaMemcpyDeviceToDevice, s));
  ++c->sch_builds;
  if (verbose()) {
    c->sync();
    fprintf(stderr, "[cvsadc] schur partial eigh n %lld p %d: %d iterations, %.1f ms, lam0 %.6f\n",
            (long long)n, p, it, now_ms() - t0, hw[0]);
  }
}

// Eigen-decomposition of sch_S into sch_U / sch_lam.  With warm set,
// sch_U holds the eigenvectors of a nearby S (the previous theta): S is
// first transformed into that basis, where it is nearly diagonal, so the
// Jacobi sweeps needed drop, and the eigenvectors are mapped back.
void schur_eigh(cvsadc_ctx* c, bool warm = false) {
  const double t0 = verbose() ? (c->sync(), now_ms()) : 0.0;
  const int64_t N1 = c->N1;
  const size_t cc_n = (size_t)(N1 / 2 + 2);
  double* part = c->sch_th.d() + 128;
  double* cc = c->sch_th.d() + 736;
  cplx* se = (cplx*)(c->sch_th.d() + 736 + ((cc_n + 1) & ~(size_t)1));
  if (warm) {
    // sch_V = S U_prev; sch_S = U_prev^H sch_V; sch_W keeps U_prev
    c->sch_W.ensure((size_t)N1 * N1 * sizeof(cplx));
    CVS_CUDA(cudaMemcpyAsync(c->sch_W.p, c->sch_U.p, (size_t)N1 * N1 * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, c->stream));
    gemm64(c, (int)N1, (int)N1, (int)N1, 1.0, view(c->sch_S.c(), N1, 1),
           view(c->sch_W.c(), N1, 1), 0.0, view(c->sch_V.c(), N1, 1));
    gemm64(c, (int)N1, (int)N1, (int)N1, 1.0,
           conj_of(trans(view(c->sch_W.c(), N1, 1))), view(c->sch_V.c(), N1, 1),
           0.0, view(c->sch_S.c(), N1, 1));
  }
  const int sweeps =
      jacobi_eigh_parallel(c->stream, c->sch_S.c(), (int)N1, c->sch_lam.d(),
                           c->sch_U.c(), c->sch_V.c(), part, cc, se, 30);
  if (warm) {
    // eigenvectors in the original basis: U = U_prev U'
    CVS_CUDA(cudaMemcpyAsync(c->sch_V.p, c->sch_U.p, (size_t)N1 * N1 * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, c->stream));
    gemm64(c, (int)N1, (int)N1, (int)N1, 1.0, view(c->sch_W.c(), N1, 1),
           view(c->sch_V.c(), N1, 1), 0.0, view(c->sch_U.c(), N1, 1));
  }
  ++c->sch_builds;
  if (verbose()) {
    c->sync();
    fprintf(stderr, "[cvsadc] schur eigh n %lld: %d sweeps, %.1f ms\n",
            (long long)N1, sweeps, now_ms() - t0);
  }
}

// Lowest eigenpair of a small Hermitian matrix (host, cyclic Jacobi);
// A is p x p row-major and is overwritten.
double small_eigh_lowest(std::vector<std::complex<double>>& A, int p,
                         std::vector<std::complex<double>>& y) {
  using C = std::complex<double>;
  std::vector<C> V((size_t)p * p, C(0, 0));
  for (int i = 0; i < p; ++i) V[(size_t)i * p + i] = C(1, 0);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < p; ++i)
      for (int j = 0; j < p; ++j) {
        const double m = std::norm(A[(size_t)i * p + j]);
        tot += m;
        if (i != j) off += m;
      }
    if (tot == 0.0 || off <= 1e-30 * tot) break;
    for (int a = 0; a < p; ++a)
      for (int b = a + 1; b < p; ++b) {
        const C apq = A[(size_t)a * p + b];
        const double r = std::abs(apq);
        if (r == 0.0) continue;
        const double app = A[(size_t)a * p + a].real(), aqq = A[(size_t)b * p + b].real();
        const double tau = (aqq - app) / (2.0 * r);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t);
        const C se = (t * cs) * (apq / r);
        for (int k = 0; k < p; ++k) {  // rows: A <- J^H A
          const C x = A[(size_t)a * p + k], z = A[(size_t)b * p + k];
          A[(size_t)a * p + k] = cs * x - se * z;
          A[(size_t)b * p + k] = std::conj(se) * x + cs * z;
        }
        for (int k = 0; k < p; ++k) {  // columns: A <- A J, V <- V J
          const C x = A[(size_t)k * p + a], z = A[(size_t)k * p + b];
          A[(size_t)k * p + a] = cs * x - std::conj(se) * z;
          A[(size_t)k * p + b] = se * x + cs * z;
          const C vx = V[(size_t)k * p + a], vz = V[(size_t)k * p + b];
          V[(size_t)k * p + a] = cs * vx - std::conj(se) * vz;
          V[(size_t)k * p + b] = se * vx + cs * vz;
        }
      }
  }
  int best = 0;
  for (int i = 1; i < p; ++i)
    if (A[(size_t)i * p + i].real() < A[(size_t)best * p + best].real()) best = i;
  y.resize(p);
  for (int k = 0; k < p; ++k) y[k] = V[(size_t)k * p + best];
  return A[(size_t)best * p + best].real();
}

// buffers of the preconditioner (sized for the prepared problem)
void schur_init(cvsadc_ctx* c) {
  const int nc = c->ncore, v = c->nvirt;
  const int64_t N1 = c->N1;
  const int jc = schur_jchunk(c);
  const int64_t v3 = (int64_t)v * v * v;
  const bool large = N1 > SCHUR_FULL_MAX;
  c->sch_p = large ? (int)std::min<int64_t>(SCHUR_PL, N1) : (int)N1;
  c->sch_S.ensure((size_t)N1 * N1 * sizeof(cplx));
  c->sch_U.ensure((size_t)N1 * c->sch_p * sizeof(cplx));
  c->sch_V.ensure((size_t)N1 * N1 * sizeof(cplx));
  c->sch_lam.ensure((size_t)N1 * sizeof(double));
  c->sch_C11.ensure((size_t)nc * v * v * sizeof(cplx));
  c->sch_C12.ensure((size_t)v * v * nc * nc * sizeof(cplx));
  c->sch_work.ensure((size_t)(2 + nc) * jc * v3 * sizeof(cplx));
  c->sch_tmp.ensure(std::max((size_t)v * v * nc * nc, (size_t)N1 * 64) * sizeof(cplx));
  c->sch_th.ensure(schur_th_doubles(N1) * sizeof(double) + 256);
}

// Finds theta0 and builds the preconditioner; false when it does not apply
// (singles space too large for the dense eigensolver, or the lowest root
// above the lowest M22 entry).  theta0 comes from Newton's method on
// f(theta) = lam0(S(theta)) - theta, which is concave and decreasing below
// the lowest M22 entry, started just below it: the iterates decrease
// monotonically towards the lowest root and stay above it.
void fold_apply(cvsadc_ctx* c, int prec, const cplx* V, int b, const double* th,
                cplx* R, cplx* D);

bool schur_setup(cvsadc_ctx* c) {
  const double t0 = now_ms();
  c->sch_on = false;
  c->sch_builds = 0;
  c->sch_couplings = 0;
  const int nc = c->ncore, nw = c->nval, v = c->nvirt, o = c->o, n = c->n;
  const int64_t N1 = c->N1, N = c->N;
  if (N1 > 3 * SCHUR_FULL_MAX || v < 2) return false;
  // large singles spaces: BF16X3 products for the build (it only steers the
  // iteration), the approximate cross term and the partial eigensystem
  const bool large = N1 > SCHUR_FULL_MAX;
  const int prec = large && tc_available() ? CVSADC_MIXED_BF16X3 : schur_precision();
  cudaStream_t s = c->stream;
  // lowest M22 entry
  std::vector<double> eps(n);
  CVS_CUDA(cudaMemcpyAsync(eps.data(), c->eps.p, n * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  c->sync();
  std::vector<double> ev(eps.begin() + o, eps.end());
  std::sort(ev.begin(), ev.end());
  const double emax_c = *std::max_element(eps.begin(), eps.begin() + nc);
  const double emax_w = *std::max_element(eps.begin() + nc, eps.begin() + o);
  const double pole = ev[0] + ev[1] - emax_c - emax_w;
  c->sch_pole = pole;
  schur_init(c);
  const int jc = schur_jchunk(c);
  const int64_t v3 = (int64_t)v * v * v;
  // keep <ab||cj> when it fits comfortably
  size_t free_b = 0, total_b = 0;
  CVS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const double gbytes = (double)nw * v3 * sizeof(cplx);
  bool cached = false;
  if (gbytes <= std::min(0.3 * (double)free_b, 48e9)) {
    c->sch_g.ensure((size_t)gbytes);
    cplx* X1 = c->sch_work.c();
    for (int j0 = 0; j0 < nw; j0 += jc)
      build_g_chunk(c, prec, j0, std::min(jc, nw - j0), X1,
                    c->sch_g.c() + (int64_t)j0 * v3);
    cached = true;
  }
  if (large) {
    // two builds: at the start point below the pole, then at the fixed point
    // of the lowest eigenvector's lift, found by Newton steps on that lift
    // (omega <- theta + (lam - theta) / (1 + ||W M21 u||^2), one fold each)
    double theta = pole - std::max(1.0, 0.03 * std::fabs(pole));
    DBuf u, R, D, MU, dots;
    u.ensure((size_t)N1 * sizeof(cplx));
    R.ensure((size_t)N1 * sizeof(cplx));
    D.ensure((size_t)N1 * sizeof(cplx));
    MU.ensure((size_t)N1 * sizeof(cplx));
    dots.ensure((size_t)(8 + 3 * TS_CHUNKS) * sizeof(cplx));
    for (int b = 0; b < 2; ++b) {
      build_schur(c, prec, theta, cached, true);
      schur_eigh_partial(c, c->sch_p);
      double lam0 = 0.0;
      CVS_CUDA(cudaMemcpyAsync(&lam0, c->sch_lam.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      c->sync();
      if (!std::isfinite(lam0) || (b == 0 && lam0 >= pole)) break;
      c->sch_theta = theta;
      c->sch_on = true;
      if (b == 1) break;
      copyv(c, 1, (int)N1, 1.0, view(c->sch_U.c(), 1, c->sch_p), view(u.p, N1, 1));
      gemm64(c, 1, (int)N1, (int)N1, 1.0, view(u.p, N1, 1), trans(view(c->M11.c(), N1, 1)),
             0.0, view(MU.p, N1, 1));
      double th = theta;
      for (int nt = 0; nt < 5; ++nt) {
        fold_apply(c, prec, u.c(), 1, &th, R.c(), D.c());
        cplx* part = dots.c() + 8;
        ts_dot(s, u.c(), 1, MU.c(), 1, N1, part, dots.c(), 1, true);
        ts_dot(s, u.c(), 1, R.c(), 1, N1, part, dots.c() + 1, 1, true);
        ts_dot(s, u.c(), 1, D.c(), 1, N1, part, dots.c() + 2, 1, true);
        cplx hv[3];
        CVS_CUDA(cudaMemcpyAsync(hv, dots.p, sizeof hv, cudaMemcpyDeviceToHost, s));
        c->sync();
        const double lam = hv[0].x + hv[1].x, nn = std::max(0.0, hv[2].x);
        double tn = th + (lam - th) / (1.0 + nn);
        if (!std::isfinite(tn)) break;
        tn = std::min(tn, 0.5 * (th + pole));
        const bool done = std::fabs(tn - th) < 1e-4 * std::max(1.0, std::fabs(th));
        th = tn;
        if (done) break;
      }
      if (verbose())
        fprintf(stderr, "[cvsadc] schur (large) theta %.6f lam0 %.6f -> next theta %.6f\n",
                theta, lam0, th);
      theta = th;
    }
    c->sync();
    c->sch_ms = now_ms() - t0;
    return c->sch_on;
  }
  // theta0: after each full build of S(theta), Newton's method runs on
  // lam0 of S projected on its p lowest eigenvectors u_i, where for any
  // theta only the small matrix
  //   S_p(theta) = U^H M11 U + W^H (theta - M22)^-1 W,  W = M21 U,
  // is needed (Rayleigh-Ritz: the projected root is never below the true
  // one).  The next full build is at the projected root; the search ends
  // when a build barely moves it.
  const int pp = (int)std::min<int64_t>(SCHUR_P, N1);
  DBuf xb, wb, zb, gb;
  xb.ensure((size_t)pp * N * sizeof(cplx));
  wb.ensure((size_t)pp * N * sizeof(cplx));
  zb.ensure((size_t)pp * N * sizeof(cplx));
  gb.ensure((size_t)(2 * pp * pp + N1 * pp) * sizeof(cplx));
  // start 1 Eh (or 3 % of |pole|) below the pole
  const double gap = std::max(1.0, 0.03 * std::fabs(pole));
  double theta = pole - gap;
  double built = theta;
  bool ok = false;
  std::vector<double> thv(pp);
  for (int it = 0; it < 6; ++it) {
    build_schur(c, prec, theta, cached);
    schur_eigh(c, it > 0);
    built = theta;
    double lam0 = 0.0;
    CVS_CUDA(cudaMemcpyAsync(&lam0, c->sch_lam.p, sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    c->sync();
    if (!std::isfinite(lam0)) break;
    if (it == 0 && lam0 >= pole) break;  // lowest root above the pole
    ok = true;
    // W = M21 U_p and A_p = U_p^H M11 U_p
    CVS_CUDA(cudaMemsetAsync(xb.p, 0, (size_t)pp * N * sizeof(cplx), s));
    copyv(c, pp, (int)N1, 1.0, view(c->sch_U.c(), 1, c->sch_p), view(xb.p, N, 1));
    sigma_impl(c, prec, xb.c(), wb.c(), pp, SIG_FWD);
    c->sch_couplings += pp;
    cplx* Gw = gb.c();
    cplx* G2 = Gw + (int64_t)pp * pp;
    cplx* T = G2 + (int64_t)pp * pp;
    gemm64(c, (int)N1, pp, (int)N1, 1.0, view(c->M11.c(), N1, 1),
           view(xb.p, 1, N), 0.0, view(T, pp, 1));
    gemm64(c, pp, pp, (int)N1, 1.0, conj_of(view(xb.p, N, 1)), view(T, pp, 1), 0.0,
           view(Gw, pp, 1));
    std::vector<std::complex<double>> Ap((size_t)pp * pp), Gh((size_t)pp * pp),
        G2h((size_t)pp * pp), Sp, y;
    CVS_CUDA(cudaMemcpyAsync(Ap.data(), Gw, (size_t)pp * pp * sizeof(cplx),
                             cudaMemcpyDeviceToHost, s));
    c->sync();
    double th = theta;
    for (int nt = 0; nt < 40; ++nt) {
      // Z = (th - M22)^-1 W;  G = Z^H W, G2 = Z^H Z over the doubles
      std::fill(thv.begin(), thv.end(), th);
      CVS_CUDA(cudaMemcpyAsync(c->sch_th.p, thv.data(), pp * sizeof(double),
                               cudaMemcpyHostToDevice, s));
      fold_doubles(s, wb.c(), nullptr, c->sch_th.d(), pp, N, N1, nc, nw, v,
                   c->eps.d(), true, zb.c());
      // rows i of conj(Z) (stride N), columns j of W and Z (stride N)
      gemm64(c, pp, pp, (int)(N - N1), 1.0, conj_of(view(zb.c() + N1, N, 1)),
             view(wb.c() + N1, 1, N), 0.0, view(Gw, pp, 1));
      gemm64(c, pp, pp, (int)(N - N1), 1.0, conj_of(view(zb.c() + N1, N, 1)),
             view(zb.c() + N1, 1, N), 0.0, view(G2, pp, 1));
      CVS_CUDA(cudaMemcpyAsync(Gh.data(), Gw, (size_t)pp * pp * sizeof(cplx),
                               cudaMemcpyDeviceToHost, s));
      CVS_CUDA(cudaMemcpyAsync(G2h.data(), G2, (size_t)pp * pp * sizeof(cplx),
                               cudaMemcpyDeviceToHost, s));
      c->sync();
      Sp.resize((size_t)pp * pp);
      for (int i = 0; i < pp; ++i)
        for (int j = 0; j < pp; ++j) {
          const std::complex<double> a = Ap[(size_t)i * pp + j] + Gh[(size_t)i * pp + j];
          const std::complex<double> b = Ap[(size_t)j * pp + i] + Gh[(size_t)j * pp + i];
          Sp[(size_t)i * pp + j] = 0.5 * (a + std::conj(b));
        }
      const double lp = small_eigh_lowest(Sp, pp, y);
      double zz = 0.0;  // y^H G2 y
      for (int i = 0; i < pp; ++i) {
        std::complex<double> t(0, 0);
        for (int j = 0; j < pp; ++j) t += G2h[(size_t)i * pp + j] * y[j];
        zz += (std::conj(y[i]) * t).real();
      }
      const double step = (lp - th) / (-1.0 - zz);
      if (!std::isfinite(step)) break;
      th = std::min(th - step, 0.5 * (th + pole));
      if (std::fabs(step) < 1e-9 * std::max(1.0, std::fabs(th))) break;
    }
    if (verbose())
      fprintf(stderr, "[cvsadc] schur theta %.8f lam0 %.8f projected root %.8f\n",
              theta, lam0, th);
    if (!std::isfinite(th)) break;
    const double move = theta - th;
    theta = th;
    // a start below the projected root is rebuilt there once (the projected
    // root is never below the true one), so the last build sits at or above
    // the lowest root
    if (std::fabs(move) < 0.05 && (move >= 0.0 || it > 0)) break;
  }
  c->sch_theta = built;
  c->sch_on = ok;
  c->sync();
  c->sch_ms = now_ms() - t0;
  return ok;
}

// ------------------------------------------------------------- Davidson
struct DavResult {
  int iters = 0, sigmas = 0, converged = 0;
  double maxres = 0.0;
  double t_sigma_ms = 0.0;
};

// Block Davidson for the lowest nroots eigenpairs of M (sigma in `prec`,
// all subspace algebra in FP64).  Restarts keep the nkeep lowest Ritz
// vectors (about a third of the subspace), which retains much of the
// Krylov information of the stiff doubles-dominated roots.  With
// stop_on_stagnation the iteration also ends when the largest residual has
// not halved over 50 iterations (the noise floor of a mixed-precision
// sigma).
DavResult davidson_impl(cvsadc_ctx* c, int prec, int nroots, int max_iter,
                        int max_sub, double tol, const cplx* X0, int nx0,
                        cplx* Xout, double* wout,
                        bool stop_on_stagnation = false, bool schur = false) {
  schur = schur && c->sch_on && c->sch_p == c->N1;
  // Gram matrices, Gram-Schmidt and Ritz combinations: plain FP64 for the
  // FP64-class precisions, double-float on the FP32 pipes for the mixed ones
  const bool a64 = prec == CVSADC_FP64 || prec == CVSADC_FP64_SLICE7;
  const int64_t N = c->N;
  const int k = nroots;
  const int msub = std::max(max_sub, 2 * k + 2);
  const int nkeep = std::max(k, std::min(msub / 3, msub - 2 * k));
  DavResult res;
  c->dv_V.ensure((size_t)msub * N * sizeof(cplx));
  c->dv_W.ensure((size_t)msub * N * sizeof(cplx));
  c->dv_X.ensure((size_t)nkeep * N * sizeof(cplx));
  c->dv_AX.ensure((size_t)nkeep * N * sizeof(cplx));
  c->dv_T.ensure((size_t)k * N * sizeof(cplx));
  c->dv_H.ensure((size_t)msub * msub * sizeof(cplx));
  c->dv_A.ensure((size_t)msub * msub * sizeof(cplx));
  c->dv_U.ensure((size_t)msub * msub * sizeof(cplx));
  c->dv_w.ensure((size_t)(msub + 64) * sizeof(double));
  // dv_misc: ts_dot partials [msub*msub*TS_CHUNKS] complex, then a
  // double work area laid out at fixed offsets
  const size_t W_PART = 0, W_RN2 = 64 * 320, W_JAC = W_RN2 + 128,
               W_KS = W_JAC + 64, W_IDX = W_KS + 1024, W_NRM = W_IDX + 128,
               W_KEPT = W_NRM + 64, W_COEF = W_KEPT + 64,
               W_TOTAL = W_COEF + 2 * (2 * 64 * 64 + 128 * 64);
  c->dv_misc.ensure((size_t)msub * msub * TS_CHUNKS * sizeof(cplx) +
                    W_TOTAL * sizeof(double));
  cplx* V = c->dv_V.c();
  cplx* W = c->dv_W.c();
  cplx* part = c->dv_misc.c();
  double* dwork = (double*)(part + (size_t)msub * msub * TS_CHUNKS);
  cplx* coef = (cplx*)(dwork + W_COEF);  // Gram, transform, projections
  cplx* Cproj = coef + 2 * 64 * 64;       // [msub][64] projection coefficients
  cudaStream_t s = c->stream;

  // initial vectors: given X0, else unit vectors at the smallest diagonal
  int m = 0;
  int nguess = std::min<int64_t>(std::max(k, std::min(2 * k, msub / 2)), N);
  if (X0 && nx0 > 0) {
    CVS_CUDA(cudaMemcpyAsync(V, X0, (size_t)nx0 * N * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, s));
    nguess = nx0;
  } else if (schur && std::min<int64_t>(std::min(nguess, 64), c->N1) >= k) {
    // the lowest eigenvectors u of S(theta0) with their folded doubles
    // (theta0 - M22)^-1 M21 u, built in W then compacted into V below (used
    // when they can cover every wanted root)
    nguess = (int)std::min<int64_t>(std::min(nguess, 64), c->N1);
    const int64_t N1 = c->N1;
    CVS_CUDA(cudaMemsetAsync(W, 0, (size_t)nguess * N * sizeof(cplx), s));
    copyv(c, nguess, (int)N1, 1.0, view(c->sch_U.c(), 1, N1), view(W, N, 1));
    sigma_impl(c, schur_precision(), W, V, nguess, SIG_FWD);
    c->sch_couplings += nguess;
    std::vector<double> th0(nguess, c->sch_theta);
    double* thd = c->sch_th.d();
    CVS_CUDA(cudaMemcpyAsync(thd, th0.data(), nguess * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    fold_doubles(s, V, nullptr, thd, nguess, N, N1, c->ncore, c->nval,
                 c->nvirt, c->eps.d(), false, W);
    CVS_CUDA(cudaMemcpyAsync(V, W, (size_t)nguess * N * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, s));
    c->sync();
  } else {
    nguess = std::min(nguess, 64);
    int64_t* idx = (int64_t*)(dwork + W_IDX);
    k_smallest(s, c->diag.d(), N, nguess, idx, dwork + W_KS);
    std::vector<int64_t> hidx(nguess);
    CVS_CUDA(cudaMemcpyAsync(hidx.data(), idx, nguess * sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemsetAsync(V, 0, (size_t)nguess * N * sizeof(cplx), s));
    c->sync();
    cplx one = cmake(1, 0);
    for (int q = 0; q < nguess; ++q)
      CVS_CUDA(cudaMemcpyAsync(V + q * N + hidx[q], &one, sizeof(cplx),
                               cudaMemcpyHostToDevice, s));
  }
  // append a block of cnt vectors (contiguous at T) to V: two passes of
  // block classical Gram-Schmidt against V, then an orthonormalising
  // transform of the block from its Gram matrix (FP64 throughout); vectors
  // whose norm falls below 1e-8 of their original norm are dropped
  cplx* G0 = coef;                     // [64][64] Gram matrix
  cplx* Xo = coef + 64 * 64;           // [64][64] transform
  double* nrm0 = dwork + W_NRM;        // [64]
  int* kept_d = (int*)(dwork + W_KEPT);
  auto orthonormalise_append = [&](cplx* T, int cnt) {
    cnt = std::min(cnt, msub - m);
    if (cnt <= 0) return 0;
    ts_dot(s, T, cnt, T, cnt, N, part, G0, cnt, a64);
    gram_diag_sqrt(s, G0, cnt, cnt, nrm0);
    if (m > 0) {
      for (int pass = 0; pass < 2; ++pass) {
        ts_dot(s, V, m, T, cnt, N, part, Cproj, cnt, a64);
        ts_subtract(s, V, m, Cproj, cnt, cnt, N, T, a64);
      }
    }
    ts_dot(s, T, cnt, T, cnt, N, part, G0, cnt, a64);
    block_orth(s, G0, cnt, cnt, nrm0, 1e-8, Xo, kept_d);
    int kept = 0;
    CVS_CUDA(cudaMemcpyAsync(&kept, kept_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    c->sync();
    if (kept > 0)
      ts_combine(s, T, Xo, nullptr, nullptr, cnt, cnt, kept, N,
                 V + (int64_t)m * N, a64);
    m += kept;
    return kept;
  };
  {
    // guesses live in V already at slots [0, nguess): compact through W
    CVS_CUDA(cudaMemcpyAsync(W, V, (size_t)nguess * N * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, s));
    m = 0;
    orthonormalise_append(W, nguess);
  }
  int m_done = 0;  // vectors whose sigma is known
  std::vector<double> theta(k), rn2(k), hist;
  std::vector<cplx> hostbuf;
  double t_it = now_ms();
  for (int it = 0; it < max_iter; ++it) {
    // sigma for new vectors
    int nnew = m - m_done;
    cudaEvent_t e0, e1;
    CVS_CUDA(cudaEventCreate(&e0));
    CVS_CUDA(cudaEventCreate(&e1));
    CVS_CUDA(cudaEventRecord(e0, s));
    sigma_impl(c, prec, V + (int64_t)m_done * N, W + (int64_t)m_done * N, nnew);
    CVS_CUDA(cudaEventRecord(e1, s));
    res.sigmas += nnew;
    // subspace matrix columns for the new vectors
    ts_dot(s, V, m, W + (int64_t)m_done * N, nnew, N, part,
           c->dv_H.c() + m_done, msub, a64);
    // the new rows against the old sigma images follow from Hermiticity
    herm_fill(s, c->dv_H.c(), msub, m_done, m);
    m_done = m;
    // A = (H + H^H)/2 over m x m (H stored with leading dimension msub)
    hermitize(s, c->dv_H.c(), msub, m, c->dv_A.c(), m);
    jacobi_eigh(s, c->dv_A.c(), m, c->dv_w.d(), c->dv_U.c(), 60,
                dwork + W_JAC);
    // Ritz vectors and their sigma images for the lowest k
    ts_combine(s, V, c->dv_U.c(), nullptr, nullptr, m, m, k, N, c->dv_X.c(), a64);
    ts_combine(s, nullptr, nullptr, W, c->dv_U.c(), m, m, k, N, c->dv_AX.c(), a64);
    residual_precond(s, c->dv_AX.c(), c->dv_X.c(), c->dv_w.d(),
                     schur ? nullptr : c->diag.d(), k, N, c->dv_T.c(),
                     dwork + W_PART, dwork + W_RN2);
    CVS_CUDA(cudaMemcpyAsync(theta.data(), c->dv_w.d(), k * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemcpyAsync(rn2.data(), dwork + W_RN2, k * sizeof(double),
                             cudaMemcpyDeviceToHost, s));
    c->sync();
    {
      float ms = 0;
      CVS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      res.t_sigma_ms += ms;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    res.iters = it + 1;
    if (verbose()) {
      double mx = 0;
      for (int r = 0; r < k; ++r) mx = std::max(mx, rn2[r]);
      fprintf(stderr, "[cvsadc] davidson it %3d m %3d theta0 %.12f max|r| %.3e  t %.1f ms\n",
              it, m, theta[0], std::sqrt(mx), now_ms() - t_it);
      t_it = now_ms();
    }
    std::vector<int> todo;
    res.maxres = 0;
    res.converged = 0;
    for (int r = 0; r < k; ++r) {
      double rn = std::sqrt(std::max(rn2[r], 0.0));
      res.maxres = std::max(res.maxres, rn);
      if (rn <= tol)
        ++res.converged;
      else
        todo.push_back(r);
    }
    if (todo.empty() || it == max_iter - 1) break;
    if (stop_on_stagnation) {
      // near the noise floor of a mixed-precision sigma the residual stops
      // falling: end when it has not halved over 30 iterations there
      hist.push_back(res.maxres);
      if (res.maxres < 100 * tol && hist.size() > 30 &&
          res.maxres > 0.5 * hist[hist.size() - 31])
        break;
      // with the Schur preconditioner the residual falls several-fold per
      // iteration until the noise floor: hand over once three iterations
      // have not halved it
      if (schur && hist.size() > 3 && res.maxres > 0.5 * hist[hist.size() - 4])
        break;
    }
    // thick restart to the nkeep lowest Ritz vectors when the block does
    // not fit
    if (m + (int)todo.size() > msub) {
      const int nk = std::min(nkeep, m);
      ts_combine(s, V, c->dv_U.c(), nullptr, nullptr, m, m, nk, N, c->dv_X.c(), a64);
      ts_combine(s, nullptr, nullptr, W, c->dv_U.c(), m, m, nk, N, c->dv_AX.c(), a64);
      CVS_CUDA(cudaMemcpyAsync(V, c->dv_X.p, (size_t)nk * N * sizeof(cplx),
                               cudaMemcpyDeviceToDevice, s));
      CVS_CUDA(cudaMemcpyAsync(W, c->dv_AX.p, (size_t)nk * N * sizeof(cplx),
                               cudaMemcpyDeviceToDevice, s));
      // H = diag(theta_0 .. theta_{nk-1})
      std::vector<double> th(nk);
      CVS_CUDA(cudaMemcpyAsync(th.data(), c->dv_w.d(), nk * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
      c->sync();
      std::vector<cplx> h((size_t)msub * msub, cmake(0, 0));
      for (int r = 0; r < nk; ++r) h[(size_t)r * msub + r] = cmake(th[r], 0);
      CVS_CUDA(cudaMemcpyAsync(c->dv_H.p, h.data(), h.size() * sizeof(cplx),
                               cudaMemcpyHostToDevice, s));
      c->sync();
      // the k wanted Ritz pairs are rows 0..k-1 of the new basis again
      m = nk;
      m_done = nk;
    }
    // append corrections of the unconverged roots
    for (size_t q = 0; q < todo.size(); ++q)
      if (todo[q] != (int)q)
        CVS_CUDA(cudaMemcpyAsync(c->dv_T.c() + (int64_t)q * N,
                                 c->dv_T.c() + (int64_t)todo[q] * N,
                                 N * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    cplx* Tn = c->dv_T.c();
    if (schur) {
      // block elimination with S(theta0) (see schur_setup): Z, Y are free
      // here (the Ritz blocks are rebuilt next iteration)
      const int cnt = (int)todo.size();
      const int64_t N1 = c->N1;
      const int pp = schur_precision();
      cplx* Z = c->dv_X.c();
      cplx* Yb = c->dv_AX.c();
      std::vector<double> tht(cnt);
      for (int q = 0; q < cnt; ++q) tht[q] = theta[todo[q]];
      double* thd = c->sch_th.d();
      CVS_CUDA(cudaMemcpyAsync(thd, tht.data(), cnt * sizeof(double),
                               cudaMemcpyHostToDevice, s));
      // z = (0, (theta - M22)^-1 r2);  y1 = r1 + M12 z2
      fold_doubles(s, Tn, nullptr, thd, cnt, N, N1, c->ncore, c->nval,
                   c->nvirt, c->eps.d(), true, Z);
      sigma_impl(c, pp, Z, Yb, cnt, SIG_ADJ);
      add_singles(s, Tn, Yb, N, N1, cnt, Yb);
      // t1 = U (theta - lam)^-1 U^H y1
      cplx* Ty = c->sch_tmp.c();
      gemm64(c, (int)N1, cnt, (int)N1, 1.0,
             conj_of(trans(view(c->sch_U.c(), N1, 1))), view(Yb, 1, N), 0.0,
             view(Ty, cnt, 1));
      eig_shift(s, Ty, N1, cnt, c->sch_lam.d(), thd);
      gemm64(c, (int)N1, cnt, (int)N1, 1.0, view(c->sch_U.c(), N1, 1),
             view(Ty, cnt, 1), 0.0, view(Z, 1, N));
      // t2 = (theta - M22)^-1 (r2 + M21 t1)
      sigma_impl(c, pp, Z, Yb, cnt, SIG_FWD);
      fold_doubles(s, Tn, Yb, thd, cnt, N, N1, c->ncore, c->nval, c->nvirt,
                   c->eps.d(), false, Z);
      c->sch_couplings += 2 * cnt;
      // roots at or above the lowest M22 entry: S(theta0) says nothing about
      // them, so they take the diagonal preconditioner
      for (int q = 0; q < cnt; ++q)
        if (tht[q] >= c->sch_pole - 1e-3)
          diag_precond(s, Tn + (int64_t)q * N, tht[q], c->diag.d(), N,
                       Z + (int64_t)q * N);
      Tn = Z;
    }
    int added = orthonormalise_append(Tn, (int)todo.size());
    if (added == 0) break;
  }
  CVS_CUDA(cudaMemcpyAsync(wout, c->dv_w.d(), k * sizeof(double),
                           cudaMemcpyDeviceToHost, s));
  CVS_CUDA(cudaMemcpyAsync(Xout, c->dv_X.p, (size_t)k * N * sizeof(cplx),
                           cudaMemcpyDeviceToDevice, s));
  c->sync();
  return res;
}

// Residual at which the mixed-precision Davidson hands over to the FP64
// correction: a few times the sigma noise of the tensor-core GEMMs
// (BF16X3 ~1e-5 relative, SLICE4 ~1e-8, on |M x| of O(10-100) Eh).
// FP64-class sigma for the residual correction: the exact-slice
// tensor-core GEMM (FP64_SLICE7, ~1e-14 relative) after SLICE4, the FP64
// FMA GEMM after BF16X3 (CVSADC_REFINE_FP64 forces FP64 FMA for both)
int refine_precision(int prec) {
  const char* e = getenv("CVSADC_REFINE_FP64");
  if (e && *e && *e != '0') return CVSADC_FP64;
  return prec == CVSADC_MIXED_SLICE4 ? CVSADC_FP64_SLICE7 : CVSADC_FP64;
}

double mixed_tolerance(int prec) {
  const char* e = getenv("CVSADC_MIXED_TOL");
  if (e && *e) return atof(e);
  return prec == CVSADC_MIXED_BF16X3 ? 3e-4 : 1e-6;
}

// Lowest k roots of the prepared problem into Xd [k][N] and w: Davidson in
// `prec`, then, for the tensor-core precisions (unless no_refine), a
// continuation with FP64-class sigma from the converged Ritz vectors, each
// sweep costing one sigma per unconverged root.  t_refine gets the time of
// the second phase.
DavResult solve_roots(cvsadc_ctx* c, int prec, int k, double tol, int max_iter,
                      int max_sub, int refine_sweeps, bool no_refine, cplx* Xd,
                      double* w, double* t_refine, bool use_schur = true) {
  const bool refine = needs_refine(prec) && !no_refine;
  const double tol_phase = refine ? std::max(tol, mixed_tolerance(prec)) : tol;
  c->sch_ms = 0.0;
  c->sch_builds = 0;
  c->sch_couplings = 0;
  const bool schur = use_schur && schur_setup(c);
  DavResult r = davidson_impl(c, prec, k, max_iter, max_sub, tol_phase, nullptr,
                              0, Xd, w, needs_refine(prec), schur);
  const double t1 = now_ms();
  if (refine) {
    DBuf X0;
    X0.ensure((size_t)k * c->N * sizeof(cplx));
    CVS_CUDA(cudaMemcpyAsync(X0.p, Xd, (size_t)k * c->N * sizeof(cplx),
                             cudaMemcpyDeviceToDevice, c->stream));
    const int sweeps = refine_sweeps > 0 ? refine_sweeps : 20;
    DavResult r2 = davidson_impl(c, refine_precision(prec), k, sweeps, max_sub,
                                 tol, X0.c(), k, Xd, w, false, schur);
    r.iters += r2.iters;
    r.sigmas += r2.sigmas;
    r.t_sigma_ms += r2.t_sigma_ms;
    r.converged = r2.converged;
    r.maxres = r2.maxres;
  }
  if (t_refine) *t_refine = refine ? now_ms() - t1 : 0.0;
  return r;
}

// ===================================================== doubles-folded solver
// M22 is diagonal, so an eigenpair (omega, z) of M with omega below the
// lowest M22 entry has z = (x1, W(omega) M21 x1), W(theta) = (theta -
// M22)^-1, where x1 solves the pseudo-eigenvalue problem S(omega) x1 =
// omega x1 with S(theta) = M11 + M12 W(theta) M21 (Eqs. 11-12; exact because
// the doubles block is diagonal).  This solver stores singles-space vectors
// only.  Its basis vectors are lifts z_j = (v_j, W_j M21 v_j), each at its
// own theta_j, represented by v_j and the two folds
//   R_j = M12 W_j M21 v_j   and   D_j = M12 W_j^2 M21 v_j,
// from which every projected matrix of M over the basis follows exactly
// (lift_assemble): the Rayleigh-Ritz step is the one of M in the full
// space, and no doubles vector outlives a fold.  A Ritz pair (omega, C) has
// the full residual r = (sum_j c_j (s_j - omega v_j),
// sum_j c_j (theta_j - omega) W_j u_j), s_j = M11 v_j + R_j, whose norm
// also follows from the projected matrices, and the folded residual
// r~ = S(omega) x1 - omega x1 ~ sum_j c_j (s_j - (omega - theta_j) D_j -
// omega v_j).  New directions are preconditioned folded residuals lifted at
// the current Ritz values; lifts made at outdated theta leave a part of the
// residual that singles directions cannot remove, so once ||r~|| falls
// below half of ||r|| the basis restarts from the Ritz singles lifted at
// their Ritz values.

// R = M12 W M21 v and D = M12 W^2 M21 v for b singles vectors (rows of V,
// [b][N1]) with theta th[b] (host); R and D are [b][N1].  Each group of g
// vectors goes through one forward coupling product (M21), two weightings
// and one adjoint product (M12) over 2g vectors.
void fold_apply(cvsadc_ctx* c, int prec, const cplx* V, int b, const double* th,
                cplx* R, cplx* D) {
  const int64_t N = c->N, N1 = c->N1;
  cudaStream_t s = c->stream;
  const double per = 4.0 * (double)N * sizeof(cplx);
  const int g = (int)std::max(1.0, std::min((double)b, 40e9 / per));
  c->fd_A.ensure((size_t)2 * g * N * sizeof(cplx));
  c->fd_B.ensure((size_t)2 * g * N * sizeof(cplx));
  c->fd_th.ensure((size_t)(2 * g + 8) * sizeof(double));
  for (int q0 = 0; q0 < b; q0 += g) {
    const int gg = std::min(g, b - q0);
    cplx* X = c->fd_A.c();   // [gg][N] lift input, later [2gg][N] adjoint output
    cplx* Sg = X + (int64_t)gg * N;
    cplx* U2 = c->fd_B.c();  // [2gg][N]: (0, W u) then (0, W^2 u)
    CVS_CUDA(cudaMemsetAsync(X, 0, (size_t)gg * N * sizeof(cplx), s));
    copyv(c, gg, (int)N1, 1.0, view(V + (int64_t)q0 * N1, N1, 1), view(X, N, 1));
    sigma_impl(c, prec, X, Sg, gg, SIG_FWD);  // doubles of Sg = M21 v
    CVS_CUDA(cudaMemcpyAsync(c->fd_th.p, th + q0, gg * sizeof(double),
                             cudaMemcpyHostToDevice, s));
    fold_doubles(s, Sg, nullptr, c->fd_th.d(), gg, N, N1, c->ncore, c->nval, c->nvirt,
                 c->eps.d(), true, U2);
    fold_doubles(s, U2, nullptr, c->fd_th.d(), gg, N, N1, c->ncore, c->nval, c->nvirt,
                 c->eps.d(), true, U2 + (int64_t)gg * N);
    sigma_impl(c, prec, U2, X, 2 * gg, SIG_ADJ);  // singles of X = M12 (.)
    copyv(c, gg, (int)N1, 1.0, view(X, N, 1), view(R + (int64_t)q0 * N1, N1, 1));
    copyv(c, gg, (int)N1, 1.0, view(X + (int64_t)gg * N, N, 1),
          view(D + (int64_t)q0 * N1, N1, 1));
    c->sync();  // fd_th is reused by the next group
  }
  c->sch_couplings += 3 * b;
}

struct FoldResult {
  int iters = 0, folds = 0, restarts = 0, converged = 0;
  double maxres = 0.0;
};

// Lowest k roots by the doubles-folded solver in precision `prec`.  Starting
// singles x0 [nx0][N1] at theta th0 (host), or (nx0 == 0) the lowest
// eigenvectors of the Schur preconditioner S(theta0).  Outputs: the Ritz
// singles X1 [k][N1] (device) and the roots w[k] (host).
FoldResult folded_davidson(cvsadc_ctx* c, int prec, int k, int max_iter, int max_sub,
                           double tol, const cplx* x0, const double* th0, int nx0,
                           cplx* X1out, double* wout, bool stop_on_stagnation,
                           bool newton_start) {
  const int64_t N1 = c->N1;
  cudaStream_t s = c->stream;
  const bool a64 = prec == CVSADC_FP64 || prec == CVSADC_FP64_SLICE7;
  const int msub = std::min(128, std::max(max_sub, 3 * k + 2));
  const double delta = 1e-3;  // partial fractions vs midpoint rule for Q
  FoldResult res;
  c->fv_V.ensure((size_t)msub * N1 * sizeof(cplx));
  c->fv_B.ensure((size_t)msub * N1 * sizeof(cplx));
  c->fv_R.ensure((size_t)msub * N1 * sizeof(cplx));
  c->fv_D.ensure((size_t)msub * N1 * sizeof(cplx));
  c->fv_MV.ensure((size_t)msub * N1 * sizeof(cplx));
  c->fv_T.ensure((size_t)4 * k * N1 * sizeof(cplx));
  c->fv_T2.ensure((size_t)4 * k * N1 * sizeof(cplx));
  // small device matrices (leading dimension msub, or the block size for
  // the orthonormalisation scratch, up to 64)
  const size_t mm = (size_t)std::max(msub, 64) * std::max(msub, 64);
  const size_t n_small = 13 * mm;
  const size_t W_PART = n_small * 2;  // in doubles
  const size_t TSP = (size_t)std::min(msub, 96) * 192 * TS_CHUNKS;
  c->fv_small.ensure(n_small * sizeof(cplx) + TSP * sizeof(cplx) +
                     (size_t)(6 * msub + 4096) * sizeof(double));
  cplx* E = c->fv_small.c();
  cplx* VD = E + mm;
  cplx* Am = VD + mm;
  cplx* VV = Am + mm;
  cplx* Q = VV + mm;
  cplx* H = Q + mm;
  cplx* O = H + mm;
  cplx* Uo = O + mm;
  cplx* Oi = Uo + mm;
  cplx* Hp = Oi + mm;
  cplx* Yp = Hp + mm;
  cplx* C = Yp + mm;
  cplx* Cp = C + mm;
  cplx* tsp = c->fv_small.c() + n_small;
  double* dw = (double*)(tsp + TSP);
  double* wo = dw;              // [msub]
  double* wp = wo + msub;       // [msub]
  double* thd = wp + msub;      // [msub]
  double* rn1 = thd + msub;     // [msub]
  double* rnt = rn1 + msub;     // [msub]
  double* jinfo = rnt + msub;   // jacobi info + misc
  cplx* V = c->fv_V.c();
  cplx* Bo = c->fv_B.c();  // orthonormal basis of span(V) (singles metric)
  cplx* Rf = c->fv_R.c();
  cplx* Df = c->fv_D.c();
  cplx* MV = c->fv_MV.c();
  cplx* T = c->fv_T.c();
  cplx* T2 = c->fv_T2.c();
  std::vector<double> th(msub, 0.0);
  int m = 0, nb = 0;  // basis size, orthonormal-basis size

  // orthonormal rows of T (cnt) against Bo[0:nb] and within, appended to
  // Bo and (when toV) V; returns how many were kept
  double* nrm0 = jinfo + 16;
  int* kept_d = (int*)(jinfo + 16 + 256);
  int* src_d = kept_d + 64;
  std::vector<int> src_h(64);
  cplx* G0 = Hp;  // scratch for the block Gram / transform (cnt <= 4k <= msub)
  cplx* Xo = Yp;
  auto orth_append = [&](cplx* Tb, int cnt, bool toV) {
    if (cnt <= 0) return 0;
    ts_dot(s, Tb, cnt, Tb, cnt, N1, tsp, G0, cnt, a64);
    gram_diag_sqrt(s, G0, cnt, cnt, nrm0);
    if (nb > 0)
      for (int pass = 0; pass < 2; ++pass) {
        ts_dot(s, Bo, nb, Tb, cnt, N1, tsp, Cp, cnt, a64);
        ts_subtract(s, Bo, nb, Cp, cnt, cnt, N1, Tb, a64);
      }
    ts_dot(s, Tb, cnt, Tb, cnt, N1, tsp, G0, cnt, a64);
    block_orth(s, G0, cnt, cnt, nrm0, 1e-10, Xo, kept_d, src_d);
    int kept = 0;
    CVS_CUDA(cudaMemcpyAsync(&kept, kept_d, sizeof(int), cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemcpyAsync(src_h.data(), src_d, 64 * sizeof(int), cudaMemcpyDeviceToHost, s));
    c->sync();
    kept = std::min(kept, msub - nb);
    if (kept > 0) {
      ts_combine(s, Tb, Xo, nullptr, nullptr, cnt, cnt, kept, N1, Bo + (int64_t)nb * N1, a64);
      if (toV)
        CVS_CUDA(cudaMemcpyAsync(V + (int64_t)m * N1, Bo + (int64_t)nb * N1,
                                 (size_t)kept * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    }
    nb += kept;
    return kept;
  };
  // lift rows [m0, m0 + cnt) of V at th[m0..], fold, and M11 V
  auto lift = [&](int m0, int cnt) {
    fold_apply(c, prec, V + (int64_t)m0 * N1, cnt, th.data() + m0, Rf + (int64_t)m0 * N1,
               Df + (int64_t)m0 * N1);
    gemm64(c, cnt, (int)N1, (int)N1, 1.0, view(V + (int64_t)m0 * N1, N1, 1),
           trans(view(c->M11.c(), N1, 1)), 0.0, view(MV + (int64_t)m0 * N1, N1, 1));
    res.folds += cnt;
  };
  // set the basis to the rows of Xs (cnt, normalised) lifted at ths
  auto restart = [&](const cplx* Xs, const double* ths, int cnt) {
    cnt = std::min(cnt, msub);
    CVS_CUDA(cudaMemcpyAsync(V, Xs, (size_t)cnt * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    row_norm2(s, V, cnt, N1, rn1);
    std::vector<double> nn(cnt), sc(cnt);
    CVS_CUDA(cudaMemcpyAsync(nn.data(), rn1, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
    c->sync();
    for (int q = 0; q < cnt; ++q) sc[q] = nn[q] > 0 ? 1.0 / std::sqrt(nn[q]) : 1.0;
    CVS_CUDA(cudaMemcpyAsync(rn1, sc.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, s));
    scale_vectors(s, V, rn1, cnt, N1);
    for (int q = 0; q < cnt; ++q) th[q] = ths[q];
    m = cnt;
    lift(0, cnt);
    // orthonormal basis of the restart singles
    nb = 0;
    CVS_CUDA(cudaMemcpyAsync(T2, V, (size_t)cnt * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    for (int q0 = 0; q0 < cnt; q0 += 64) orth_append(T2 + (int64_t)q0 * N1, std::min(64, cnt - q0), false);
    ++res.restarts;
  };

  // ---- initial basis
  int nguess;
  if (x0 && nx0 > 0) {
    nguess = std::min(nx0, msub);
    restart(x0, th0, nguess);
    --res.restarts;
  } else {
    CVS_REQUIRE(c->sch_on, CVSADC_EINVAL, "folded solver: no initial vectors");
    // the lowest eigenvectors of S(theta0), lifted at theta0
    nguess = (int)std::min<int64_t>(std::min(std::min(2 * k, msub), c->sch_p), N1);
    copyv(c, nguess, (int)N1, 1.0, view(c->sch_U.c(), 1, c->sch_p), view(T, N1, 1));
    std::vector<double> t0(nguess, c->sch_theta);
    restart(T, t0.data(), nguess);
    --res.restarts;
    newton_start = true;
  }
  if (newton_start) {
    // one Newton step on each starting vector u lifted at theta,
    // omega ~ theta + (lam - theta) / (1 + ||W M21 u||^2) (the Rayleigh
    // quotient of the lift), gives the theta it is lifted at next
    ts_dot(s, V, m, Rf, m, N1, tsp, E, msub, a64);
    ts_dot(s, V, m, MV, m, N1, tsp, Am, msub, a64);
    ts_dot(s, V, m, Df, m, N1, tsp, VD, msub, a64);
    std::vector<cplx> he((size_t)m * msub), ha((size_t)m * msub), hd((size_t)m * msub);
    CVS_CUDA(cudaMemcpyAsync(he.data(), E, he.size() * sizeof(cplx), cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemcpyAsync(ha.data(), Am, ha.size() * sizeof(cplx), cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemcpyAsync(hd.data(), VD, hd.size() * sizeof(cplx), cudaMemcpyDeviceToHost, s));
    c->sync();
    std::vector<double> est(m);
    for (int q = 0; q < m; ++q) {
      const double lam = he[(size_t)q * msub + q].x + ha[(size_t)q * msub + q].x;
      const double nq = hd[(size_t)q * msub + q].x;
      est[q] = th[q] + (lam - th[q]) / (1.0 + nq);
      if (!std::isfinite(est[q])) est[q] = th[q];
    }
    if (c->sch_on && x0 == nullptr) {
      // first-order drift of the Schur eigenvalues with theta: d_i = ||W(theta0)
      // M21 u_i||^2 for the guesses u_i (lifted at theta0 just now); the
      // higher eigenvectors take the last of these
      std::vector<double> dd(c->sch_p, std::max(0.0, hd[(size_t)(m - 1) * msub + (m - 1)].x));
      for (int q = 0; q < m && q < c->sch_p; ++q) dd[q] = std::max(0.0, hd[(size_t)q * msub + q].x);
      c->sch_d.ensure((size_t)c->sch_p * sizeof(double));
      CVS_CUDA(cudaMemcpyAsync(c->sch_d.p, dd.data(), c->sch_p * sizeof(double),
                               cudaMemcpyHostToDevice, s));
      c->sch_d_on = true;
    }
    CVS_CUDA(cudaMemcpyAsync(T, V, (size_t)m * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    restart(T, est.data(), m);
    --res.restarts;
  }

  std::vector<double> w(msub), r1(k), rt(k), hist;
  std::vector<cplx> g2((size_t)k * k);
  for (int it = 0; it < max_iter; ++it) {
    // projected matrices over the lifted basis
    CVS_CUDA(cudaMemcpyAsync(thd, th.data(), m * sizeof(double), cudaMemcpyHostToDevice, s));
    ts_dot(s, V, m, Rf, m, N1, tsp, E, msub, a64);
    ts_dot(s, V, m, MV, m, N1, tsp, Am, msub, a64);
    ts_dot(s, V, m, Df, m, N1, tsp, VD, msub, a64);
    ts_dot(s, V, m, V, m, N1, tsp, VV, msub, a64);
    lift_assemble(s, E, VD, Am, VV, thd, m, msub, delta, Q, H, O);
    // generalised eigenproblem H c = w O c through O^-1/2 (eigenvalues of O
    // below 1e-12 of the largest are dropped)
    hermitize(s, O, msub, m, Hp, m);
    jacobi_eigh(s, Hp, m, wo, Uo, 60, jinfo);
    std::vector<double> hw(m);
    CVS_CUDA(cudaMemcpyAsync(hw.data(), wo, m * sizeof(double), cudaMemcpyDeviceToHost, s));
    c->sync();
    int off = 0;
    while (off < m - 1 && !(hw[off] > 1e-12 * hw[m - 1])) ++off;
    const int kept = m - off;
    // Uo is [m][m] dense (ld m); Oi [m][kept] with ld msub
    inv_sqrt_cols(s, Uo, wo, m, off, kept, m, Oi);
    // Hp = Oi^H H Oi (kept x kept)
    gemm64(c, m, kept, m, 1.0, view(H, msub, 1), view(Oi, m, 1), 0.0, view(Cp, msub, 1));
    gemm64(c, kept, kept, m, 1.0, conj_of(trans(view(Oi, m, 1))), view(Cp, msub, 1), 0.0,
           view(Hp, kept, 1));
    jacobi_eigh(s, Hp, kept, wp, Yp, 60, jinfo);
    const int kk = std::min(k, kept);
    // C = Oi Yp[:, :kk]  ([m][kk], ld msub)
    gemm64(c, m, kk, kept, 1.0, view(Oi, m, 1), view(Yp, kept, 1), 0.0, view(C, msub, 1));
    CVS_CUDA(cudaMemcpyAsync(w.data(), wp, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
    // Ritz singles X1 = C^T V, S C = C^T (MV + R), residuals
    gemm64(c, kk, (int)N1, m, 1.0, trans(view(C, msub, 1)), view(V, N1, 1), 0.0, view(T2, N1, 1));
    gemm64(c, kk, (int)N1, m, 1.0, trans(view(C, msub, 1)), view(MV, N1, 1), 0.0, view(T, N1, 1));
    gemm64(c, kk, (int)N1, m, 1.0, trans(view(C, msub, 1)), view(Rf, N1, 1), 1.0, view(T, N1, 1));
    lift_coef(s, C, m, kk, msub, wp, thd, Cp);
    // r1 = SC - w X1 (into T), the folded residual r~ = r1 - Cp^T D (into T + k N1)
    row_axpy(s, T, T2, wp, kk, N1, T);
    cplx* Rt = T + (int64_t)k * N1;
    CVS_CUDA(cudaMemcpyAsync(Rt, T, (size_t)kk * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    gemm64(c, kk, (int)N1, m, -1.0, trans(view(Cp, msub, 1)), view(Df, N1, 1), 1.0, view(Rt, N1, 1));
    row_norm2(s, T, kk, N1, rn1);
    row_norm2(s, Rt, kk, N1, rnt);
    // ||r2||^2 = Cp^H Q Cp (diagonal): G = Q Cp, then Cp^H G
    gemm64(c, m, kk, m, 1.0, view(Q, msub, 1), view(Cp, msub, 1), 0.0, view(Hp, msub, 1));
    gemm64(c, kk, kk, m, 1.0, conj_of(trans(view(Cp, msub, 1))), view(Hp, msub, 1), 0.0,
           view(Yp, kk, 1));
    CVS_CUDA(cudaMemcpyAsync(r1.data(), rn1, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemcpyAsync(rt.data(), rnt, kk * sizeof(double), cudaMemcpyDeviceToHost, s));
    CVS_CUDA(cudaMemcpyAsync(g2.data(), Yp, (size_t)kk * kk * sizeof(cplx), cudaMemcpyDeviceToHost, s));
    c->sync();
    res.iters = it + 1;
    std::vector<double> rn(kk), rtn(kk);
    std::vector<int> todo;
    res.maxres = 0.0;
    res.converged = 0;
    for (int q = 0; q < kk; ++q) {
      rn[q] = std::sqrt(std::max(0.0, r1[q] + std::max(0.0, g2[(size_t)q * kk + q].x)));
      rtn[q] = std::sqrt(std::max(0.0, rt[q]));
      res.maxres = std::max(res.maxres, rn[q]);
      if (rn[q] <= tol) ++res.converged; else todo.push_back(q);
    }
    if (verbose())
      fprintf(stderr, "[cvsadc] folded it %3d m %3d w0 %.12f max|r| %.3e folds %d\n", it, m,
              w[0], res.maxres, res.folds);
    if (todo.empty() || it == max_iter - 1) break;
    if (stop_on_stagnation) {
      // the noise floor of a mixed-precision sigma: no 10 % gain over 8
      // iterations (slow linear convergence of clustered roots keeps going;
      // restarts keep the Ritz vectors, so the history runs through them)
      hist.push_back(res.maxres);
      if (hist.size() > 8 && res.maxres > 0.9 * hist[hist.size() - 9]) break;
    }
    bool stale = false;
    for (int q : todo) stale = stale || rtn[q] < 0.5 * rn[q];
    if (stale || m + (int)todo.size() > msub) {
      // the Ritz singles, re-lifted at their Ritz values
      CVS_CUDA(cudaMemcpyAsync(T, T2, (size_t)kk * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
      restart(T, w.data(), kk);
      continue;
    }
    // preconditioned folded residuals of the unconverged roots
    const int cnt = (int)todo.size();
    for (int q = 0; q < cnt; ++q)
      if (todo[q] != q)
        CVS_CUDA(cudaMemcpyAsync(Rt + (int64_t)q * N1, Rt + (int64_t)todo[q] * N1,
                                 N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    std::vector<double> wt(cnt);
    for (int q = 0; q < cnt; ++q) wt[q] = w[todo[q]];
    if (c->sch_on && c->sch_p < N1) {
      // partial eigensystem: t = U_p (w - lam)^-1 U_p^H r~ plus
      // (1 - U_p U_p^H) r~ / (w - lam_c), lam_c the highest computed
      const int pp = c->sch_p;
      double lam_c = 0.0;
      CVS_CUDA(cudaMemcpyAsync(&lam_c, c->sch_lam.d() + pp - 1, sizeof(double),
                               cudaMemcpyDeviceToHost, s));
      cplx* Ty = c->sch_tmp.c();
      CVS_CUDA(cudaMemcpyAsync(rn1, wt.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, s));
      c->sync();
      gemm64(c, pp, cnt, (int)N1, 1.0, conj_of(trans(view(c->sch_U.c(), pp, 1))),
             view(Rt, 1, N1), 0.0, view(Ty, cnt, 1));
      if (!c->sch_d_on) {
        c->sch_d.ensure((size_t)pp * sizeof(double));
        CVS_CUDA(cudaMemsetAsync(c->sch_d.p, 0, (size_t)pp * sizeof(double), s));
        c->sch_d_on = true;
      }
      eig_shift_partial(s, Ty, pp, cnt, c->sch_lam.d(), c->sch_d.d(), c->sch_theta, rn1, lam_c);
      gemm64(c, (int)N1, cnt, pp, 1.0, view(c->sch_U.c(), pp, 1), view(Ty, cnt, 1), 0.0,
             view(T, 1, N1));
      std::vector<double> sc(cnt);
      for (int q = 0; q < cnt; ++q) {
        const double dc = wt[q] - lam_c;
        sc[q] = -1.0 / (std::fabs(dc) < 1e-8 ? (dc < 0 ? -1e-8 : 1e-8) : dc);
      }
      CVS_CUDA(cudaMemcpyAsync(rnt, sc.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, s));
      row_axpy(s, T, Rt, rnt, cnt, N1, T);
      c->sync();
    } else if (c->sch_on) {
      // t = U (w - lam)^-1 U^H r~   (S(theta0) = U diag(lam) U^H)
      cplx* Ty = c->sch_tmp.c();
      CVS_CUDA(cudaMemcpyAsync(rn1, wt.data(), cnt * sizeof(double), cudaMemcpyHostToDevice, s));
      gemm64(c, (int)N1, cnt, (int)N1, 1.0, conj_of(trans(view(c->sch_U.c(), N1, 1))),
             view(Rt, 1, N1), 0.0, view(Ty, cnt, 1));
      if (c->sch_d_on)
        eig_shift_d(s, Ty, N1, cnt, c->sch_lam.d(), c->sch_d.d(), c->sch_theta, rn1);
      else
        eig_shift(s, Ty, N1, cnt, c->sch_lam.d(), rn1);
      gemm64(c, (int)N1, cnt, (int)N1, 1.0, view(c->sch_U.c(), N1, 1), view(Ty, cnt, 1), 0.0,
             view(T, 1, N1));
    } else {
      CVS_CUDA(cudaMemcpyAsync(T, Rt, (size_t)cnt * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    }
    const int m0 = m;
    const int added = orth_append(T, cnt, true);
    if (added == 0) break;
    // each new direction is lifted at the Ritz value of the root whose
    // correction it was started from (the block Gram-Schmidt is triangular)
    for (int q = 0; q < added; ++q) th[m0 + q] = wt[std::min(std::max(src_h[q], 0), cnt - 1)];
    m += added;
    lift(m0, added);
  }
  CVS_CUDA(cudaMemcpyAsync(X1out, T2, (size_t)std::min(k, m) * N1 * sizeof(cplx),
                           cudaMemcpyDeviceToDevice, s));
  for (int q = 0; q < k; ++q) wout[q] = w[std::min(q, (int)w.size() - 1)];
  c->sync();
  return res;
}

// Oscillator strengths f_n = 2/3 w_n sum_x |X_n^H F^x|^2 (section
// "Properties in ISR formulation") of nvec full vectors X [nvec][N] into f.
void osc_strengths(cvsadc_ctx* c, const cplx* X, int nvec, const double* w, double* f) {
  c->fd_th.ensure((size_t)(nvec * 3 * TS_CHUNKS + nvec * 3 + 8) * sizeof(cplx));
  cplx* part = (cplx*)c->fd_th.p;
  cplx* Tn = part + (size_t)nvec * 3 * TS_CHUNKS;
  ts_dot(c->stream, X, nvec, c->F.c(), 3, c->N, part, Tn, 3, true);
  std::vector<cplx> T((size_t)nvec * 3);
  CVS_CUDA(cudaMemcpyAsync(T.data(), Tn, T.size() * sizeof(cplx), cudaMemcpyDeviceToHost,
                           c->stream));
  c->sync();
  for (int r0 = 0; r0 < nvec; ++r0) {
    double s2 = 0;
    for (int x = 0; x < 3; ++x) {
      const cplx t = T[(size_t)r0 * 3 + x];
      s2 += t.x * t.x + t.y * t.y;
    }
    f[r0] = 2.0 / 3.0 * w[r0] * s2;
  }
}

// Would the full-space Davidson (V, W [msub][N], X, AX [nkeep][N], T [k][N])
// plus a sigma group fit in 85 % of the free device memory?
bool full_space_fits(cvsadc_ctx* c, int k, int max_sub) {
  const int msub = std::max(max_sub, 2 * k + 2);
  const int nkeep = std::max(k, std::min(msub / 3, msub - 2 * k));
  const double vec = (double)c->N * sizeof(cplx);
  const double need = vec * (2.0 * msub + 2.0 * nkeep + k + 2.0 * 3 * k) +
                      4.0 * (double)c->N1 * c->nval * c->nvirt * sizeof(cplx);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    (void)cudaGetLastError();
    return true;
  }
  return need < 0.85 * (double)free_b;
}

// The doubles-folded solver behind cvsadc_davidson: roots, and (when asked)
// the full eigenvectors (x1, W(w) M21 x1) normalised, and oscillator
// strengths.
void folded_entry(cvsadc_ctx* c, const cvsadc_params* p, double* omega, void* X,
                  double* osc, cvsadc_info* info, double tol, int max_iter, int max_sub) {
  const int k = p->nroots;
  const int64_t N1 = c->N1, N = c->N;
  cudaStream_t s = c->stream;
  CVS_REQUIRE(k <= N1, CVSADC_EINVAL, "the folded solver finds at most N1 roots");
  const bool dev = (p->flags & CVSADC_FLAG_DEVICE_PTRS) != 0;
  const double t0 = now_ms();
  c->sch_ms = 0.0;
  c->sch_builds = 0;
  c->sch_couplings = 0;
  const bool use_schur = (p->flags & CVSADC_FLAG_DIAG_PRECOND) == 0;
  c->sch_d_on = false;
  if (!(use_schur && schur_setup(c))) c->sch_on = false;
  const int prec = p->precision;
  const bool refine = needs_refine(prec) && (p->flags & CVSADC_FLAG_NO_REFINE) == 0;
  const double tol_phase = refine ? std::max(tol, mixed_tolerance(prec)) : tol;
  DBuf X1, x0;
  X1.ensure((size_t)k * N1 * sizeof(cplx));
  std::vector<double> w(k), th0;
  const cplx* start = nullptr;
  int nstart = 0;
  if (!c->sch_on) {
    // no Schur eigenvectors: unit vectors at the smallest diagonal entries
    // of M11, lifted 1 Eh (or 3 %) below the lowest M22 entry
    nstart = (int)std::min<int64_t>(2 * k, N1);
    c->dv_misc.ensure((size_t)(64 * 320 + 2048) * sizeof(double));
    double* dwork = c->dv_misc.d();
    int64_t* idx = (int64_t*)(dwork + 1024);
    k_smallest(s, c->diag.d(), N1, nstart, idx, dwork);
    std::vector<int64_t> hidx(nstart);
    CVS_CUDA(cudaMemcpyAsync(hidx.data(), idx, nstart * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    x0.ensure((size_t)nstart * N1 * sizeof(cplx));
    CVS_CUDA(cudaMemsetAsync(x0.p, 0, (size_t)nstart * N1 * sizeof(cplx), s));
    c->sync();
    const cplx one = cmake(1, 0);
    for (int q = 0; q < nstart; ++q)
      CVS_CUDA(cudaMemcpyAsync(x0.c() + (int64_t)q * N1 + hidx[q], &one, sizeof(cplx),
                               cudaMemcpyHostToDevice, s));
    std::vector<double> eps(c->n);
    CVS_CUDA(cudaMemcpyAsync(eps.data(), c->eps.p, c->n * sizeof(double), cudaMemcpyDeviceToHost, s));
    c->sync();
    std::vector<double> ev(eps.begin() + c->o, eps.end());
    std::sort(ev.begin(), ev.end());
    const double pole = ev[0] + ev[1] - *std::max_element(eps.begin(), eps.begin() + c->ncore) -
                        *std::max_element(eps.begin() + c->ncore, eps.begin() + c->o);
    th0.assign(nstart, pole - std::max(1.0, 0.03 * std::fabs(pole)));
    start = x0.c();
  }
  FoldResult r = folded_davidson(c, prec, k, max_iter, max_sub, tol_phase, start,
                                 th0.empty() ? nullptr : th0.data(), nstart, X1.c(), w.data(),
                                 refine, true);
  const double t1 = now_ms();
  double t_ref = 0.0;
  if (refine) {
    // FP64-class continuation from the converged Ritz singles, lifted at
    // their roots
    DBuf xs;
    xs.ensure((size_t)k * N1 * sizeof(cplx));
    CVS_CUDA(cudaMemcpyAsync(xs.p, X1.p, (size_t)k * N1 * sizeof(cplx), cudaMemcpyDeviceToDevice, s));
    std::vector<double> wr = w;
    const int sweeps = p->refine_sweeps > 0 ? p->refine_sweeps : 20;
    FoldResult r2 = folded_davidson(c, refine_precision(prec), k, sweeps, max_sub, tol, xs.c(),
                                    wr.data(), k, X1.c(), w.data(), false, false);
    r.iters += r2.iters;
    r.folds += r2.folds;
    r.converged = r2.converged;
    r.maxres = r2.maxres;
    t_ref = now_ms() - t1;
  }
  // full vectors when asked for: z = (x1, W(w) M21 x1) / ||.||, in groups
  std::vector<double> f(k, 0.0);
  const bool want_x = X && (p->flags & CVSADC_FLAG_RETURN_X);
  const bool want_f = osc && c->has_dip;
  if (want_x || want_f) {
    const double per = 2.0 * (double)N * sizeof(cplx);
    const int g = (int)std::max(1.0, std::min((double)k, 24e9 / per));
    DBuf Z, Sg, th, nr;
    Z.ensure((size_t)g * N * sizeof(cplx));
    Sg.ensure((size_t)g * N * sizeof(cplx));
    th.ensure((size_t)(g + 8) * sizeof(double));
    nr.ensure((size_t)(g + 8) * sizeof(double));
    for (int q0 = 0; q0 < k; q0 += g) {
      const int gg = std::min(g, k - q0);
      CVS_CUDA(cudaMemsetAsync(Z.p, 0, (size_t)gg * N * sizeof(cplx), s));
      copyv(c, gg, (int)N1, 1.0, view(X1.c() + (int64_t)q0 * N1, N1, 1), view(Z.p, N, 1));
      sigma_impl(c, prec == CVSADC_FP64 || !tc_available() ? CVSADC_FP64 : CVSADC_FP64_SLICE7,
                 Z.c(), Sg.c(), gg, SIG_FWD);
      CVS_CUDA(cudaMemcpyAsync(th.p, w.data() + q0, gg * sizeof(double), cudaMemcpyHostToDevice, s));
      // doubles of Z = W(w) M21 x1 (singles kept)
      fold_doubles(s, Sg.c(), nullptr, th.d(), gg, N, N1, c->ncore, c->nval, c->nvirt,
                   c->eps.d(), false, Z.c());
      copyv(c, gg, (int)N1, 1.0, view(X1.c() + (int64_t)q0 * N1, N1, 1), view(Z.p, N, 1));
      row_norm2(s, Z.c(), gg, N, nr.d());
      std::vector<double> hn(gg);
      CVS_CUDA(cudaMemcpyAsync(hn.data(), nr.p, gg * sizeof(double), cudaMemcpyDeviceToHost, s));
      c->sync();
      for (double& x : hn) x = x > 0 ? 1.0 / std::sqrt(x) : 1.0;
      CVS_CUDA(cudaMemcpyAsync(nr.p, hn.data(), gg * sizeof(double), cudaMemcpyHostToDevice, s));
      scale_vectors(s, Z.c(), nr.d(), gg, N);
      c->dv_misc.ensure((size_t)(152 * gg * 4 + 64) * sizeof(cplx));
      phase_fix(s, Z.c(), gg, N, c->dv_misc.d());
      if (want_f) osc_strengths(c, Z.c(), gg, w.data() + q0, f.data() + q0);
      if (want_x)
        download(c, (cplx*)X + (int64_t)q0 * N, Z.p, (size_t)gg * N * sizeof(cplx), dev);
      c->sync();
    }
  }
  if (dev) {
    CVS_CUDA(cudaMemcpyAsync(omega, w.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
    if (want_f)
      CVS_CUDA(cudaMemcpyAsync(osc, f.data(), k * sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    std::memcpy(omega, w.data(), k * sizeof(double));
    if (want_f) std::memcpy(osc, f.data(), k * sizeof(double));
  }
  c->sync();
  if (info) {
    info->iterations = r.iters;
    info->sigma_vectors = 0;
    info->converged = r.converged;
    info->max_residual = r.maxres;
    info->t_davidson_ms = t1 - t0 - c->sch_ms;
    info->t_refine_ms = t_ref;
    info->t_sigma_ms = 0.0;
    info->emp2 = c->emp2;
    info->nvirt_kept = c->nvirt;
    info->t_schur_ms = c->sch_ms;
    info->schur_theta = c->sch_on ? c->sch_theta : 0.0;
    info->coupling_vectors = c->sch_couplings;
    info->schur_builds = c->sch_builds;
  }
  if (r.converged < k) throw Error{CVSADC_ENOTCONV, "folded solver did not converge"};
}

void davidson_entry(cvsadc_ctx* c, const cvsadc_params* p, double* omega,
                    void* X, double* osc, cvsadc_info* info) {
  CVS_REQUIRE(c->prepared, CVSADC_ESTATE, "no prepared problem");
  CVS_REQUIRE(omega, CVSADC_EINVAL, "omega is required");
  const int k = p->nroots;
  CVS_REQUIRE(k >= 1 && k <= 64 && k <= c->N, CVSADC_EINVAL, "bad nroots");
  bool dev = (p->flags & CVSADC_FLAG_DEVICE_PTRS) != 0;
  double tol = p->conv_residual > 0 ? p->conv_residual : 1e-6;
  int max_iter = p->max_iter > 0 ? p->max_iter : 400;
  int max_sub = p->max_subspace > 0 ? p->max_subspace : std::max(8 * k, 48);
  max_sub = std::min(max_sub, 128);
  if ((p->flags & CVSADC_FLAG_FOLDED) || !full_space_fits(c, k, max_sub)) {
    folded_entry(c, p, omega, X, osc, info, tol, max_iter, max_sub);
    return;
  }
  double t0 = now_ms();
  DBuf Xd;
  Xd.ensure((size_t)k * c->N * sizeof(cplx));
  std::vector<double> w(k);
  double t_ref = 0;
  DavResult r = solve_roots(c, p->precision, k, tol, max_iter, max_sub,
                            p->refine_sweeps,
                            (p->flags & CVSADC_FLAG_NO_REFINE) != 0, Xd.c(),
                            w.data(), &t_ref,
                            (p->flags & CVSADC_FLAG_DIAG_PRECOND) == 0);
  double t1 = now_ms() - t_ref;
  phase_fix(c->stream, Xd.c(), k, c->N, c->dv_misc.d());
  if (dev)
    CVS_CUDA(cudaMemcpyAsync(omega, w.data(), k * sizeof(double),
                             cudaMemcpyHostToDevice, c->stream));
  else
    std::memcpy(omega, w.data(), k * sizeof(double));
  if (X && (p->flags & CVSADC_FLAG_RETURN_X))
    download(c, X, Xd.p, (size_t)k * c->N * sizeof(cplx), dev);
  if (osc && c->has_dip) {
    // T_n^x = X_n^H F^x, f_n = 2/3 w_n sum_x |T|^2
    cplx* part = c->dv_misc.c();
    cplx* Tn = part + (size_t)k * 3 * TS_CHUNKS;
    ts_dot(c->stream, Xd.c(), k, c->F.c(), 3, c->N, part, Tn, 3, true);
    std::vector<cplx> T((size_t)k * 3);
    CVS_CUDA(cudaMemcpyAsync(T.data(), Tn, T.size() * sizeof(cplx),
                             cudaMemcpyDeviceToHost, c->stream));
    c->sync();
    std::vector<double> f(k);
    for (int r0 = 0; r0 < k; ++r0) {
      double s2 = 0;
      for (int x = 0; x < 3; ++x) {
        cplx t = T[(size_t)r0 * 3 + x];
        s2 += t.x * t.x + t.y * t.y;
      }
      f[r0] = 2.0 / 3.0 * w[r0] * s2;
    }
    if (dev)
      CVS_CUDA(cudaMemcpyAsync(osc, f.data(), k * sizeof(double),
                               cudaMemcpyHostToDevice, c->stream));
    else
      std::memcpy(osc, f.data(), k * sizeof(double));
  }
  c->sync();
  if (info) {
    info->iterations = r.iters;
    info->sigma_vectors = r.sigmas;
    info->converged = r.converged;
    info->max_residual = r.maxres;
    info->t_davidson_ms = t1 - t0;
    info->t_refine_ms = t_ref;
    info->t_sigma_ms = r.t_sigma_ms;
    info->emp2 = c->emp2;
    info->nvirt_kept = c->nvirt;
    info->t_schur_ms = c->sch_ms;
    info->schur_theta = c->sch_on ? c->sch_theta : 0.0;
    info->coupling_vectors = c->sch_couplings;
    info->schur_builds = c->sch_builds;
  }
  if (r.converged < k) throw Error{CVSADC_ENOTCONV, "Davidson did not converge"};
}

void check_device_error(cvsadc_ctx* c) {
  if (!c->err.p) return;
  int e = 0;
  CVS_CUDA(cudaMemcpyAsync(&e, c->err.p, sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
  CVS_CUDA(cudaStreamSynchronize(c->stream));
  if (e != 0) {
    CVS_CUDA(cudaMemsetAsync(c->err.p, 0, sizeof(int), c->stream));
    char b[128];
    snprintf(b, sizeof b, "a bounded device wait expired (code %d)", e);
    throw Error{CVSADC_ETIMEOUT, b};
  }
}


// ===================================================================== S10
// Gradient of E = sum of selected roots with respect to the spinor energies
// and the Cholesky vectors.  M is Hermitian and the eigenvectors are
// normalised, so dE/dtheta = sum_n x_n^H (dM/dtheta) x_n (Hellmann-Feynman)
// with the x_n held fixed: the reverse pass below differentiates
//   f = sum_n [x1^H M11 x1 + 2 Re x2^H M21 x1 + x2^H M22 x2]
// through every forward contraction (M11 pieces, t2 and its energy
// denominators, the B^P couplings).  Complex gradients follow
// g_z = df/dRe z + i df/dIm z; grad_B is projected on Hermitian matrices
// (the inputs' manifold).

// a view with the same geometry into the gradient of the tensor it reads
View mirror(const View& v, const cplx* base, cplx* gbase) {
  View g = v;
  g.p = gbase + (v.p - base);
  g.conj = 0;
  g.ext = -1;
  return g;
}

// backward of C = alpha * A B: gradients into the tensors A and B read
// (either may be skipped with a null mirror); gC is C's gradient view.
void gemm_backward(cvsadc_ctx* c, int M, int N, int K, double alpha, View A,
                   View gA, View B, View gB, View gC) {
  if (gA.p) {
    // d/dA: gC B^H (A read plain) or conj(gC) B^T (A read conjugated)
    View Bh = A.conj ? trans(B) : conj_of(trans(B));
    View g = A.conj ? conj_of(gC) : gC;
    gemm64(c, M, K, N, alpha, g, Bh, 1.0, gA);
  }
  if (gB.p) {
    View Ah = B.conj ? trans(A) : conj_of(trans(A));
    View g = B.conj ? conj_of(gC) : gC;
    gemm64(c, K, N, M, alpha, Ah, g, 1.0, gB);
  }
}

void grad_impl(cvsadc_ctx* c, const cplx* X, int k, double* gE, cplx* gB) {
  const int nc = c->ncore, nw = c->nval, v = c->nvirt, o = c->o, n = c->n,
            L = c->naux;
  const int64_t nn = (int64_t)n * n, N1 = c->N1, N = c->N, vv = (int64_t)v * v,
                ovv = (int64_t)o * vv, vo = (int64_t)v * o;
  const cplx* B = c->B.c();
  const cplx* t2 = c->t2.c();
  const cplx* g2 = c->g2.c();
  cudaStream_t s = c->stream;
  CVS_CUDA(cudaMemsetAsync(gE, 0, n * sizeof(double), s));
  CVS_CUDA(cudaMemsetAsync(gB, 0, (size_t)L * nn * sizeof(cplx), s));
  auto mB = [&](const View& vw) { return mirror(vw, B, gB); };

  // ---------------------------------------------------- M11 (singles)
  DBuf rho, gC1, gC2, gX, gY, gZ, gt2, gg2;
  rho.ensure(N1 * N1 * sizeof(cplx));
  // rho[s][t] = sum_q conj(x_s) x_t
  gemm64(c, (int)N1, (int)N1, k, 1.0, conj_of(view(X, 1, N)), view(X, N, 1), 0.0,
         view(rho.p, N1, 1));
  gC1.ensure(vv * nc * nc * sizeof(cplx));
  gC2.ensure(N1 * N1 * sizeof(cplx));
  gZ.ensure(N1 * N1 * sizeof(cplx));
  gX.ensure(vv * sizeof(cplx));
  gY.ensure((size_t)nc * nc * sizeof(cplx));
  m11_backward(s, rho.c(), nc, v, o, gC1.c(), gC2.c(), gX.c(), gY.c(), gZ.c(), gE);
  // C1[(a,b),(J,I)] = (ab|JI)
  {
    View A = rows2(view(B + (int64_t)o * n + o, 0, nn), n, 1, v);
    View Bv = cols2(view(B, nn, 0), n, 1, nc);
    gemm_backward(c, v * v, nc * nc, L, 1.0, A, mB(A), Bv, mB(Bv),
                  view(gC1.p, nc * nc, 1));
  }
  // C2[(I,a),(J,b)] = (aI|Jb)
  {
    View A = rows2(view(B + (int64_t)o * n, 0, nn), 1, n, v);
    View Bv = cols2(view(B + o, nn, 0), n, 1, v);
    gemm_backward(c, (int)N1, (int)N1, L, 1.0, A, mB(A), Bv, mB(Bv),
                  view(gC2.p, N1, 1));
  }
  // X, Y, Z through t2 and <ab||ij>
  gt2.ensure((size_t)o * ovv * sizeof(cplx));
  gg2.ensure((size_t)o * ovv * sizeof(cplx));
  CVS_CUDA(cudaMemsetAsync(gt2.p, 0, (size_t)o * ovv * sizeof(cplx), s));
  CVS_CUDA(cudaMemsetAsync(gg2.p, 0, (size_t)o * ovv * sizeof(cplx), s));
  auto mT = [&](const View& vw) { return mirror(vw, t2, gt2.c()); };
  auto mG = [&](const View& vw) { return mirror(vw, g2, gg2.c()); };
  {
    View A = cols2(view(t2, v, 0), vv, 1, v);
    View Bv = conj_of(rows2(view(g2, 0, v), vv, 1, v));
    gemm_backward(c, v, v, o * o * v, 1.0, A, mT(A), Bv, mG(Bv), view(gX.p, v, 1));
  }
  {
    View A = view(t2, ovv, 1);
    View Bv = conj_of(view(g2, 1, ovv));
    gemm_backward(c, nc, nc, (int)ovv, 1.0, A, mT(A), Bv, mG(Bv), view(gY.p, nc, 1));
  }
  {
    View A = cols2(rows2(view(t2, 0, 0), ovv, v, v), vv, 1, v);
    View Bv = conj_of(cols2(rows2(view(g2, 0, 0), vv, 1, v), ovv, v, v));
    gemm_backward(c, (int)N1, (int)N1, o * v, 1.0, A, mT(A), Bv, mG(Bv),
                  view(gZ.p, N1, 1));
  }
  rho.release();
  gC1.release();
  gC2.release();
  gZ.release();
  // t2 = g/D, g = (ai|bj) - (aj|bi): gR in gg2
  t2_backward(s, gt2.c(), gg2.c(), g2, o, v, c->eps.d(), gE);
  gt2.release();
  {
    int64_t per_a = (int64_t)o * vo * sizeof(cplx);
    int na = (int)std::max<int64_t>(1, std::min<int64_t>(v, (2LL << 30) / per_a));
    DBuf gQ;
    gQ.ensure((size_t)na * per_a);
    for (int a0 = 0; a0 < v; a0 += na) {
      const int nb = std::min(na, v - a0);
      q_backward_band(s, gg2.c(), a0, nb, o, v, gQ.c());
      View A = rows2(view(B + (int64_t)(o + a0) * n, 0, nn), n, 1, o);
      View Bv = cols2(view(B + (int64_t)o * n, nn, 0), n, 1, o);
      gemm_backward(c, nb * o, (int)vo, L, 1.0, A, mB(A), Bv, mB(Bv),
                    view(gQ.p, vo, 1));
    }
  }
  gg2.release();

  // --------------------------------------------- couplings, by root groups
  const int64_t wv = (int64_t)nw * v, vL = (int64_t)v * L, wvL = wv * L;
  const int64_t N1L = N1 * L, N1wv = N1 * wv;
  const double per_vec = (3.0 * N1wv + 2.0 * N1L + 2.0 * wvL) * sizeof(cplx);
  const int gmax = (int)std::max(1.0, std::min((double)k, 32e9 / per_vec));
  DBuf Yt, Yb, Vv, gY2, gV2;
  for (int q0 = 0; q0 < k; q0 += gmax) {
    const int g = std::min(gmax, k - q0);
    const cplx* x = X + (int64_t)q0 * N;
    Yt.ensure((size_t)g * N1wv * sizeof(cplx));
    Yb.ensure((size_t)g * N1L * sizeof(cplx));
    Vv.ensure((size_t)g * wvL * sizeof(cplx));
    gY2.ensure((size_t)g * N1L * sizeof(cplx));
    gV2.ensure((size_t)g * wvL * sizeof(cplx));
    for (int q = 0; q < g; ++q)
      unpack_doubles(s, x + q * N + N1, nc, nw, v, Yt.c() + q * N1wv);
    // forward intermediates Y and Vv (as in sigma)
    View A1 = rows2(view(x, 0, 1), N, v, nc);
    View B1 = cols2(view(B + (int64_t)o * n + o, 1, 0), n, nn, L);
    gemm64(c, g * nc, (int)vL, v, 1.0, A1, B1, 0.0, view(Yb.p, vL, 1));
    View A2 = rows2(view(x, 0, v), N, 1, v);
    View B2 = cols2(view(B, n, 0), 1, nn, L);
    View CY2 = cols2(rows2(view(Yb.p, 0, 0), N1L, L, v), vL, 1, L);
    gemm64(c, g * v, nc * L, nc, -1.0, A2, B2, 1.0, CY2);
    View B3 = cols2(view(B + nc, n, 0), 1, nn, L);
    View CV = cols2(rows2(view(Vv.p, 0, 0), wvL, L, v), vL, 1, L);
    gemm64(c, g * v, nw * L, nc, 1.0, A2, B3, 0.0, CV);
    // f_coup = Re(-2 sum conj(y) G) -> gG = -2 y (the unpacked doubles)
    View gG1 = view(Yt.p, wv, 1);
    View gG2 = cols2(view(Yt.p, wv, 0), N1wv, 1, (int)wv);
    // G1 = Y B4: gY = gG B4^H, gB(B4) += Y^H gG
    View B4 = cols2(view(B + (int64_t)o * n + nc, nn, 0), 1, n, v);
    gemm64(c, (int)(g * N1), L, (int)wv, -2.0, gG1, conj_of(trans(B4)), 0.0,
           view(gY2.p, L, 1));
    gemm64(c, L, (int)wv, (int)(g * N1), -2.0, conj_of(trans(view(Yb.p, L, 1))),
           gG1, 1.0, mB(B4));
    // G2 = -A5 Vv: gB(A5) += -gG Vv^H, gVv = -A5^H gG
    View A5 = rows2(view(B + (int64_t)o * n, 0, nn), 1, n, v);
    gemm64(c, (int)N1, L, (int)(g * wv), 2.0, gG2, conj_of(trans(view(Vv.p, 1, L))),
           1.0, mB(A5));
    gemm64(c, L, (int)(g * wv), (int)N1, 2.0, conj_of(trans(A5)), gG2, 0.0,
           view(gV2.p, 1, L));
    // Vv = A2 B3: gB(B3) += A2^H gVv
    View gCV = cols2(rows2(view(gV2.p, 0, 0), wvL, L, v), vL, 1, L);
    gemm64(c, nc, nw * L, g * v, 1.0, conj_of(trans(A2)), gCV, 1.0, mB(B3));
    // Y = A1 B1 - A2 B2: gB(B1) += A1^H gY, gB(B2) -= A2^H gY
    gemm64(c, v, (int)vL, g * nc, 1.0, conj_of(trans(A1)), view(gY2.p, vL, 1), 1.0,
           mB(B1));
    View gCY2 = cols2(rows2(view(gY2.p, 0, 0), N1L, L, v), vL, 1, L);
    gemm64(c, nc, nc * L, g * v, -1.0, conj_of(trans(A2)), gCY2, 1.0, mB(B2));
  }
  // M22
  m22_backward(s, X, k, N, N1, nc, nw, v, gE);
  herm_project(s, gB, n, L);
  c->sync();
}

void grad_entry(cvsadc_ctx* c, const cvsadc_params* p, const double* eps,
                const void* B, const int32_t* root_mask, double* omega,
                double* grad_eps, void* grad_B) {
  CVS_REQUIRE(p && eps && B && omega && grad_eps && grad_B, CVSADC_EINVAL,
              "NULL argument");
  CVS_REQUIRE(p->fns_threshold <= 0, CVSADC_EINVAL,
              "gradients are defined for the untruncated virtual space (tau <= 0)");
  CVS_REQUIRE(p->precision >= CVSADC_FP64 && p->precision <= CVSADC_FP64_SLICE7,
              CVSADC_EINVAL, "bad precision");
  // the problem (t2, M11) is always built in FP64, so that the eigenpairs
  // and the adjoint below belong to the same matrix; params->precision only
  // selects the sigma of the Davidson phase, which for the tensor-core
  // precisions is followed by the FP64-class refinement
  cvsadc_params q = *p;
  q.precision = CVSADC_FP64;
  q.flags = (p->flags & CVSADC_FLAG_DEVICE_PTRS);
  prepare_impl(c, &q, eps, B, nullptr, nullptr, true);
  const int k = q.nroots;
  CVS_REQUIRE(k >= 1 && k <= 64 && k <= c->N, CVSADC_EINVAL, "bad nroots");
  const double tol = p->conv_residual > 0 ? p->conv_residual : 1e-8;
  const int max_iter = p->max_iter > 0 ? p->max_iter : 400;
  const int max_sub = std::min(p->max_subspace > 0 ? p->max_subspace : std::max(8 * k, 48), 128);
  DBuf Xd;
  Xd.ensure((size_t)k * c->N * sizeof(cplx));
  std::vector<double> w(k);
  // the gradient needs converged eigenvectors, so the refinement may run
  // as long as the first phase
  DavResult r = solve_roots(c, p->precision, k, tol, max_iter, max_sub,
                            p->refine_sweeps > 0 ? p->refine_sweeps : max_iter,
                            false, Xd.c(), w.data(), nullptr,
                            (p->flags & CVSADC_FLAG_DIAG_PRECOND) == 0);
  CVS_REQUIRE(r.converged == k, CVSADC_ENOTCONV, "Davidson did not converge");
  // selected roots, contiguous
  std::vector<int> sel;
  for (int i = 0; i < k; ++i)
    if (!root_mask || root_mask[i]) sel.push_back(i);
  CVS_REQUIRE(!sel.empty(), CVSADC_EINVAL, "root_mask selects no root");
  for (size_t i = 0; i < sel.size(); ++i)
    if (sel[i] != (int)i)
      CVS_CUDA(cudaMemcpyAsync(Xd.c() + i * c->N, Xd.c() + sel[i] * c->N,
                               c->N * sizeof(cplx), cudaMemcpyDeviceToDevice,
                               c->stream));
  DBuf gE, gBd;
  gE.ensure(c->n * sizeof(double));
  gBd.ensure((size_t)c->naux * c->n * c->n * sizeof(cplx));
  grad_impl(c, Xd.c(), (int)sel.size(), gE.d(), gBd.c());
  const bool dev = (p->flags & CVSADC_FLAG_DEVICE_PTRS) != 0;
  download(c, grad_eps, gE.p, c->n * sizeof(double), dev);
  download(c, grad_B, gBd.p, (size_t)c->naux * c->n * c->n * sizeof(cplx), dev);
  if (dev)
    CVS_CUDA(cudaMemcpyAsync(omega, w.data(), k * sizeof(double),
                             cudaMemcpyHostToDevice, c->stream));
  else
    std::memcpy(omega, w.data(), k * sizeof(double));
  c->sync();
}

template <typename F>
int guarded(cvsadc_ctx* c, F&& f) {
  try {
    if (c) CVS_CUDA(cudaSetDevice(c->device));
    f();
    if (c) check_device_error(c);
    if (c) c->last_error.clear();
    return CVSADC_OK;
  } catch (const Error& e) {
    if (c) c->last_error = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    if (c) c->last_error = "host allocation failed";
    return CVSADC_ENOMEM;
  } catch (...) {
    if (c) c->last_error = "unexpected internal error";
    return CVSADC_ECUDA;
  }
}

}  // namespace

// =================================================================== C ABI
// ------------------------------------------------------ batched solves
namespace {

// Device bytes one solve of `p` holds at its peak: inputs, the t2 band
// buffers, the moment accumulators, M11 and its build scratch, the
// eigensolver's vectors (the full-space Davidson subspace and block, or
// with CVSADC_FLAG_FOLDED the folded solver's singles-space vectors and
// the lift of the eigenvectors), the sigma intermediates of its largest
// group, the preconditioner, the tensor-core packing workspace of the
// largest contraction, the kept operand packs and the split-K scratch.
// Host arithmetic only; used to admit instances of a batch to the GPU and
// offered to callers that size their own memory.
double estimate_bytes(const cvsadc_params* p) {
  const double z = sizeof(cplx);
  const double nc = p->ncore, nw = p->nval, v = p->nvirt, L = p->naux;
  const double o = nc + nw, n = o + v;
  const double N1 = nc * v, wv = nw * v, N = N1 + nc * nw * v * (v - 1) / 2;
  const int k = std::max(1, p->nroots);
  const int msub = std::min(p->max_subspace > 0 ? p->max_subspace
                                                : std::max(8 * k, 48), 128);
  const int ms = std::max(msub, 2 * k + 2);
  const int nkeep = std::max(k, std::min(ms / 3, ms - 2 * k));
  const bool schur_on = N1 <= 4096 && !(p->flags & CVSADC_FLAG_DIAG_PRECOND);
  const bool folded = (p->flags & CVSADC_FLAG_FOLDED) != 0;
  double g = std::min(64, std::max(k, std::min(2 * k, ms / 2)));
  if (schur_on) g = std::max(g, std::min<double>(SCHUR_P, N1));
  // sigma_impl runs at most as many vectors at once as fit its budget
  {
    const double per_vec = (2.0 * N1 * wv + 2.0 * N1 * L + 2.0 * wv * L) * z;
    g = std::max(1.0, std::min(g, std::floor(SIGMA_BUDGET / per_vec)));
  }
  double b = 8 * n + z * L * n * n;
  b += 3 * z * n * n;                       // dipoles
  // t2 bands: the in-place (ai|bj) / <ab||ij> block and the t2 block
  const double band = std::min(16e9, 2 * z * o * o * v * v);
  b += band;
  b += 6 * z * nc * nw * v * v;             // moment accumulators (with dipoles)
  if (p->fns_threshold > 0) b += z * L * n * n + 2 * z * v * v;  // rotated B^P
  b += z * g * N1 * wv;                     // s_big1
  b += std::max({z * (v * v * nc * nc + 2 * N1 * N1 + v * v + nc * nc),
                 z * g * N1 * wv, 2 * z * nc * nw * v * v});  // s_big2
  b += z * N1 * N1 + 8 * N;                 // M11, diagonal
  b += 2 * z * g * N1 * L + 2 * z * g * wv * L;  // S, Y, R, V
  if (folded) {
    // the folded solver: singles-space V, B, R, D, M11 V and block scratch,
    // and the lift of the full eigenvectors (groups within 24 GB)
    const double fms = std::min(128, std::max(p->max_subspace, 3 * k + 2));
    b += z * N1 * (5.0 * fms + 9.0 * k);
    b += std::min(24e9, 2.0 * z * N * k);
  } else {
    b += z * N * (2.0 * ms + 2.0 * nkeep + k);  // Davidson V, W, X, AX, T
  }
  b += z * (double)ms * ms * 320 + 1e6;     // subspace matrices, partials
  if (N1 > SCHUR_FULL_MAX && !(p->flags & CVSADC_FLAG_DIAG_PRECOND))
    // the large-space preconditioner: partial eigenbasis, j-chunk buffers,
    // S(theta) and its cross-term blocks
    b += z * N1 * SCHUR_PL * 4.0 + 6.5e9 + 2.0 * z * N1 * N1 + z * v * v * nc * nc;
  b += 3 * z * N;                           // moments
  if (p->precision != CVSADC_FP64 || schur_on) {
    const int ns = p->precision == CVSADC_MIXED_SLICE4 ? 4
                   : p->precision == CVSADC_FP64_SLICE7 ? 7
                   : p->precision == CVSADC_FP64 ? 4 : 0;
    auto ws = [&](double M, double Nn, double K, int nsl) {
      if (M < 32 || K < 64 || M * Nn * K < 1e7) return 0.0;
      return (double)(nsl ? slice_workspace_bytes((int)M, (int)Nn, (int)K, nsl)
                          : tc_workspace_bytes((int)M, (int)Nn, (int)K, 3));
    };
    const double na = std::max(1.0, std::min(v, std::floor(band / (2 * z * o * v * o))));
    double w = 0;
    for (double s : {ws(na * o, v * o, L, ns), ws(N1, N1, L, ns), ws(N1, N1, o * v, ns),
                     ws(g * N1, L, wv, ns), ws(g * wv, L, N1, ns), ws(g * N1, wv, L, ns),
                     ws(N1, g * wv, L, ns)})
      w = std::max(w, s);
    // the preconditioner's contractions run as 4-slice products
    if (schur_on) {
      const double v3 = v * v * v;
      const double jc = std::max(1.0, std::min(nw, std::floor(6e9 / ((3.0 + nc) * v3 * z))));
      for (double s : {ws(v * v, jc * v, L, 4), ws(jc * v, v * v, L, 4),
                       ws(nc * v, v, jc * v * v, 4), ws(g * N1, L, wv, 4),
                       ws(g * wv, L, N1, 4), ws(g * N1, wv, L, 4), ws(N1, g * wv, L, 4)})
        w = std::max(w, s);
    }
    // a mixed precision is refined with the 7-slice product
    if (needs_refine(p->precision))
      for (double s : {ws(k * N1, L, wv, 7), ws(k * wv, L, N1, 7), ws(k * N1, wv, L, 7),
                       ws(N1, k * wv, L, 7)})
        w = std::max(w, s);
    b += w;
  }
  b += (double)(8 << 20) * z + 1024;        // split-K scratch, error flag
  // cached slice packs of B^P views (at most min(35 % of free, 64 GB)): the
  // B operands of the sigma's S and G products, the A operands of its
  // sigma1^T and Y^T products, and the preconditioner's (aj|bc) product
  {
    const double pairs = (p->precision == CVSADC_FP64_SLICE7 || needs_refine(p->precision))
                             ? 10.0 + 28.0 : 10.0;
    double cb = schur_on ? 8.0 * 10.0 * v * v * L : 0.0;
    if (p->precision != CVSADC_FP64) cb += 2.0 * 8.0 * pairs * v * v * L;
    if (p->precision != CVSADC_FP64) cb += 32.0 * v * v * L;
    b += std::min(64e9, cb);
  }
  // Schur-complement preconditioner (when the singles space allows it)
  if (N1 <= 4096 && !(p->flags & CVSADC_FLAG_DIAG_PRECOND)) {
    const double v3 = v * v * v;
    const double per_j = (2.0 + nc) * v3 * z;
    const double jc = std::max(1.0, std::min(nw, std::floor(6e9 / per_j)));
    b += z * (nc * v * nc * nw * 2 + nc * nc * v * nw);  // <Kb||Ij>, temps
    b += std::min(nw * v3 * z, 48e9);          // cached <ab||cj>
    b += 4 * z * N1 * N1 + 8 * N1 + z * nc * v * v + z * v * v * nc * nc;
    b += (2.0 + nc) * jc * v3 * z;             // chunk workspace
    b += z * std::max(v * v * nc * nc, N1 * 64.0) + 8 * (800 + 2 * N1) + 2 * z * N;
  }
  return 1.1 * b + (64 << 20);
}

struct BatchJob {
  int idx;
  double bytes;
  bool solo;  // admitted only onto an otherwise idle GPU
};

// Runs the instances on `lanes` worker contexts (each its own stream and
// host thread).  Jobs are taken largest first; a job is admitted when its
// estimated footprint fits next to the running ones within `budget`, or
// when nothing else runs.  A job that still runs out of memory beside
// others is put back to run alone.
void solve_batched_impl(cvsadc_ctx* c, int ninst, const cvsadc_params* params,
                        const double* const* eps, const void* const* B,
                        const void* const* dip, double* const* omega,
                        void* const* X, double* const* osc, cvsadc_info* info,
                        int32_t* status, int lanes) {
  std::vector<BatchJob> queue;
  for (int i = 0; i < ninst; ++i) {
    validate(&params[i]);
    CVS_REQUIRE(eps[i] && B[i] && omega[i], CVSADC_EINVAL,
                "batched: eps, B and omega are required for every instance");
    queue.push_back({i, estimate_bytes(&params[i]), false});
  }
  std::stable_sort(queue.begin(), queue.end(),
                   [](const BatchJob& a, const BatchJob& b) { return a.bytes > b.bytes; });
  size_t free_b = 0, total_b = 0;
  CVS_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const double budget = 0.9 * (double)free_b;
  lanes = std::max(1, std::min(lanes, ninst));
  while ((int)c->lanes.size() < lanes) {
    cvsadc_ctx* l = nullptr;
    int rc = cvsadc_create(&l, c->device, nullptr);
    CVS_REQUIRE(rc == CVSADC_OK, rc, "batched: could not create a worker context");
    c->lanes.push_back(l);
  }
  std::vector<int> rcs(ninst, CVSADC_OK);
  std::vector<std::string> msgs(ninst);
  std::mutex mu;
  std::condition_variable cv;
  double in_use = 0;
  int running = 0;
  auto worker = [&](cvsadc_ctx* lane) {
    cudaSetDevice(c->device);
    for (;;) {
      BatchJob job{-1, 0, false};
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (queue.empty()) return;
          auto it = queue.end();
          if (running == 0) {
            it = queue.begin();
          } else {
            for (auto q = queue.begin(); q != queue.end(); ++q)
              if (!q->solo && in_use + q->bytes <= budget) {
                it = q;
                break;
              }
          }
          if (it != queue.end()) {
            job = *it;
            queue.erase(it);
            break;
          }
          cv.wait(lk);
        }
        in_use += job.bytes;
        ++running;
      }
      const int i = job.idx;
      int rc = cvsadc_solve(lane, &params[i], eps[i], B[i], dip ? dip[i] : nullptr,
                            omega[i], X ? X[i] : nullptr, osc ? osc[i] : nullptr,
                            info ? &info[i] : nullptr);
      std::string msg = rc == CVSADC_OK ? "" : lane->last_error;
      lane->trim();
      {
        std::lock_guard<std::mutex> lk(mu);
        in_use -= job.bytes;
        --running;
        if (rc == CVSADC_ENOMEM && !job.solo) {
          job.solo = true;
          queue.insert(queue.begin(), job);
        } else {
          rcs[i] = rc;
          msgs[i] = msg;
        }
      }
      cv.notify_all();
    }
  };
  std::vector<std::thread> th;
  for (int l = 0; l < lanes; ++l) th.emplace_back(worker, c->lanes[l]);
  for (auto& t : th) t.join();
  int worst = CVSADC_OK;
  for (int i = 0; i < ninst; ++i) {
    if (status) status[i] = rcs[i];
    if (rcs[i] < 0 && worst >= 0) {
      worst = rcs[i];
      c->last_error = "instance " + std::to_string(i) + ": " + msgs[i];
    } else if (rcs[i] == CVSADC_ENOTCONV && worst == CVSADC_OK) {
      worst = CVSADC_ENOTCONV;
    }
  }
  if (worst < 0) throw Error{worst, c->last_error};
  if (worst == CVSADC_ENOTCONV)
    throw Error{CVSADC_ENOTCONV, "some instances did not converge"};
}

}  // namespace

extern "C" {

int cvsadc_create(cvsadc_ctx** ctx, int device, void* cuda_stream) {
  if (!ctx) return CVSADC_EINVAL;
  *ctx = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    (void)cudaGetLastError();
    return CVSADC_ECUDA;
  }
  if (device < 0 || device >= ndev) return CVSADC_EINVAL;
  cvsadc_ctx* c = new (std::nothrow) cvsadc_ctx();
  if (!c) return CVSADC_ENOMEM;
  c->device = device;
  int rc = guarded(c, [&] {
    init_kernel_attributes();
    init_gemm_attributes();
    c->s_kpart.ensure((size_t)8 << 20 << 4);  // 8 Mi complex = 128 MB
    c->err.ensure(256);
    CVS_CUDA(cudaMemset(c->err.p, 0, 256));
    if (cuda_stream) {
      c->stream = (cudaStream_t)cuda_stream;
    } else {
      CVS_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
  });
  if (rc != CVSADC_OK) {
    delete c;
    return rc;
  }
  *ctx = c;
  return CVSADC_OK;
}

void cvsadc_destroy(cvsadc_ctx* c) {
  if (!c) return;
  for (cvsadc_ctx* l : c->lanes) cvsadc_destroy(l);
  c->lanes.clear();
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* cvsadc_strerror(int status) {
  switch (status) {
    case CVSADC_OK: return "ok";
    case CVSADC_EINVAL: return "invalid argument";
    case CVSADC_ENONHERM: return "input matrix is not Hermitian";
    case CVSADC_ENOMEM: return "out of memory";
    case CVSADC_ECUDA: return "CUDA error";
    case CVSADC_ETIMEOUT: return "device wait timed out";
    case CVSADC_ESTATE: return "no prepared problem";
    case CVSADC_ENOTCONV: return "not converged";
    default: return "unknown status";
  }
}

const char* cvsadc_last_error(cvsadc_ctx* c) {
  return c ? c->last_error.c_str() : "";
}

int cvsadc_prepare(cvsadc_ctx* c, const cvsadc_params* p, const double* eps,
                   const void* B, const void* dip, cvsadc_info* info) {
  if (!c) return CVSADC_EINVAL;
  return guarded(c, [&] { prepare_impl(c, p, eps, B, dip, info); });
}

int cvsadc_prepared_sizes(cvsadc_ctx* c, int32_t* nvirt, int64_t* N1,
                          int64_t* N2) {
  if (!c) return CVSADC_EINVAL;
  if (!c->prepared) return CVSADC_ESTATE;
  if (nvirt) *nvirt = c->nvirt;
  if (N1) *N1 = c->N1;
  if (N2) *N2 = c->N2;
  return CVSADC_OK;
}

int cvsadc_get_t2(cvsadc_ctx* c, int32_t flags, void* t2, double* emp2) {
  if (!c) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(c->prepared, CVSADC_ESTATE, "no prepared problem");
    if (emp2) *emp2 = c->emp2;
    if (t2) {
      // built on request: the prepared problem does not keep t2 whole
      if (!c->t2.p) {
        double e = 0.0;
        build_t2(c, c->prep_prec, c->B.c(), c->eps.d(), c->o, c->nvirt, c->naux,
                 c->t2, c->g2, &e);
      }
      download(c, t2, c->t2.p, (size_t)c->o * c->o * c->nvirt * c->nvirt * sizeof(cplx),
               flags & CVSADC_FLAG_DEVICE_PTRS);
    }
    c->sync();
  });
}

int cvsadc_get_m11(cvsadc_ctx* c, int32_t flags, void* m11) {
  if (!c || !m11) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(c->prepared, CVSADC_ESTATE, "no prepared problem");
    download(c, m11, c->M11.p, (size_t)c->N1 * c->N1 * sizeof(cplx),
             flags & CVSADC_FLAG_DEVICE_PTRS);
    c->sync();
  });
}

int cvsadc_get_fns(cvsadc_ctx* c, int32_t flags, double* occ, void* U) {
  if (!c) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(c->prepared && c->has_fns, CVSADC_ESTATE, "no FNS in the prepared problem");
    bool dev = flags & CVSADC_FLAG_DEVICE_PTRS;
    if (occ) download(c, occ, c->fns_occ.p, c->nvirt_in * sizeof(double), dev);
    if (U)
      download(c, U, c->fns_U.p, (size_t)c->nvirt_in * c->nvirt * sizeof(cplx), dev);
    c->sync();
  });
}

int cvsadc_get_moments(cvsadc_ctx* c, int32_t flags, void* F) {
  if (!c || !F) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(c->prepared && c->has_dip, CVSADC_ESTATE, "no dipoles in the prepared problem");
    download(c, F, c->F.p, (size_t)3 * c->N * sizeof(cplx),
             flags & CVSADC_FLAG_DEVICE_PTRS);
    c->sync();
  });
}

int cvsadc_sigma(cvsadc_ctx* c, int32_t precision, int32_t flags,
                 const void* x, void* sigma, int32_t nvec) {
  if (!c || !x || !sigma || nvec < 0) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(c->prepared, CVSADC_ESTATE, "no prepared problem");
    CVS_REQUIRE(valid_precision(precision), CVSADC_EINVAL, "unknown precision");
    if (nvec == 0) return;
    bool dev = flags & CVSADC_FLAG_DEVICE_PTRS;
    size_t bytes = (size_t)nvec * c->N * sizeof(cplx);
    if (dev) {
      RegGuard gx(x, bytes), gs(sigma, bytes);
      sigma_impl(c, precision, (const cplx*)x, (cplx*)sigma, nvec);
    } else {
      DBuf xd, sd;
      xd.ensure(bytes);
      sd.ensure(bytes);
      CVS_CUDA(cudaMemcpyAsync(xd.p, x, bytes, cudaMemcpyHostToDevice, c->stream));
      sigma_impl(c, precision, xd.c(), sd.c(), nvec);
      CVS_CUDA(cudaMemcpyAsync(sigma, sd.p, bytes, cudaMemcpyDeviceToHost, c->stream));
      c->sync();
    }
    c->sync();
  });
}

void cvsadc_kernel_timing(int32_t enable) { kstats_set(enable != 0); }

int cvsadc_kernel_stats(int32_t kernel, int64_t* launches, double* ms,
                        double* flops) {
  if (kernel < 0 || kernel >= K_NKERNELS || !launches || !ms || !flops)
    return CVSADC_EINVAL;
  return guarded(nullptr, [&] { kstats_collect(kernel, launches, ms, flops); });
}

void cvsadc_kernel_stats_reset(void) {
  try {
    kstats_reset();
  } catch (...) {
  }
}

int64_t cvsadc_launch_count(void) {
  return (int64_t)__atomic_load_n(&g_launch_count, __ATOMIC_RELAXED);
}

int cvsadc_wait_probe(cvsadc_ctx* c, int64_t limit_ns) {
  if (!c) return CVSADC_EINVAL;
  return guarded(c, [&] { wait_probe(c->stream, limit_ns, c->err.as<int>()); });
}

int cvsadc_zgemm(cvsadc_ctx* c, int32_t precision, int32_t flags, int32_t M,
                 int32_t N, int32_t K, const void* A, int64_t lda,
                 const void* B, int64_t ldb, void* C, int64_t ldc) {
  if (!c || !A || !B || !C || M < 0 || N < 0 || K < 0) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(valid_precision(precision), CVSADC_EINVAL, "unknown precision");
    CVS_REQUIRE(lda >= std::max(K, 1) && ldb >= std::max(N, 1) &&
                    ldc >= std::max(N, 1),
                CVSADC_EINVAL, "leading dimension too small");
    if (M == 0 || N == 0) return;
    bool dev = flags & CVSADC_FLAG_DEVICE_PTRS;
    size_t ab = (size_t)M * lda * sizeof(cplx), bb = (size_t)K * ldb * sizeof(cplx),
           cb = (size_t)M * ldc * sizeof(cplx);
    DBuf da, db, dc;
    const void *pa = A, *pb = B;
    void* pc = C;
    std::unique_ptr<RegGuard> ga, gb, gc;
    if (dev) {
      ga.reset(new RegGuard(A, ab));
      gb.reset(new RegGuard(B, bb));
      gc.reset(new RegGuard(C, cb));
    } else {
      upload(c, da, A, ab, false);
      upload(c, db, B, bb, false);
      dc.ensure(cb);
      pa = da.p;
      pb = db.p;
      pc = dc.p;
    }
    if (K == 0) {
      CVS_CUDA(cudaMemsetAsync(pc, 0, cb, c->stream));
    } else {
      gemm(c, precision, M, N, K, 1.0, view(pa, lda, 1), view(pb, ldb, 1), 0.0,
           view(pc, ldc, 1));
    }
    if (!dev) download(c, C, dc.p, cb, false);
    c->sync();
  });
}

int cvsadc_spectrum(cvsadc_ctx* c, int32_t flags, int32_t nroots, const double* omega,
                    const double* osc, double e0_ev, double de_ev, int32_t npts,
                    double fwhm_ev, double shift_ev, double* out) {
  if (!c || nroots < 0 || npts < 0 || (nroots > 0 && (!omega || !osc)) ||
      (npts > 0 && !out) || !(fwhm_ev > 0.0))
    return CVSADC_EINVAL;
  return guarded(c, [&] {
    if (npts == 0) return;
    const bool dev = (flags & CVSADC_FLAG_DEVICE_PTRS) != 0;
    DBuf w, f, o;
    w.ensure((size_t)(nroots + 1) * sizeof(double));
    f.ensure((size_t)(nroots + 1) * sizeof(double));
    o.ensure((size_t)npts * sizeof(double));
    if (nroots > 0) {
      upload(c, w, omega, nroots * sizeof(double), dev);
      upload(c, f, osc, nroots * sizeof(double), dev);
    }
    lorentz_spectrum(c->stream, w.d(), f.d(), nroots, e0_ev, de_ev, npts, fwhm_ev, shift_ev,
                     27.211386245988, o.d());
    download(c, out, o.p, (size_t)npts * sizeof(double), dev);
    c->sync();
  });
}

int cvsadc_block_dot(cvsadc_ctx* c, int32_t precision, const void* A,
                     int32_t ma, const void* B, int32_t mb, int64_t N, void* out) {
  if (!c || !A || !B || !out || ma < 1 || mb < 1 || N < 1) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(valid_precision(precision), CVSADC_EINVAL, "unknown precision");
    const size_t ab = (size_t)ma * N * sizeof(cplx), bb = (size_t)mb * N * sizeof(cplx);
    RegGuard ga(A, ab), gb(B, bb);
    const bool f64 = precision == CVSADC_FP64 || precision == CVSADC_FP64_SLICE7;
    DBuf part, o;
    part.ensure((size_t)std::min(ma, 96) * std::min(mb, 192) * TS_CHUNKS * sizeof(cplx) +
                (size_t)ma * mb * sizeof(cplx));
    o.ensure((size_t)ma * mb * sizeof(cplx));
    ts_dot(c->stream, (const cplx*)A, ma, (const cplx*)B, mb, N, part.c(), o.c(), mb, f64);
    CVS_CUDA(cudaMemcpyAsync(out, o.p, (size_t)ma * mb * sizeof(cplx),
                             cudaMemcpyDeviceToHost, c->stream));
    c->sync();
  });
}

int cvsadc_davidson(cvsadc_ctx* c, const cvsadc_params* p, double* omega,
                    void* X, double* osc, cvsadc_info* info) {
  if (!c || !p) return CVSADC_EINVAL;
  return guarded(c, [&] { davidson_entry(c, p, omega, X, osc, info); });
}

int cvsadc_grad(cvsadc_ctx* c, const cvsadc_params* p, const double* eps,
                const void* B, const int32_t* root_mask, double* omega,
                double* grad_eps, void* grad_B) {
  if (!c || !p) return CVSADC_EINVAL;
  return guarded(c, [&] {
    grad_entry(c, p, eps, B, root_mask, omega, grad_eps, grad_B);
  });
}

int cvsadc_solve(cvsadc_ctx* c, const cvsadc_params* p, const double* eps,
                 const void* B, const void* dip, double* omega, void* X,
                 double* osc, cvsadc_info* info) {
  if (!c || !p) return CVSADC_EINVAL;
  double t0 = now_ms();
  int rc = guarded(c, [&] { prepare_impl(c, p, eps, B, dip, info); });
  if (rc != CVSADC_OK) return rc;
  rc = guarded(c, [&] { davidson_entry(c, p, omega, X, osc, info); });
  if (info) info->t_total_ms = now_ms() - t0;
  return rc;
}

int cvsadc_estimate_bytes(const cvsadc_params* p, int64_t* bytes) {
  if (!p || !bytes) return CVSADC_EINVAL;
  try {
    validate(p);
    *bytes = (int64_t)estimate_bytes(p);
    return CVSADC_OK;
  } catch (const Error& e) {
    return e.code;
  } catch (...) {
    return CVSADC_EINVAL;
  }
}

int cvsadc_device_bytes(cvsadc_ctx* c, int64_t* bytes) {
  if (!c || !bytes) return CVSADC_EINVAL;
  *bytes = (int64_t)c->held_bytes();
  return CVSADC_OK;
}

int cvsadc_solve_batched(cvsadc_ctx* c, int32_t ninst, const cvsadc_params* params,
                         const double* const* eps, const void* const* B,
                         const void* const* dip, double* const* omega,
                         void* const* X, double* const* osc, cvsadc_info* info,
                         int32_t* status, int32_t lanes) {
  if (!c || ninst < 0 || (ninst > 0 && (!params || !eps || !B || !omega)))
    return CVSADC_EINVAL;
  if (ninst == 0) return CVSADC_OK;
  return guarded(c, [&] {
    solve_batched_impl(c, ninst, params, eps, B, dip, omega, X, osc, info, status,
                       lanes > 0 ? lanes : 4);
  });
}

int cvsadc_get_schur(cvsadc_ctx* c, double theta, int32_t flags, void* S) {
  if (!c || !S) return CVSADC_EINVAL;
  return guarded(c, [&] {
    CVS_REQUIRE(c->prepared, CVSADC_ESTATE, "no prepared problem");
    c->sch_on = false;
    schur_init(c);
    build_schur(c, CVSADC_FP64, theta, false);
    download(c, S, c->sch_S.p, (size_t)c->N1 * c->N1 * sizeof(cplx),
             (flags & CVSADC_FLAG_DEVICE_PTRS) != 0);
    c->sync();
  });
}

}  // extern "C"
