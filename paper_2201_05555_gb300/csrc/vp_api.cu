// C ABI of libvp: argument checks, workspace, and the composition of the
// kernels into the calls declared in include/vp.h.
#include "vp_internal.cuh"

#include <cstdarg>
#include <cmath>
#include <vector>

using namespace vpk;

// ------------------------------------------------------------ context glue
vp_status vp_fail(vp_ctx* ctx, vp_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->last_error = buf;
  }
  return s;
}

vp_status vp_cuda_check(vp_ctx* ctx, cudaError_t e, const char* what) {
  return vp_fail(ctx, e == cudaErrorMemoryAllocation ? VP_ENOMEM : VP_ECUDA, "%s: %s", what,
                 cudaGetErrorString(e));
}

vp_status vp_workspace(vp_ctx* ctx, size_t bytes, void** out) {
  if (bytes > ctx->budget)
    return vp_fail(ctx, VP_ENOMEM, "workspace of %zu bytes exceeds the context budget %zu", bytes,
                   ctx->budget);
  if (bytes > ctx->ws_bytes) {
    if (ctx->ws) {
      VP_CUDA(cudaDeviceSynchronize());
      VP_CUDA(cudaFree(ctx->ws));
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
    }
    size_t want = bytes + bytes / 4;
    if (want > ctx->budget) want = bytes;
    VP_CUDA(cudaMalloc(&ctx->ws, want));
    ctx->ws_bytes = want;
  }
  *out = ctx->ws;
  return VP_OK;
}

void comm_sum_f64(vp_ctx* ctx, double* buf, int64_t count, cudaStream_t st) {
  if (!ctx->comm_on || ctx->comm_failed || count <= 0) return;
  if (ctx->comm.sum_f64(ctx->comm.user, buf, count, (void*)st) != 0) ctx->comm_failed = true;
}
void comm_sum_u64(vp_ctx* ctx, unsigned long long* buf, int64_t count, cudaStream_t st) {
  if (!ctx->comm_on || ctx->comm_failed || count <= 0) return;
  if (ctx->comm.sum_u64(ctx->comm.user, reinterpret_cast<uint64_t*>(buf), count, (void*)st) != 0)
    ctx->comm_failed = true;
}

namespace {
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

#define VP_ENTER()                                              \
  if (!ctx) return VP_EINVAL;                                   \
  std::lock_guard<std::mutex> lock_(ctx->mu);                   \
  DeviceGuard guard_(ctx->device);                              \
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);     \
  (void)st;

// Reduced-model calls that do not sum over ranks refuse while a communicator
// is attached (their results would be this rank's rows only).
#define VP_NO_COMM()                                                                  \
  if (ctx->comm_on)                                                                   \
    return vp_fail(ctx, VP_EUNSUPPORTED, "%s: not available with a communicator attached", \
                   __func__)

vp_status check_grid(vp_ctx* ctx, const vp_grid* g) {
  if (!g) return vp_fail(ctx, VP_EINVAL, "grid is NULL");
  if (g->Nx < 3 || g->Nx > VP_MAX_NX)
    return vp_fail(ctx, VP_EINVAL, "Nx = %d outside [3, %d]", g->Nx, VP_MAX_NX);
  if (!(g->L > 0.0) || !std::isfinite(g->L)) return vp_fail(ctx, VP_EINVAL, "L must be > 0");
  if (!(g->mp > 0.0) || !std::isfinite(g->mp)) return vp_fail(ctx, VP_EINVAL, "mp must be > 0");
  if (!std::isfinite(g->Mq) || !std::isfinite(g->background))
    return vp_fail(ctx, VP_EINVAL, "Mq and background must be finite");
  return VP_OK;
}

vp_status check_np(vp_ctx* ctx, int64_t N, int32_t p) {
  if (N < 1 || N >= (int64_t(1) << 31)) return vp_fail(ctx, VP_EINVAL, "N = %lld outside [1, 2^31)", (long long)N);
  if (p < 1 || p > 65535) return vp_fail(ctx, VP_EINVAL, "p = %d outside [1, 65535]", p);
  return VP_OK;
}

vp_status check_n(vp_ctx* ctx, int32_t n, int64_t N) {
  if (n < 1 || n > 40) return vp_fail(ctx, VP_EUNSUPPORTED, "n = %d outside [1, 40] (2n <= 80)", n);
  if (n > N) return vp_fail(ctx, VP_EINVAL, "n = %d exceeds N = %lld", n, (long long)N);
  return VP_OK;
}


// Workspace of the reduced-model calls.
struct RedWS {
  unsigned long long* counts;
  double *F, *Efield, *part, *gX, *k, *kr, *Ze, *Z0, *Z1, *GVraw, *aux;
  double2 *grams, *cay, *C, *tmp;
  int* flags;  // [0] done, [1] iters, [2] ticket, [3] period of the cycle stopped on
  double* rows[5];
  float2 *Q2a, *Q2b;  // row-format shadows of Q0 and Q_half (float2 or float)
  uint16_t* jcell;    // cell index per (particle, sample), N x p
  float* bop;         // operand of the tensor-core row products (FP32 form)
  float2* frows[5];   // row blocks of the FP32-based step
  float2 *Z2, *Zh2, *F2;
  double* phi_out = nullptr;  // when set, the FP32-based field also writes the potentials
  int gx_proj, gx_gram;
  // parameter subsample of the basis stages (Sec. 4.1): per-sample buffers
  // for the nsub selected columns; N-row buffers are shared
  struct Sub {
    int nsub = 0;
    const int32_t* idx = nullptr;
    unsigned long long* counts = nullptr;
    double *F = nullptr, *Efield = nullptr, *Zs = nullptr;
    float2 *Z2 = nullptr, *Zh2 = nullptr, *F2 = nullptr;
    uint16_t* jcell = nullptr;
  } sub;
};

// Cell-index entries of the tile-by-tile layout (jt_block): whole tiles and
// whole sample chunks.
static size_t jcell_count(int64_t N, int p, int Nx) {
  const int pc = chunk_pc(p, Nx > 0 ? Nx : 3);
  return (size_t)ceil_div(N, TILE_ROWS) * ceil_div(p, pc) * TILE_ROWS * pc;
}

// Bytes of the subsample buffers (RedWS::Sub) for nsub columns.
static size_t sub_ws_bytes(int64_t N, int n, int nsub, int Nx) {
  if (nsub <= 0) return 0;
  const size_t pn = (size_t)nsub * (Nx > 0 ? Nx : 1), zn = (size_t)2 * n * nsub;
  return arena_bytes(pn, 8) * 2 + arena_bytes(nsub, 8) + arena_bytes(zn, 8) +
         2 * arena_bytes(zn, 8) + arena_bytes(pn, 8) + arena_bytes(jcell_count(N, nsub, Nx), 2);
}

// f32rows: the FP32 form (arith 2) keeps its row blocks (Q2a, frows) as FP32,
// half the double-float size; the double-float shadow Q2b of its energy
// check and re-orthonormalisation keeps the full size.
size_t red_ws_bytes(int sms, int64_t N, int n, int p, int Nx, int nrows, bool df, int* gx_proj,
                    int* gx_gram, const int* tune = nullptr, int nsub = 0, bool f32rows = false) {
  const int n2 = 2 * n, nn = n * n;
  const int chunks = project_chunks(p, Nx > 0 ? Nx : 3);
  // the FP32-based path sizes its grids by the context's launch-shape knobs
  const int* tn = tune ? tune : kTuneDefault;
  const int gp = df ? grid_bps(ceil_div(N, TILE_ROWS), chunks, tn[TUNE_PROJECT], sms)
                    : tile_grid_x(N, chunks, sms);
  const int gg = df ? grid_bps(ceil_div(N, 32), 1, tn[TUNE_GRAM], sms) : gram_grid_x(N, sms);
  if (gx_proj) *gx_proj = gp;
  if (gx_gram) *gx_gram = gg;
  size_t part_d = std::max<size_t>((size_t)gp * n2 * p,
                                   std::max<size_t>((size_t)gg * 12 * nn * 2, (size_t)gg * n2 * n2));
  size_t pn = (size_t)p * (Nx > 0 ? Nx : 1);
  return arena_bytes(pn, 8) * 2 + arena_bytes(p, 8) + arena_bytes(part_d, 8) +
         arena_bytes((size_t)n2 * p, 8) * 5 + arena_bytes((size_t)3 * n2 * p, 8) +
         arena_bytes((size_t)n2 * n2, 8) + arena_bytes((size_t)(n2 + 5) * p + 64, 8) + arena_bytes(12 * nn, 16) + arena_bytes(4 * nn, 16) +
         arena_bytes(4 * nn, 16) + arena_bytes(17 * nn, 16) + arena_bytes(8, 4) +
         (size_t)nrows * arena_bytes((size_t)N * n2, 8) +
         (df ? arena_bytes((size_t)N * n2, 8) + 6 * arena_bytes((size_t)N * n2, f32rows ? 4 : 8) +
                   arena_bytes(jcell_count(N, p, Nx), 2) +
                   2 * arena_bytes((size_t)n2 * p, 8) + arena_bytes(pn, 8) +
                   arena_bytes(rows_tc_bop_floats(n, p), 4) + sub_ws_bytes(N, n, nsub, Nx)
             : 0);
}

vp_status red_ws(vp_ctx* ctx, int64_t N, int n, int p, int Nx, int nrows, RedWS& w,
                 bool df = false, int nsub = 0, bool f32rows = false) {
  const int n2 = 2 * n, nn = n * n;
  size_t pn = (size_t)p * (Nx > 0 ? Nx : 1);
  f32rows = f32rows && df;
  size_t bytes = red_ws_bytes(ctx->num_sms, N, n, p, Nx, nrows, df, &w.gx_proj, &w.gx_gram,
                              ctx->tune, df ? nsub : 0, f32rows);
  size_t part_d = std::max<size_t>((size_t)w.gx_proj * n2 * p,
                                   std::max<size_t>((size_t)w.gx_gram * 12 * nn * 2,
                                                    (size_t)w.gx_gram * n2 * n2));
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, bytes, &base));
  Arena a{(char*)base, 0, bytes};
  w.counts = a.take<unsigned long long>(pn);
  w.F = a.take<double>(pn);
  w.Efield = a.take<double>(p);
  w.part = a.take<double>(part_d);
  w.gX = a.take<double>((size_t)n2 * p);
  w.k = a.take<double>((size_t)n2 * p);
  w.kr = a.take<double>((size_t)3 * n2 * p);  // ring of earlier fixed-point iterates
  w.Ze = a.take<double>((size_t)n2 * p);
  w.Z0 = a.take<double>((size_t)n2 * p);
  w.Z1 = a.take<double>((size_t)n2 * p);
  w.GVraw = a.take<double>((size_t)n2 * n2);
  w.aux = a.take<double>((size_t)(n2 + 5) * p + 64);
  w.grams = a.take<double2>(12 * nn);
  w.cay = a.take<double2>(4 * nn);
  w.C = a.take<double2>(4 * nn);
  w.tmp = a.take<double2>(17 * nn);  // small dense scratch (see dense.cu)
  w.flags = a.take<int>(8);
  for (int r = 0; r < 5; ++r) w.rows[r] = r < nrows ? a.take<double>((size_t)N * n2) : nullptr;
  // the row blocks of the df / FP32 step: float2 (double-float) elements, or
  // float with f32rows, N x 2n each
  auto rowblk = [&]() -> float2* {
    if (!df) return nullptr;
    if (f32rows) return reinterpret_cast<float2*>(a.take<float>((size_t)N * n2));
    return a.take<float2>((size_t)N * n2);
  };
  w.Q2a = rowblk();
  for (int r = 0; r < 5; ++r) w.frows[r] = rowblk();
  w.Q2b = df ? a.take<float2>((size_t)N * n2) : nullptr;
  w.jcell = df ? a.take<uint16_t>(jcell_count(N, p, Nx)) : nullptr;
  w.Z2 = df ? a.take<float2>((size_t)n2 * p) : nullptr;
  w.Zh2 = df ? a.take<float2>((size_t)n2 * p) : nullptr;
  w.F2 = df ? a.take<float2>(pn) : nullptr;
  w.bop = df ? a.take<float>(rows_tc_bop_floats(n, p)) : nullptr;
  w.sub = RedWS::Sub();
  if (df && nsub > 0) {
    const size_t ps = (size_t)nsub * (Nx > 0 ? Nx : 1), zs = (size_t)n2 * nsub;
    w.sub.nsub = nsub;
    w.sub.counts = a.take<unsigned long long>(ps);
    w.sub.F = a.take<double>(ps);
    w.sub.Efield = a.take<double>(nsub);
    w.sub.Zs = a.take<double>(zs);
    w.sub.Z2 = a.take<float2>(zs);
    w.sub.Zh2 = a.take<float2>(zs);
    w.sub.F2 = a.take<float2>(ps);
    w.sub.jcell = a.take<uint16_t>(jcell_count(N, nsub, Nx));
  }
  return VP_OK;
}

// ------------------------------------------------------- reduced building blocks
struct Red {
  vp_ctx* ctx;
  GridC g;
  int64_t N;
  int n, p;
  RedWS w;
  cudaStream_t st;
  bool df = false;

  // deposit X_r = Re(Q Z) and solve: F, Efield (counts zeroed again by the solve).
  // With df, Q2 is the double-float shadow of Q and the cell indices are kept.
  void field(const double* Q, const double* Z, const int* skip = nullptr,
             const float2* Q2 = nullptr) {
    (void)Q2;
    VP_K(VP_K_DEPOSIT_REDUCED, deposit_reduced(g, N, n, p, Q, Z, w.counts, skip, ctx->num_sms, st));
    comm_sum_u64(ctx, w.counts, (int64_t)p * g.Nx, st);
    VP_K(VP_K_POISSON, poisson(g, p, nullptr, w.counts, nullptr, w.F, w.Efield, w.counts, skip, ctx->d_status, st));
  }
  // Grams out_s = blk[pa]^H blk[pb] into `out` (npairs x n x n double2)
  void grams(std::initializer_list<const double*> blks,
             std::initializer_list<std::pair<int, int>> pairs, double2* out) {
    GramArgs a{};
    a.nblk = 0;
    for (const double* b : blks) a.blk[a.nblk++] = b;
    a.npairs = 0;
    for (auto pr : pairs) {
      a.pa[a.npairs] = pr.first;
      a.pb[a.npairs] = pr.second;
      ++a.npairs;
    }
    VP_K(VP_K_GRAM, gram(N, n, a, reinterpret_cast<double2*>(w.part), w.gx_gram, st));
    VP_K(VP_K_REDUCE, reduce_partials(w.gx_gram, (int64_t)a.npairs * n * n * 2, w.part,
                    reinterpret_cast<double*>(out), nullptr, st));
    comm_sum_f64(ctx, reinterpret_cast<double*>(out), (int64_t)a.npairs * n * n * 2, st);
  }
  void gv(const double* Q, double* GVraw) {
    VP_K(VP_K_GRAM_REAL, gram_real(N, 2 * n, Q, w.part, w.gx_gram, st));
    VP_K(VP_K_REDUCE, reduce_partials(w.gx_gram, (int64_t)4 * n * n, w.part, GVraw, nullptr, st));
    comm_sum_f64(ctx, GVraw, (int64_t)4 * n * n, st);
  }
  void comb(std::initializer_list<const double*> xs, const double2* C, double* out) {
    AffineArgs a{};
    a.nterms = 0;
    for (const double* x : xs) a.X[a.nterms++] = x;
    VP_K(VP_K_AFFINE, affine(N, n, a, C, out, ctx->num_sms, st));
  }
  // X(Q, Z) * scale into out, using M as scratch (F must hold the field at (Q, Z))
  void basis_velocity_from_field(const double* Q, const double* Z, double scale, double* M,
                                 double* out, const float2* Q2 = nullptr) {
    (void)Q2;
    VP_K(VP_K_BASIS_M, basis_M(g, N, n, p, Q, Z, w.F, M, ctx->num_sms, st));
    grams({Q, M}, {{0, 1}}, w.grams);
    VP_K(VP_K_SMALL_BASIS, small_basis_coeffs(n, p, w.grams, Z, scale, w.C, w.tmp, ctx->d_status, st));
    comb({M, Q}, w.C, out);
  }
  // Qout = R_Q0(xi); leaves G0, P, XX in w.cay[0..3n^2)
  void cayley(const double* Q0, const double* xi, double* Qout) {
    grams({Q0, xi}, {{0, 0}, {0, 1}, {1, 1}}, w.cay);
    const int nn = n * n;
    VP_K(VP_K_SMALL_CAYLEY, small_cayley_coeffs(n, w.cay, w.cay + nn, w.cay + 2 * nn, w.C, w.tmp, ctx->d_status, st));
    comb({Q0, xi}, w.C, Qout);
  }
  // Y(xi, Z) * scale with Qh = R_Q0(xi) and Xp = X(Qh, Z) given; w.cay must hold
  // the Cayley Grams of (Q0, xi).
  void tangent(const double* Q0, const double* xi, const double* Qh, const double* Xp, double scale,
               double* out) {
    grams({Q0, xi, Qh, Xp}, {{0, 3}, {1, 3}, {0, 2}, {2, 3}, {2, 1}}, w.grams);
    const int nn = n * n;
    VP_K(VP_K_SMALL_TANGENT, small_tangent_coeffs(n, w.grams, w.cay, w.cay + nn, scale, w.C, w.tmp, ctx->d_status, st));
    comb({Xp, xi, Q0}, w.C, out);
  }
};

vp_status red_setup(vp_ctx* ctx, const vp_grid* grid, int64_t N, int n, int p, int nrows,
                    cudaStream_t st, Red& R, bool df = false, int nsub = 0,
                    bool f32rows = false) {
  R.ctx = ctx;
  R.df = df;
  R.N = N;
  R.n = n;
  R.p = p;
  R.st = st;
  // fixed-point scales bound the sums over all ranks' particles
  if (grid) R.g = make_gridc(*grid, ctx->comm_on ? ctx->comm.n_global : N);
  VP_TRY(red_ws(ctx, N, n, p, grid ? grid->Nx : 0, nrows, R.w, df, nsub, f32rows));
  if (grid) VP_CUDA(cudaMemsetAsync(R.w.counts, 0, sizeof(unsigned long long) * p * grid->Nx, st));
  if (grid && R.w.sub.nsub)
    VP_CUDA(cudaMemsetAsync(R.w.sub.counts, 0, sizeof(unsigned long long) * nsub * grid->Nx, st));
  return VP_OK;
}

// The Red of the subsample: the subset's per-sample buffers, the rest shared.
Red sub_red(const Red& R) {
  Red Rs = R;
  const RedWS::Sub& b = R.w.sub;
  Rs.p = b.nsub;
  Rs.w.counts = b.counts;
  Rs.w.F = b.F;
  Rs.w.Efield = b.Efield;
  Rs.w.Z2 = b.Z2;
  Rs.w.Zh2 = b.Zh2;
  Rs.w.F2 = b.F2;
  Rs.w.jcell = b.jcell;
  return Rs;
}
}  // namespace

// ------------------------------------------- double-float partitioned RK2
// The same stage structure as the FP64 path: every N-row intermediate (M,
// xi_half, Q_half, X(Q_half, Z_mid), xi_1) is kept as double-float rows,
// Gram matrices and the small dense algebra are FP64, and Q is written back
// in FP64.
namespace {
// FP32-based composition (arith 1 double-float, 2 FP32); rows are stored in
// buffers sized for double-float and used as float2 or float.
struct RedDF {
  Red& R;
  vp_ctx* ctx;
  cudaStream_t st;
  int64_t N;
  int n, p, arith;
  bool diag = false;  // the FP64-accurate energy diagnostic of the FP32 form (own profiling id)
  LpArgs base() const {
    LpArgs a;
    a.g = &R.g;
    a.N = N;
    a.n = n;
    a.p = p;
    a.num_sms = ctx->num_sms;
    a.tune = ctx->tune;
    a.status = ctx->d_status;
    a.tc = ctx->tensor_cores;
    return a;
  }
  // field at (Q2, Z): Z2 = Z and Zh2 = Z / h in row format (skipped when the
  // caller already wrote them), deposit, Poisson writing F and (q/m) F in row format
  void field(const void* Q2, const double* Z, const int* skip, bool z_ready = false) {
    RedWS& w = R.w;
    LpArgs a = base();
    if (!z_ready) {
      a.dsrc = Z;
      a.v0 = w.Z2;
      a.v1 = w.Zh2;
      a.skip = skip;
      VP_K(VP_K_PREP_LP, lp_launch(arith, LP_PREP, a, st));
    }
    a = base();
    a.v0 = const_cast<void*>(Q2);
    a.v1 = w.Zh2;
    a.counts = w.counts;
    // the energy check's cell indices would be overwritten unread by the
    // step's own field evaluation: not stored
    a.j = diag ? nullptr : w.jcell;
    a.skip = skip;
    const bool tc = (a.tc & VP_TC_DEPOSIT) && arith == 2 && deposit_tc_supported(n, p, R.g.Nx, R.g.Kp);
    VP_K(diag ? VP_K_DEPOSIT_DIAG : (tc ? VP_K_DEPOSIT_TC : VP_K_DEPOSIT_LP),
         lp_launch(arith, LP_DEPOSIT, a, st));
    comm_sum_u64(ctx, w.counts, (int64_t)p * R.g.Nx, st);
    VP_K(VP_K_POISSON, poisson(R.g, p, nullptr, w.counts, w.phi_out, w.F, w.Efield, w.counts, skip,
                               ctx->d_status, st, w.F2, arith));
  }
  void project(const void* Q2, const int* skip) {
    LpArgs a = base();
    a.v0 = const_cast<void*>(Q2);
    a.v1 = R.w.F2;
    a.j = R.w.jcell;
    a.part = R.w.part;
    a.gridx = R.w.gx_proj;
    a.skip = skip;
    const bool tc = (a.tc & VP_TC_PROJECT) && arith == 2 && project_tc_supported(n, p, R.g.Nx);
    VP_K(tc ? VP_K_PROJECT_TC : VP_K_PROJECT_LP, lp_launch(arith, LP_PROJECT, a, st));
  }
  // one or two CTAs per SM (shared memory), at most one per 32-row tile and
  // within the partial buffer
  int gram_tc_grid(int nblk) const {
    int64_t g = (int64_t)ctx->num_sms * (nblk <= 2 ? 2 : 1);
    g = std::min<int64_t>(g, (N + 31) / 32);
    g = std::min<int64_t>(g, R.w.gx_gram);
    return (int)std::max<int64_t>(g, 1);
  }
  void grams(std::initializer_list<const void*> blks,
             std::initializer_list<std::pair<int, int>> pairs, double2* out) {
    LpArgs a = base();
    for (const void* b : blks) a.gram.blk[a.gram.nblk++] = b;
    for (auto pr : pairs) {
      a.gram.pa[a.gram.npairs] = pr.first;
      a.gram.pb[a.gram.npairs] = pr.second;
      ++a.gram.npairs;
    }
    a.part = R.w.part;
    const bool tc = (a.tc & VP_TC_GRAM) && arith == 2 && gram_tc_supported(n, a.gram.nblk, a.gram.npairs);
    a.gridx = tc ? gram_tc_grid(a.gram.nblk) : R.w.gx_gram;
    VP_K(tc ? VP_K_GRAM_TC : VP_K_GRAM_LP, lp_launch(arith, LP_GRAM, a, st));
    VP_K(VP_K_REDUCE, reduce_partials(a.gridx, (int64_t)a.gram.npairs * n * n * 2, R.w.part,
                                      reinterpret_cast<double*>(out), nullptr, st));
    comm_sum_f64(ctx, reinterpret_cast<double*>(out), (int64_t)a.gram.npairs * n * n * 2, st);
  }
  void gv(const void* Q2, double* GVraw) {
    LpArgs a = base();
    a.v0 = const_cast<void*>(Q2);
    a.part = R.w.part;
    const bool tc = (a.tc & VP_TC_GRAM) && arith == 2 && gram_tc_supported(n, 1, 1);
    a.gridx = tc ? gram_tc_grid(1) : R.w.gx_gram;
    VP_K(tc ? VP_K_GRAM_TC : VP_K_GRAM_REAL_LP, lp_launch(arith, LP_GRAM_REAL, a, st));
    VP_K(VP_K_REDUCE, reduce_partials(a.gridx, (int64_t)4 * n * n, R.w.part, GVraw, nullptr, st));
    comm_sum_f64(ctx, GVraw, (int64_t)4 * n * n, st);
  }
  void comb(std::initializer_list<const void*> xs, const double2* C, double* out_d, void* out_v,
            const double* base_d = nullptr) {
    LpArgs a = base();
    for (const void* x : xs) a.aff.X[a.aff.nterms++] = x;
    a.aff.base = base_d;
    a.C = C;
    a.dout = out_d;
    a.v0 = out_v;
    a.bop = R.w.bop;
    const bool tc = (a.tc & VP_TC_AFFINE) && arith == 2 && R.w.bop && affine_tc_supported(n, a.aff.nterms);
    VP_K(tc ? VP_K_AFFINE_TC : VP_K_AFFINE_LP, lp_launch(arith, LP_AFFINE, a, st));
  }
  void split(const double* Q, void* Q2) {
    LpArgs a = base();
    a.m = N * 2 * n;
    a.dsrc = Q;
    a.v0 = Q2;
    VP_K(VP_K_SPLIT, lp_launch(arith, LP_SPLIT, a, st));
  }
  // scale * X(Q, Z) into out (F2, jcell, Z2 must hold the field at (Q, Z))
  void basis_velocity(const void* Q2, const double* Z, double scale, void* M, void* out) {
    RedWS& w = R.w;
    LpArgs a = base();
    a.v0 = const_cast<void*>(Q2);
    a.v1 = w.Z2;
    a.v2 = w.F2;
    a.v3 = M;
    a.j = w.jcell;
    a.bop = w.bop;
    const bool tc = (a.tc & VP_TC_BASIS_M) && arith == 2 && w.bop && basis_tc_supported(n, p);
    VP_K(tc ? VP_K_BASIS_M_TC : VP_K_BASIS_M_LP, lp_launch(arith, LP_BASIS_M, a, st));
    grams({Q2, M}, {{0, 1}}, w.grams);
    VP_K(VP_K_SMALL_BASIS, small_basis_coeffs(n, p, w.grams, Z, scale, w.C, w.tmp, ctx->d_status, st,
                                              arith == 2));
    comb({M, Q2}, w.C, nullptr, out);
  }
  // Cayley retraction of Q0 along xi; leaves G0, P, XX in w.cay.  Q0d (FP64
  // rows of Q0, nullable): out_d = Q0d + the increment (see AffineArgsLP)
  void cayley(const void* Q0, const void* xi, double* out_d, void* out_v,
              const double* Q0d = nullptr) {
    RedWS& w = R.w;
    grams({Q0, xi}, {{0, 0}, {0, 1}, {1, 1}}, w.cay);
    const int nn = n * n;
    VP_K(VP_K_SMALL_CAYLEY, small_cayley_coeffs(n, w.cay, w.cay + nn, w.cay + 2 * nn, w.C, w.tmp,
                                                ctx->d_status, st, arith == 2));
    comb({Q0, xi}, w.C, out_d, out_v, Q0d);
  }
};
}  // namespace

namespace {
// Lowest fixed-point tolerance of the FP32 form (about 8 FP32 ulps).
constexpr double kTolFP32 = 1e-6;
struct DFStep {
  vp_ctx* ctx;
  Red& R;
  double* Q;
  double* Z;
  double dt;
  vp_step_opts o;
  double* kstate;
  cudaStream_t st;
  const void* Qm = nullptr;  // rows the fixed point evaluates at (Q_half, or Q0 when frozen)
  Red Rs;                    // parameter subsample of the basis stages (Rs.p = 0: none)
  cudaEvent_t field_event = nullptr;  // recorded after the subsample's field, when set
  DFStep(vp_ctx* c, Red& r, double* q, double* z, double d, const vp_step_opts& opt, double* ks,
         cudaStream_t s);
  vp_status pre(double* trace_step);
  vp_status rounds(int count);
  vp_status post();
};
}  // namespace

// One step of the FP32-based path in three phases, so that the host-steered
// loop below and the batched engine (batch.cu, CUDA graphs) issue the same
// kernel sequence: pre (field at the entering state, energies, basis stage,
// fixed-point set-up), rounds (fixed-point iterations; after convergence the
// kernels see the done flag and return at once), post (Z update, tangent
// velocity, Cayley retraction, re-orthonormalisation).
DFStep::DFStep(vp_ctx* c, Red& r, double* q, double* z, double d, const vp_step_opts& opt,
               double* ks, cudaStream_t s)
    : ctx(c), R(r), Q(q), Z(z), dt(d), o(opt), kstate(ks), st(s) {
  // the FP32 form evaluates the fixed-point map with FP32 rows: its updates
  // stop shrinking near the FP32 rounding level (~1e-7 relative), so the stop
  // tolerance is at least kTolFP32
  if (o.arith == 2 && o.tol < kTolFP32) o.tol = kTolFP32;
  Rs = sub_red(R);
  Rs.w.sub.idx = opt.sub_idx;
}

// scale X(Q2, Zsrc) of the basis stage into out, on all samples or on the
// parameter subsample (field and basis kernels on the selected columns)
static vp_status basis_stage(DFStep& S, const void* Q2, const double* Zsrc, double scale,
                             void* M, void* out, bool field_ready) {
  vp_ctx* ctx = S.ctx;
  cudaStream_t st = S.st;
  const int n = S.R.n;
  if (S.Rs.p > 0) {
    RedDF Ds{S.Rs, ctx, st, S.R.N, n, S.Rs.p, S.o.arith};
    VP_K(VP_K_SUBSET, gather_cols(2 * n, S.R.p, Zsrc, S.o.sub_idx, S.Rs.p, S.R.w.sub.Zs,
                                  ctx->d_status, st));
    Ds.field(Q2, S.R.w.sub.Zs, nullptr);
    if (S.field_event) VP_CUDA(cudaEventRecord(S.field_event, st));
    Ds.basis_velocity(Q2, S.R.w.sub.Zs, scale, M, out);
  } else {
    RedDF D{S.R, ctx, st, S.R.N, n, S.R.p, S.o.arith};
    if (!field_ready) D.field(Q2, Zsrc, nullptr);
    D.basis_velocity(Q2, Zsrc, scale, M, out);
  }
  return VP_OK;
}

vp_status DFStep::pre(double* trace_step) {
  RedWS& w = R.w;
  const int n = R.n, p = R.p;
  const int64_t N = R.N;
  RedDF D{R, ctx, st, N, n, p, o.arith};
  RedDF DD{R, ctx, st, N, n, p, 1, true};  // double-float diagnostics
  void *Q0 = w.Q2a, *M = w.frows[0], *xih = w.frows[1], *Qh = w.frows[2];
  const int64_t zsz = (int64_t)2 * n * p;
  if (trace_step && o.arith == 2) {  // FP64-accurate diagnostic in the precision form
    DD.split(Q, w.Q2b);
    DD.field(w.Q2b, Z, nullptr);
    DD.gv(w.Q2b, w.GVraw);
    VP_K(VP_K_ENERGIES, energies(n, p, w.GVraw, Z, w.Efield, trace_step, trace_step + 1, 2, nullptr,
                                 nullptr, ctx->d_status, st));
  }
  D.split(Q, Q0);
  // the field of all samples at the entering state serves the energies and,
  // without a subsample, the basis stage
  const bool full_field = Rs.p == 0 || (trace_step && o.arith != 2);
  if (full_field) D.field(Q0, Z, nullptr);
  if (trace_step && o.arith != 2) {
    D.gv(Q0, w.GVraw);
    VP_K(VP_K_ENERGIES, energies(n, p, w.GVraw, Z, w.Efield, trace_step, trace_step + 1, 2, nullptr,
                                 nullptr, ctx->d_status, st));
  }
  Qm = Q0;
  if (!o.freeze_basis) {
    VP_TRY(basis_stage(*this, Q0, Z, 0.5 * dt, M, xih, full_field));  // xi_half = dt/2 X(Q0, Z0)
    D.cayley(Q0, xih, nullptr, Qh);                                   // Q_half = R_Q0(xi_half)
    Qm = Qh;
  }
  D.gv(Qm, w.GVraw);
  VP_CUDA(cudaMemcpyAsync(w.Z0, Z, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
  if (kstate) {
    VP_CUDA(cudaMemcpyAsync(w.k, kstate, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
    VP_K(VP_K_AXPY, axpy(zsz, 0.5 * dt, w.k, w.Z0, w.Ze, st));
  } else {
    VP_CUDA(cudaMemcpyAsync(w.Ze, Z, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
    VP_CUDA(cudaMemsetAsync(w.k, 0, sizeof(double) * zsz, st));
  }
  VP_CUDA(cudaMemsetAsync(w.flags, 0, 4 * sizeof(int), st));
  LpArgs a = D.base();  // Ze in row format for the first round's deposit
  a.dsrc = w.Ze;
  a.v0 = w.Z2;
  a.v1 = w.Zh2;
  VP_K(VP_K_PREP_LP, lp_launch(o.arith, LP_PREP, a, st));
  return VP_OK;
}

vp_status DFStep::rounds(int count) {
  RedWS& w = R.w;
  const int n = R.n, p = R.p;
  RedDF D{R, ctx, st, R.N, n, p, o.arith};
  const int64_t zsz = (int64_t)2 * n * p;
  (void)zsz;
  // Ze in row format (Z2, Zh2) comes from pre() for the first round and from
  // the coefficient update (which also sums the projection partials) after it
  for (int r = 0; r < count; ++r) {
    D.field(Qm, w.Ze, w.flags, true);
    D.project(Qm, w.flags);
    if (ctx->comm_on) {  // the projection summed over the ranks before the update
      VP_K(VP_K_REDUCE, reduce_partials(w.gx_proj, zsz, w.part, w.gX, w.flags, st));
      comm_sum_f64(ctx, w.gX, zsz, st);
      VP_K(VP_K_COEFF_UPDATE,
           coeff_update(n, p, w.gX, w.GVraw, w.Z0, w.k, w.kr, w.Ze, dt, o.tol, o.maxit,
                        o.cycle_max, o.cycle_ratio, w.aux, w.flags, w.flags + 1, ctx->d_status,
                        st, nullptr, 0, w.Z2, w.Zh2, R.g.inv_h, o.arith));
      continue;
    }
    VP_K(VP_K_COEFF_UPDATE,
         coeff_update(n, p, nullptr, w.GVraw, w.Z0, w.k, w.kr, w.Ze, dt, o.tol, o.maxit,
                      o.cycle_max, o.cycle_ratio, w.aux, w.flags, w.flags + 1, ctx->d_status, st, w.part,
                      w.gx_proj, w.Z2, w.Zh2, R.g.inv_h, o.arith));
  }
  return VP_OK;
}

vp_status DFStep::post() {
  RedWS& w = R.w;
  const int n = R.n, p = R.p;
  const int64_t N = R.N;
  RedDF D{R, ctx, st, N, n, p, o.arith};
  RedDF DD{R, ctx, st, N, n, p, 1};
  void *Q0 = w.Q2a, *M = w.frows[0], *xih = w.frows[1], *Qh = w.frows[2], *Xp = w.frows[3],
       *xi1 = w.frows[4];
  const int64_t zsz = (int64_t)2 * n * p;
  VP_K(VP_K_AXPY, axpy(zsz, dt, w.k, w.Z0, w.Z1, st));
  if (kstate) VP_CUDA(cudaMemcpyAsync(kstate, w.k, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
  if (!o.freeze_basis) {
    VP_TRY(basis_stage(*this, Qh, w.Ze, 1.0, M, Xp, false));  // X(Q_half, Z_mid)
    D.grams({Q0, xih, Qh, Xp}, {{0, 3}, {1, 3}, {0, 2}, {2, 3}, {2, 1}}, w.grams);
    const int nn = n * n;
    VP_K(VP_K_SMALL_TANGENT, small_tangent_coeffs(n, w.grams, w.cay, w.cay + nn, dt, w.C, w.tmp,
                                                  ctx->d_status, st, o.arith == 2));
    D.comb({Xp, xih, Q0}, w.C, nullptr, xi1);  // xi_1 = dt Y(xi_half, Z_mid)
    // Q_1 = R_Q0(xi_1) in FP64; in the FP32 form as Q_0 + (Q_1 - Q_0), the
    // increment from FP32 rows added to the FP64 Q_0, so that Q does not take
    // an FP32 rounding error every step
    D.cayley(Q0, xi1, Q, nullptr, o.arith == 2 ? Q : nullptr);
    if (o.reortho) {                           // Q <- Q (Q^H Q)^-1/2
      DD.split(Q, w.Q2b);
      DD.grams({w.Q2b}, {{0, 0}}, w.grams);
      VP_K(VP_K_INIT, lowdin(n, w.grams, w.C, ctx->d_status, st));
      DD.comb({w.Q2b}, w.C, Q, nullptr);
    }
  }
  VP_CUDA(cudaMemcpyAsync(Z, w.Z1, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
  return VP_OK;
}

static vp_status basis_update_df(vp_ctx* ctx, Red& R, double* Q, double* Z, double dt,
                                 int nsteps, const vp_step_opts& o, double* trace, int32_t* iters,
                                 double* kstate, cudaStream_t st) {
  RedWS& w = R.w;
  const int64_t tstride = (int64_t)R.p * 2;
  DFStep S(ctx, R, Q, Z, dt, o, kstate, st);
  int round = 4;
  for (int step = 0; step < nsteps; ++step) {
    VP_TRY(S.pre(trace ? trace + step * tstride : nullptr));
    int done_h = 0, total = 0;
    while (!done_h) {
      const int r = std::min(round, o.maxit - total);
      VP_TRY(S.rounds(r));
      total += r;
      VP_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, w.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      VP_CUDA(cudaStreamSynchronize(st));
      if (!ctx->pending.empty()) vp_prof_collect(ctx);
      done_h = ctx->h_pinned[1];
      if (!done_h && total >= o.maxit) break;
      round = 2;
    }
    const int its = ctx->h_pinned[2];
    round = its > 2 ? its : 2;
    if (iters) VP_CUDA(cudaMemcpyAsync(iters + step, w.flags + 1, sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (!done_h || its >= o.maxit) {
      VP_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      VP_CUDA(cudaStreamSynchronize(st));
      if (ctx->h_pinned[0] != 0 || !done_h)
        return vp_fail(ctx, VP_ENOCONV, "fixed point did not converge in %d iterations (step %d)",
                       o.maxit, step);
    }
    VP_TRY(S.post());
  }
  VP_LAUNCHED();
  return VP_OK;
}

// ------------------------------------------ DMD-DEIM reduced dynamics
// Algorithm 2 on the device: windows, DMD and DEIM operators of one reduced
// problem (see vp_hyper_* in vp.h).  All buffers are owned by the object
// (one allocation), apart from the step workspace of the context.
struct vp_hyper {
  vp_ctx* ctx = nullptr;
  vp_grid grid{};
  GridC g{};
  int64_t N = 0;
  int n = 0, p = 0, nsub = 0, dim = 0, T = 0, d = 0, n_up = 0, k_deim = 1, r_max = 0;
  double dmd_tol = 0.0;
  void* mem = nullptr;
  int32_t *sub = nullptr, *idx = nullptr;
  double *eta = nullptr, *eta_s = nullptr, *eps = nullptr;
  double* phi_ring = nullptr;  // 2 (T+1) slots of nsub x Nx (each written twice, so
                               // every window of T+1 consecutive entries is contiguous)
  double* y_ring = nullptr;    // (T+1) slots of nsub x N (DEIM data; order is immaterial)
  double *B = nullptr, *Bp = nullptr, *A = nullptr, *S = nullptr, *beta_s = nullptr,
         *beta = nullptr, *phi_half = nullptr, *F = nullptr, *Psi = nullptr, *Psi_prev = nullptr,
         *c = nullptr, *Qd = nullptr;
  void* scratch = nullptr;       // DMD scratch (main stream)
  void* scratch_deim = nullptr;  // DEIM scratch (side stream)
  cudaStream_t side = nullptr;   // DEIM data and construction
  cudaStream_t side2 = nullptr;  // DMD chain
  cudaEvent_t ev_data = nullptr, ev_deim = nullptr, ev_dmd = nullptr;
  int64_t entries = 0;  // potentials written to the windows
  int intervals = 0, hyper_intervals = 0, r = 0;
};

namespace {
__global__ void k_gather_eta(int dim, int nsub, const int32_t* __restrict__ sub,
                             const double* __restrict__ eta, int p, double* __restrict__ eta_s,
                             int* status) {
  for (int e = threadIdx.x; e < nsub * dim; e += blockDim.x) {
    const int i = e / dim, a = e - i * dim;
    const int c = sub[i];
    if (c < 0 || c >= p) {
      vp_set_status(status, VP_EINVAL);
      eta_s[e] = 0.0;
    } else {
      eta_s[e] = eta[c * dim + a];
    }
  }
}

// One interval of Algorithm 2 (see vp.h); S is the step of this call.
vp_status hyper_interval(vp_hyper* h, Red& R, DFStep& S, double* trace_step, int round_hint,
                         int* its_out) {
  vp_ctx* ctx = h->ctx;
  cudaStream_t st = S.st;
  RedWS& w = R.w;
  const int n = h->n, p = h->p, q = h->nsub, Nx = h->grid.Nx, T = h->T;
  const int64_t N = h->N;
  const vp_step_opts& o = S.o;
  // 1. field of the sampled parameters at the entering state writes Phi_{tau-1};
  // the windows and operators below start as soon as it is done (event
  // ev_data, recorded inside the first basis stage) and overlap the rest of
  // the stage on two more streams: DEIM data and construction (N-row work)
  // on `side`, the single-block DMD chain on `side2`
  const int slot = (int)(h->entries % (T + 1));
  double* phi_slot = h->phi_ring + (size_t)slot * q * Nx;
  S.Rs.w.phi_out = phi_slot;
  S.field_event = h->ev_data;
  VP_TRY(S.pre(trace_step));
  S.Rs.w.phi_out = nullptr;
  S.field_event = nullptr;
  ++h->entries;
  const bool hyper = h->entries >= T + 1;
  {
    cudaStream_t st = h->side;
    VP_CUDA(cudaStreamWaitEvent(st, h->ev_data, 0));
    VP_K(VP_K_HYPER, phi_at_qz(h->g, N, n, q, S.Q, w.sub.Zs, phi_slot,
                               h->y_ring + (size_t)slot * q * N, ctx->num_sms, st));
    if (hyper) {  // DEIM basis, indices (all, or the n_up most rotated), weights
      std::swap(h->Psi, h->Psi_prev);
      VP_TRY(deim_basis_run(ctx, N, (T + 1) * q, h->y_ring, N, h->d, h->Psi, nullptr,
                            h->scratch_deim, st));
      const bool full = h->hyper_intervals % h->k_deim == 0;
      VP_TRY(deim_indices_run(ctx, N, h->d, h->Psi, h->idx, full ? nullptr : h->Psi_prev, h->n_up,
                              h->scratch_deim, st));
      VP_TRY(deim_weights_run(ctx, N, h->d, h->Psi, h->idx, h->g.Mq, h->c, h->scratch_deim, st));
    }
    VP_CUDA(cudaEventRecord(h->ev_deim, st));
  }
  {
    cudaStream_t st = h->side2;
    VP_CUDA(cudaStreamWaitEvent(st, h->ev_data, 0));
    VP_CUDA(cudaMemcpyAsync(phi_slot + (size_t)(T + 1) * q * Nx, phi_slot, sizeof(double) * q * Nx,
                            cudaMemcpyDeviceToDevice, st));
    if (hyper) {  // DMD of the window (oldest entry first), coordinates, RBF, Phi at t + dt/2
      const int oldest = (int)((h->entries - (T + 1)) % (T + 1));
      const double* Y = h->phi_ring + (size_t)oldest * q * Nx;
      int r = 0;
      VP_TRY(dmd_fit_run(ctx, Nx, T * q, Y, Y + (size_t)q * Nx, h->dmd_tol, h->r_max, &r, h->B,
                         h->Bp, h->A, h->S, nullptr, h->scratch, st));
      h->r = r;
      VP_K(VP_K_HYPER, dmd_coords_run(Nx, r, h->Bp, q, phi_slot, h->beta_s, st));
      VP_K(VP_K_HYPER, rbf_run(h->dim, q, h->eta_s, r, h->beta_s, p, h->eta, 0.0, h->eps, h->beta,
                               ctx->d_status, st));
      VP_K(VP_K_HYPER, dmd_potential_run(Nx, r, h->B, h->A, h->S, p, h->beta, 0, 1, h->phi_half,
                                         st));
      VP_K(VP_K_CELL_GRADIENT, cell_gradient(h->g, p, h->phi_half, h->F, st));
    }
    VP_CUDA(cudaEventRecord(h->ev_dmd, st));
  }
  // the main stream continues after both (the side stream reads the
  // subsample's coefficients, which the last basis stage overwrites)
  VP_CUDA(cudaStreamWaitEvent(st, h->ev_deim, 0));
  VP_CUDA(cudaStreamWaitEvent(st, h->ev_dmd, 0));
  if (hyper) {
    // the d DEIM rows of the basis at the coefficient stage (U_1/2)
    VP_K(VP_K_HYPER, gather_rows_lp(S.Qm, o.arith, N, 2 * n, h->idx, h->d, h->Qd, ctx->d_status, st));
    ++h->hyper_intervals;
  }
  // fixed point of the coefficient stage
  int round = round_hint, done_h = 0, total = 0;
  while (!done_h) {
    const int rr = std::min(round, o.maxit - total);
    if (hyper) {
      for (int k = 0; k < rr; ++k) {
        VP_K(VP_K_DEIM_ROUND, deim_round(h->g, n, p, h->d, h->Qd, w.Ze, h->F, h->c, w.gX, w.flags, st));
        VP_K(VP_K_COEFF_UPDATE,
             coeff_update(n, p, w.gX, w.GVraw, w.Z0, w.k, w.kr, w.Ze, S.dt, o.tol, o.maxit,
                          o.cycle_max, o.cycle_ratio, w.aux, w.flags, w.flags + 1, ctx->d_status, st));
      }
    } else {
      VP_TRY(S.rounds(rr));
    }
    total += rr;
    VP_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, w.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    VP_CUDA(cudaStreamSynchronize(st));
    if (!ctx->pending.empty()) vp_prof_collect(ctx);
    done_h = ctx->h_pinned[1];
    if (!done_h && total >= o.maxit) break;
    round = 2;
  }
  const int its = ctx->h_pinned[2];
  *its_out = its;
  if (!done_h || its >= o.maxit) {
    VP_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    VP_CUDA(cudaStreamSynchronize(st));
    if (ctx->h_pinned[0] != 0 || !done_h)
      return vp_fail(ctx, VP_ENOCONV, "fixed point did not converge in %d iterations (interval %d)",
                     o.maxit, h->intervals);
  }
  VP_TRY(S.post());
  ++h->intervals;
  return VP_OK;
}
}  // namespace

vp_status vp_hyper_create(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                          const vp_hyper_opts* opts, vp_hyper** out) {
  void* stream = nullptr;
  VP_ENTER();
  VP_NO_COMM();
  if (!out || !opts) return vp_fail(ctx, VP_EINVAL, "null pointer");
  *out = nullptr;
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  const vp_hyper_opts& o = *opts;
  if (o.nsub < n || o.nsub > p || !o.sub_idx)
    return vp_fail(ctx, VP_EINVAL, "subsample of %d outside [n, p] = [%d, %d] or no indices", o.nsub,
                   n, p);
  if (o.dim < 1 || !o.eta) return vp_fail(ctx, VP_EINVAL, "parameters eta (p x dim) are required");
  if (o.T < 1 || (int64_t)o.T * o.nsub > 256)
    return vp_fail(ctx, VP_EUNSUPPORTED, "window T = %d with p* = %d: need T >= 1, p* T <= 256", o.T,
                   o.nsub);
  const int m = (o.T + 1) * o.nsub;
  if (o.d < 1 || o.d > 128 || o.d > m || (int64_t)m * o.d > 25600 || o.d > N)
    return vp_fail(ctx, VP_EINVAL, "d = %d outside [1, min(p* (T+1), 128, N)] or m d > 25600", o.d);
  if (o.n_up < 0 || o.n_up > o.d || o.k_deim < 1)
    return vp_fail(ctx, VP_EINVAL, "n_up outside [0, d] or k_deim < 1");
  if (o.r_max < 1 || o.r_max > 64 || !(o.dmd_tol >= 0.0))
    return vp_fail(ctx, VP_EINVAL, "r_max outside [1, 64] or dmd_tol < 0");
  if ((int64_t)o.nsub * (o.nsub + o.r_max) * 8 > 200 * 1024)
    return vp_fail(ctx, VP_EUNSUPPORTED, "RBF system of p* = %d too large", o.nsub);
  auto* h = new vp_hyper();
  h->ctx = ctx;
  h->grid = *grid;
  h->g = make_gridc(*grid, N);
  h->N = N;
  h->n = n;
  h->p = p;
  h->nsub = o.nsub;
  h->dim = o.dim;
  h->T = o.T;
  h->d = o.d;
  h->n_up = o.n_up;
  h->k_deim = o.k_deim;
  h->r_max = o.r_max;
  h->dmd_tol = o.dmd_tol;
  const int q = o.nsub, Nx = grid->Nx, n2 = 2 * n, rm = o.r_max;
  const size_t scratch = dmd_fit_scratch(Nx, o.T * q, rm);
  const size_t scratch_deim = std::max(deim_basis_scratch(ctx->num_sms, N, m),
                                       std::max(deim_indices_scratch(ctx->num_sms, N, o.d),
                                                deim_weights_scratch(ctx->num_sms, N, o.d)));
  const size_t bytes = arena_bytes(q, 4) + arena_bytes(o.d, 4) + arena_bytes((size_t)p * o.dim, 8) +
                       arena_bytes((size_t)q * o.dim, 8) + arena_bytes(1, 8) +
                       arena_bytes((size_t)2 * (o.T + 1) * q * Nx, 8) +
                       arena_bytes((size_t)(o.T + 1) * q * N, 8) + 2 * arena_bytes((size_t)rm * Nx, 8) +
                       2 * arena_bytes((size_t)rm * rm, 8) + arena_bytes((size_t)q * rm, 8) +
                       arena_bytes((size_t)p * rm, 8) + 2 * arena_bytes((size_t)p * Nx, 8) +
                       2 * arena_bytes((size_t)o.d * N, 8) + arena_bytes(o.d, 8) +
                       arena_bytes((size_t)o.d * n2, 8) + arena_bytes(scratch, 8) +
                       arena_bytes(scratch_deim, 8);
  cudaError_t e = cudaMalloc(&h->mem, bytes);
  if (e != cudaSuccess) {
    delete h;
    return vp_cuda_check(ctx, e, "cudaMalloc (DMD-DEIM state)");
  }
  Arena a{(char*)h->mem, 0, bytes};
  h->sub = a.take<int32_t>(q);
  h->idx = a.take<int32_t>(o.d);
  h->eta = a.take<double>((size_t)p * o.dim);
  h->eta_s = a.take<double>((size_t)q * o.dim);
  h->eps = a.take<double>(1);
  h->phi_ring = a.take<double>((size_t)2 * (o.T + 1) * q * Nx);
  h->y_ring = a.take<double>((size_t)(o.T + 1) * q * N);
  h->B = a.take<double>((size_t)rm * Nx);
  h->Bp = a.take<double>((size_t)rm * Nx);
  h->A = a.take<double>((size_t)rm * rm);
  h->S = a.take<double>((size_t)rm * rm);
  h->beta_s = a.take<double>((size_t)q * rm);
  h->beta = a.take<double>((size_t)p * rm);
  h->phi_half = a.take<double>((size_t)p * Nx);
  h->F = a.take<double>((size_t)p * Nx);
  h->Psi = a.take<double>((size_t)o.d * N);
  h->Psi_prev = a.take<double>((size_t)o.d * N);
  h->c = a.take<double>(o.d);
  h->Qd = a.take<double>((size_t)o.d * n2);
  h->scratch = a.take<char>(scratch);
  h->scratch_deim = a.take<char>(scratch_deim);
  e = cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->side2, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_data, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_deim, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_dmd, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    if (h->ev_deim) cudaEventDestroy(h->ev_deim);
    if (h->ev_data) cudaEventDestroy(h->ev_data);
    if (h->side2) cudaStreamDestroy(h->side2);
    if (h->side) cudaStreamDestroy(h->side);
    cudaFree(h->mem);
    delete h;
    return vp_cuda_check(ctx, e, "DMD-DEIM streams and events");
  }
  e = cudaMemcpyAsync(h->sub, o.sub_idx, sizeof(int32_t) * q, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->eta, o.eta, sizeof(double) * p * o.dim, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->phi_half, 0, sizeof(double) * p * Nx, st);
  if (e == cudaSuccess) {
    k_gather_eta<<<1, 256, 0, st>>>(o.dim, q, h->sub, h->eta, p, h->eta_s, ctx->d_status);
    rbf_width_run(o.dim, q, h->eta_s, h->eps, st);
    e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaEventDestroy(h->ev_dmd);
    cudaEventDestroy(h->ev_deim);
    cudaEventDestroy(h->ev_data);
    cudaStreamDestroy(h->side2);
    cudaStreamDestroy(h->side);
    cudaFree(h->mem);
    delete h;
    return vp_cuda_check(ctx, e, "DMD-DEIM set-up");
  }
  *out = h;
  return VP_OK;
}

vp_status vp_hyper_step(vp_hyper* h, double* Q, double* Z, double dt, int32_t nsteps,
                        const vp_step_opts* opts, double* trace, int32_t* iters, double* kstate,
                        void* stream) {
  if (!h) return VP_EINVAL;
  vp_ctx* ctx = h->ctx;
  VP_ENTER();
  VP_NO_COMM();
  if (!Q || !Z) return vp_fail(ctx, VP_EINVAL, "Q and Z are required");
  if (nsteps < 0 || !std::isfinite(dt)) return vp_fail(ctx, VP_EINVAL, "nsteps < 0 or dt not finite");
  vp_step_opts o{1e-9, 100, 0, 1e-3, 1e-2, 1, 0, 0, nullptr};
  if (opts) o = *opts;
  if (!(o.tol >= 0.0) || o.maxit < 1) return vp_fail(ctx, VP_EINVAL, "tol < 0 or maxit < 1");
  if (o.arith < 1 || o.arith > 2)
    return vp_fail(ctx, VP_EUNSUPPORTED, "the DMD-DEIM step needs arith 1 or 2");
  if (o.freeze_basis) return vp_fail(ctx, VP_EUNSUPPORTED, "the DMD-DEIM step evolves the basis");
  const int n = h->n, p = h->p;
  if ((int64_t)4 * n * n + (int64_t)2 * n * p > 25600)
    return vp_fail(ctx, VP_EUNSUPPORTED, "4n^2 + 2n p exceeds 25600");
  o.nsub = h->nsub;
  o.sub_idx = h->sub;
  Red R;
  VP_TRY(red_setup(ctx, &h->grid, h->N, n, p, 0, st, R, true, h->nsub));
  DFStep S(ctx, R, Q, Z, dt, o, kstate, st);
  const int64_t tstride = (int64_t)p * 2;
  int round = 4;
  for (int step = 0; step < nsteps; ++step) {
    int its = 0;
    VP_TRY(hyper_interval(h, R, S, trace ? trace + step * tstride : nullptr, round, &its));
    if (iters)
      VP_CUDA(cudaMemcpyAsync(iters + step, R.w.flags + 1, sizeof(int), cudaMemcpyDeviceToDevice, st));
    round = its > 2 ? its : 2;
  }
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_hyper_info(vp_hyper* h, int32_t* intervals, int32_t* hyper_intervals, int32_t* r_dmd,
                        int32_t* idx, double* Phi, void* stream) {
  if (!h) return VP_EINVAL;
  vp_ctx* ctx = h->ctx;
  VP_ENTER();
  if (intervals) *intervals = h->intervals;
  if (hyper_intervals) *hyper_intervals = h->hyper_intervals;
  if (r_dmd) *r_dmd = h->r;
  if (idx) VP_CUDA(cudaMemcpyAsync(idx, h->idx, sizeof(int32_t) * h->d, cudaMemcpyDeviceToDevice, st));
  if (Phi)
    VP_CUDA(cudaMemcpyAsync(Phi, h->phi_half, sizeof(double) * h->p * h->grid.Nx,
                            cudaMemcpyDeviceToDevice, st));
  return VP_OK;
}

vp_status vp_hyper_destroy(vp_hyper* h) {
  if (!h) return VP_OK;
  {
    std::lock_guard<std::mutex> lock(h->ctx->mu);
    DeviceGuard guard(h->ctx->device);
    cudaStreamSynchronize(h->side);
    cudaStreamSynchronize(h->side2);
    cudaEventDestroy(h->ev_dmd);
    cudaEventDestroy(h->ev_deim);
    cudaEventDestroy(h->ev_data);
    cudaStreamDestroy(h->side2);
    cudaStreamDestroy(h->side);
    cudaFree(h->mem);
  }
  delete h;
  return VP_OK;
}

// ------------------------------------------------------------------ tuning
vp_status vp_ctx_set_comm(vp_ctx* ctx, const vp_comm* comm) {
  if (!ctx) return VP_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  if (!comm) {
    ctx->comm_on = false;
    ctx->comm = vp_comm{};
    return VP_OK;
  }
  if (!comm->sum_f64 || !comm->sum_u64 || comm->n_global < 1)
    return vp_fail(ctx, VP_EINVAL, "communicator needs sum_f64, sum_u64 and n_global >= 1");
  ctx->comm = *comm;
  ctx->comm_on = true;
  ctx->comm_failed = false;
  return VP_OK;
}

vp_status vp_tensor_cores(vp_ctx* ctx, int32_t mask) {
  if (!ctx || mask < 0 || mask > VP_TC_ALL) return VP_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->tensor_cores = mask;
  return VP_OK;
}

vp_status vp_tune_set(vp_ctx* ctx, int32_t knob, int32_t blocks_per_sm) {
  if (!ctx || knob < 0 || knob >= TUNE_COUNT || blocks_per_sm < 1 || blocks_per_sm > 32)
    return VP_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->tune[knob] = blocks_per_sm;
  return VP_OK;
}

vp_status vp_tune_get(vp_ctx* ctx, int32_t knob, int32_t* blocks_per_sm) {
  if (!ctx || knob < 0 || knob >= TUNE_COUNT || !blocks_per_sm) return VP_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  *blocks_per_sm = ctx->tune[knob];
  return VP_OK;
}

// Times each FP32-based particle kernel at candidate grid sizes on the
// caller's state (one field evaluation sets up the cell indices and the
// field) and keeps the fastest per knob.  Reads Q and Z only.
vp_status vp_autotune(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                      const double* Q, const double* Z, int32_t arith, int32_t reps,
                      int32_t* chosen, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z) return vp_fail(ctx, VP_EINVAL, "Q and Z are required");
  if (arith < 1 || arith > 2) return vp_fail(ctx, VP_EINVAL, "arith must be 1 or 2");
  if (reps < 1 || reps > 1000) return vp_fail(ctx, VP_EINVAL, "reps outside [1, 1000]");
  static const int cand[] = {1, 2, 3, 4, 6, 8};
  const int ncand = 6;
  const int saved[TUNE_COUNT] = {ctx->tune[0], ctx->tune[1], ctx->tune[2], ctx->tune[3], ctx->tune[4]};
  const uint64_t mask = ctx->prof_mask;
  ctx->prof_mask = 0;
  // workspace for the largest grids
  for (int k = 0; k < TUNE_COUNT; ++k) ctx->tune[k] = cand[ncand - 1];
  Red R;
  vp_status s = red_setup(ctx, grid, N, n, p, 0, st, R, true);
  for (int k = 0; k < TUNE_COUNT; ++k) ctx->tune[k] = saved[k];
  if (s != VP_OK) {
    ctx->prof_mask = mask;
    return s;
  }
  RedWS& w = R.w;
  RedDF D{R, ctx, st, N, n, p, arith};
  D.split(Q, w.Q2a);
  D.field(w.Q2a, Z, nullptr);  // cell indices, (q/m) F, Z2, Zh2 at (Q, Z)
  VP_CUDA(cudaMemsetAsync(w.C, 0, sizeof(double2) * 4 * n * n, st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  VP_CUDA(cudaEventCreate(&e0));
  VP_CUDA(cudaEventCreate(&e1));
  const int chunks = project_chunks(p, grid->Nx);
  int best_all[TUNE_COUNT];
  for (int knob = 0; knob < TUNE_COUNT; ++knob) {
    float best = 1e30f;
    int bestc = saved[knob];
    for (int ci = 0; ci < ncand; ++ci) {
      ctx->tune[knob] = cand[ci];
      LpArgs a = D.base();
      auto launch = [&]() {
        switch (knob) {
          case TUNE_DEPOSIT:
            a.v0 = w.Q2a;
            a.v1 = w.Zh2;
            a.counts = w.counts;
            a.j = w.jcell;
            lp_launch(arith, LP_DEPOSIT, a, st);
            break;
          case TUNE_PROJECT:
            a.v0 = w.Q2a;
            a.v1 = w.F2;
            a.j = w.jcell;
            a.part = w.part;
            a.gridx = grid_bps(ceil_div(N, TILE_ROWS), chunks, cand[ci], ctx->num_sms);
            lp_launch(arith, LP_PROJECT, a, st);
            break;
          case TUNE_BASIS_M:
            a.v0 = w.Q2a;
            a.v1 = w.Z2;
            a.v2 = w.F2;
            a.v3 = w.frows[0];
            a.j = w.jcell;
            lp_launch(arith, LP_BASIS_M, a, st);
            break;
          case TUNE_GRAM:
            a.gram.blk[0] = w.Q2a;
            a.gram.blk[1] = w.frows[1];
            a.gram.nblk = 2;
            a.gram.pa[0] = 0;
            a.gram.pb[0] = 1;
            a.gram.pa[1] = 1;
            a.gram.pb[1] = 1;
            a.gram.npairs = 2;
            a.part = w.part;
            a.gridx = grid_bps(ceil_div(N, 32), 1, cand[ci], ctx->num_sms);
            lp_launch(arith, LP_GRAM, a, st);
            break;
          default:
            a.aff.X[0] = w.Q2a;
            a.aff.X[1] = w.frows[1];
            a.aff.nterms = 2;
            a.C = w.C;
            a.v0 = w.frows[2];
            lp_launch(arith, LP_AFFINE, a, st);
            break;
        }
      };
      launch();  // warm-up
      VP_CUDA(cudaEventRecord(e0, st));
      for (int r = 0; r < reps; ++r) launch();
      VP_CUDA(cudaEventRecord(e1, st));
      VP_CUDA(cudaEventSynchronize(e1));
      VP_LAUNCHED();
      float ms = 0.f;
      VP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) {
        best = ms;
        bestc = cand[ci];
      }
    }
    ctx->tune[knob] = bestc;
    best_all[knob] = bestc;
  }
  VP_CUDA(cudaMemsetAsync(w.counts, 0, sizeof(unsigned long long) * p * grid->Nx, st));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->prof_mask = mask;
  if (chosen)
    for (int k = 0; k < TUNE_COUNT; ++k) chosen[k] = best_all[k];
  return VP_OK;
}

// ------------------------------------------------ per-instance step objects
// The batched engine (batch.cu) drives one of these per instance; each owns
// its workspace (in its context) and issues the same kernels as
// vp_basis_update with arith 1 or 2.
struct InstanceStep {
  Red R;
  DFStep* S = nullptr;
};

vp_status step_setup(vp_ctx* ctx, const vp_grid* grid, int64_t N, int n, int p, double* Q,
                     double* Z, double dt, const vp_step_opts* opts, double* kstate,
                     cudaStream_t st, InstanceStep** out) {
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !out) return vp_fail(ctx, VP_EINVAL, "Q, Z and out are required");
  if (!std::isfinite(dt)) return vp_fail(ctx, VP_EINVAL, "dt not finite");
  if (!opts || opts->arith < 1 || opts->arith > 2)
    return vp_fail(ctx, VP_EINVAL, "batched steps need arith 1 or 2");
  if ((int64_t)4 * n * n + (int64_t)2 * n * p > 25600)
    return vp_fail(ctx, VP_EUNSUPPORTED, "4n^2 + 2n p exceeds 25600");
  InstanceStep* is = new InstanceStep();
  if (opts->nsub != 0 && (opts->nsub < n || opts->nsub > p || !opts->sub_idx)) {
    delete is;
    return vp_fail(ctx, VP_EINVAL, "subsample outside [n, p] or no indices");
  }
  vp_status s = red_setup(ctx, grid, N, n, p, 0, st, is->R, true, opts->nsub, opts->arith == 2);
  if (s != VP_OK) {
    delete is;
    return s;
  }
  is->S = new DFStep(ctx, is->R, Q, Z, dt, *opts, kstate, st);
  *out = is;
  return VP_OK;
}
vp_status step_pre(InstanceStep* is, double* trace_step) { return is->S->pre(trace_step); }
vp_status step_rounds(InstanceStep* is, int count) { return is->S->rounds(count); }
vp_status step_post(InstanceStep* is) { return is->S->post(); }
int* step_flags(InstanceStep* is) { return is->R.w.flags; }
void step_free(InstanceStep* is) {
  if (!is) return;
  delete is->S;
  delete is;
}

// ============================================================== profiling
static const char* kKernelNames[VP_K_COUNT] = {
    "k_deposit", "k_counts_to_rho", "k_poisson", "k_gather", "k_full_step", "k_reconstruct",
    "k_deposit_reduced", "k_project", "k_basis_M", "k_gram", "k_gram_real", "k_reduce_partials",
    "k_affine", "k_cell_gradient", "k_small_basis_coeffs", "k_small_cayley", "k_small_tangent",
    "k_coeff_update", "k_axpy", "k_add_linear", "k_energies", "k_split", "k_deposit_lp",
    "k_project_lp", "k_basis_M_lp", "k_prep_lp", "k_gram_lp", "k_gram_real_lp", "k_affine_lp",
    "k_init", "k_load", "k_subset", "k_hyper", "k_deim_round", "k_deim", "k_dmd",
    "k_jacobi_sym", "k_deposit_lp_diag", "k_project_tc", "k_deposit_tc", "k_gram_tc",
    "k_basis_M_tc", "k_affine_tc"};

static cudaEvent_t take_event(vp_ctx* ctx) {
  if (ctx->event_pool.empty()) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = ctx->event_pool.back();
  ctx->event_pool.pop_back();
  return e;
}

void vp_prof_begin(vp_ctx* ctx, int id, cudaStream_t st, cudaEvent_t* a) {
  ctx->launches[id] += 1;
  *a = nullptr;
  if (!(ctx->prof_mask >> id & 1ull)) return;
  if (ctx->pending.size() > 4096) vp_prof_collect(ctx);
  *a = take_event(ctx);
  if (*a) cudaEventRecord(*a, st);
}

void vp_prof_end(vp_ctx* ctx, int id, cudaStream_t st, cudaEvent_t a) {
  if (!a) return;
  cudaEvent_t b = take_event(ctx);
  if (!b) {
    ctx->event_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, st);
  ctx->pending.push_back({id, a, b});
}

void vp_prof_collect(vp_ctx* ctx) {
  for (auto& q : ctx->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(q.b) == cudaSuccess && cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      ctx->ms[q.id] += ms;
      ctx->timed[q.id] += 1;
    }
    ctx->event_pool.push_back(q.a);
    ctx->event_pool.push_back(q.b);
  }
  ctx->pending.clear();
  (void)cudaGetLastError();
}

// ================================================================ context
// Rank at t = 0 (reading of the paper's constant-rank observation): the
// smallest n in [n_min, n_max] whose relative tail energy
// sum_{j>n} sigma_j^2 / sum_j sigma_j^2 is below tol (n_max if none), then
// lowered while sigma_n < 1e-6 sigma_1 (even below n_min): S(Z) = Z Z^T then
// has condition number <= 1e12, and sigma_n stays above the resolution of
// singular values taken from the Gram matrix R0^H R0 (~1e-8 sigma_1).
// Returns 0 when all singular values vanish.
int vp_choose_rank(const double* sig, int p, int n_min, int n_max, double tol) {
  n_max = std::min(n_max, p);
  double total = 0.0;
  for (int k = 0; k < p; ++k) total += sig[k] * sig[k];
  if (!(total > 0.0)) return 0;
  int n = n_max;
  double tail = total;
  for (int k = 1; k <= n_max; ++k) {
    tail -= sig[k - 1] * sig[k - 1];
    if (k >= n_min && tail < tol * total) {
      n = k;
      break;
    }
  }
  while (n > 0 && !(sig[n - 1] >= 1e-6 * sig[0])) --n;
  return n;
}

namespace {
size_t init_ws_bytes(int sms, int64_t N, int p, int n, int* gx_out) {
  const int64_t pp = (int64_t)p * p;
  int gx = ceil_div(N, 32);
  int gmax = (int)std::max<int64_t>(1, (64ll << 20) / (pp * 16));  // partials <= 64 MiB
  gx = std::min(gx, std::min(2 * sms, gmax));
  if (gx_out) *gx_out = gx;
  const int nn = n * n;
  return arena_bytes((size_t)gx * pp, 16) + 4 * arena_bytes(pp, 16) + arena_bytes(p, 8) +
         arena_bytes((size_t)p * n, 16) + 2 * arena_bytes(nn, 16) + arena_bytes(n, 8) +
         arena_bytes((size_t)gx * n * p, 16) + arena_bytes((size_t)n * p, 16) +
         arena_bytes((size_t)N * 2 * n, 8) + arena_bytes(4 * nn, 16) +
         arena_bytes((size_t)2 * sms * 4 * nn, 16);
}
}  // namespace

// Workspace one serving query needs: the larger of the start and the steps.
size_t vp_query_ws_bytes(int sms, int64_t N, int n, int p, int Nx, int arith) {
  const bool df = arith != 0;
  return std::max(init_ws_bytes(sms, N, p, n, nullptr),
                  red_ws_bytes(sms, N, n, p, Nx, df ? 0 : 5, df, nullptr, nullptr, nullptr, 0,
                               arith == 2));
}

// Free a context's workspace arena (synchronises the device).
void vp_workspace_release(vp_ctx* ctx) {
  if (!ctx || !ctx->ws) return;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
}

extern "C" {

vp_status vp_profile_enable(vp_ctx* ctx, uint64_t mask) {
  if (!ctx) return VP_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  ctx->prof_mask = mask;
  return VP_OK;
}

vp_status vp_profile_read(vp_ctx* ctx, int32_t kernel, int64_t* launches, int64_t* timed,
                          double* ms_total) {
  if (!ctx || kernel < 0 || kernel >= VP_K_COUNT) return VP_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard guard(ctx->device);
  vp_prof_collect(ctx);
  if (launches) *launches = ctx->launches[kernel];
  if (timed) *timed = ctx->timed[kernel];
  if (ms_total) *ms_total = ctx->ms[kernel];
  return VP_OK;
}

vp_status vp_profile_reset(vp_ctx* ctx) {
  if (!ctx) return VP_EINVAL;
  std::lock_guard<std::mutex> lock(ctx->mu);
  DeviceGuard guard(ctx->device);
  vp_prof_collect(ctx);
  for (int k = 0; k < VP_K_COUNT; ++k) {
    ctx->launches[k] = 0;
    ctx->timed[k] = 0;
    ctx->ms[k] = 0.0;
  }
  return VP_OK;
}

const char* vp_kernel_name(int32_t kernel) {
  return (kernel >= 0 && kernel < VP_K_COUNT) ? kKernelNames[kernel] : "unknown";
}


int32_t vp_version(void) { return 10000; }

const char* vp_status_string(vp_status s) {
  switch (s) {
    case VP_OK: return "ok";
    case VP_EINVAL: return "invalid argument";
    case VP_ENOMEM: return "out of memory / over budget";
    case VP_EBUSY: return "busy";
    case VP_EAGAIN: return "not ready";
    case VP_ETIMEDOUT: return "timed out";
    case VP_ENOCONV: return "fixed point did not converge";
    case VP_ENUMERIC: return "non-finite value or singular system";
    case VP_EDRIFT: return "basis left the ortho-symplectic manifold";
    case VP_ECUDA: return "CUDA error";
    case VP_EUNSUPPORTED: return "unsupported size or call";
    case VP_ECOMM: return "sum over the ranks failed";
  }
  return "unknown status";
}

vp_status vp_ctx_create(vp_ctx** out, int device, size_t scratch_bytes) {
  if (!out) return VP_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return VP_ECUDA;
  vp_ctx* ctx = new vp_ctx();
  ctx->device = device;
  ctx->budget = scratch_bytes ? scratch_bytes : (size_t(16) << 30);
  DeviceGuard guard(device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (cudaMalloc(&ctx->d_status, 64) != cudaSuccess ||
      cudaMallocHost(&ctx->h_pinned, 64) != cudaSuccess) {
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return VP_ENOMEM;
  }
  cudaMemset(ctx->d_status, 0, 64);
  memset(ctx->h_pinned, 0, 64);
  pic_init();
  reduced_init();
  dense_init();
  df_init();
  tc_init();
  tc_deposit_init();
  tc_gram_init();
  tc_rows_init();
  init_kernels_init();
  deim_init();
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_pinned);
    delete ctx;
    return VP_ECUDA;
  }
  *out = ctx;
  return VP_OK;
}

vp_status vp_ctx_destroy(vp_ctx* ctx) {
  if (!ctx) return VP_EINVAL;
  {
    DeviceGuard guard(ctx->device);
    cudaDeviceSynchronize();
    vp_prof_collect(ctx);
    for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  }
  delete ctx;
  return VP_OK;
}

const char* vp_last_error(const vp_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

size_t vp_ctx_workspace_bytes(const vp_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

vp_status vp_ctx_sync_status(vp_ctx* ctx, void* stream) {
  VP_ENTER();
  VP_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  VP_CUDA(cudaMemsetAsync(ctx->d_status, 0, sizeof(int), st));
  VP_CUDA(cudaStreamSynchronize(st));
  int s = ctx->h_pinned[0];
  if (s != 0) return vp_fail(ctx, (vp_status)s, "device reported: %s", vp_status_string((vp_status)s));
  return VP_OK;
}

// ======================================================= particle-grid maps
vp_status vp_deposit_cic(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, const double* X,
                         int64_t ldx, double* rho, void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  if (!X || !rho || ldx < N) return vp_fail(ctx, VP_EINVAL, "null pointer or ldx < N");
  GridC g = make_gridc(*grid, N);
  void* base;
  size_t cb = sizeof(unsigned long long) * p * grid->Nx;
  VP_TRY(vp_workspace(ctx, cb, &base));
  auto* counts = (unsigned long long*)base;
  VP_CUDA(cudaMemsetAsync(counts, 0, cb, st));
  VP_K(VP_K_DEPOSIT, deposit_samples(g, N, p, X, ldx, counts, ctx->num_sms, st));
  VP_K(VP_K_RHO, counts_to_rho(g, p, counts, rho, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_poisson_periodic(vp_ctx* ctx, const vp_grid* grid, int32_t p, const double* rho,
                              double* phi, double* F, double* energy, void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, 1, p));
  if (!rho || !F) return vp_fail(ctx, VP_EINVAL, "rho and F are required");
  GridC g = make_gridc(*grid, 1);
  VP_K(VP_K_POISSON, poisson(g, p, rho, nullptr, phi, F, energy, nullptr, nullptr, ctx->d_status, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_gather_E(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, const double* X,
                      int64_t ldx, const double* F, const int32_t* idx, int64_t d, double* GX,
                      void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  if (!X || !F || !GX || ldx < N) return vp_fail(ctx, VP_EINVAL, "null pointer or ldx < N");
  if (idx && (d < 1 || d > N)) return vp_fail(ctx, VP_EINVAL, "d = %lld outside [1, N]", (long long)d);
  GridC g = make_gridc(*grid, N);
  VP_K(VP_K_GATHER, gather(g, N, p, X, ldx, F, idx, d, GX, ctx->num_sms, ctx->d_status, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_full_step(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, double* X, double* V,
                       double dt, int32_t nsteps, double* trace, void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  if (!X || !V) return vp_fail(ctx, VP_EINVAL, "X and V are required");
  if (nsteps < 0 || !std::isfinite(dt)) return vp_fail(ctx, VP_EINVAL, "nsteps < 0 or dt not finite");
  if (nsteps == 0) return VP_OK;
  GridC g = make_gridc(*grid, N);
  cudaError_t fe = cudaSuccess;
  VP_K(VP_K_FULL_STEP, fe = full_step(g, N, p, X, V, dt, nsteps, trace, ctx->d_status, st));
  VP_CUDA(fe);
  VP_LAUNCHED();
  return VP_OK;
}

// ============================================================ reduced model
vp_status vp_reconstruct(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q,
                         const double* Z, double* X, double* V, void* stream) {
  VP_ENTER();
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !X) return vp_fail(ctx, VP_EINVAL, "Q, Z and X are required");
  VP_K(VP_K_RECONSTRUCT, reconstruct(N, n, p, Q, Z, X, V, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_project_grad(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q,
                          const double* GX, const double* Z, double* g_out, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !g_out) return vp_fail(ctx, VP_EINVAL, "Q, Z and g are required");
  Red R;
  vp_grid dummy{3, 1.0, 0.0, 1.0, 0.0};
  VP_TRY(red_setup(ctx, &dummy, N, n, p, 0, st, R));
  if (GX) {
    VP_K(VP_K_PROJECT, project(R.g, N, n, p, Q, Z, nullptr, GX, N, nullptr, nullptr, N, R.w.part, R.w.gx_proj,
            nullptr, ctx->d_status, st));
    VP_K(VP_K_REDUCE, reduce_partials(R.w.gx_proj, (int64_t)2 * n * p, R.w.part, R.w.gX, nullptr, st));
  }
  R.gv(Q, R.w.GVraw);
  VP_K(VP_K_ADD_LINEAR, add_linear(n, p, GX ? R.w.gX : nullptr, R.w.GVraw, Z, g_out, st));
  VP_LAUNCHED();
  return VP_OK;
}

// ------------------------------------------------- typed per-step calls
static vp_status check_dtype(vp_ctx* ctx, int32_t dtype, std::initializer_list<const void*> ptrs) {
  if (dtype < VP_F64 || dtype > VP_BF16) return vp_fail(ctx, VP_EINVAL, "dtype %d", dtype);
  const uintptr_t a = (uintptr_t)vp_dtype_size(dtype);
  for (const void* q : ptrs)
    if (q && ((uintptr_t)q % a)) return vp_fail(ctx, VP_EINVAL, "pointer not aligned to its dtype");
  return VP_OK;
}

vp_status vp_deposit_cic_t(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, const void* X,
                           int64_t ldx, int32_t dtype, double* rho, int32_t flags, void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  if (!X || !rho || ldx < N) return vp_fail(ctx, VP_EINVAL, "null pointer or ldx < N");
  if (flags & ~VP_DEPOSIT_FIXEDPOINT) return vp_fail(ctx, VP_EINVAL, "unknown deposit flags");
  VP_TRY(check_dtype(ctx, dtype, {X}));
  GridC g = make_gridc(*grid, N);
  void* base;
  size_t cb = sizeof(unsigned long long) * p * grid->Nx;
  VP_TRY(vp_workspace(ctx, cb, &base));
  auto* counts = (unsigned long long*)base;
  VP_CUDA(cudaMemsetAsync(counts, 0, cb, st));
  VP_K(VP_K_DEPOSIT, deposit_typed(g, N, p, X, ldx, dtype, counts, ctx->num_sms, st));
  VP_K(VP_K_RHO, counts_to_rho(g, p, counts, rho, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_gather_E_t(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, const void* X,
                        int64_t ldx, int32_t dtype, const double* F, const int32_t* idx, int64_t d,
                        void* GX, void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  if (!X || !F || !GX || ldx < N) return vp_fail(ctx, VP_EINVAL, "null pointer or ldx < N");
  if (idx && (d < 1 || d > N)) return vp_fail(ctx, VP_EINVAL, "d = %lld outside [1, N]", (long long)d);
  VP_TRY(check_dtype(ctx, dtype, {X, GX}));
  GridC g = make_gridc(*grid, N);
  VP_K(VP_K_GATHER, gather_typed(g, N, p, X, ldx, dtype, F, idx, d, GX, ctx->num_sms,
                                 ctx->d_status, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_reconstruct_t(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const void* Q,
                           int64_t ldq, int32_t dtype, const double* Z, void* X, void* V,
                           int64_t ldx, void* stream) {
  VP_ENTER();
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !X) return vp_fail(ctx, VP_EINVAL, "Q, Z and X are required");
  if (ldq < 2 * n || ldx < N) return vp_fail(ctx, VP_EINVAL, "ldq < 2n or ldx < N");
  VP_TRY(check_dtype(ctx, dtype, {Q, X, V}));
  VP_K(VP_K_RECONSTRUCT, reconstruct_typed(N, n, p, Q, ldq, dtype, Z, X, V, ldx, ctx->num_sms, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_project_grad_t(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const void* Q,
                            int64_t ldq, int32_t dtype, const void* GX, int64_t ldg,
                            const double* Z, double* g_out, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !g_out) return vp_fail(ctx, VP_EINVAL, "Q, Z and g are required");
  if (ldq < 2 * n || (GX && ldg < N)) return vp_fail(ctx, VP_EINVAL, "ldq < 2n or ldg < N");
  VP_TRY(check_dtype(ctx, dtype, {Q, GX}));
  const int n2 = 2 * n, ch = ceil_div(p, 32);
  const int gp = typed_grid_x(N, ch, ctx->num_sms), gg = typed_grid_x(N, 1, ctx->num_sms);
  const size_t zsz = (size_t)n2 * p, gsz = (size_t)n2 * n2;
  const size_t part = std::max((size_t)gp * zsz, (size_t)gg * gsz);
  void* base;
  VP_TRY(vp_workspace(ctx, sizeof(double) * (part + zsz + gsz), &base));
  double* P = (double*)base;
  double* gX = P + part;
  double* GV = gX + zsz;
  if (GX) {
    VP_K(VP_K_PROJECT, project_typed(N, n, p, Q, ldq, dtype, GX, ldg, P, gp, st));
    VP_K(VP_K_REDUCE, reduce_partials(gp, (int64_t)zsz, P, gX, nullptr, st));
  }
  VP_K(VP_K_GRAM_REAL, gram_real_typed(N, n2, Q, ldq, dtype, P, gg, st));
  VP_K(VP_K_REDUCE, reduce_partials(gg, (int64_t)gsz, P, GV, nullptr, st));
  VP_K(VP_K_ADD_LINEAR, add_linear(n, p, GX ? gX : nullptr, GV, Z, g_out, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_basis_velocity(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                            const double* Q, const double* Z, double* Xi, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !Xi) return vp_fail(ctx, VP_EINVAL, "Q, Z and Xi are required");
  Red R;
  VP_TRY(red_setup(ctx, grid, N, n, p, 1, st, R));
  R.field(Q, Z);
  R.basis_velocity_from_field(Q, Z, 1.0, R.w.rows[0], Xi);
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_cayley_retract(vp_ctx* ctx, int64_t N, int32_t n, const double* Q0, const double* xi,
                            double* Qout, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_np(ctx, N, 1));
  VP_TRY(check_n(ctx, n, N));
  if (!Q0 || !xi || !Qout) return vp_fail(ctx, VP_EINVAL, "Q0, xi and Qout are required");
  Red R;
  VP_TRY(red_setup(ctx, nullptr, N, n, 1, 0, st, R));
  R.cayley(Q0, xi, Qout);
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_tangent_velocity(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                              const double* Q0, const double* xi, const double* Z, double* Y,
                              void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q0 || !xi || !Z || !Y) return vp_fail(ctx, VP_EINVAL, "Q0, xi, Z and Y are required");
  Red R;
  VP_TRY(red_setup(ctx, grid, N, n, p, 3, st, R));
  double *Qh = R.w.rows[0], *M = R.w.rows[1], *Xp = R.w.rows[2];
  R.cayley(Q0, xi, Qh);
  R.field(Qh, Z);
  R.basis_velocity_from_field(Qh, Z, 1.0, M, Xp);
  R.tangent(Q0, xi, Qh, Xp, 1.0, Y);
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_reduced_energy(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                            const double* Q, const double* Z, double* E, double* H, double* resid,
                            void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z) return vp_fail(ctx, VP_EINVAL, "Q and Z are required");
  if (ctx->comm_on && N > ctx->comm.n_global)
    return vp_fail(ctx, VP_EINVAL, "N = %lld rows exceed n_global", (long long)N);
  ctx->comm_failed = false;
  Red R;
  VP_TRY(red_setup(ctx, grid, N, n, p, 0, st, R));
  R.field(Q, Z);
  R.gv(Q, R.w.GVraw);
  if (resid) R.grams({Q}, {{0, 0}}, R.w.grams);
  VP_K(VP_K_ENERGIES, energies(n, p, R.w.GVraw, Z, R.w.Efield, E, H, 1, resid ? R.w.grams : nullptr, resid,
           ctx->d_status, st));
  VP_LAUNCHED();
  if (ctx->comm_failed) return vp_fail(ctx, VP_ECOMM, "a sum over the ranks failed");
  return VP_OK;
}

// ------------------------------------------------- accuracy diagnostics
static vp_status init_csvd_impl(vp_ctx* ctx, int64_t N, int32_t p, int32_t n_min, int32_t n_max,
                                double rank_tol, const double* X0, const double* V0, double* Q,
                                double* Z, double* sigma, int32_t* n_out, cudaStream_t st);

static vp_status rel_errors_impl(vp_ctx* ctx, int64_t N, int n, int p, const double* Q,
                                 const double* Z, const double* X, const double* V, double* eps,
                                 cudaStream_t st) {
  const int nb = diag_blocks(N, ctx->num_sms);
  const size_t bytes = arena_bytes((size_t)nb * 4, 8) + arena_bytes(4, 8);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, bytes, &base));
  Arena a{(char*)base, 0, bytes};
  double* part = a.take<double>((size_t)nb * 4);
  double* sums = a.take<double>(4);
  VP_K(VP_K_REDUCE, rel_err_parts(N, n, p, Q, Z, X, V, part, nb, st));
  VP_K(VP_K_REDUCE, reduce_partials(nb, 4, part, sums, nullptr, st));
  VP_K(VP_K_REDUCE, ratio_sqrt(2, sums, eps, st));
  return VP_OK;
}

vp_status vp_rel_errors(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q,
                        const double* Z, const double* X, const double* V, double* eps,
                        void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !X || !V || !eps) return vp_fail(ctx, VP_EINVAL, "null pointer");
  VP_TRY(rel_errors_impl(ctx, N, n, p, Q, Z, X, V, eps, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_target_errors(vp_ctx* ctx, int64_t N, int32_t p, int32_t n, const double* X,
                           const double* V, double* eps, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_np(ctx, N, p));
  if (n < 1 || n > 40 || n > p || n > N) return vp_fail(ctx, VP_EINVAL, "n outside [1, min(p, N, 40)]");
  if (!X || !V || !eps) return vp_fail(ctx, VP_EINVAL, "null pointer");
  // the rank-n complex SVD state of the snapshots (stream-ordered buffers),
  // then the relative errors of its reconstruction
  double *Qt = nullptr, *Zt = nullptr;
  VP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&Qt), sizeof(double) * N * 2 * n, st));
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&Zt), sizeof(double) * 2 * n * p, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(Qt, st);
    return vp_cuda_check(ctx, e, "cudaMallocAsync");
  }
  int32_t nn = n;
  vp_status s = init_csvd_impl(ctx, N, p, n, n, -1.0, X, V, Qt, Zt, nullptr, &nn, st);
  if (s == VP_OK) s = rel_errors_impl(ctx, N, n, p, Qt, Zt, X, V, eps, st);
  cudaFreeAsync(Zt, st);
  cudaFreeAsync(Qt, st);
  VP_TRY(s);
  VP_LAUNCHED();
  return VP_OK;
}

static vp_status rank_indicator_impl(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n,
                                     int32_t p, const double* Q, const double* Z, double* out,
                                     cudaStream_t st) {
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !out) return vp_fail(ctx, VP_EINVAL, "null pointer");
  Red R;
  VP_TRY(red_setup(ctx, grid, N, n, p, 0, st, R));
  RedWS& w = R.w;
  const int64_t zsz = (int64_t)2 * n * p;
  R.field(Q, Z);
  VP_K(VP_K_PROJECT, project(R.g, N, n, p, Q, Z, w.F, nullptr, 0, nullptr, nullptr, N, w.part,
                             w.gx_proj, nullptr, ctx->d_status, st));
  VP_K(VP_K_REDUCE, reduce_partials(w.gx_proj, zsz, w.part, w.gX, nullptr, st));
  R.gv(Q, w.GVraw);
  VP_K(VP_K_ADD_LINEAR, add_linear(n, p, w.gX, w.GVraw, Z, w.k, st));  // g = U^T G
  const int nb = diag_blocks(N, ctx->num_sms);
  if ((int64_t)nb * 2 + 2 > (int64_t)w.gx_proj * zsz)
    return vp_fail(ctx, VP_EUNSUPPORTED, "partial buffer too small");
  VP_K(VP_K_REDUCE, normal_parts(R.g, N, n, p, Q, Z, w.F, w.k, w.part, nb, st));
  VP_K(VP_K_REDUCE, reduce_partials(nb, 2, w.part, w.aux, nullptr, st));
  VP_K(VP_K_REDUCE, ratio_sqrt(1, w.aux, out, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_rank_indicator(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                            const double* Q, const double* Z, double* out, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  return rank_indicator_impl(ctx, grid, N, n, p, Q, Z, out, st);
}

// Re-initialisation at a larger rank (Sec. 6.4): the indicator of the current
// reduced state decides on the host; the new start is the truncated complex
// SVD of the full-order states, as at t = 0.
vp_status vp_restart_csvd(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                          const double* Q, const double* Z, const double* X, const double* V,
                          double threshold, int32_t n_new, double* Q_new, double* Z_new,
                          double* indicator, int32_t* restarted, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  if (!restarted || !X || !V || !Q_new || !Z_new) return vp_fail(ctx, VP_EINVAL, "null pointer");
  if (threshold != threshold) return vp_fail(ctx, VP_EINVAL, "threshold is NaN");
  *restarted = 0;
  double* d_ind = nullptr;
  VP_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_ind), sizeof(double), st));
  vp_status s = rank_indicator_impl(ctx, grid, N, n, p, Q, Z, d_ind, st);
  double ind = 0.0;
  if (s == VP_OK) {
    cudaError_t e = cudaMemcpyAsync(&ind, d_ind, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = vp_cuda_check(ctx, e, "indicator read");
  }
  cudaFreeAsync(d_ind, st);
  VP_TRY(s);
  if (indicator) *indicator = ind;
  if (!(ind <= threshold)) {  // a NaN indicator (a broken state) restarts as well
    VP_TRY(init_csvd_impl(ctx, N, p, 1, n_new, -1.0, X, V, Q_new, Z_new, nullptr, nullptr, st));
    *restarted = 1;
  }
  return VP_OK;
}

vp_status vp_half_basis(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                        const double* Q0, const double* Z0, double dt, double* Qh, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q0 || !Z0 || !Qh) return vp_fail(ctx, VP_EINVAL, "null pointer");
  Red R;
  VP_TRY(red_setup(ctx, grid, N, n, p, 2, st, R));
  R.field(Q0, Z0);
  R.basis_velocity_from_field(Q0, Z0, 0.5 * dt, R.w.rows[0], R.w.rows[1]);
  R.cayley(Q0, R.w.rows[1], Qh);
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_hamiltonian_error_terms(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n,
                                     int32_t p, const double* Q0, const double* Z0,
                                     const double* Qh, const double* Q1, const double* Z1,
                                     double* out, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q0 || !Z0 || !Qh || !Q1 || !Z1 || !out) return vp_fail(ctx, VP_EINVAL, "null pointer");
  Red R;
  VP_TRY(red_setup(ctx, grid, N, n, p, 1, st, R));
  RedWS& w = R.w;
  // H at (U0, Z0), (U1, Z1), (U_1/2, Z0), (U_1/2, Z1) into four p-vectors
  // (in the row buffer, which neither the field nor the Grams use)
  double* hv = w.rows[0];
  if (4 * (int64_t)p > N * 2 * n) return vp_fail(ctx, VP_EUNSUPPORTED, "4 p > 2 n N");
  const double* Qs[4] = {Q0, Q1, Qh, Qh};
  const double* Zs[4] = {Z0, Z1, Z0, Z1};
  for (int k = 0; k < 4; ++k) {
    R.field(Qs[k], Zs[k]);
    R.gv(Qs[k], w.GVraw);
    VP_K(VP_K_ENERGIES, energies(n, p, w.GVraw, Zs[k], w.Efield, nullptr, hv + (int64_t)k * p, 1,
                                 nullptr, nullptr, ctx->d_status, st));
  }
  VP_K(VP_K_REDUCE, ham_terms(p, hv, hv + p, hv + 2 * p, hv + 3 * p, out, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_deim_gather_project(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                                 const double* Q, const double* Z, int64_t d, const int32_t* idx,
                                 const double* c, const double* phi, double* gX, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z || !idx || !c || !phi || !gX) return vp_fail(ctx, VP_EINVAL, "null pointer");
  if (d < 1 || d > N) return vp_fail(ctx, VP_EINVAL, "d = %lld outside [1, N]", (long long)d);
  Red R;
  VP_TRY(red_setup(ctx, grid, d, n, p, 0, st, R));
  R.g = make_gridc(*grid, N);
  VP_K(VP_K_CELL_GRADIENT, cell_gradient(R.g, p, phi, R.w.F, st));
  VP_K(VP_K_PROJECT, project(R.g, d, n, p, Q, Z, R.w.F, nullptr, 0, idx, c, N, R.w.part, R.w.gx_proj, nullptr,
          ctx->d_status, st));
  VP_K(VP_K_REDUCE, reduce_partials(R.w.gx_proj, (int64_t)2 * n * p, R.w.part, gX, nullptr, st));
  VP_LAUNCHED();
  return VP_OK;
}

// Truncated complex SVD start.  rank_tol < 0: n = n_max as given; otherwise
// the eigenvalues of R0^H R0 are copied to the host after the Jacobi sweep
// (one stream synchronisation) and n is chosen by vp_choose_rank.
static vp_status init_csvd_impl(vp_ctx* ctx, int64_t N, int32_t p, int32_t n_min, int32_t n_max,
                                double rank_tol, const double* X0, const double* V0, double* Q,
                                double* Z, double* sigma, int32_t* n_out, cudaStream_t st) {
  VP_TRY(check_np(ctx, N, p));
  if (p > 256) return vp_fail(ctx, VP_EUNSUPPORTED, "p = %d > 256", p);
  if (n_max < 1 || n_max > 40 || n_max > p || n_max > N)
    return vp_fail(ctx, VP_EINVAL, "n = %d outside [1, min(p, N, 40)]", n_max);
  if (n_min < 1 || n_min > n_max) return vp_fail(ctx, VP_EINVAL, "n_min = %d outside [1, n_max]", n_min);
  if (!X0 || !V0 || !Q || !Z) return vp_fail(ctx, VP_EINVAL, "null pointer");
  const int64_t pp = (int64_t)p * p;
  int gx = 0;
  size_t bytes = init_ws_bytes(ctx->num_sms, N, p, n_max, &gx);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, bytes, &base));
  Arena a{(char*)base, 0, bytes};
  const int nnx = n_max * n_max;
  double2* part = a.take<double2>((size_t)gx * pp);
  double2* A = a.take<double2>(pp);
  double2* Wj = a.take<double2>(pp);
  double2* Ws = a.take<double2>(pp);
  double* lam = a.take<double>(p);
  double2* Cn = a.take<double2>((size_t)p * n_max);
  double2* G = a.take<double2>(nnx);
  double2* Gs = a.take<double2>(nnx);
  double* lamG = a.take<double>(n_max);
  double2* zpart = a.take<double2>((size_t)gx * n_max * p);
  double2* zeta = a.take<double2>((size_t)n_max * p);
  double* Q0 = a.take<double>((size_t)N * 2 * n_max);
  double2* WG = a.take<double2>(4 * nnx);
  double2* gpart = a.take<double2>((size_t)2 * ctx->num_sms * 4 * nnx);
  (void)gpart;
  // 1. A = R0^H R0
  VP_K(VP_K_INIT, init_launch_rgram(N, p, X0, V0, part, gx, st));
  VP_K(VP_K_REDUCE, reduce_partials(gx, pp * 2, reinterpret_cast<double*>(part),
                                    reinterpret_cast<double*>(A), nullptr, st));
  // 2. A = W diag(lambda) W^H, lambda descending
  VP_K(VP_K_INIT, init_launch_jacobi(p, A, Wj, lam, Ws, ctx->d_status, st));
  int n = n_max;
  if (rank_tol >= 0.0) {
    std::vector<double> lh(p), sh(p);
    VP_CUDA(cudaMemcpyAsync(lh.data(), lam, sizeof(double) * p, cudaMemcpyDeviceToHost, st));
    VP_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < p; ++k) sh[k] = lh[k] > 0.0 ? std::sqrt(lh[k]) : 0.0;
    n = vp_choose_rank(sh.data(), p, n_min, n_max, rank_tol);
    if (n < 1) return vp_fail(ctx, VP_ENUMERIC, "no usable rank: the snapshot matrix is zero");
  }
  if (n_out) *n_out = n;
  const int nn = n * n;
  // 3. Q0 = R0 W_n diag(lambda_n)^-1/2
  VP_K(VP_K_INIT, init_launch_coeff(p, n, Ws, lam, Cn, ctx->d_status, st));
  VP_K(VP_K_INIT, init_launch_r_times(N, p, n, X0, V0, Cn, Q0, ctx->num_sms, st));
  // 4. Q = Q0 (Q0^H Q0)^-1/2
  {
    GramArgs ga{};
    ga.blk[0] = Q0;
    ga.nblk = 1;
    ga.pa[0] = 0;
    ga.pb[0] = 0;
    ga.npairs = 1;
    int ggx = gram_grid_x(N, ctx->num_sms);
    VP_K(VP_K_GRAM, gram(N, n, ga, gpart, ggx, st));
    VP_K(VP_K_REDUCE, reduce_partials(ggx, (int64_t)nn * 2, reinterpret_cast<double*>(gpart),
                                      reinterpret_cast<double*>(G), nullptr, st));
    VP_K(VP_K_INIT, init_launch_jacobi(n, G, WG, lamG, WG + nn, ctx->d_status, st));
    VP_K(VP_K_INIT, init_launch_inv_sqrt(n, WG + nn, lamG, Gs, ctx->d_status, st));
    AffineArgs aa{};
    aa.X[0] = Q0;
    aa.nterms = 1;
    VP_K(VP_K_AFFINE, affine(N, n, aa, Gs, Q, ctx->num_sms, st));
  }
  // 5. zeta = Q^H R0
  VP_K(VP_K_INIT, init_launch_zeta(N, p, n, Q, X0, V0, zpart, gx, st));
  VP_K(VP_K_REDUCE, reduce_partials(gx, (int64_t)n * p * 2, reinterpret_cast<double*>(zpart),
                                    reinterpret_cast<double*>(zeta), nullptr, st));
  VP_K(VP_K_INIT, init_launch_zeta_to_Z(n, p, zeta, Z, st));
  if (sigma) {
    // sigma = sqrt(max(lambda, 0)), computed on the device
    VP_K(VP_K_INIT, sqrt_nonneg(p, lam, sigma, st));
  }
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_init_csvd(vp_ctx* ctx, int64_t N, int32_t p, int32_t n, const double* X0,
                       const double* V0, double* Q, double* Z, double* sigma, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  return init_csvd_impl(ctx, N, p, 1, n, -1.0, X0, V0, Q, Z, sigma, nullptr, st);
}

vp_status vp_param_subsample(vp_ctx* ctx, int32_t n, int32_t p, const double* Z0, int32_t p_max,
                             double tol, int32_t* idx, int32_t* count, void* stream) {
  VP_ENTER();
  if (n < 1 || p < 1 || p > 1024 || p_max < 1 || !Z0 || !idx || !count || !(tol >= 0.0))
    return vp_fail(ctx, VP_EINVAL, "subsample arguments (n %d, p %d, p_max %d)", n, p, p_max);
  int32_t* d_count = reinterpret_cast<int32_t*>(ctx->d_status) + 4;  // spare words of the status block
  VP_K(VP_K_SUBSET, param_subsample(2 * n, p, Z0, std::min(p_max, p), tol, idx, d_count, st));
  VP_LAUNCHED();
  VP_CUDA(cudaMemcpyAsync(ctx->h_pinned + 4, d_count, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  VP_CUDA(cudaStreamSynchronize(st));
  *count = ctx->h_pinned[4];
  return VP_OK;
}

vp_status vp_init_csvd_rank(vp_ctx* ctx, int64_t N, int32_t p, int32_t n_min, int32_t n_max,
                            double tail_tol, const double* X0, const double* V0, double* Q,
                            double* Z, double* sigma, int32_t* n_out, void* stream) {
  VP_ENTER();
  VP_NO_COMM();
  if (!(tail_tol >= 0.0)) return vp_fail(ctx, VP_EINVAL, "tail_tol must be >= 0");
  return init_csvd_impl(ctx, N, p, n_min, n_max, tail_tol, X0, V0, Q, Z, sigma, n_out, st);
}

// One partitioned RK2 step per iteration (Sec. 5; stage structure as in the
// oracle's prk2_step).  Buffers: rows[0] = M / M', rows[1] = xi_half,
// rows[2] = Q_half, rows[3] = X(Q_half, Z_mid), rows[4] = xi_1 = dt Y.
vp_status vp_basis_update(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                          double* Q, double* Z, double dt, int32_t nsteps, const vp_step_opts* opts,
                          double* trace, int32_t* iters, double* kstate, void* stream) {
  VP_ENTER();
  VP_TRY(check_grid(ctx, grid));
  VP_TRY(check_np(ctx, N, p));
  VP_TRY(check_n(ctx, n, N));
  if (!Q || !Z) return vp_fail(ctx, VP_EINVAL, "Q and Z are required");
  if (nsteps < 0 || !std::isfinite(dt)) return vp_fail(ctx, VP_EINVAL, "nsteps < 0 or dt not finite");
  vp_step_opts o{1e-9, 100, 0, 1e-3, 1e-2, 0, 0, 0, nullptr};
  if (opts) o = *opts;
  if (!(o.tol >= 0.0) || o.maxit < 1) return vp_fail(ctx, VP_EINVAL, "tol < 0 or maxit < 1");
  if (o.arith < 0 || o.arith > 2) return vp_fail(ctx, VP_EINVAL, "arith must be 0, 1 or 2");
  if ((int64_t)4 * n * n + (int64_t)2 * n * p > 25600)
    return vp_fail(ctx, VP_EUNSUPPORTED, "4n^2 + 2n p = %lld exceeds 25600 (shared memory of the "
                   "fixed-point update)", (long long)(4 * n * n + 2 * n * p));
  if (o.nsub != 0) {
    if (o.arith == 0)
      return vp_fail(ctx, VP_EUNSUPPORTED, "the parameter subsample needs arith 1 or 2");
    if (o.nsub < n || o.nsub > p || !o.sub_idx)
      return vp_fail(ctx, VP_EINVAL, "subsample of %d columns outside [n, p] = [%d, %d] or no indices",
                     o.nsub, n, p);
  }
  if (ctx->comm_on && N > ctx->comm.n_global)
    return vp_fail(ctx, VP_EINVAL, "N = %lld rows exceed n_global", (long long)N);
  ctx->comm_failed = false;
  const bool df = o.arith != 0;
  Red R;
  VP_TRY(red_setup(ctx, grid, N, n, p, df ? 0 : 5, st, R, df, o.nsub, o.arith == 2));
  if (df) {
    VP_TRY(basis_update_df(ctx, R, Q, Z, dt, nsteps, o, trace, iters, kstate, st));
    if (ctx->comm_failed) return vp_fail(ctx, VP_ECOMM, "a sum over the ranks failed");
    return VP_OK;
  }
  RedWS& w = R.w;
  double *M = w.rows[0], *xih = w.rows[1], *Qh = w.rows[2], *Xp = w.rows[3], *xi1 = w.rows[4];
  const int64_t zsz = (int64_t)2 * n * p;
  const int64_t tstride = (int64_t)p * 2;
  int round = 4;
  for (int step = 0; step < nsteps; ++step) {
    // stage 1: field at (Q0, Z0); energies of the entering state
    R.field(Q, Z);
    if (trace) {
      R.gv(Q, w.GVraw);
      VP_K(VP_K_ENERGIES, energies(n, p, w.GVraw, Z, w.Efield, trace + step * tstride, trace + step * tstride + 1, 2,
               nullptr, nullptr, ctx->d_status, st));
    }
    const double* Qmid = Q;
    if (!o.freeze_basis) {
      R.basis_velocity_from_field(Q, Z, 0.5 * dt, M, xih);  // xi_half = dt/2 X(Q0, Z0)
      R.cayley(Q, xih, Qh);                                        // Q_half = R_Q0(xi_half)
      Qmid = Qh;

    }
    // stage 2: fixed point for k2 at Q_half
    R.gv(Qmid, w.GVraw);
    VP_CUDA(cudaMemcpyAsync(w.Z0, Z, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
    if (kstate) {  // warm start: k^0 = previous k2, Ze = Z0 + dt/2 k^0
      VP_CUDA(cudaMemcpyAsync(w.k, kstate, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
      VP_K(VP_K_AXPY, axpy(zsz, 0.5 * dt, w.k, w.Z0, w.Ze, st));
    } else {
      VP_CUDA(cudaMemcpyAsync(w.Ze, Z, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
      VP_CUDA(cudaMemsetAsync(w.k, 0, sizeof(double) * zsz, st));
    }
    VP_CUDA(cudaMemsetAsync(w.flags, 0, 4 * sizeof(int), st));
    int done_h = 0, total = 0;
    while (!done_h) {
      for (int r = 0; r < round && total < o.maxit; ++r, ++total) {
        R.field(Qmid, w.Ze, w.flags);
        VP_K(VP_K_PROJECT, project(R.g, N, n, p, Qmid, w.Ze, w.F, nullptr, 0, nullptr, nullptr, N,
                                   w.part, w.gx_proj, w.flags, ctx->d_status, st));
        VP_K(VP_K_REDUCE, reduce_partials(w.gx_proj, zsz, w.part, w.gX, w.flags, st));
        comm_sum_f64(ctx, w.gX, zsz, st);
        VP_K(VP_K_COEFF_UPDATE, coeff_update(n, p, w.gX, w.GVraw, w.Z0, w.k, w.kr, w.Ze, dt, o.tol,
                                             o.maxit, o.cycle_max, o.cycle_ratio, w.aux, w.flags,
                                             w.flags + 1, ctx->d_status, st));
      }
      VP_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, w.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
      VP_CUDA(cudaStreamSynchronize(st));
      if (!ctx->pending.empty()) vp_prof_collect(ctx);
      done_h = ctx->h_pinned[1];
      if (!done_h && total >= o.maxit) break;
      round = 2;
    }
    const int its = ctx->h_pinned[2];
    round = its > 2 ? its : 2;
    if (iters) VP_CUDA(cudaMemcpyAsync(iters + step, w.flags + 1, sizeof(int), cudaMemcpyDeviceToDevice, st));
    if (!done_h || its >= o.maxit) {
      // status word carries VP_ENOCONV or VP_ENUMERIC
      VP_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
      VP_CUDA(cudaStreamSynchronize(st));
      if (ctx->h_pinned[0] != 0 || !done_h)
        return vp_fail(ctx, VP_ENOCONV, "fixed point did not converge in %d iterations (step %d)",
                       o.maxit, step);
    }
    // Z_mid = w.Ze (= Z0 + dt/2 k2), Z1 = Z0 + dt k2
    VP_K(VP_K_AXPY, axpy(zsz, dt, w.k, w.Z0, w.Z1, st));
    if (kstate)
      VP_CUDA(cudaMemcpyAsync(kstate, w.k, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
    if (!o.freeze_basis) {
      // stage 3: basis velocity at (Q_half, Z_mid), tangent velocity, retraction
      R.field(Qh, w.Ze);
      R.basis_velocity_from_field(Qh, w.Ze, 1.0, M, Xp);
      R.tangent(Q, xih, Qh, Xp, dt, xi1);  // xi_1 = dt Y(xi_half, Z_mid)
      R.cayley(Q, xi1, Q);                 // Q_1 = R_Q0(xi_1), in place
    }
    VP_CUDA(cudaMemcpyAsync(Z, w.Z1, sizeof(double) * zsz, cudaMemcpyDeviceToDevice, st));
  }
  VP_LAUNCHED();
  if (ctx->comm_failed) return vp_fail(ctx, VP_ECOMM, "a sum over the ranks failed");
  return VP_OK;
}

}  // extern "C"
