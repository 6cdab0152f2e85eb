// Internal definitions shared by the translation units of libvp.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "../../include/vp.h"

#define VP_MAX_NX 1024
#define VP_MAX_N2 128  // 2n <= 128
#define VP_NSM_DEFAULT 152

// Launch-shape knobs of the FP32-based particle kernels: resident blocks per
// SM the grid is sized for (vp_tune_set / vp_autotune).
enum TuneKnob { TUNE_DEPOSIT = 0, TUNE_PROJECT, TUNE_BASIS_M, TUNE_GRAM, TUNE_AFFINE, TUNE_COUNT };
constexpr int kTuneDefault[TUNE_COUNT] = {4, 4, 4, 8, 8};

// ----------------------------------------------------------------- context
struct vp_ctx {
  int device = 0;
  int num_sms = VP_NSM_DEFAULT;
  size_t budget = 0;
  // workspace arena: one device allocation, grown on demand within budget
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // device status word (int32) and a pinned mirror used by host-steered loops
  int* d_status = nullptr;
  int* h_pinned = nullptr;  // pinned host ints: [0] status, [1] done flag, [2] iterations
  std::string last_error;
  std::mutex mu;
  // profiling: launch counters and event timers per kernel (vp_kernel ids)
  uint64_t prof_mask = 0;
  int64_t launches[VP_K_COUNT] = {};
  int64_t timed[VP_K_COUNT] = {};
  double ms[VP_K_COUNT] = {};
  struct Pending { int id; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  int tune[TUNE_COUNT] = {kTuneDefault[0], kTuneDefault[1], kTuneDefault[2], kTuneDefault[3],
                         kTuneDefault[4]};
  int tensor_cores = VP_TC_DEFAULT;  // vp_tensor_cores mask: tcgen05 kernels where they apply
  // particle sharding (vp_ctx_set_comm): sums over the rows of all ranks
  vp_comm comm{};
  bool comm_on = false;
  bool comm_failed = false;
};

// Sum over the ranks of the attached communicator, in place on the device
// buffer, ordered on st; no-op without one.  A failure is recorded in the
// context (the entry point then returns VP_ECOMM).
void comm_sum_f64(vp_ctx* ctx, double* buf, int64_t count, cudaStream_t st);
void comm_sum_u64(vp_ctx* ctx, unsigned long long* buf, int64_t count, cudaStream_t st);

// Blocks of a grid sized for `bps` resident blocks per SM over `chunks`
// column chunks, at most one per tile.
inline int grid_bps(int64_t tiles, int chunks, int bps, int num_sms) {
  int64_t want = ((int64_t)bps * num_sms + chunks - 1) / chunks;
  int64_t g = tiles < want ? tiles : want;
  return g < 1 ? 1 : (int)g;
}

// Count (and, if enabled, event-time) one kernel launch made by `expr`.
void vp_prof_begin(vp_ctx* ctx, int id, cudaStream_t st, cudaEvent_t* a);
void vp_prof_end(vp_ctx* ctx, int id, cudaStream_t st, cudaEvent_t a);
void vp_prof_collect(vp_ctx* ctx);  // resolve pending event pairs (synchronises them)
#define VP_K(id, expr)                               \
  do {                                               \
    cudaEvent_t ev_a_ = nullptr;                     \
    vp_prof_begin(ctx, id, st, &ev_a_);              \
    expr;                                            \
    vp_prof_end(ctx, id, st, ev_a_);                 \
  } while (0)

vp_status vp_fail(vp_ctx* ctx, vp_status s, const char* fmt, ...);
vp_status vp_cuda_check(vp_ctx* ctx, cudaError_t e, const char* what);
// Ensure the arena holds at least `bytes`; grows (synchronously) if needed.
vp_status vp_workspace(vp_ctx* ctx, size_t bytes, void** out);
// Workspace bytes of one serving query (start + steps) and arena release.
size_t vp_query_ws_bytes(int sms, int64_t N, int n, int p, int Nx, int arith);
void vp_workspace_release(vp_ctx* ctx);
// One reduced step of one instance in phases (vp_api.cu), for the batched
// engine: the kernel sequence of vp_basis_update with arith 1 or 2.
struct InstanceStep;
vp_status step_setup(vp_ctx* ctx, const vp_grid* grid, int64_t N, int n, int p, double* Q,
                     double* Z, double dt, const vp_step_opts* opts, double* kstate,
                     cudaStream_t st, InstanceStep** out);
vp_status step_pre(InstanceStep* is, double* trace_step);
vp_status step_rounds(InstanceStep* is, int count);
vp_status step_post(InstanceStep* is);
int* step_flags(InstanceStep* is);  // device [done, iterations]
void step_free(InstanceStep* is);
// Rank at t = 0 from the singular values (tail energy rule).
int vp_choose_rank(const double* sig, int p, int n_min, int n_max, double tol);

#define VP_CUDA(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return vp_cuda_check(ctx, e_, #call);   \
  } while (0)

#define VP_TRY(x)               \
  do {                          \
    vp_status s_ = (x);         \
    if (s_ != VP_OK) return s_; \
  } while (0)

#define VP_LAUNCHED()                                              \
  do {                                                             \
    cudaError_t e_ = cudaGetLastError();                           \
    if (e_ != cudaSuccess) return vp_cuda_check(ctx, e_, "launch"); \
  } while (0)

// Device status word: the first error wins.
__device__ __forceinline__ void vp_set_status(int* st, int code) {
  if (st) atomicCAS(st, 0, code);
}

// ------------------------------------------------- bulk copies (TMA engine)
// One-dimensional bulk copies global -> shared completed on an mbarrier
// (cp.async.bulk with complete_tx).  Addresses and sizes must be multiples of
// 16 bytes.  Waits are bounded: after kMbarSpins polls the waiting thread sets
// VP_ETIMEDOUT in the status word and goes on, so every thread still reaches
// the same barriers and the kernel ends.
constexpr int kMbarSpins = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make initialised barriers visible to the bulk-copy engine
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// order this CTA's earlier generic-proxy accesses of shared memory before
// later bulk-copy writes into it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* status,
                                          int spins = kMbarSpins) {
  for (int i = 0; i < spins; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  vp_set_status(status, VP_ETIMEDOUT);
  return false;
}

// Double-float split of an FP64 value: hi = rn(d), lo = rn(d - hi).
__device__ __forceinline__ float2 df_split(double d) {
  float h = __double2float_rn(d);
  float l = __double2float_rn(d - (double)h);
  return make_float2(h, l);
}
// The same split by integer operations on the bit pattern, for an exponent
// of d in [-70, 126]: this part issues FP64 conversions at 1/64 of the FP32
// rate, and the row splits of the FP32-based forms were bound by them.
// hi = d rounded to 24 significant bits (to nearest, ties to even); the
// remainder r = d - hi, an integer multiple of 2^(e-52) with |r| <= 2^(e-24),
// is rounded to FP32 by the int-to-float conversion and scaled by a power of
// two (exact).  The same bits as df_split; zero, tiny, huge and non-finite d
// take df_split.
__device__ __forceinline__ float2 df_split_bits(double d) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(d);
  const int e = (int)((u >> 52) & 0x7ffull) - 1023;
  if (e < -70 || e > 126) return df_split(d);
  const unsigned long long mant = u & ((1ull << 52) - 1);
  const unsigned int low = (unsigned int)(mant & ((1ull << 29) - 1));
  unsigned int m23 = (unsigned int)(mant >> 29);
  const unsigned int up = (low > (1u << 28) || (low == (1u << 28) && (m23 & 1u))) ? 1u : 0u;
  const int r = (int)low - (int)(up << 29);
  m23 += up;
  unsigned int fe = (unsigned int)(e + 127);
  if (m23 == (1u << 23)) {
    m23 = 0;
    fe += 1;
  }
  const unsigned int sgn = (unsigned int)(u >> 63);
  const float hi = __uint_as_float((sgn << 31) | (fe << 23) | m23);
  const float lo = (float)(sgn ? -r : r) * __uint_as_float((unsigned int)(e - 52 + 127) << 23);
  return make_float2(hi, lo);
}
// Store d in the row format of the FP32-based forms: mode 1 double-float
// (float2), mode 2 FP32 (float).
__device__ __forceinline__ void store_lp(void* base, int64_t e, double d, int mode) {
  if (mode == 1) reinterpret_cast<float2*>(base)[e] = df_split(d);
  else reinterpret_cast<float*>(base)[e] = __double2float_rn(d);
}

// Sub-allocation inside the arena (256-byte aligned).
struct Arena {
  char* base;
  size_t off;
  size_t cap;
  template <typename T>
  T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};
inline size_t arena_bytes(size_t count, size_t elem) { return (count * elem + 255) & ~size_t(255); }

// ------------------------------------------------------- fixed-point charge
// Deposit weights lambda in [0,1] are accumulated as integers lambda*2^S.
// A node receives at most N*2^S < 2^62 (S = 62 - bitlength(N), capped at 52),
// so the int64 sums never overflow and do not depend on the summation order.
inline int fixed_point_bits(int64_t N) {
  int b = 0;
  while ((int64_t(1) << b) <= N) ++b;  // bitlength(N)
  int S = 62 - b;
  return S > 52 ? 52 : S;
}

// Wrapped cell index and fraction of an unwrapped position x (cell units
// t = x/h, periodic with period Nx).
__device__ __forceinline__ void cell_of(double x, double inv_h, int Nx, double dNx, double inv_Nx,
                                        int& j, double& s) {
  double t = x * inv_h;
  double w = floor(t * inv_Nx);
  double tt = fma(-w, dNx, t);
  if (tt < 0.0) tt += dNx;
  if (tt >= dNx) tt -= dNx;
  double fl = floor(tt);
  j = (int)fl;
  if (j > Nx - 1) j = Nx - 1;
  if (j < 0) j = 0;
  s = tt - (double)j;
}

// ----------------------------------------------------------- launch helpers
inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Complex FP64 helpers (double2 = re, im).
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {  // conj(a) * b
  return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.x, b.y, -a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// ------------------------------------------------------------ shared state
// Launch configuration shared by the reduced-model tile kernels.
#define TILE_ROWS 64     // particles (rows of Q) per tile
#define TILE_THREADS 256 // threads per block of the tile kernels

// -------------------------------------------------------- internal entry
// (implemented in the .cu files; used by the API layer)
namespace vpk {

struct GridC {
  int Nx;
  double L, h, inv_h, inv_Nx, dNx, Mq, mp, qm, bg_load, fp_scale, fp_inv;  // fp_*: 2^S, 2^-S
  int S;
  // FP32 row form: one packed count per particle, (1 << Kp) + round(frac 2^Sp)
  // into its cell (the count field above bit Kp, the weight sum below it);
  // Kp = 0 when N is too large for packing
  int Sp, Kp;
};
GridC make_gridc(const vp_grid& g, int64_t N);

struct GramArgs {  // out_s = blk[pa[s]]^H blk[pb[s]]
  const double* blk[6];
  int pa[12], pb[12];
  int nblk, npairs;
};
struct AffineArgs {  // out = sum_t X[t] C_t
  const double* X[4];
  int nterms;
};
// FP32-based row kernels (reduced_df.cu): rows stored as float2 (double-float)
// or float (FP32), selected by the arithmetic policy at launch.
struct GramArgsLP {
  const void* blk[4];
  int pa[8], pb[8];
  int nblk, npairs;
};
struct AffineArgsLP {
  const void* X[4];
  int nterms;
  // FP64 rows of term 0 (nullable): the FP64 output is then written as
  // base + sum_t X_t C_t - X_0, i.e. term 0's coefficient less the identity
  // in the row arithmetic and the base added in FP64 (increment form)
  const double* base = nullptr;
};
enum LpOp { LP_SPLIT, LP_PREP, LP_DEPOSIT, LP_PROJECT, LP_BASIS_M, LP_GRAM, LP_GRAM_REAL, LP_AFFINE };
struct LpArgs {
  const GridC* g = nullptr;
  int64_t N = 0;
  int n = 0, p = 0, num_sms = 0, gridx = 0;
  int64_t m = 0;
  const double* dsrc = nullptr;
  const double* F = nullptr;
  void *v0 = nullptr, *v1 = nullptr, *v2 = nullptr, *v3 = nullptr;
  unsigned long long* counts = nullptr;
  uint16_t* j = nullptr;
  double* part = nullptr;
  const int* skip = nullptr;
  GramArgsLP gram{};
  AffineArgsLP aff{};
  const double2* C = nullptr;
  double* dout = nullptr;
  const int* tune = nullptr;  // vp_ctx::tune (null: defaults)
  int* status = nullptr;      // device status word
  int tc = 0;                 // vp_tc_kernel mask: tensor-core kernels where they apply
  float* bop = nullptr;       // scratch of the tensor-core row products (rows_tc_bop_floats)
};

// Cell indices of the FP32-based path are stored tile by tile: for row tile
// t (TILE_ROWS particles) and sample chunk c (PC samples) one contiguous
// TILE_ROWS x PC block, so a kernel fetches its (tile, chunk) indices, or all
// chunks of a tile, with one bulk copy.  Entries past N or p are padding.
__host__ __device__ __forceinline__ int64_t jt_block(int64_t tile, int chunk, int nchunks, int PC) {
  return (tile * nchunks + chunk) * (int64_t)TILE_ROWS * PC;
}

// pic_kernels.cu
void deposit_samples(const GridC& g, int64_t N, int p, const double* X, int64_t ldx,
                     unsigned long long* counts, int num_sms, cudaStream_t st);
void counts_to_rho(const GridC& g, int p, const unsigned long long* counts, double* rho,
                   cudaStream_t st);
// the same launches, returning the launch's own error
cudaError_t deposit_samples_launch(const GridC& g, int64_t N, int p, const double* X, int64_t ldx,
                                   unsigned long long* counts, int num_sms, cudaStream_t st);
cudaError_t counts_to_rho_launch(const GridC& g, int p, const unsigned long long* counts,
                                 double* rho, cudaStream_t st);
void poisson(const GridC& g, int p, const double* rho, const unsigned long long* counts,
             double* phi, double* F, double* energy, unsigned long long* zero_counts,
             const int* skip, int* status, cudaStream_t st, void* F2 = nullptr, int f2mode = 0);
void gather(const GridC& g, int64_t N, int p, const double* X, int64_t ldx, const double* F,
            const int32_t* idx, int64_t d, double* GX, int num_sms, int* status, cudaStream_t st);
cudaError_t full_step(const GridC& g, int64_t N, int p, double* X, double* V, double dt,
                      int nsteps, double* trace, int* status, cudaStream_t st);

// reduced_kernels.cu
int tile_grid_x(int64_t N, int chunks, int num_sms);
int gram_grid_x(int64_t N, int num_sms);
int project_chunks(int p, int Nx);
int chunk_pc(int p, int Nx);  // samples per column chunk of the particle kernels
void reconstruct(int64_t N, int n, int p, const double* Q, const double* Z, double* X, double* V,
                 cudaStream_t st);
void deposit_reduced(const GridC& g, int64_t N, int n, int p, const double* Q, const double* Z,
                     unsigned long long* counts, const int* skip, int num_sms, cudaStream_t st);
void project(const GridC& g, int64_t count, int n, int p, const double* Q, const double* Z,
             const double* F, const double* GX, int64_t ldg, const int32_t* idx, const double* cw,
             int64_t nrows, double* part, int gridx, const int* skip, int* status,
             cudaStream_t st);
void basis_M(const GridC& g, int64_t N, int n, int p, const double* Q, const double* Z,
             const double* F, double* M, int num_sms, cudaStream_t st);
void gram(int64_t N, int n, const GramArgs& a, double2* part, int gridx, cudaStream_t st);
void gram_real(int64_t N, int m, const double* X, double* part, int gridx, cudaStream_t st);
void reduce_partials(int nparts, int64_t elems, const double* part, double* out, const int* skip,
                     cudaStream_t st);
void affine(int64_t N, int n, const AffineArgs& a, const double2* C, double* out, int num_sms,
            cudaStream_t st);
void cell_gradient(const GridC& g, int p, const double* phi, double* F, cudaStream_t st);
void reduced_init();

// dense.cu (single-block small dense algebra, FP64; df: in double-float on
// the FP32 pipes, for the FP32 form)
void small_basis_coeffs(int n, int p, const double2* QhM, const double* Z, double scale,
                        double2* C, double2* tmp, int* status, cudaStream_t st, bool df = false);
void small_cayley_coeffs(int n, const double2* G0, const double2* P, const double2* XX, double2* C,
                         double2* tmp, int* status, cudaStream_t st, bool df = false);
void small_tangent_coeffs(int n, const double2* grams, const double2* G0, const double2* P,
                          double scale, double2* C, double2* tmp, int* status, cudaStream_t st,
                          bool df = false);
// gX: the projection (2n x p), or nullptr with `part` (nparts x 2n x p block
// partials of it, summed here in block order).  kr (3 x 2n x p): ring of
// the iterates two to four iterations back (no initial value needed).
// partials: 5 p + 8 doubles (block sums, then the last 8 relative updates).
// Z2/Zh2 (nullable): the new evaluation point Ze and Ze / h in the row format
// `zmode` (1 double-float, 2 FP32) for the next deposit.
void coeff_update(int n, int p, const double* gX, const double* GVraw, const double* Z0, double* k,
                  double* kr, double* Ze, double dt, double tol, int maxit, double cycle_max,
                  double cycle_ratio, double* partials, int* done, int* iters, int* status,
                  cudaStream_t st, const double* part = nullptr, int nparts = 0,
                  void* Z2 = nullptr, void* Zh2 = nullptr, double inv_h = 0.0, int zmode = 0);
void axpy(int64_t m, double a, const double* x, const double* y, double* out, cudaStream_t st);
void sqrt_nonneg(int m, const double* x, double* out, cudaStream_t st);
void add_linear(int n, int p, const double* gX, const double* GVraw, const double* Z, double* g,
                cudaStream_t st);
void energies(int n, int p, const double* GVraw, const double* Z, const double* Efield,
              double* E_out, double* H_out, int64_t stride, const double2* QhQ, double* resid,
              int* status, cudaStream_t st);
void lowdin(int n, const double2* G, double2* C, int* status, cudaStream_t st);
void gather_cols(int rows, int p, const double* Z, const int32_t* idx, int nsub, double* Zs,
                 int* status, cudaStream_t st);
void param_subsample(int rows, int p, const double* Z, int p_max, double tol, int32_t* idx,
                     int32_t* count, cudaStream_t st);
void dense_init();
void pic_init();

// reduced_df.cu: arith 1 = double-float, 2 = FP32
void lp_launch(int arith, LpOp op, const LpArgs& a, cudaStream_t st);
void df_init();
// tc_project.cu: projection of the FP32 form on the tensor cores
bool project_tc_supported(int n, int p, int Nx);
void project_tc(const GridC& g, int64_t N, int n, int p, const float* Q2, const float* F2,
                const uint16_t* jt, double* part, int gridx, const int* skip, int* status,
                cudaStream_t st);
void tc_init();
// tc_deposit.cu: deposit of the FP32 form with the reconstruction on the tensor cores
bool deposit_tc_supported(int n, int p, int Nx, int Kp);
void deposit_tc(const GridC& g, int64_t N, int n, int p, const float* Q2, const float* Zh2,
                unsigned long long* counts, uint16_t* jout, int gridx, const int* skip,
                int* status, cudaStream_t st);
void tc_deposit_init();
// Gram matrices of the FP32 rows on the tensor cores: the complex pairs of
// a GramArgsLP (real_out = 0) or the real Gram of block 0 (real_out = 1),
// per-block partials in the layout of the SIMT kernels.
bool gram_tc_supported(int n, int nblk, int npairs);
void gram_tc(int64_t N, int n, const GramArgsLP& a, int real_out, double* part, int gridx,
             int* status, cudaStream_t st);
void tc_gram_init();
// Row-block products of the FP32 rows on the tensor cores: M = Gamma zeta^H
// (the split form [Q | G] [W ; a^T | -b^T]) and the combinations
// sum_t X_t C_t of LP_AFFINE; bop holds rows_tc_bop_floats(n, p) floats.
bool basis_tc_supported(int n, int p);
bool affine_tc_supported(int n, int nterms);
size_t rows_tc_bop_floats(int n, int p);
void basis_tc(const GridC& g, int64_t N, int n, int p, int PC, const float* Q2, const float* Z2,
              const float* F2, const uint16_t* jt, float* M, float* bop, int num_sms,
              int* status, cudaStream_t st);
void affine_tc(const GridC& g, int64_t N, int n, const AffineArgsLP& aff, const double2* C,
               double* out_d, float* out_v, float* bop, int num_sms, int* status,
               cudaStream_t st);
void tc_rows_init();
// typed.cu: per-step calls on FP64 / FP32 / BF16 inputs (dtype 0 / 1 / 2)
int vp_dtype_size(int dtype);
void deposit_typed(const GridC& g, int64_t N, int p, const void* X, int64_t ldx, int dtype,
                   unsigned long long* counts, int num_sms, cudaStream_t st);
void gather_typed(const GridC& g, int64_t N, int p, const void* X, int64_t ldx, int dtype,
                  const double* F, const int32_t* idx, int64_t d, void* GX, int num_sms,
                  int* status, cudaStream_t st);
void reconstruct_typed(int64_t N, int n, int p, const void* Q, int64_t ldq, int dtype,
                       const double* Z, void* X, void* V, int64_t ldx, int num_sms,
                       cudaStream_t st);
void project_typed(int64_t N, int n, int p, const void* Q, int64_t ldq, int dtype, const void* GX,
                   int64_t ldg, double* part, int gridx, cudaStream_t st);
void gram_real_typed(int64_t N, int m, const void* Q, int64_t ldq, int dtype, double* part,
                     int gridx, cudaStream_t st);
int typed_grid_x(int64_t N, int chunks, int num_sms);

// init.cu (complex SVD start)
void init_launch_rgram(int64_t N, int p, const double* X, const double* V, double2* part, int gx,
                       cudaStream_t st);
void init_launch_jacobi(int m, double2* A, double2* W, double* lambda, double2* Wout, int* status,
                        cudaStream_t st);
void init_launch_coeff(int p, int n, const double2* W, const double* lambda, double2* C, int* status,
                       cudaStream_t st);
void init_launch_r_times(int64_t N, int p, int n, const double* X, const double* V, const double2* C,
                         double* Q, int num_sms, cudaStream_t st);
void init_launch_inv_sqrt(int n, const double2* W, const double* lambda, double2* out, int* status,
                          cudaStream_t st);
void init_launch_zeta(int64_t N, int p, int n, const double* Q, const double* X, const double* V,
                      double2* part, int gx, cudaStream_t st);
void init_launch_zeta_to_Z(int n, int p, const double2* zeta, double* Z, cudaStream_t st);
void init_kernels_init();  // kernel attributes of init.cu
void deim_init();          // kernel attributes of deim.cu
// diag.cu: accuracy diagnostics (partial sums per block, reduced in order)
int diag_blocks(int64_t N, int sms);
void rel_err_parts(int64_t N, int n, int p, const double* Q, const double* Z, const double* X,
                   const double* V, double* part, int nb, cudaStream_t st);
void normal_parts(const GridC& g, int64_t N, int n, int p, const double* Q, const double* Z,
                  const double* F, const double* gproj, double* part, int nb, cudaStream_t st);
void ratio_sqrt(int pairs, const double* s, double* out, cudaStream_t st);
void ham_terms(int p, const double* h00, const double* h11, const double* hh0, const double* hh1,
               double* out, cudaStream_t st);
// deim.cu: DEIM construction and DMD on caller-owned scratch (sizes below)
size_t deim_basis_scratch(int sms, int64_t N, int m);
vp_status deim_basis_run(vp_ctx* ctx, int64_t N, int m, const double* Y, int64_t ldy, int d,
                         double* Psi, double* sigma, void* scratch, cudaStream_t st);
size_t deim_indices_scratch(int sms, int64_t N, int d);
// Psi_prev == nullptr: all d indices by the greedy rule; else idx holds the
// previous indices and the n_up most rotated positions are renewed
vp_status deim_indices_run(vp_ctx* ctx, int64_t N, int d, const double* Psi, int32_t* idx,
                           const double* Psi_prev, int n_up, void* scratch, cudaStream_t st);
size_t deim_weights_scratch(int sms, int64_t N, int d);
vp_status deim_weights_run(vp_ctx* ctx, int64_t N, int d, const double* Psi, const int32_t* idx,
                           double Mq, double* c, void* scratch, cudaStream_t st);
size_t dmd_fit_scratch(int nx, int m, int r_max);
vp_status dmd_fit_run(vp_ctx* ctx, int nx, int m, const double* Y, const double* Yp, double tol,
                      int r_max, int* r_out, double* B, double* Bpinv, double* A, double* S,
                      double* sigma, void* scratch, cudaStream_t st);
void dmd_coords_run(int nx, int r, const double* Bpinv, int q, const double* Phi, double* beta,
                    cudaStream_t st);
void rbf_run(int dim, int q, const double* eta_s, int K, const double* values, int p,
             const double* eta, double eps, const double* eps_dev, double* out, int* status,
             cudaStream_t st);
void rbf_width_run(int dim, int q, const double* eta_s, double* eps, cudaStream_t st);
void dmd_potential_run(int nx, int r, const double* B, const double* A, const double* S, int p,
                       const double* beta, int ksteps, int half, double* Phi, cudaStream_t st);
void phi_at_qz(const GridC& g, int64_t N, int n, int q, const double* Q, const double* Zs,
               const double* phi, double* Y, int sms, cudaStream_t st);
void gather_rows_lp(const void* Q2, int mode, int64_t N, int n2, const int32_t* idx, int d,
                    double* out, int* status, cudaStream_t st);
void deim_round(const GridC& g, int n, int p, int d, const double* Qd, const double* Ze,
                const double* F, const double* c, double* gX, const int* done, cudaStream_t st);
// Particle loading (load.cu): eta p x 3, X and V p x N; mode 0 quiet start,
// mode 1 Philox4x32-10 keyed by seed.
void load_particles(int family, int mode, unsigned long long seed, double k, int64_t N, int p,
                    const double* eta, double* X, double* V, int num_sms, cudaStream_t st);

}  // namespace vpk
