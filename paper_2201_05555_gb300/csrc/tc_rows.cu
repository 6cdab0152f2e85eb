// Row-block products of the FP32 form on the tensor cores (tcgen05,
// kind::tf32): for every 128-row tile of the N particle rows,
//   out_tile (128 x 2n) = [X_0 | .. | X_{T-1} | G] (K = T 2n + p)  x  Bop,
// with the row blocks X_t (N x 2n FP32 rows [Re | Im]) and, for the basis
// velocity only, the gathered field values G.  Two uses:
//
// 1. M = Gamma zeta^H, the basis velocity of Sec. 3.2 (the derivative of U
//    under the PRK2 step of Sec. 5), Gamma_li = (q/m) F_i[j_li] + i V_li,
//    V_li = Im(Q_l zeta_i), M_lk = sum_i Gamma_li conj(zeta_ki).  Split form:
//    with zeta = a + i b, Q_l = x_l + i y_l and V_li = x_l b_i + y_l a_i,
//      Re M_lk =  sum_i G_li a_ki + [x_l | y_l] W[:, k],
//      Im M_lk = -sum_i G_li b_ki + [x_l | y_l] W[:, n + k],
//    W = Y Y^T, Y = [b; a] (2n x p), because sum_i V_li b_ki and
//    sum_i V_li a_ki are [x_l | y_l] times the columns of W.  So T = 1,
//    X_0 = Q, Bop = [W ; a^T | -b^T] (rows m < 2n: W, rows 2n + i: sample i),
//    V_r is never formed, and G_li is gathered with the cell j_li that the
//    deposit stored.
// 2. out_l = sum_t X_t,l C_t with complex n x n coefficients C_t (the
//    combinations of the basis velocity, the Cayley retraction and the
//    tangent velocity, Sec. 3.2 and Sec. 5): Bop stacks the real forms
//    [[Re C_t, Im C_t], [-Im C_t, Re C_t]]; with an FP64 base (the rows of
//    term 0) the output is base + sum_t X_t C_t - X_0, term 0's coefficient
//    taken less the identity, so that the increment keeps its own relative
//    accuracy and the base its FP64 one.
//
// Precision: every FP32 value v (row value or coefficient) is split into
// v_hi = v rounded to TF32 and v_lo = v - v_hi rounded to TF32
// (|v - v_hi - v_lo| <= 2^-22 |v|, tf32_split); the accumulator (128 x 2NB,
// NB = 2n rounded up to 16) takes a_s [B_hi | B_lo] for s = hi, lo, and
// out = D[:, :NB] + D[:, NB:] (FP32 accumulation in tensor memory).  An exact
// three-piece split of the row values measured no difference in the step's
// error against the oracle, so kBmPieces = 2.  Bop is built and split
// once per call by a prep kernel into 32-row K chunks in the K-major
// no-swizzle canonical layout (element (c, k) of a chunk at byte (c / 8) *
// 1024 + (k / 4) * 128 + (c % 8) * 16 + (k % 4) * 4, B_hi in rows c < NB,
// B_lo in rows NB + c); W is accumulated in FP64.
//
// Pipeline (512 threads, one CTA per SM, three stages of [A_hi | A_lo | B
// chunk | cell indices]): thread 0 bulk-copies a step's B chunk (and, for the
// sample steps, its two 64-row blocks of cell indices) S - 1 steps ahead; all
// threads load the step's A values one step ahead (row blocks of the next
// tile prefetched into L2 a tile ahead, field values through L1), split them
// and store them; thread 0 issues the MMAs and commits each stage;
// accumulators alternate between two tensor-memory buffers so that warps 0-3
// write tile t's rows while tile t+1 accumulates.  Every wait is bounded
// (VP_ETIMEDOUT).
#include "tc_common.cuh"

namespace vpk {
namespace {

constexpr int kBmRows = 128;     // MMA M
constexpr int kBmK = 32;         // K per step
constexpr int kBmThreads = 512;
constexpr int kBmStages = 3;
constexpr int kBmTerms = 4;      // row blocks of one product
constexpr int kBmPieces = 2;       // TF32 pieces of a row value
constexpr uint32_t kBmA = 16384;   // one TF32 piece of A of one step
constexpr uint32_t kBmB = 16384;   // B chunk, at most 2 NB = 128 rows
constexpr uint32_t kBmJ = 8192;    // two 64-row blocks of up to 32 cell indices
constexpr uint32_t kBmStage = kBmPieces * kBmA + kBmB + kBmJ;

__device__ __forceinline__ uint32_t bm_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}
__device__ __forceinline__ void bm_put(float* chunk, int NB, int c, int k, double v) {
  const float2 sp = tf32_split((float)v);
  chunk[bm_off(c, k) / 4] = sp.x;
  chunk[bm_off(NB + c, k) / 4] = sp.y;
}

struct RowsArgs {
  const float* X[kBmTerms];  // row blocks, N x 2n
  int nterms;
  int p, PC;                 // sample part (p = 0: none)
  const float* F2;           // (q/m) F rows, p x Nx
  const uint16_t* jt;        // cells, tile layout (jt_block)
  float* out_v;              // FP32 rows (nullable)
  double* out_d;             // FP64 rows (nullable)
  const double* base;        // FP64 rows added to out_d (nullable)
};

// Bop of Gamma zeta^H: chunk kt < KTq holds W rows m = 32 kt + k, chunk
// kt >= KTq the sample rows i = 32 (kt - KTq) + k; block (kt, c) writes row c
// of chunk kt (B_hi) and row NB + c (B_lo), thread k one element.
__global__ void k_basis_tc_prep(int n, int p, int NB, int KTq, const float* __restrict__ Z2,
                                float* __restrict__ Bg) {
  const int n2 = 2 * n, kt = blockIdx.x, c = blockIdx.y, k = threadIdx.x;
  double v = 0.0;
  if (c < n2) {
    if (kt < KTq) {
      const int m = kt * kBmK + k;
      if (m < n2) {  // W_mc = sum_i Y_m,i Y_c,i, Y row m = zeta row (m + n) mod 2n
        const float* ym = Z2 + (size_t)((m + n) % n2) * p;
        const float* yc = Z2 + (size_t)((c + n) % n2) * p;
        for (int i = 0; i < p; ++i) v = fma((double)ym[i], (double)yc[i], v);
      }
    } else {
      const int i = (kt - KTq) * kBmK + k;
      if (i < p) v = (c < n) ? (double)Z2[(size_t)c * p + i] : -(double)Z2[(size_t)c * p + i];
    }
  }
  bm_put(Bg + (size_t)kt * 2 * NB * kBmK, NB, c, k, v);
}

// Bop of the combinations: chunk kt covers rows m = 32 (kt % KTq) + k of term
// kt / KTq, whose real form has rows q (Re of the input) [Re C_qk | Im C_qk]
// and n + q (Im of the input) [-Im C_qk | Re C_qk]; with sub_id, term 0's
// coefficient less the identity.
__global__ void k_affine_tc_prep(int n, int NB, int KTq, const double2* __restrict__ C, int sub_id,
                                 float* __restrict__ Bg) {
  const int n2 = 2 * n, kt = blockIdx.x, c = blockIdx.y, k = threadIdx.x;
  const int tt = kt / KTq, m = (kt - tt * KTq) * kBmK + k;
  double v = 0.0;
  if (c < n2 && m < n2) {
    const int q = m < n ? m : m - n, kk = c < n ? c : c - n;
    double2 cv = C[(size_t)tt * n * n + (size_t)q * n + kk];
    if (sub_id && tt == 0 && q == kk) cv.x -= 1.0;
    v = (m < n) ? (c < n ? cv.x : cv.y) : (c < n ? -cv.y : cv.x);
  }
  bm_put(Bg + (size_t)kt * 2 * NB * kBmK, NB, c, k, v);
}

template <bool kSamples>
__device__ __forceinline__ void rows_tc_body(const GridC& g, int64_t N, int n, int NB,
                                             const RowsArgs& a, const float* __restrict__ Bg,
                                             int* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smraw + kBmStages * kBmStage);  // copies landed
  uint64_t* mdone = full + kBmStages;   // stage read by the MMAs (commit)
  uint64_t* accb = mdone + kBmStages;   // [2] accumulator complete (commit)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(accb + 2);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int n2 = 2 * n, Nx = g.Nx;
  const int KTq = (n2 + kBmK - 1) / kBmK, KTr = a.nterms * KTq;
  const int p = kSamples ? a.p : 0, PC = kSamples ? a.PC : 1;
  const int KT = KTr + (p + kBmK - 1) / kBmK;
  const int nch = kSamples ? (p + PC - 1) / PC : 1, pcs = __ffs(PC) - 1;
  const int64_t ntiles = (N + kBmRows - 1) / kBmRows, nt64 = (N + 63) / 64;
  const int64_t T = (int64_t)blockIdx.x < ntiles
                        ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  const int64_t G = T * KT;  // steps of this CTA: KT per tile
  const uint32_t bbytes = 256u * (uint32_t)NB;
  const bool vec = (n2 & 3) == 0;
  if (t == 0) {
    for (int s = 0; s < 2 * kBmStages + 2; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
  }
  if (warp == 0) tc_alloc(tslot, 256);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  auto stage = [&](int64_t gs) { return smraw + (uint32_t)(gs % kBmStages) * kBmStage; };
  auto tile_of = [&](int64_t tl) { return (int64_t)blockIdx.x + tl * gridDim.x; };
  // row block tt (a select chain keeps the pointers in registers)
  auto xblk = [&](int tt) {
    return tt == 0 ? a.X[0] : tt == 1 ? a.X[1] : tt == 2 ? a.X[2] : a.X[3];
  };
  // thread 0: the B chunk and, for a sample step, the cell indices of step gs
  auto issue = [&](int64_t gs) {
    const int64_t tl = gs / KT;
    const int kt = (int)(gs - tl * KT);
    const int64_t tile = tile_of(tl);
    unsigned char* S = stage(gs);
    uint64_t* bar = &full[gs % kBmStages];
    uint32_t jbytes = 0;
    int c0 = 0;
    if (kSamples && kt >= KTr) {
      c0 = ((kt - KTr) * kBmK) >> pcs;
      const int m = min(kBmK >> pcs, nch - c0);
      jbytes = 128u * (uint32_t)PC * (uint32_t)m;  // 64 rows x PC x m indices
    }
    const bool h1 = 2 * tile + 1 < nt64;
    fence_proxy_async_smem();
    mbar_expect_tx(bar, bbytes + jbytes * (h1 ? 2u : 1u));
    bulk_g2s(S + kBmPieces * kBmA, Bg + (size_t)kt * 2 * NB * kBmK, bbytes, bar);
    if (jbytes) {
      bulk_g2s(S + kBmPieces * kBmA + kBmB, a.jt + jt_block(2 * tile, c0, nch, PC), jbytes, bar);
      if (h1)
        bulk_g2s(S + kBmPieces * kBmA + kBmB + 4096, a.jt + jt_block(2 * tile + 1, c0, nch, PC), jbytes,
                 bar);
    }
  };
  // thread t: row r of the tile, K columns 8 kq + e (e < 8) of each step
  const int r = t & (kBmRows - 1), kq = t >> 7;
  auto fetch = [&](int64_t gs, float* o) {
    const int64_t tl = gs / KT;
    const int kt = (int)(gs - tl * KT);
    const int64_t R = tile_of(tl) * kBmRows + r;
    if (kt < KTr) {  // columns of a row block
      const int tt = kt / KTq;
      const float* X = xblk(tt);
      const int c = (kt - tt * KTq) * kBmK + 8 * kq;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (R < N && vec && c + 4 * u < n2) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(X + R * n2 + c + 4 * u));
          o[4 * u] = q.x; o[4 * u + 1] = q.y; o[4 * u + 2] = q.z; o[4 * u + 3] = q.w;
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            o[4 * u + v] = (R < N && c + 4 * u + v < n2) ? __ldg(X + R * n2 + c + 4 * u + v) : 0.f;
        }
      }
    } else if (kSamples) {  // field values G_li = (q/m) F_i[j_li]
      const uint16_t* J = reinterpret_cast<const uint16_t*>(stage(gs) + kBmPieces * kBmA + kBmB) +
                          (r >> 6) * 2048;
      const int i0 = (kt - KTr) * kBmK + 8 * kq;
      uint16_t jj[8];
      if (PC >= 8) {  // the thread's 8 samples lie in one chunk: one 16-byte load
        const int k = 8 * kq;
        const uint4 w = *reinterpret_cast<const uint4*>(
            J + (((k >> pcs) << 6) + (r & 63)) * PC + (k & (PC - 1)));
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          jj[2 * e] = (uint16_t)(ws[e] & 0xFFFFu);
          jj[2 * e + 1] = (uint16_t)(ws[e] >> 16);
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = 8 * kq + e;
          jj[e] = J[(((k >> pcs) << 6) + (r & 63)) * PC + (k & (PC - 1))];
        }
      }
      const float* f = a.F2 + i0 * Nx;  // p x Nx field rows: offsets fit 32 bits
#pragma unroll
      for (int e = 0; e < 8; ++e) o[e] = (R < N && i0 + e < p) ? __ldg(f + e * Nx + jj[e]) : 0.f;
    }
  };
  // warps 0-3: rows 32 w + lane of local tile tl from accumulator tl % 2
  auto epilogue = [&](int64_t tl) {
    const int b = (int)(tl & 1);
    mbar_wait(&accb[b], (uint32_t)((tl >> 1) & 1), status);
    tc_fence_after();
    const int64_t R = tile_of(tl) * kBmRows + 32 * warp + lane;
    const uint32_t tb = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(128 * b);
    for (int c0 = 0; c0 < NB; c0 += 16) {
      uint32_t h[16], l[16];
      tc_ld16(tb + c0, h);
      tc_ld16(tb + NB + c0, l);
      if (R >= N) continue;
      if (a.out_v) {
        float* dst = a.out_v + R * n2 + c0;
        if (vec) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (c0 + 4 * q < n2)
              *reinterpret_cast<float4*>(dst + 4 * q) = make_float4(
                  __uint_as_float(h[4 * q]) + __uint_as_float(l[4 * q]),
                  __uint_as_float(h[4 * q + 1]) + __uint_as_float(l[4 * q + 1]),
                  __uint_as_float(h[4 * q + 2]) + __uint_as_float(l[4 * q + 2]),
                  __uint_as_float(h[4 * q + 3]) + __uint_as_float(l[4 * q + 3]));
        } else {
#pragma unroll
          for (int jj = 0; jj < 16; ++jj)
            if (c0 + jj < n2) dst[jj] = __uint_as_float(h[jj]) + __uint_as_float(l[jj]);
        }
      }
      if (a.out_d) {  // n2 even: pairs of columns as double2
        double* dst = a.out_d + R * n2 + c0;
        const double* bs = a.base ? a.base + R * n2 + c0 : nullptr;
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (c0 + 2 * q < n2) {
            double2 v = make_double2(
                (double)__uint_as_float(h[2 * q]) + (double)__uint_as_float(l[2 * q]),
                (double)__uint_as_float(h[2 * q + 1]) + (double)__uint_as_float(l[2 * q + 1]));
            if (bs) {
              const double2 b2 = *reinterpret_cast<const double2*>(bs + 2 * q);
              v.x += b2.x;
              v.y += b2.y;
            }
            *reinterpret_cast<double2*>(dst + 2 * q) = v;
          }
      }
    }
    tc_fence_before();
  };
  if (t == 0)
    for (int64_t gs = 0; gs < G && gs < kBmStages; ++gs) issue(gs);
  float val[8], valn[8];
  if (G > 0) fetch(0, val);  // step 0 reads row-block columns
  const uint32_t idesc = tc_idesc_tf32(kBmRows, 2 * NB);
  for (int64_t gs = 0; gs < G; ++gs) {
    const int64_t tl = gs / KT;
    const int kt = (int)(gs - tl * KT);
    const int s = (int)(gs % kBmStages);
    if (kt == 0 && tl + 1 < T) {  // the next tile's rows of every block into L2
      const int64_t left = N - tile_of(tl + 1) * kBmRows;
      const int64_t nb = (left < kBmRows ? left : (int64_t)kBmRows) * n2 * 4;
      const int64_t b0 = tile_of(tl + 1) * kBmRows * n2;
      for (int tt = 0; tt < a.nterms; ++tt)
        if ((int64_t)t * 128 < nb)
          asm volatile("prefetch.global.L2 [%0];" ::"l"(reinterpret_cast<const char*>(xblk(tt) + b0) +
                                                         t * 128));
    }
    if (gs + 1 < G) {
      const int ktn = (int)((gs + 1) % KT);
      if (kSamples && ktn >= KTr)
        mbar_wait(&full[(gs + 1) % kBmStages], (uint32_t)(((gs + 1) / kBmStages) & 1), status);
      fetch(gs + 1, valn);
    }
    if (gs >= kBmStages) mbar_wait(&mdone[s], (uint32_t)((gs / kBmStages - 1) & 1), status);
    unsigned char* S = stage(gs);
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int k = 8 * kq + 4 * u;
      const float2 v0 = tf32_split(val[4 * u]), v1 = tf32_split(val[4 * u + 1]),
                   v2 = tf32_split(val[4 * u + 2]), v3 = tf32_split(val[4 * u + 3]);
      *reinterpret_cast<float4*>(S + bm_off(r, k)) = make_float4(v0.x, v1.x, v2.x, v3.x);
      *reinterpret_cast<float4*>(S + kBmA + bm_off(r, k)) = make_float4(v0.y, v1.y, v2.y, v3.y);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      mbar_wait(&full[s], (uint32_t)((gs / kBmStages) & 1), status);
      tc_fence_after();
      const uint32_t sa = smem_u32(S), sb = sa + kBmPieces * kBmA;
      const uint32_t d = tmem + (uint32_t)(128 * (tl & 1));
#pragma unroll
      for (int j = 0; j < kBmK / 8; ++j) {
        const uint64_t bd = tc_sdesc(sb + 256 * j, 128, 1024);
#pragma unroll
        for (int piece = 0; piece < kBmPieces; ++piece)
          tc_mma_tf32(d, tc_sdesc(sa + piece * kBmA + 256 * j, 128, 1024), bd, idesc,
                      (kt > 0 || j > 0 || piece > 0));
      }
      tc_commit(&mdone[s]);
      if (kt == KT - 1) tc_commit(&accb[tl & 1]);
      if (gs >= 1 && gs + kBmStages - 1 < G) {
        mbar_wait(&mdone[(gs - 1) % kBmStages], (uint32_t)(((gs - 1) / kBmStages) & 1), status);
        issue(gs + kBmStages - 1);
      }
    }
    __syncwarp();
    if (kt == 0 && tl > 0 && warp < 4) epilogue(tl - 1);
#pragma unroll
    for (int e = 0; e < 8; ++e) val[e] = valn[e];
  }
  if (T > 0 && warp < 4) epilogue(T - 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 256);
}

__global__ void __launch_bounds__(kBmThreads, 1)
k_basis_M_tc(GridC g, int64_t N, int n, int NB, RowsArgs a, const float* __restrict__ Bg,
             int* status) {
  rows_tc_body<true>(g, N, n, NB, a, Bg, status);
}

__global__ void __launch_bounds__(kBmThreads, 1)
k_affine_tc(GridC g, int64_t N, int n, int NB, RowsArgs a, const float* __restrict__ Bg,
            int* status) {
  rows_tc_body<false>(g, N, n, NB, a, Bg, status);
}

size_t rows_tc_smem() {
  return (size_t)kBmStages * kBmStage + sizeof(uint64_t) * (2 * kBmStages + 2) + 16;
}
int rows_nb(int n) { return (2 * n + 15) & ~15; }
int rows_ktq(int n) { return (2 * n + kBmK - 1) / kBmK; }

}  // namespace

bool basis_tc_supported(int n, int p) { return n >= 1 && 2 * n <= 64 && p >= 1; }
bool affine_tc_supported(int n, int nterms) {
  return n >= 1 && 2 * n <= 64 && nterms >= 1 && nterms <= kBmTerms;
}

// scratch of both products: the larger of kBmTerms row blocks and one row
// block plus the p sample rows
size_t rows_tc_bop_floats(int n, int p) {
  const int KTq = rows_ktq(n);
  const int kt = std::max(kBmTerms * KTq, KTq + (p + kBmK - 1) / kBmK);
  return (size_t)kt * 2 * rows_nb(n) * kBmK;
}

// M (N x 2n FP32 rows [Re | Im]) = Gamma zeta^H from the FP32 Q rows, the
// coefficient rows Z2 (2n x p), the (q/m) F rows F2 (p x Nx) and the cells
// jt (tile layout, chunks of PC samples); bop: rows_tc_bop_floats(n, p).
void basis_tc(const GridC& g, int64_t N, int n, int p, int PC, const float* Q2, const float* Z2,
              const float* F2, const uint16_t* jt, float* M, float* bop, int num_sms,
              int* status, cudaStream_t st) {
  const int NB = rows_nb(n), KTq = rows_ktq(n), KT = KTq + (p + kBmK - 1) / kBmK;
  k_basis_tc_prep<<<dim3(KT, NB), kBmK, 0, st>>>(n, p, NB, KTq, Z2, bop);
  if (N <= 0) return;
  RowsArgs a{};
  a.X[0] = Q2;
  a.nterms = 1;
  a.p = p;
  a.PC = PC;
  a.F2 = F2;
  a.jt = jt;
  a.out_v = M;
  const int gx = (int)std::min<int64_t>((N + kBmRows - 1) / kBmRows, num_sms);
  k_basis_M_tc<<<gx, kBmThreads, rows_tc_smem(), st>>>(g, N, n, NB, a, bop, status);
}

// out = sum_t X_t C_t (C: nterms x n x n complex), as FP64 rows (out_d, plus
// aff.base in the increment form) and/or FP32 rows (out_v).
void affine_tc(const GridC& g, int64_t N, int n, const AffineArgsLP& aff, const double2* C,
               double* out_d, float* out_v, float* bop, int num_sms, int* status,
               cudaStream_t st) {
  const int NB = rows_nb(n), KTq = rows_ktq(n), KT = aff.nterms * KTq;
  k_affine_tc_prep<<<dim3(KT, NB), kBmK, 0, st>>>(n, NB, KTq, C, aff.base ? 1 : 0, bop);
  if (N <= 0) return;
  RowsArgs a{};
  for (int tt = 0; tt < aff.nterms; ++tt) a.X[tt] = static_cast<const float*>(aff.X[tt]);
  a.nterms = aff.nterms;
  a.out_v = out_v;
  a.out_d = out_d;
  a.base = out_d ? aff.base : nullptr;
  const int gx = (int)std::min<int64_t>((N + kBmRows - 1) / kBmRows, num_sms);
  k_affine_tc<<<gx, kBmThreads, rows_tc_smem(), st>>>(g, N, n, NB, a, bop, status);
}

void tc_rows_init() {
  cudaFuncSetAttribute(k_basis_M_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)rows_tc_smem());
  cudaFuncSetAttribute(k_affine_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)rows_tc_smem());
}

}  // namespace vpk
