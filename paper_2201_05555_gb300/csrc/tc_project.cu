// Projection g_X = U_X^T G of the FP32 form on the tensor cores (tcgen05,
// kind::tf32), Sec. 3.2, eq. grads: for every sample i and basis column k,
// g_ki = sum_l U_X,lk G_li with G_li = (q/m) F_i[j_li], the field of sample i
// at the cell j_li of particle l (written by the deposit at the same state).
//
// The sum over the N particles is the K dimension of the MMA.  Each CTA owns
// one chunk of PC samples (16 or 32) and a strided set of 32-row tiles; its
// accumulator D lives in tensor memory for the CTA's whole life:
//   D (128 x PC) = A (128 x K) B (K x PC),
//   A = [Q_hi^T; Q_lo^T]  (rows 0..63: the FP32 row Q_l split as
//                          Q_hi = Q rounded to TF32; rows 64..127: Q_lo =
//                          Q - Q_hi rounded to TF32, tf32_split),
//   B = G_hi + G_lo       (two MMAs with the same A, G split the same way),
// so rows m and m + 64 of D hold Q_hi G and Q_lo G, whose sum (taken in FP64
// in the epilogue) is Q G up to the split (2^-22 of each operand) and the
// FP32 accumulation: close to the accuracy of FP32 row arithmetic.  2n <= 64
// (zero-padded to 64).
//
// Operands are staged by all 256 threads in the K-major, no-swizzle canonical
// layout of tcgen05 (8 x 16-byte core matrices: element (r, k) of a tile at
// byte (r / 8) * 1024 + (k / 4) * 128 + (r % 8) * 16 + (k % 4) * 4), in three
// stages; thread 0 issues the MMAs of a stage and commits them to the stage's
// mbarrier, which the producers wait on before they overwrite it.  Every wait
// is bounded (VP_ETIMEDOUT, then the kernel runs to its end and frees its
// tensor memory).  Output: per-block partial sums part[bx][k][p] (FP64), the
// layout of k_project_lp, summed in block order by the coefficient update.
#include "tc_common.cuh"

namespace vpk {
namespace {

constexpr int kTcRows = 32;     // rows of Q (the K extent) per stage
constexpr int kTcStages = 3;
constexpr int kTcM = 128;       // MMA M: 64 hi rows + 64 lo rows
constexpr int kTcThreads = 256;

// byte offset of element (r, k) in a canonical K-major tile of 32 K columns
__device__ __forceinline__ uint32_t cm_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

template <int PC>
__global__ void __launch_bounds__(kTcThreads)
k_project_tc(GridC g, int64_t N, int n, int p, const float* __restrict__ Q2,
             const float* __restrict__ F2, const uint16_t* __restrict__ jt,
             double* __restrict__ part, const int* skip, int* status) {
  static_assert(PC == 16 || PC == 32, "MMA N is the sample chunk");
  if (skip && *skip) return;
  constexpr uint32_t kABytes = kTcM * kTcRows * 4;  // 16 KB
  constexpr uint32_t kBBytes = PC * kTcRows * 4;    // G_hi or G_lo
  constexpr uint32_t kStage = kABytes + 2 * kBBytes;
  constexpr uint32_t kCols = 32;                    // TMEM columns (>= PC, power of 2)
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int n2 = 2 * n, Nx = g.Nx;
  const int nch = gridDim.y, chunk = blockIdx.y, c0 = chunk * PC;
  const int t = threadIdx.x, warp = t >> 5;
  // layout: stages (1024-aligned), then F (PC x Nx) and the barriers; the
  // epilogue stages D (kTcM x (PC + 1) floats) in the stage buffers
  unsigned char* stages = smraw;
  float* Fs = reinterpret_cast<float*>(smraw + kTcStages * kStage);
  float* Ds = reinterpret_cast<float*>(smraw);
  uint64_t* bars = reinterpret_cast<uint64_t*>(Fs + PC * Nx);  // stages + done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kTcStages + 1);
  static_assert(kTcM * (PC + 1) * 4 <= kTcStages * kStage, "D staging fits the stages");

  for (int e = t; e < PC * Nx; e += kTcThreads) {
    const int c = e / Nx;
    Fs[e] = (c0 + c < p) ? F2[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : 0.f;
  }
  // A rows for basis columns >= 2n (both halves) stay zero in every stage
  for (int e = t; e < kTcStages * (int)(kABytes / 4); e += kTcThreads) {
    const int s = e / (kABytes / 4), w = e - s * (kABytes / 4);
    reinterpret_cast<float*>(stages + s * kStage)[w] = 0.f;
  }
  if (t == 0) {
    for (int s = 0; s <= kTcStages; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  if (warp == 0) tc_alloc(tslot, kCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc_idesc_tf32(kTcM, PC);
  const int64_t ntiles = (N + kTcRows - 1) / kTcRows;
  const int pc_eff = min(PC, p - c0);

  // The global loads of a tile (its Q values and cell indices) are issued one
  // iteration ahead into registers, so their latency overlaps the split and
  // the stores of the tile before.  Thread roles: A, basis column m = t % 64
  // and row groups (t / 64) + {0, 4}; B, sample column c = t % PC and row
  // group t / PC (PC = 32: all threads; PC = 16: threads < 128).
  const int m = t & 63;
  const bool b_role = t < PC * (kTcRows / 4);
  const int bc = t % PC, bkq = t / PC;
  float qa[2][4];
  uint16_t jb[4];
  // per-thread offsets within a tile, 32-bit: Q row 4 kq + u of column m,
  // and the cell of row 4 bkq + u, sample bc, inside the tile's index block
  // (a 32-row tile lies in one TILE_ROWS-row block of the cell layout)
  const int qo = 4 * (t >> 6) * n2 + m;
  const bool q_role = m < n2, j_role = b_role && bc < pc_eff;
  auto load = [&](int64_t tile) {
    const int64_t r0 = tile * kTcRows;
    const int rows = N - r0 < (int64_t)kTcRows ? (int)(N - r0) : kTcRows;  // >= 1
    const float* q = Q2 + r0 * n2 + qo;
    const int64_t tl = r0 / TILE_ROWS;
    const uint16_t* jp =
        jt + jt_block(tl, chunk, nch, PC) + ((int)(r0 - tl * TILE_ROWS) + 4 * bkq) * PC + bc;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int r = 4 * ((t >> 6) + 4 * h) + u;
        qa[h][u] = (q_role && r < rows) ? __ldg(q + (16 * h + u) * n2) : 0.f;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      jb[u] = (j_role && 4 * bkq + u < rows) ? __ldg(jp + u * PC) : (uint16_t)0xFFFFu;
  };
  if (blockIdx.x < ntiles) load(blockIdx.x);
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = it % kTcStages;
    unsigned char* A = stages + s * kStage;
    unsigned char* Bh = A + kABytes;
    unsigned char* Bl = Bh + kBBytes;
    if (it >= kTcStages)  // the MMAs that read this stage last time are done
      mbar_wait(&bars[s], (uint32_t)((it / kTcStages - 1) & 1), status);
    // A: Q_hi in rows m, Q_lo in rows m + 64 (columns >= 2n stay zero)
    if (m < n2) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kq = (t >> 6) + 4 * h;
        const float2 a0 = tf32_split(qa[h][0]), a1 = tf32_split(qa[h][1]),
                     a2 = tf32_split(qa[h][2]), a3 = tf32_split(qa[h][3]);
        *reinterpret_cast<float4*>(A + cm_off(m, 4 * kq)) = make_float4(a0.x, a1.x, a2.x, a3.x);
        *reinterpret_cast<float4*>(A + cm_off(m + 64, 4 * kq)) =
            make_float4(a0.y, a1.y, a2.y, a3.y);
      }
    }
    // B: G = (q/m) F of the sample at the particle's cell, split
    if (b_role) {
      float v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = jb[u] != 0xFFFFu ? Fs[bc * Nx + jb[u]] : 0.f;
      const float2 b0 = tf32_split(v[0]), b1 = tf32_split(v[1]), b2 = tf32_split(v[2]),
                   b3 = tf32_split(v[3]);
      *reinterpret_cast<float4*>(Bh + cm_off(bc, 4 * bkq)) = make_float4(b0.x, b1.x, b2.x, b3.x);
      *reinterpret_cast<float4*>(Bl + cm_off(bc, 4 * bkq)) = make_float4(b0.y, b1.y, b2.y, b3.y);
    }
    if (tile + gridDim.x < ntiles) load(tile + gridDim.x);  // next tile, in flight now
    fence_proxy_async_smem();  // generic-proxy writes before the MMAs read them
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(A), bh0 = smem_u32(Bh), bl0 = smem_u32(Bl);
#pragma unroll
      for (int j = 0; j < kTcRows / 8; ++j) {  // K steps of 8 rows (two core matrices)
        const uint64_t ad = tc_sdesc(a0 + 256 * j, 128, 1024);
        tc_mma_tf32(tmem, ad, tc_sdesc(bh0 + 256 * j, 128, 1024), idesc, (it > 0 || j > 0));
        tc_mma_tf32(tmem, ad, tc_sdesc(bl0 + 256 * j, 128, 1024), idesc, 1u);
      }
      tc_commit(&bars[s]);
    }
  }
  // all MMAs done: D holds the sums of this block's rows
  if (t == 0) {
    if (it > 0) tc_commit(&bars[kTcStages]);
    else mbar_expect_tx(&bars[kTcStages], 0);  // nothing issued: complete the phase
  }
  mbar_wait(&bars[kTcStages], 0u, status);
  tc_fence_after();
  if (warp < 4) {
    uint32_t v[32];
    if (it > 0) {
      tc_ld32(tmem + ((uint32_t)(32 * warp) << 16), v);
    } else {
#pragma unroll
      for (int c = 0; c < 32; ++c) v[c] = 0u;
    }
    const int row = 32 * warp + (t & 31);
#pragma unroll
    for (int c = 0; c < PC; ++c) Ds[row * (PC + 1) + c] = __uint_as_float(v[c]);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, kCols);
  for (int e = t; e < n2 * PC; e += kTcThreads) {
    const int m = e / PC, c = e - m * PC;
    if (c >= pc_eff) continue;
    const double v = (double)Ds[m * (PC + 1) + c] + (double)Ds[(m + 64) * (PC + 1) + c];
    part[(int64_t)blockIdx.x * n2 * p + (int64_t)m * p + c0 + c] = (m < n) ? v : -v;
  }
}

template <int PC>
size_t tc_smem(int Nx) {
  return (size_t)kTcStages * (kTcM * kTcRows * 4 + 2 * PC * kTcRows * 4) +
         sizeof(float) * (size_t)PC * Nx + sizeof(uint64_t) * (kTcStages + 1) + 16;
}

}  // namespace

bool project_tc_supported(int n, int p, int Nx) {
  const int PC = chunk_pc(p, Nx);
  return 2 * n <= 64 && (PC == 16 || PC == 32);
}

// Same grid and partials as the FP32 k_project_lp: (gridx, ceil(p / PC)).
void project_tc(const GridC& g, int64_t N, int n, int p, const float* Q2, const float* F2,
                const uint16_t* jt, double* part, int gridx, const int* skip, int* status,
                cudaStream_t st) {
  const int PC = chunk_pc(p, g.Nx), ch = ceil_div(p, PC);
  if (PC == 32)
    k_project_tc<32><<<dim3(gridx, ch), kTcThreads, tc_smem<32>(g.Nx), st>>>(
        g, N, n, p, Q2, F2, jt, part, skip, status);
  else
    k_project_tc<16><<<dim3(gridx, ch), kTcThreads, tc_smem<16>(g.Nx), st>>>(
        g, N, n, p, Q2, F2, jt, part, skip, status);
}

void tc_init() {
  cudaFuncSetAttribute(k_project_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc_smem<32>(VP_MAX_NX));
  cudaFuncSetAttribute(k_project_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)tc_smem<16>(VP_MAX_NX));
}

}  // namespace vpk
