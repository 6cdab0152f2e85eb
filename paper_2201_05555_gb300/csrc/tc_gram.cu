// Gram matrices of the FP32 form on the tensor cores (tcgen05, kind::tf32):
// for pairs (X, Y) of row blocks (N x n complex rows stored [Re | Im] in FP32)
// the sums over the N rows X^H Y (n x n complex; the basis velocity, the
// Cayley retraction and the tangent velocity, Sec. 3.2 and Sec. 5), or the
// real X^T X of one block (G_V = U_V^T U_V of the stored rows).
//
// All of them come from the real product P = [Xr Xi]^T [Yr Yi] (2n x 2n):
// X^H Y = (P11 + P22) + i (P12 - P21).  Per CTA (a strided set of 32-row
// tiles) and pair s the accumulator D_s (128 x 64) = [X_hi; X_lo]^T (Y_hi +
// Y_lo) lives in tensor memory (64 columns per pair), with every FP32 value
// v split into v_hi = v rounded to TF32 and v_lo = v - v_hi rounded to TF32;
// rows c and c + 64 of D_s add up, in FP64, to P's row c.  2n <= 64,
// zero-padded.
//
// One staged buffer per row block and stage, [hi | lo] in the K-major
// no-swizzle canonical layout (element (c, k) of the hi half at byte
// (c / 8) * 1024 + (k / 4) * 128 + (c % 8) * 16 + (k % 4) * 4, the lo half
// 8 KB after it), serves at once as A (M = 128: hi rows then lo rows) and as
// the two B operands (N = 64: the hi half, then the lo half).  Three stages,
// the next tile's global loads issued before the current one is split; thread
// 0 issues the MMAs and commits each stage; every wait is bounded.  Output:
// per-block partials in the layout of the SIMT kernels (complex pairs:
// part[bx][s][k1][k2] as (re, im); real: part[bx][i][j]), summed in block
// order by the partial reduction.
#include "tc_common.cuh"

namespace vpk {
namespace {

constexpr int kGRows = 32;           // rows (the K extent) per stage
constexpr int kGStages = 3;
constexpr int kGBlock = 16384;       // one block's staged tile: hi (8 KB) + lo (8 KB)
constexpr int kGThreads = 256;
constexpr int kGMaxBlocks = 4;
constexpr int kGMaxPairs = 7;        // 64 TMEM columns per pair

__device__ __forceinline__ uint32_t g_off(int c, int k) {
  return (uint32_t)((c >> 3) * 1024 + (k >> 2) * 128 + (c & 7) * 16 + (k & 3) * 4);
}

__global__ void __launch_bounds__(kGThreads, 2)
k_gram_tc(int64_t N, int n, GramArgsLP a, int real_out, double* __restrict__ part, int* status) {
  extern __shared__ __align__(1024) unsigned char smraw[];
  const int n2 = 2 * n, nb = a.nblk, np = a.npairs;
  const uint32_t stage_bytes = (uint32_t)nb * kGBlock;
  unsigned char* stages = smraw;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smraw + kGStages * stage_bytes);  // stages + done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kGStages + 1);
  const int t = threadIdx.x, warp = t >> 5;
  // columns >= 2n of every block stay zero in every stage
  for (int e = t; e < kGStages * (int)stage_bytes / 4; e += kGThreads)
    reinterpret_cast<float*>(stages)[e] = 0.f;
  if (t == 0) {
    for (int s = 0; s <= kGStages; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
  }
  const uint32_t ncols = np <= 1 ? 64 : np <= 2 ? 128 : np <= 4 ? 256 : 512;
  if (warp == 0) tc_alloc(tslot, ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = tc_idesc_tf32(128, 64);
  const int64_t ntiles = (N + kGRows - 1) / kGRows;
  // thread roles: column c = t % 64, row groups (t / 64) + {0, 4} of the tile
  const int c = t & 63;
  float qv[kGMaxBlocks][2][4];
  // 32-bit offsets within a tile: row 4 kq + u, column c
  const int co = 4 * (t >> 6) * n2 + c;
  auto load = [&](int64_t tile) {
    const int64_t r0 = tile * kGRows;
    const int rows = N - r0 < (int64_t)kGRows ? (int)(N - r0) : kGRows;  // >= 1
#pragma unroll
    for (int b = 0; b < kGMaxBlocks; ++b) {
      if (b >= nb) {  // blocks past nb stage zeros
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int u = 0; u < 4; ++u) qv[b][h][u] = 0.f;
        continue;
      }
      const float* x = static_cast<const float*>(a.blk[b]) + r0 * n2 + co;
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int r = 4 * ((t >> 6) + 4 * h) + u;
          qv[b][h][u] = (c < n2 && r < rows) ? __ldg(x + (16 * h + u) * n2) : 0.f;
        }
    }
  };
  if (blockIdx.x < ntiles) load(blockIdx.x);
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int s = it % kGStages;
    unsigned char* S = stages + s * stage_bytes;
    if (it >= kGStages) mbar_wait(&bars[s], (uint32_t)((it / kGStages - 1) & 1), status);
    if (c < n2) {
#pragma unroll
      for (int b = 0; b < kGMaxBlocks; ++b) {
        if (b >= nb) break;
        unsigned char* B = S + b * kGBlock;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int kq = (t >> 6) + 4 * h;
          const float2 v0 = tf32_split(qv[b][h][0]), v1 = tf32_split(qv[b][h][1]),
                       v2 = tf32_split(qv[b][h][2]), v3 = tf32_split(qv[b][h][3]);
          *reinterpret_cast<float4*>(B + g_off(c, 4 * kq)) = make_float4(v0.x, v1.x, v2.x, v3.x);
          *reinterpret_cast<float4*>(B + 8192 + g_off(c, 4 * kq)) =
              make_float4(v0.y, v1.y, v2.y, v3.y);
        }
      }
    }
    if (tile + gridDim.x < ntiles) load(tile + gridDim.x);  // next tile, in flight now
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
      const uint32_t s0 = smem_u32(S);
      for (int q = 0; q < np; ++q) {
        const uint32_t xa = s0 + (uint32_t)a.pa[q] * kGBlock, yb = s0 + (uint32_t)a.pb[q] * kGBlock;
        const uint32_t dq = tmem + (uint32_t)(64 * q);
#pragma unroll
        for (int j = 0; j < kGRows / 8; ++j) {
          const uint64_t ad = tc_sdesc(xa + 256 * j, 128, 1024);
          tc_mma_tf32(dq, ad, tc_sdesc(yb + 256 * j, 128, 1024), idesc, (it > 0 || j > 0));
          tc_mma_tf32(dq, ad, tc_sdesc(yb + 8192 + 256 * j, 128, 1024), idesc, 1u);
        }
      }
      tc_commit(&bars[s]);
    }
  }
  if (t == 0) {
    if (it > 0) tc_commit(&bars[kGStages]);
    else mbar_expect_tx(&bars[kGStages], 0);
  }
  mbar_wait(&bars[kGStages], 0u, status);
  tc_fence_after();
  // epilogue, pair by pair: D_q staged as floats (128 x 65) in the stage buffers
  float* Ds = reinterpret_cast<float*>(stages);
  const int out_per = real_out ? n2 * n2 : n * n;
  for (int q = 0; q < np; ++q) {
    if (warp < 4) {
      uint32_t v[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (it > 0) {
          tc_ld32(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(64 * q + 32 * half), v);
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) v[j] = 0u;
        }
        const int row = 32 * warp + (t & 31);
#pragma unroll
        for (int j = 0; j < 32; ++j) Ds[row * 65 + 32 * half + j] = __uint_as_float(v[j]);
      }
    }
    __syncthreads();
    auto P = [&](int i, int j) { return (double)Ds[i * 65 + j] + (double)Ds[(i + 64) * 65 + j]; };
    for (int e = t; e < out_per; e += kGThreads) {
      if (real_out) {
        const int i = e / n2, j = e - i * n2;
        part[(int64_t)blockIdx.x * out_per + e] = P(i, j);
      } else {
        const int k1 = e / n, k2 = e - k1 * n;
        const double re = P(k1, k2) + P(n + k1, n + k2), im = P(k1, n + k2) - P(n + k1, k2);
        double2* o = reinterpret_cast<double2*>(part);
        o[((int64_t)blockIdx.x * np + q) * out_per + e] = make_double2(re, im);
      }
    }
    __syncthreads();
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, ncols);
}

size_t gram_tc_smem(int nblk) {
  return (size_t)kGStages * nblk * kGBlock + sizeof(uint64_t) * (kGStages + 1) + 16;
}

}  // namespace

bool gram_tc_supported(int n, int nblk, int npairs) {
  return 2 * n <= 64 && nblk >= 1 && nblk <= kGMaxBlocks && npairs >= 1 && npairs <= kGMaxPairs;
}

// Complex pairs (real_out = 0, part as double2 [gridx][npairs][n][n]) or the
// real Gram of block 0 (real_out = 1, part [gridx][2n][2n]).
void gram_tc(int64_t N, int n, const GramArgsLP& a, int real_out, double* part, int gridx,
             int* status, cudaStream_t st) {
  k_gram_tc<<<gridx, kGThreads, gram_tc_smem(a.nblk), st>>>(N, n, a, real_out, part, status);
}

void tc_gram_init() {
  cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)gram_tc_smem(kGMaxBlocks));
}

}  // namespace vpk
