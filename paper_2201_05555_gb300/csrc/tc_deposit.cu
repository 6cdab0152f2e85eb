// Cloud-in-cell deposit of the FP32 form with the reconstruction on the
// tensor cores (tcgen05, kind::tf32), Sec. 2.1 eq. PoissonSystem with
// X_r = U_X Z (Sec. 3.2): for particle l and sample i the position in cell
// units x_li = Re(Q_l zeta_i) / h = sum_k A_lk a_ki / h - B_lk b_ki / h, then
// its cell j and fraction s, deposited as one packed count (1 << Kp) +
// round(s 2^Sp) into cell j of sample i (decoded exactly by the Poisson
// solve), and j stored for the projection and the basis kernel.
//
// Per 128-row tile of Q and chunk of PC samples (one CTA owns a chunk and a
// strided set of tiles):
//   D (128 x 2 PC) = Q_hi [z_hi | z_lo] + Q_lo [z_hi | z_lo]   (K = 2n),
// with z = zeta / h and the B half of its rows negated, every FP32 value v
// split into v_hi = v rounded to TF32 and v_lo = v - v_hi rounded to TF32
// (|v - v_hi - v_lo| <= 2^-22 |v|); x_li = D[l][i] + D[l][PC + i], close to
// the accuracy of FP32 row arithmetic (FP32 accumulation in tensor memory).
//
// Warp roles (21 warps): warps 16-19 stage the Q tiles (split, K-major
// canonical layout, two stages); warp 20 allocates tensor memory and its lane
// 0 issues the MMAs into one of two accumulators; warps 0-15 read an
// accumulator (warp w: lanes 32 (w % 4) .. + 31, samples of quarter w / 4),
// release it and deposit.  Counts accumulate in shared memory (int64,
// order-free) and go to the global counts once per CTA.  Every mbarrier wait
// is bounded (VP_ETIMEDOUT; the kernel then runs to its end and frees its
// tensor memory).
#include "tc_common.cuh"

namespace vpk {
namespace {

constexpr int kDepRows = 128;  // MMA M: particles per tile
constexpr int kDepWarps = 21;  // 16 epilogue, 4 producer, 1 MMA
constexpr int kDepThreads = 32 * kDepWarps;
constexpr int kDepStages = 2;

// byte offset of element (r, k) in a canonical K-major tile with kp K columns
__device__ __forceinline__ uint32_t cmk_off(int r, int k, int kp) {
  return (uint32_t)((r >> 3) * (kp * 32) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

template <int PC>
__global__ void __launch_bounds__(kDepThreads, 1)
k_deposit_tc(GridC g, int64_t N, int n, int p, const float* __restrict__ Q2,
             const float* __restrict__ Zh2, unsigned long long* __restrict__ counts,
             uint16_t* __restrict__ jout, const int* skip, int* status) {
  static_assert(PC == 16 || PC == 32, "four quarters of PC / 4 samples");
  if (skip && *skip) return;
  constexpr int NB = 2 * PC;  // MMA N: [z_hi | z_lo]
  constexpr int SUB = PC / 4;  // samples per epilogue warp
  const int n2 = 2 * n, kp = (n2 + 7) & ~7, Nx = g.Nx;
  const uint32_t aBytes = (uint32_t)kDepRows * kp * 4;  // Q_hi or Q_lo tile
  const uint32_t bBytes = (uint32_t)NB * kp * 4;
  extern __shared__ __align__(1024) unsigned char smraw[];
  unsigned char* A0 = smraw;                              // stages x (hi, lo)
  unsigned char* Bs = smraw + kDepStages * 2 * aBytes;    // [z_hi | z_lo]
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(Bs + bBytes);  // PC x Nx
  uint64_t* bars = reinterpret_cast<uint64_t*>(cnt + PC * Nx);
  uint64_t* full = bars;       // [2] tile staged (128 producer arrivals)
  uint64_t* afree = bars + 2;  // [2] stage read by the MMAs (commit)
  uint64_t* dfull = bars + 4;  // [2] accumulator ready (commit)
  uint64_t* dfree = bars + 6;  // [2] accumulator drained (512 epilogue arrivals)
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 8);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int nch = gridDim.y, chunk = blockIdx.y, c0 = chunk * PC;
  const int pc_eff = min(PC, p - c0);

  // B operand: column c < PC holds z_hi of sample c0 + c, column PC + c its
  // z_lo; rows k >= n take -b (x = sum A a - B b); K padding and missing
  // samples are zero.  Counts start at zero.
  for (int e = t; e < NB * kp; e += kDepThreads) {
    const int c = e / kp, k = e - c * kp, cs = c % PC;
    float v = 0.f;
    if (k < n2 && cs < pc_eff) {
      const float z = Zh2[(int64_t)k * p + c0 + cs];
      const float2 zs = tf32_split(k < n ? z : -z);
      v = c < PC ? zs.x : zs.y;
    }
    *reinterpret_cast<float*>(Bs + cmk_off(c, k, kp)) = v;
  }
  for (int e = t; e < PC * Nx; e += kDepThreads) cnt[e] = 0ull;
  if (t == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&full[s], 128);
      mbar_init(&afree[s], 1);
      mbar_init(&dfull[s], 1);
      mbar_init(&dfree[s], 512);
    }
    mbar_fence_init();
  }
  if (warp == 20) tc_alloc(tslot, 4 * PC);  // two accumulators of 2 PC columns
  fence_proxy_async_smem();                  // B written by the generic proxy
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t ntiles = (N + kDepRows - 1) / kDepRows;
  const int my_tiles = blockIdx.x < ntiles ? (int)((ntiles - 1 - blockIdx.x) / gridDim.x) + 1 : 0;

  if (warp >= 16 && warp < 20) {
    // ---- producers: warp pw stages rows 32 pw .. 32 pw + 31 of the tile.  In
    // iteration i lane l takes row 32 pw + 8 (i % 4) + l % 8 and float4 column
    // 4 (i / 4) + l / 8: the warp's stores fill one contiguous 512-byte run of
    // the canonical layout (conflict-free), its loads 8 rows x 64 bytes; all
    // loads are in flight before the splits and stores
    const int pw = warp - 16, nq = kp / 4;
    for (int it = 0; it < my_tiles; ++it) {
      const int s = it & 1;
      if (it >= 2) mbar_wait(&afree[s], (uint32_t)(((it >> 1) - 1) & 1), status);
      const int64_t base = (int64_t)(blockIdx.x + (int64_t)it * gridDim.x) * kDepRows;
      unsigned char* Ah = A0 + s * 2 * aBytes;
      unsigned char* Al = Ah + aBytes;
#pragma unroll
      for (int ph = 0; ph < 2; ++ph) {  // two phases of eight loads in flight
        float4 v[8];
#pragma unroll
        for (int i2 = 0; i2 < 8; ++i2) {
          const int i = 8 * ph + i2;
          const int r = 32 * pw + 8 * (i & 3) + (lane & 7), q = 4 * (i >> 2) + (lane >> 3);
          const int64_t R = base + r;
          v[i2] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (q < nq && R < N && 4 * q < n2)
            v[i2] = __ldg(reinterpret_cast<const float4*>(Q2 + R * n2) + q);
        }
#pragma unroll
        for (int i2 = 0; i2 < 8; ++i2) {
          const int i = 8 * ph + i2;
          const int r = 32 * pw + 8 * (i & 3) + (lane & 7), q = 4 * (i >> 2) + (lane >> 3);
          if (q < nq) {
            const float2 a = tf32_split(v[i2].x), b = tf32_split(v[i2].y),
                         c = tf32_split(v[i2].z), d = tf32_split(v[i2].w);
            *reinterpret_cast<float4*>(Ah + cmk_off(r, 4 * q, kp)) = make_float4(a.x, b.x, c.x, d.x);
            *reinterpret_cast<float4*>(Al + cmk_off(r, 4 * q, kp)) = make_float4(a.y, b.y, c.y, d.y);
          }
        }
      }
      fence_proxy_async_smem();
      mbar_arrive(&full[s]);
    }
  } else if (warp == 20) {
    // ---- MMA issue
    if (lane == 0) {
      const uint32_t idesc = tc_idesc_tf32(kDepRows, NB);
      const uint32_t sbo = (uint32_t)kp * 32;  // 8 rows of kp floats
      const uint32_t b0 = smem_u32(Bs);
      for (int it = 0; it < my_tiles; ++it) {
        const int s = it & 1, d = it & 1;
        mbar_wait(&full[s], (uint32_t)((it >> 1) & 1), status);
        if (it >= 2) mbar_wait(&dfree[d], (uint32_t)(((it >> 1) - 1) & 1), status);
        tc_fence_after();
        const uint32_t ah = smem_u32(A0 + s * 2 * aBytes), al = ah + aBytes;
        const uint32_t dt = tmem + (uint32_t)(d * NB);
        for (int j = 0; j < kp / 8; ++j) {  // K steps of 8 (two core matrices)
          const uint64_t bd = tc_sdesc(b0 + 256 * j, 128, sbo);
          tc_mma_tf32(dt, tc_sdesc(ah + 256 * j, 128, sbo), bd, idesc, j > 0);
          tc_mma_tf32(dt, tc_sdesc(al + 256 * j, 128, sbo), bd, idesc, 1u);
        }
        tc_commit(&afree[s]);
        tc_commit(&dfull[d]);
      }
    }
    __syncwarp();
  } else {
    // ---- epilogue: warp w reads lanes 32 (w % 4) .. + 31, samples of quarter w / 4
    const int quarter = warp >> 2, row = 32 * (warp & 3) + lane;
    const long long one = 1ll << g.Sp;
    const float pscale = (float)one, inv_Nx = (float)g.inv_Nx;
    const unsigned long long pbit = 1ull << g.Kp;
    for (int it = 0; it < my_tiles; ++it) {
      const int d = it & 1;
      mbar_wait(&dfull[d], (uint32_t)((it >> 1) & 1), status);
      tc_fence_after();
      const uint32_t ta =
          tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(d * NB + quarter * SUB);
      uint32_t vh[SUB], vl[SUB];
      if constexpr (SUB == 8) {
        tc_ld8(ta, vh);       // z_hi part of samples quarter * SUB ..
        tc_ld8(ta + PC, vl);  // z_lo part
      } else {
        tc_ld4(ta, vh);
        tc_ld4(ta + PC, vl);
      }
      tc_wait_ld();
      tc_fence_before();
      mbar_arrive(&dfree[d]);
      const int64_t tile = blockIdx.x + (int64_t)it * gridDim.x;
      const int64_t R = tile * kDepRows + row;
      if (R < N) {
        uint32_t js[SUB / 2];
#pragma unroll
        for (int u = 0; u < SUB; ++u) {
          const int c = quarter * SUB + u;
          // cell and fraction in FP32 (both exact), as the FP32 SIMT deposit
          const float th = __uint_as_float(vh[u]) + __uint_as_float(vl[u]);
          const float fl = floorf(th);
          const int q = __float2int_rn((th - fl) * pscale);
          int jr = (int)fl;
          const int wq = (int)floorf((float)jr * inv_Nx);
          jr -= wq * Nx;
          if (jr < 0) jr += Nx;
          if (jr >= Nx) jr -= Nx;
          if (u & 1) js[u >> 1] |= (uint32_t)jr << 16;
          else js[u >> 1] = (uint32_t)jr;
          if (c < pc_eff) atomicAdd(cnt + c * Nx + jr, pbit + (unsigned long long)q);
        }
        const int64_t tl = R / TILE_ROWS;
        uint16_t* dst = jout + jt_block(tl, chunk, nch, PC) + (R - tl * TILE_ROWS) * PC + quarter * SUB;
        if constexpr (SUB == 8)
          *reinterpret_cast<uint4*>(dst) = make_uint4(js[0], js[1], js[2], js[3]);
        else
          *reinterpret_cast<uint2*>(dst) = make_uint2(js[0], js[1]);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 20) tc_dealloc(tmem, 4 * PC);
  for (int e = t; e < PC * Nx; e += kDepThreads) {
    const int c = e / Nx;
    if (c < pc_eff && cnt[e]) atomicAdd(&counts[(int64_t)(c0 + c) * Nx + (e - c * Nx)], cnt[e]);
  }
}

template <int PC>
size_t dep_smem(int n2, int Nx) {
  const int kp = (n2 + 7) & ~7;
  return (size_t)kDepStages * 2 * kDepRows * kp * 4 + (size_t)2 * PC * kp * 4 +
         sizeof(unsigned long long) * (size_t)PC * Nx + sizeof(uint64_t) * 8 + 16;
}

}  // namespace

// Tensor-core deposit: FP32 rows with n2 a multiple of 4 and at most 64, the
// packed counts of the FP32 form, sample chunks of 16 or 32 and the shared
// memory of one CTA per SM.
bool deposit_tc_supported(int n, int p, int Nx, int Kp) {
  const int PC = chunk_pc(p, Nx), n2 = 2 * n;
  if (Kp <= 0 || (n2 & 3) || n2 > 64 || (PC != 16 && PC != 32)) return false;
  const size_t sm = PC == 32 ? dep_smem<32>(n2, Nx) : dep_smem<16>(n2, Nx);
  return sm <= 227 * 1024;
}

// Grid (gridx, ceil(p / PC)); cell indices in the layout of k_deposit_lp.
void deposit_tc(const GridC& g, int64_t N, int n, int p, const float* Q2, const float* Zh2,
                unsigned long long* counts, uint16_t* jout, int gridx, const int* skip,
                int* status, cudaStream_t st) {
  const int PC = chunk_pc(p, g.Nx), ch = ceil_div(p, PC);
  if (PC == 32)
    k_deposit_tc<32><<<dim3(gridx, ch), kDepThreads, dep_smem<32>(2 * n, g.Nx), st>>>(
        g, N, n, p, Q2, Zh2, counts, jout, skip, status);
  else
    k_deposit_tc<16><<<dim3(gridx, ch), kDepThreads, dep_smem<16>(2 * n, g.Nx), st>>>(
        g, N, n, p, Q2, Zh2, counts, jout, skip, status);
}

void tc_deposit_init() {
  cudaFuncSetAttribute(k_deposit_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       227 * 1024);
  cudaFuncSetAttribute(k_deposit_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       227 * 1024);
}

}  // namespace vpk
