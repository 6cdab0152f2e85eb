// Particle-loop, Gram and affine kernels of the reduced model in FP32-based
// arithmetic, for two arithmetic policies:
//
// ArithDF  double-float: every FP64 operand is an unevaluated sum hi + lo of
//          two floats (|lo| <= ulp(hi)/2, about 48 significant bits) and every
//          dot product uses the compensated algorithm "Dot2" of Ogita, Rump
//          and Oishi (SIAM J. Sci. Comput. 26, 2005): an error-free product
//          (FMA) and an error-free sum (TwoSum) per term, the rounding errors
//          accumulated separately, as if computed in twice the precision.
//          GB300 executes FP32 at 58x its FP64 rate (measured 68.8 vs 1.19
//          TFLOP/s), so this meets the FP64 tolerance several times faster.
// ArithF32 plain FP32 storage of the N-row quantities and FP32 accumulation
//          (the precision form); per-block partial sums, reductions, the small
//          dense algebra and the energies stay FP64.
//
// Storage of Q and zeta stays FP64 in both; Q is split once per change into
// the policy's row format.  The cell index of every (particle, sample) is
// written by the deposit and reused by the projection and the basis kernel
// at the same (Q, zeta).
#include "vp_internal.cuh"

#include <algorithm>

namespace vpk {

struct ArithDF {
  using V = float2;
  static constexpr bool kVec4 = false;
  static __device__ __forceinline__ V from(double d) { return df_split_bits(d); }
  // an FP32 value as V, without the FP64 pipe: (f, 0)
  static __device__ __forceinline__ V from_f(float f) { return make_float2(f, 0.f); }
  static __device__ __forceinline__ V zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ V neg(V a) { return make_float2(-a.x, -a.y); }
  static __device__ __forceinline__ float hi(V a) { return a.x; }
  static __device__ __forceinline__ float lo(V a) { return a.y; }
  // running compensated sum s + c
  struct A {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void fma2(V a, V b) {
      float p = a.x * b.x;
      float e = fmaf(a.x, b.x, -p);
      e = fmaf(a.x, b.y, e);
      e = fmaf(a.y, b.x, e);
      float t = s + p;
      float bp = t - s;
      float es = (s - (t - bp)) + (p - bp);
      s = t;
      c += es + e;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)c; }
    __device__ __forceinline__ V out() const {
      float h = s + c;
      return make_float2(h, c - (h - s));
    }
  };
};

struct ArithF32 {
  using V = float;
  static constexpr bool kVec4 = true;  // rows of plain floats: float4 loads apply
  static __device__ __forceinline__ V from(double d) { return df_split_bits(d).x; }
  static __device__ __forceinline__ V from_f(float f) { return f; }
  static __device__ __forceinline__ V zero() { return 0.f; }
  static __device__ __forceinline__ V neg(V a) { return -a; }
  static __device__ __forceinline__ float hi(V a) { return a; }
  static __device__ __forceinline__ float lo(V) { return 0.f; }
  struct A {
    float s;
    __device__ __forceinline__ void zero() { s = 0.f; }
    __device__ __forceinline__ void fma2(V a, V b) { s = fmaf(a, b, s); }
    __device__ __forceinline__ double value() const { return (double)s; }
    __device__ __forceinline__ V out() const { return s; }
  };
};

// Cell index and fixed-point fraction of t = th + tl (cell units,
// unwrapped): j in [0, Nx), w1 = round(frac * 2^S) in [0, 2^S], S >= 24.
// Only 32-bit conversions: with the exact sums th - floor(th) = a + e and
// a + tl = b + be (TwoSum), frac = b + (be + e); b1 = round(b 2^24) and the
// exact remainder b2 = b - b1 2^-24 give w1 = b1 2^(S-24) + round((b2 + be + e) 2^S),
// whose second term is below 2^(S-23) <= 2^29 in magnitude.
__device__ __forceinline__ void cell_fixed(float th, float tl, int Nx, float inv_Nx, float scale,
                                           int S, long long one, int& j, long long& w1) {
  float fl = floorf(th);
  float a = th - fl;
  float z = a - th;
  float e = (th - (a - z)) + (-fl - z);
  float b = a + tl;
  float bz = b - a;
  float be = (a - (b - bz)) + (tl - bz);
  int b1 = __float2int_rn(b * 16777216.0f);
  float b2 = fmaf(-(float)b1, 5.9604644775390625e-08f, b);
  long long q = (long long)b1 * (1ll << (S - 24)) + (long long)__float2int_rn((b2 + (be + e)) * scale);
  int jr = (int)fl;
  if (q < 0) { q += one; jr -= 1; }
  if (q > one) { q -= one; jr += 1; }
  int wq = (int)floorf((float)jr * inv_Nx);
  jr -= wq * Nx;
  if (jr < 0) jr += Nx;
  if (jr >= Nx) jr -= Nx;
  j = jr;
  w1 = q;
}

// register-resident coefficients in the deposit: instances for n up to each
// bound (double-float rows; FP32 rows with n % 4 == 0), the smallest that
// holds n is launched so that small ranks keep a small register count
static constexpr int kDepNrDF[2] = {4, 10};
static constexpr int kDepNrF32[3] = {8, 16, 32};

// the register bound launched for rank n, 0 for the shared-memory operands
template <class AR>
static inline int dep_nr(int n) {
  if constexpr (AR::kVec4) {
    if (n & 3) return 0;
    for (int b : kDepNrF32)
      if (n <= b) return b;
  } else {
    for (int b : kDepNrDF)
      if (n <= b) return b;
  }
  return 0;
}

static inline int chunk_w(int p, int Nx) {
  int pc = 1;
  while (pc < p && pc < 32) pc <<= 1;
  while (pc > 1 && (size_t)pc * Nx * 8 > 96 * 1024) pc >>= 1;
  return pc;
}

// ------------------------------------------------------------- conversions
template <class AR>
__global__ void k_split(int64_t m, const double* __restrict__ x, typename AR::V* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < m) out[e] = AR::from(x[e]);
}

// once per field evaluation: Z2 = Z, Zh2 = Z / h (2n x p), F2 = q/m F (p x Nx)
template <class AR>
__global__ void k_prep(GridC g, int64_t nz, const double* __restrict__ Z, typename AR::V* Z2,
                       typename AR::V* Zh2, int64_t nf, const double* __restrict__ F,
                       typename AR::V* F2, const int* skip) {
  if (skip && *skip) return;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nz) {
    double z = Z[e];
    if (Z2) Z2[e] = AR::from(z);
    if (Zh2) Zh2[e] = AR::from(z * g.inv_h);
  } else if (F && e - nz < nf) {
    F2[e - nz] = AR::from(g.qm * F[e - nz]);
  }
}

template <class V>
__device__ __forceinline__ void load_rows(V* Qs, int ldq, const V* __restrict__ Q2, int n2,
                                          int64_t base, int rows) {
  for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
    int r = e / n2, k = e - r * n2;
    Qs[r * ldq + k] = Q2[(base + r) * n2 + k];
  }
}

template <class AR>
__device__ __forceinline__ void load_zc(typename AR::V* Zs, int ldz,
                                        const typename AR::V* __restrict__ Z2, int n2, int p,
                                        int c0, int PC) {
  for (int e = threadIdx.x; e < n2 * PC; e += blockDim.x) {
    int k = e / PC, ii = e - k * PC;
    Zs[k * ldz + ii] = (c0 + ii < p) ? Z2[(int64_t)k * p + c0 + ii] : AR::zero();
  }
}

// ------------------------------------------------------------------ deposit
// X_r = Re(Q zeta) / h per (particle, sample) in the policy's arithmetic,
// then the cell index and fixed-point weights: charge counts accumulate in
// shared memory (int64, order-free) and go to the global counts once per
// block.  Full tiles of Q rows arrive by bulk copies into two stages, the
// copy of the block's next tile running during the current one; a partial
// last tile is read with plain loads.  With NR > 0 (n <= NR; for FP32 rows
// also n % 4 == 0) each thread keeps its sample's coefficients in registers
// for the whole launch, so the dot product reads only Q from shared memory
// (broadcast within the warp); the terms are summed in the same order as
// with the shared-memory operands.
template <class AR, int NR>
__global__ void k_deposit_lp(GridC g, int64_t N, int n, int p, int PC,
                             const typename AR::V* __restrict__ Q2,
                             const typename AR::V* __restrict__ Zh2,
                             unsigned long long* __restrict__ counts, uint16_t* __restrict__ jout,
                             const int* skip, int* status) {
  using V = typename AR::V;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, ldz = PC + 1, Nx = g.Nx;
  const uint32_t qbytes = (uint32_t)(sizeof(V) * TILE_ROWS * n2);
  const size_t qst = (qbytes + 15) & ~size_t(15);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  unsigned char* Qs0 = smraw + 16;
  V* Zs = reinterpret_cast<V*>(Qs0 + 2 * qst);
  // FP32 rows with n % 4 == 0: the coefficients also go sample-major (Zt,
  // rows padded to a multiple of 4) so that both operands of the dot
  // product arrive as float4 (one shared-memory load per 4 multiply-adds)
  const bool vec = AR::kVec4 && (n & 3) == 0;
  const bool zt = vec && NR == 0;  // Zt only when the coefficients stay in shared memory
  const int ldk = n2 + 4;
  const size_t zto = (16 + 2 * qst + sizeof(V) * n2 * ldz + 15) & ~size_t(15);
  const size_t zoff = zto + (zt ? ((sizeof(float) * PC * ldk + 15) & ~size_t(15)) : 0);
  float* Zt = reinterpret_cast<float*>(smraw + zto);
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smraw + zoff);
  const int c0 = blockIdx.y * PC;
  load_zc<AR>(Zs, ldz, Zh2, n2, p, c0, PC);
  if (zt) {
    __syncthreads();
    for (int e = threadIdx.x; e < n2 * PC; e += blockDim.x) {
      const int k = e / PC, i = e - k * PC;
      Zt[i * ldk + k] = AR::hi(Zs[k * ldz + i]);
    }
  }
  for (int e = threadIdx.x; e < PC * Nx; e += blockDim.x) cnt[e] = 0ull;
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const bool active = c0 + ii < p;
  const long long one = 1ll << g.S;
  const float scale = (float)g.fp_scale, inv_Nx = (float)g.inv_Nx;
  const bool pack = AR::kVec4 && g.Kp > 0;  // the Poisson solve decodes the same form
  const float pscale = (float)(1 << (g.Sp > 0 ? g.Sp : 0));
  const unsigned long long pbit = g.Kp > 0 ? (1ull << g.Kp) : 0ull;
  unsigned long long* mycnt = cnt + ii * Nx;
  const int64_t ntiles = (N + TILE_ROWS - 1) / TILE_ROWS;
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // registers: za[k] = a_k / h, zb[k] = b_k / h of sample c0 + ii
  V za[NR > 0 ? NR : 1], zb[NR > 0 ? NR : 1];
  if constexpr (NR > 0) {
#pragma unroll
    for (int k = 0; k < NR; ++k) {
      za[k] = k < n ? Zs[k * ldz + ii] : AR::zero();
      zb[k] = k < n ? Zs[(n + k) * ldz + ii] : AR::zero();
    }
  }
  auto issue = [&](int64_t tl, int st) {
    if (t != 0 || tl >= ntiles || (tl + 1) * TILE_ROWS > N) return;
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[st], qbytes);
    bulk_g2s(Qs0 + st * qst, Q2 + tl * TILE_ROWS * n2, qbytes, &bar[st]);
  };
  int it = 0;
  issue(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int stg = it & 1;
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    V* Qs = reinterpret_cast<V*>(Qs0 + stg * qst);
    issue(tile + gridDim.x, stg ^ 1);
    if (rows == TILE_ROWS) {
      mbar_wait(&bar[stg], (it >> 1) & 1, status);
    } else {  // partial last tile: plain loads
      for (int e = t; e < rows * n2; e += blockDim.x) Qs[e] = Q2[base * n2 + e];
      __syncthreads();
    }
    // cell and weight of position tt (cell units) of row r: charge counts and
    // the stored cell index
    auto put = [&](int r, V tt) {
      int j;
      if (pack) {
        // FP32 rows: cell and fraction in FP32 (both exact), one packed
        // count (1 << Kp) + round(frac 2^Sp) into the particle's cell
        const float th = AR::hi(tt), fl = floorf(th);
        const int q = __float2int_rn((th - fl) * pscale);
        int jr = (int)fl;
        const int wq = (int)floorf((float)jr * inv_Nx);
        jr -= wq * Nx;
        if (jr < 0) jr += Nx;
        if (jr >= Nx) jr -= Nx;
        j = jr;
        atomicAdd(mycnt + j, pbit + (unsigned long long)q);
      } else {
        long long w1;
        cell_fixed(AR::hi(tt), AR::lo(tt), Nx, inv_Nx, scale, g.S, one, j, w1);
        int j1 = (j + 1 == Nx) ? 0 : j + 1;
        atomicAdd(mycnt + j, (unsigned long long)(one - w1));
        atomicAdd(mycnt + j1, (unsigned long long)w1);
      }
      if (jout) jout[jt_block(tile, blockIdx.y, gridDim.y, PC) + r * PC + ii] = (uint16_t)j;
    };
    if (active) {
      int r0 = rsub;
      if constexpr (NR == 0 && !AR::kVec4) {
        // double-float rows with the coefficients in shared memory: two rows
        // per pass share every coefficient load, each row summed in the same
        // order as the loop below
        for (; r0 + RP < rows; r0 += 2 * RP) {
          const V* qa = Qs + r0 * n2;
          const V* qb = Qs + (r0 + RP) * n2;
          typename AR::A x, y;
          x.zero();
          y.zero();
          for (int k = 0; k < n; ++k) {
            const V za = Zs[k * ldz + ii], zb = Zs[(n + k) * ldz + ii];
            x.fma2(qa[k], za);
            y.fma2(qb[k], za);
            x.fma2(AR::neg(qa[n + k]), zb);
            y.fma2(AR::neg(qb[n + k]), zb);
          }
          put(r0, x.out());
          put(r0 + RP, y.out());
        }
      }
      for (int r = r0; r < rows; r += RP) {
        const V* q = Qs + r * n2;
        V tt;
        if constexpr (NR > 0 && AR::kVec4) {  // x = sum_k A_k a_k - B_k b_k, coefficients in registers
          const float4* q4 = reinterpret_cast<const float4*>(q);
          const int n4 = n >> 2;
          float s0 = 0.f, s1 = 0.f;
#pragma unroll
          for (int k = 0; k < NR / 4; ++k)
            if (k < n4) {
              const float4 a = q4[k], b = q4[n4 + k];
              s0 = fmaf(a.x, za[4 * k], s0);
              s1 = fmaf(a.y, za[4 * k + 1], s1);
              s0 = fmaf(a.z, za[4 * k + 2], s0);
              s1 = fmaf(a.w, za[4 * k + 3], s1);
              s0 = fmaf(-b.x, zb[4 * k], s0);
              s1 = fmaf(-b.y, zb[4 * k + 1], s1);
              s0 = fmaf(-b.z, zb[4 * k + 2], s0);
              s1 = fmaf(-b.w, zb[4 * k + 3], s1);
            }
          tt = AR::from_f(s0 + s1);
        } else if (vec) {  // x = sum_k A_k a_k - B_k b_k in two partial sums
          const float4* q4 = reinterpret_cast<const float4*>(q);
          const float4* z4 = reinterpret_cast<const float4*>(Zt + ii * ldk);
          const int n4 = n >> 2;
          float s0 = 0.f, s1 = 0.f;
          for (int k = 0; k < n4; ++k) {
            const float4 a = q4[k], za = z4[k], b = q4[n4 + k], zb = z4[n4 + k];
            s0 = fmaf(a.x, za.x, s0);
            s1 = fmaf(a.y, za.y, s1);
            s0 = fmaf(a.z, za.z, s0);
            s1 = fmaf(a.w, za.w, s1);
            s0 = fmaf(-b.x, zb.x, s0);
            s1 = fmaf(-b.y, zb.y, s1);
            s0 = fmaf(-b.z, zb.z, s0);
            s1 = fmaf(-b.w, zb.w, s1);
          }
          tt = AR::from_f(s0 + s1);
        } else if constexpr (NR > 0) {
          typename AR::A x;
          x.zero();
          if ((n & 1) == 0) {  // n even: two terms of A and of B per 16-byte load
            static_assert(NR % 2 == 0, "pairs of terms");
#pragma unroll
            for (int k = 0; k < NR; k += 2)
              if (k < n) {
                const float4 qa = *reinterpret_cast<const float4*>(q + k);
                const float4 qb = *reinterpret_cast<const float4*>(q + n + k);
                x.fma2(make_float2(qa.x, qa.y), za[k]);
                x.fma2(AR::neg(make_float2(qb.x, qb.y)), zb[k]);
                x.fma2(make_float2(qa.z, qa.w), za[k + 1]);
                x.fma2(AR::neg(make_float2(qb.z, qb.w)), zb[k + 1]);
              }
          } else {
#pragma unroll
            for (int k = 0; k < NR; ++k)
              if (k < n) {
                x.fma2(q[k], za[k]);
                x.fma2(AR::neg(q[n + k]), zb[k]);
              }
          }
          tt = x.out();
        } else {
          typename AR::A x;
          x.zero();
          for (int k = 0; k < n; ++k) {
            x.fma2(q[k], Zs[k * ldz + ii]);
            x.fma2(AR::neg(q[n + k]), Zs[(n + k) * ldz + ii]);
          }
          tt = x.out();
        }
        put(r, tt);
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < PC * Nx; e += blockDim.x) {
    int c = e / Nx;
    if (c0 + c < p && cnt[e]) atomicAdd(&counts[(int64_t)(c0 + c) * Nx + (e - c * Nx)], cnt[e]);
  }
}

// ---------------------------------------------- projection g_X = U_X^T G
// G_li = (q/m) F_i[j_li] with j from the deposit at the same (Q, zeta).
// Thread t owns sample column c = t % PC and rows k = t / PC + a (256 / PC).
// Full tiles of Q rows and of cell indices arrive by bulk copies into two
// shared-memory stages: the copy of the block's next tile runs while the
// current one is used.  A partial last tile is read with plain loads.
template <class AR, int MAXACC>
__global__ void __launch_bounds__(TILE_THREADS)
k_project_lp(GridC g, int64_t N, int n, int p, int PC, const typename AR::V* __restrict__ Q2,
             const typename AR::V* __restrict__ F2, const uint16_t* __restrict__ jt,
             double* __restrict__ part, const int* skip, int* status) {
  using V = typename AR::V;
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, Nx = g.Nx, ldG = PC + 1;
  const int nch = gridDim.y, chunk = blockIdx.y, c0 = chunk * PC;
  const uint32_t qbytes = (uint32_t)(sizeof(V) * TILE_ROWS * n2);
  const uint32_t jbytes = (uint32_t)(sizeof(uint16_t) * TILE_ROWS * PC);
  const size_t qst = (qbytes + 15) & ~size_t(15), jst = (jbytes + 15) & ~size_t(15);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);  // 2 stages
  V* Qs0 = reinterpret_cast<V*>(smraw + 16);
  uint16_t* Js0 = reinterpret_cast<uint16_t*>(smraw + 16 + 2 * qst);
  V* Fs = reinterpret_cast<V*>(smraw + 16 + 2 * qst + 2 * jst);  // PC x Nx
  V* Gs = Fs + PC * Nx;                                           // TILE_ROWS x ldG
  const int t = threadIdx.x;
  const int64_t ntiles = (N + TILE_ROWS - 1) / TILE_ROWS;
  for (int e = t; e < PC * Nx; e += blockDim.x) {
    int c = e / Nx;
    Fs[e] = (c0 + c < p) ? F2[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : AR::zero();
  }
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // thread 0: start the bulk copies of full tile `tl` into stage `st`
  auto issue = [&](int64_t tl, int st) {
    if (t != 0 || tl >= ntiles || (tl + 1) * TILE_ROWS > N) return;
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[st], qbytes + jbytes);
    bulk_g2s(reinterpret_cast<unsigned char*>(Qs0) + st * qst, Q2 + tl * TILE_ROWS * n2, qbytes, &bar[st]);
    bulk_g2s(reinterpret_cast<unsigned char*>(Js0) + st * jst, jt + jt_block(tl, chunk, nch, PC),
             jbytes, &bar[st]);
  };
  const int cc = t % PC, kk0 = t / PC, kstep = blockDim.x / PC;
  // FP32 rows with n2 % 4 == 0: thread owns contiguous groups of four
  // columns, read as float4 (one shared-memory load per 4 multiply-adds)
  const bool vec = AR::kVec4 && (n2 & 3) == 0 && n2 <= 4 * kstep * (MAXACC / 4);
  auto kof = [&](int a) { return vec ? 4 * (kk0 + (a >> 2) * kstep) + (a & 3) : kk0 + a * kstep; };
  typename AR::A acc[MAXACC];
#pragma unroll
  for (int a = 0; a < MAXACC; ++a) acc[a].zero();
  const int pc_eff = min(PC, p - c0);
  int it = 0;
  issue(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int stg = it & 1;
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    V* Qs = reinterpret_cast<V*>(reinterpret_cast<unsigned char*>(Qs0) + stg * qst);
    uint16_t* Js = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(Js0) + stg * jst);
    issue(tile + gridDim.x, stg ^ 1);  // stage stg^1 was released by the barrier ending the last tile
    if (rows == TILE_ROWS) {
      mbar_wait(&bar[stg], (it >> 1) & 1, status);
    } else {  // partial last tile: plain loads
      for (int e = t; e < rows * n2; e += blockDim.x) Qs[e] = Q2[base * n2 + e];
      const uint16_t* js = jt + jt_block(tile, chunk, nch, PC);
      for (int e = t; e < rows * PC; e += blockDim.x) Js[e] = js[e];
      __syncthreads();
    }
    for (int e = t; e < rows * PC; e += blockDim.x) {
      int r = e / PC, c = e - r * PC;
      Gs[r * ldG + c] = (c < pc_eff) ? Fs[c * Nx + Js[e]] : AR::zero();
    }
    __syncthreads();
    // rows in groups of four: the loads of a group are issued together
    int r = 0;
    if constexpr (AR::kVec4) {
      for (; vec && r + 4 <= rows; r += 4) {
        const float G0 = AR::hi(Gs[r * ldG + cc]), G1 = AR::hi(Gs[(r + 1) * ldG + cc]);
        const float G2 = AR::hi(Gs[(r + 2) * ldG + cc]), G3 = AR::hi(Gs[(r + 3) * ldG + cc]);
        const float* Qf = reinterpret_cast<const float*>(Qs);
#pragma unroll
        for (int b = 0; b < MAXACC / 4; ++b) {
          const int k = 4 * (kk0 + b * kstep);
          if (k < n2) {
            const float4 q0 = *reinterpret_cast<const float4*>(Qf + r * n2 + k);
            const float4 q1 = *reinterpret_cast<const float4*>(Qf + (r + 1) * n2 + k);
            const float4 q2 = *reinterpret_cast<const float4*>(Qf + (r + 2) * n2 + k);
            const float4 q3 = *reinterpret_cast<const float4*>(Qf + (r + 3) * n2 + k);
            acc[4 * b + 0].fma2(q0.x, G0);
            acc[4 * b + 1].fma2(q0.y, G0);
            acc[4 * b + 2].fma2(q0.z, G0);
            acc[4 * b + 3].fma2(q0.w, G0);
            acc[4 * b + 0].fma2(q1.x, G1);
            acc[4 * b + 1].fma2(q1.y, G1);
            acc[4 * b + 2].fma2(q1.z, G1);
            acc[4 * b + 3].fma2(q1.w, G1);
            acc[4 * b + 0].fma2(q2.x, G2);
            acc[4 * b + 1].fma2(q2.y, G2);
            acc[4 * b + 2].fma2(q2.z, G2);
            acc[4 * b + 3].fma2(q2.w, G2);
            acc[4 * b + 0].fma2(q3.x, G3);
            acc[4 * b + 1].fma2(q3.y, G3);
            acc[4 * b + 2].fma2(q3.z, G3);
            acc[4 * b + 3].fma2(q3.w, G3);
          }
        }
      }
    }
    for (; !vec && r + 4 <= rows; r += 4) {
      const V G0 = Gs[r * ldG + cc], G1 = Gs[(r + 1) * ldG + cc];
      const V G2 = Gs[(r + 2) * ldG + cc], G3 = Gs[(r + 3) * ldG + cc];
#pragma unroll
      for (int a = 0; a < MAXACC; ++a) {
        int k = kk0 + a * kstep;
        if (k < n2) {
          const V q0 = Qs[r * n2 + k], q1 = Qs[(r + 1) * n2 + k];
          const V q2 = Qs[(r + 2) * n2 + k], q3 = Qs[(r + 3) * n2 + k];
          acc[a].fma2(q0, G0);
          acc[a].fma2(q1, G1);
          acc[a].fma2(q2, G2);
          acc[a].fma2(q3, G3);
        }
      }
    }
    for (; r < rows; ++r) {
      const V G = Gs[r * ldG + cc];
#pragma unroll
      for (int a = 0; a < MAXACC; ++a) {
        int k = kof(a);
        if (k < n2) acc[a].fma2(Qs[r * n2 + k], G);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < MAXACC; ++a) {
    int k = kof(a);
    if (k < n2 && c0 + cc < p) {
      double v = acc[a].value();
      part[(int64_t)blockIdx.x * n2 * p + (int64_t)k * p + c0 + cc] = (k < n) ? v : -v;
    }
  }
}

// -------------------------------------------------------- M = Gamma zeta^H
// Gamma_li = (q/m) F_i[j_li] + i Im(Q_l zeta_i); M_lk = sum_i Gamma_li conj(zeta_ki).
// Needs TILE_THREADS = 256 and TILE_ROWS = 64 (the product's thread map).
#define BM_KJ 5  // columns per thread: k0 + 8 j < n <= 40
static_assert(TILE_THREADS == 256 && TILE_ROWS == 64, "k_basis_M_lp thread map");
template <class AR>
__global__ void __launch_bounds__(TILE_THREADS)
k_basis_M_lp(GridC g, int64_t N, int n, int p, int PC, const typename AR::V* __restrict__ Q2,
             const typename AR::V* __restrict__ Z2, const typename AR::V* __restrict__ F2,
             const uint16_t* __restrict__ jin, typename AR::V* __restrict__ M) {
  using V = typename AR::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  // FP32 rows with n % 4 == 0: unpadded Q rows and a sample-major copy of
  // the coefficient chunk (Zt), so that V_r = Im(Q zeta) reads float4 operands
  const bool vec = AR::kVec4 && (n & 3) == 0;
  const int n2 = 2 * n, ldq = vec ? n2 : n2 + 1, ldz = PC + 1, Nx = g.Nx, ldG = PC + 1;
  const int ldk = n2 + 4;
  V* Qs = reinterpret_cast<V*>(smraw);
  V* Zs = Qs + TILE_ROWS * ldq;
  V* Gr = Zs + n2 * ldz;         // TILE_ROWS x ldG, real part of Gamma
  V* Gi = Gr + TILE_ROWS * ldG;  // imaginary part
  float* Zt = reinterpret_cast<float*>(
      smraw + ((reinterpret_cast<unsigned char*>(Gi + TILE_ROWS * ldG) - smraw + 15) & ~size_t(15)));
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const int nch = (p + PC - 1) / PC;
  // product Gamma zeta^H: thread t owns rows r0, r0 + 32 (r0 = t / 8) and
  // columns k0 + 8 j (k0 = t % 8, j < BM_KJ), so every value read from shared
  // memory feeds several multiply-adds (register tiling)
  const int r0 = t >> 3, k0 = t & 7;
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    typename AR::A ar[2][BM_KJ], ai[2][BM_KJ];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int j = 0; j < BM_KJ; ++j) { ar[h][j].zero(); ai[h][j].zero(); }
    __syncthreads();
    load_rows(Qs, ldq, Q2, n2, base, rows);
    for (int c0 = 0; c0 < p; c0 += PC) {
      __syncthreads();
      load_zc<AR>(Zs, ldz, Z2, n2, p, c0, PC);
      __syncthreads();
      if (vec) {
        for (int e = t; e < n2 * PC; e += blockDim.x) {
          const int k = e / PC, i = e - k * PC;
          Zt[i * ldk + k] = AR::hi(Zs[k * ldz + i]);
        }
        __syncthreads();
      }
      const bool active = c0 + ii < p;
      for (int r = rsub; r < rows; r += RP) {
        V gr = AR::zero(), gi = AR::zero();
        if (active) {
          const V* q = Qs + r * ldq;
          if (vec) {  // v = sum_k B_k a_k + A_k b_k
            const float4* q4 = reinterpret_cast<const float4*>(q);
            const float4* z4 = reinterpret_cast<const float4*>(Zt + ii * ldk);
            const int n4 = n >> 2;
            float s0 = 0.f, s1 = 0.f;
            for (int k = 0; k < n4; ++k) {
              const float4 qa = q4[k], qb = q4[n4 + k], za = z4[k], zb = z4[n4 + k];
              s0 = fmaf(qb.x, za.x, s0);
              s1 = fmaf(qb.y, za.y, s1);
              s0 = fmaf(qb.z, za.z, s0);
              s1 = fmaf(qb.w, za.w, s1);
              s0 = fmaf(qa.x, zb.x, s0);
              s1 = fmaf(qa.y, zb.y, s1);
              s0 = fmaf(qa.z, zb.z, s0);
              s1 = fmaf(qa.w, zb.w, s1);
            }
            gi = AR::from_f(s0 + s1);
          } else {
            typename AR::A v;
            v.zero();
            for (int k = 0; k < n; ++k) {
              v.fma2(q[n + k], Zs[k * ldz + ii]);   // B a
              v.fma2(q[k], Zs[(n + k) * ldz + ii]); // A b
            }
            gi = v.out();
          }
          // the chunk's field rows (PC x Nx) stay in L1 across the tiles
          gr = __ldg(F2 + (int64_t)(c0 + ii) * Nx + jin[jt_block(tile, c0 / PC, nch, PC) + r * PC + ii]);
        }
        Gr[r * ldG + ii] = gr;
        Gi[r * ldG + ii] = gi;
      }
      __syncthreads();
      const int pc_eff = min(PC, p - c0);
      // rows past the tile end hold zeros in Gr, Gi; columns past n are not stored
      for (int c = 0; c < pc_eff; ++c) {
        V grc[2], gic[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          grc[h] = Gr[(r0 + 32 * h) * ldG + c];
          gic[h] = Gi[(r0 + 32 * h) * ldG + c];
        }
#pragma unroll
        for (int j = 0; j < BM_KJ; ++j) {
          const int k = k0 + 8 * j;
          if (k < n) {
            const V za = Zs[k * ldz + c], zb = Zs[(n + k) * ldz + c];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              // Gamma conj(zeta) = (Gr a + Gi b) + i (Gi a - Gr b)
              ar[h][j].fma2(grc[h], za);
              ar[h][j].fma2(gic[h], zb);
              ai[h][j].fma2(gic[h], za);
              ai[h][j].fma2(AR::neg(grc[h]), zb);
            }
          }
        }
      }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = r0 + 32 * h;
      if (r >= rows) continue;
#pragma unroll
      for (int j = 0; j < BM_KJ; ++j) {
        const int k = k0 + 8 * j;
        if (k < n) {
          M[(base + r) * n2 + k] = ar[h][j].out();
          M[(base + r) * n2 + n + k] = ai[h][j].out();
        }
      }
    }
  }
}

// M = Gamma zeta^H in the split form used when all p field rows fit in
// shared memory.  With Gamma = G + i V_r and V_r = Im(Q zeta):
//   Re M_k = sum_i G_i a_ki + [x | y] W[:, k],  Im M_k = -sum_i G_i b_ki + [x | y] W[:, n+k],
// where zeta = a + i b, Q_l = x + i y and W = Y Y^T with Y = [b; a] (2n x p), because
// sum_i V_i b_ki = sum_m x_m (b b^T)_mk + y_m (a b^T)_mk and likewise for a.
// Per row this is 2 n p + 4 n^2 multiply-adds instead of 6 n p, and V_r is
// never formed.  W is computed by every block from zeta in shared memory.
// F_i[j] is gathered from global memory (p x Nx values, cached in L1).
// Threads: TPR = 4 per row of a 64-row tile; thread (r, s) owns k = s, s+4, ...
// Q rows and the tile's cell indices (all chunks) arrive by bulk copies into
// two stages, the next tile's copies running during the current tile.
template <class AR, int KPT>
__global__ void __launch_bounds__(TILE_THREADS)
k_basis_M2_lp(GridC g, int64_t N, int n, int p, int PC, const typename AR::V* __restrict__ Q2,
              const typename AR::V* __restrict__ Z2, const typename AR::V* __restrict__ F2,
              const uint16_t* __restrict__ jt, typename AR::V* __restrict__ M, int* status) {
  using V = typename AR::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, Nx = g.Nx, ldz = p + 1, ldg = p + 1;
  const int nch = (p + PC - 1) / PC;
  const uint32_t qbytes = (uint32_t)(sizeof(V) * TILE_ROWS * n2);
  const uint32_t jbytes = (uint32_t)(sizeof(uint16_t) * TILE_ROWS * nch * PC);
  const size_t qst = (qbytes + 15) & ~size_t(15), jst = (jbytes + 15) & ~size_t(15);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  unsigned char* Qs0 = smraw + 16;
  unsigned char* Js0 = Qs0 + 2 * qst;
  V* Zs = reinterpret_cast<V*>(Js0 + 2 * jst);  // n2 x ldz: [a; b]
  V* Ws = Zs + (size_t)n2 * ldz;                // n2 x n2
  V* Gt = Ws + (size_t)n2 * n2;                 // TILE_ROWS x ldg
  const int t = threadIdx.x;
  const int64_t ntiles = (N + TILE_ROWS - 1) / TILE_ROWS;
  for (int e = t; e < n2 * p; e += blockDim.x) {
    int k = e / p, i = e - k * p;
    Zs[k * ldz + i] = Z2[e];
  }
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  // W = Y Y^T, Y = [b; a]: row m of Y is row (m + n) mod 2n of Z
  for (int e = t; e < n2 * n2; e += blockDim.x) {
    int m = e / n2, k = e - m * n2;
    const V* ym = Zs + ((m + n) % n2) * ldz;
    const V* yk = Zs + ((k + n) % n2) * ldz;
    typename AR::A acc;
    acc.zero();
    for (int i = 0; i < p; ++i) acc.fma2(ym[i], yk[i]);
    Ws[e] = acc.out();
  }
  auto issue = [&](int64_t tl, int st) {
    if (t != 0 || tl >= ntiles || (tl + 1) * TILE_ROWS > N) return;
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[st], qbytes + jbytes);
    bulk_g2s(Qs0 + st * qst, Q2 + tl * TILE_ROWS * n2, qbytes, &bar[st]);
    bulk_g2s(Js0 + st * jst, jt + jt_block(tl, 0, nch, PC), jbytes, &bar[st]);
  };
  const int r = t >> 2, sub = t & 3;
  int it = 0;
  issue(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int stg = it & 1;
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    const V* Qs = reinterpret_cast<const V*>(Qs0 + stg * qst);
    uint16_t* Js = reinterpret_cast<uint16_t*>(Js0 + stg * jst);
    issue(tile + gridDim.x, stg ^ 1);
    if (rows == TILE_ROWS) {
      mbar_wait(&bar[stg], (it >> 1) & 1, status);
    } else {  // partial last tile: plain loads
      V* Qw = reinterpret_cast<V*>(Qs0 + stg * qst);
      for (int e = t; e < rows * n2; e += blockDim.x) Qw[e] = Q2[base * n2 + e];
      const uint16_t* js = jt + jt_block(tile, 0, nch, PC);
      for (int e = t; e < TILE_ROWS * nch * PC; e += blockDim.x) Js[e] = js[e];
      __syncthreads();
    }
    // G_ri = (q/m) F_i[j_ri] of the tile, gathered from the p x Nx field
    // rows (read-only path; they stay in L1 next to this block's shared memory)
    for (int e = t; e < rows * p; e += blockDim.x) {
      int rr = e / p, i = e - rr * p;
      int c = i / PC, ci = i - c * PC;
      Gt[rr * ldg + i] = __ldg(F2 + (size_t)i * Nx + Js[(c * TILE_ROWS + rr) * PC + ci]);
    }
    __syncthreads();
    if (r < rows) {
      typename AR::A ar[KPT], ai[KPT];
#pragma unroll
      for (int q = 0; q < KPT; ++q) { ar[q].zero(); ai[q].zero(); }
      const V* gr = Gt + r * ldg;
      for (int i = 0; i < p; ++i) {
        const V gv = gr[i];
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
          const int k = sub + 4 * q;
          if (k < n) {
            ar[q].fma2(gv, Zs[k * ldz + i]);
            ai[q].fma2(AR::neg(gv), Zs[(n + k) * ldz + i]);
          }
        }
      }
      const V* qr = Qs + r * n2;
      for (int m = 0; m < n2; ++m) {
        const V qm = qr[m];
#pragma unroll
        for (int q = 0; q < KPT; ++q) {
          const int k = sub + 4 * q;
          if (k < n) {
            ar[q].fma2(qm, Ws[m * n2 + k]);
            ai[q].fma2(qm, Ws[m * n2 + n + k]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < KPT; ++q) {
        const int k = sub + 4 * q;
        if (k < n) {
          M[(base + r) * n2 + k] = ar[q].out();
          M[(base + r) * n2 + n + k] = ai[q].out();
        }
      }
    }
    __syncthreads();
  }
}

// -------------------------------------------------------------------- Gram
// out_s = blk[pa[s]]^H blk[pb[s]] (n x n complex); part[blockIdx.x][s][k1][k2].
#define GDF_ROWS 32
#define GDF_EPT 4
// Full 32-row tiles of every block arrive by bulk copies into two stages (the
// next tile's copies run during the current tile); a partial last tile is
// read with plain loads.
// Entries of a Gram launch, enumerated compactly: per pair s its full n x n
// block, or for a Hermitian pair (pa == pb) only k1 <= k2, the lower half
// written as the conjugate.  gram_entries: their count.
__host__ __device__ __forceinline__ int gram_entries(const GramArgsLP& a, int n) {
  int c = 0;
  for (int s = 0; s < a.npairs; ++s) c += (a.pa[s] == a.pb[s]) ? n * (n + 1) / 2 : n * n;
  return c;
}
// index e < n (n + 1) / 2 of the upper triangle, row by row -> (k1, k2),
// k1 <= k2: row k1 holds the n - k1 entries k2 = k1 .. n - 1 from start(k1)
__device__ __forceinline__ void tri_entry(int n, int e, int& k1, int& k2) {
  auto start = [n](int k) { return k * n - k * (k - 1) / 2; };
  const float b = (float)(2 * n + 1);
  int r = (int)(0.5f * (b - sqrtf(b * b - 8.0f * (float)e)));
  r = r < 0 ? 0 : (r > n - 1 ? n - 1 : r);
  while (r > 0 && start(r) > e) --r;
  while (r + 1 < n && start(r + 1) <= e) ++r;
  k1 = r;
  k2 = r + (e - start(r));
}
// compact index e -> (s, k1, k2); false past the last entry
__device__ __forceinline__ bool gram_entry(const GramArgsLP& a, int n, int e, int& s, int& k1,
                                           int& k2) {
  for (s = 0; s < a.npairs; ++s) {
    const bool herm = a.pa[s] == a.pb[s];
    const int cnt = herm ? n * (n + 1) / 2 : n * n;
    if (e < cnt) {
      if (herm) {
        tri_entry(n, e, k1, k2);
      } else {
        k1 = e / n;
        k2 = e - k1 * n;
      }
      return true;
    }
    e -= cnt;
  }
  return false;
}

template <class AR>
__global__ void k_gram_lp(int64_t N, int n, GramArgsLP a, double2* __restrict__ part, int* status) {
  using V = typename AR::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n;
  const uint32_t bbytes = (uint32_t)(sizeof(V) * GDF_ROWS * n2);  // one block's tile
  const size_t sst = (size_t)bbytes * a.nblk;                     // one stage, 16-aligned
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  unsigned char* S0 = smraw + 16;
  const int total = a.npairs * n * n;  // entries of the partial layout
  const int e0 = blockIdx.y * blockDim.x * GDF_EPT;
  const int t = threadIdx.x;
  const int64_t ntiles = (N + GDF_ROWS - 1) / GDF_ROWS;
  typename AR::A re[GDF_EPT], im[GDF_EPT];
  int es[GDF_EPT], ek1[GDF_EPT], ek2[GDF_EPT];
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) {
    re[q].zero();
    im[q].zero();
    if (!gram_entry(a, n, e0 + q * blockDim.x + t, es[q], ek1[q], ek2[q])) es[q] = -1;
  }
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int64_t tl, int st) {
    if (t != 0 || tl >= ntiles || (tl + 1) * GDF_ROWS > N) return;
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[st], (uint32_t)sst);
    for (int b = 0; b < a.nblk; ++b)
      bulk_g2s(S0 + st * sst + b * bbytes,
               reinterpret_cast<const V*>(a.blk[b]) + tl * GDF_ROWS * n2, bbytes, &bar[st]);
  };
  int it = 0;
  issue(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int stg = it & 1;
    const int64_t base = tile * GDF_ROWS;
    const int rows = (int)((int64_t)GDF_ROWS < N - base ? (int64_t)GDF_ROWS : N - base);
    V* sm = reinterpret_cast<V*>(S0 + stg * sst);
    issue(tile + gridDim.x, stg ^ 1);
    if (rows == GDF_ROWS) {
      mbar_wait(&bar[stg], (it >> 1) & 1, status);
    } else {
      for (int b = 0; b < a.nblk; ++b) {
        const V* src = reinterpret_cast<const V*>(a.blk[b]);
        for (int e = t; e < rows * n2; e += blockDim.x) sm[b * GDF_ROWS * n2 + e] = src[base * n2 + e];
      }
      __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < GDF_EPT; ++q) {
      if (es[q] >= 0) {
        const int s = es[q], k1 = ek1[q], k2 = ek2[q];
        const V* X = sm + a.pa[s] * GDF_ROWS * n2;
        const V* Y = sm + a.pb[s] * GDF_ROWS * n2;
        for (int r = 0; r < rows; ++r) {
          V xr = X[r * n2 + k1], xi = X[r * n2 + n + k1];
          V yr = Y[r * n2 + k2], yi = Y[r * n2 + n + k2];
          // conj(x) y = (xr yr + xi yi) + i (xr yi - xi yr)
          re[q].fma2(xr, yr);
          re[q].fma2(xi, yi);
          im[q].fma2(xr, yi);
          im[q].fma2(AR::neg(xi), yr);
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) {
    if (es[q] >= 0) {
      const int s = es[q], k1 = ek1[q], k2 = ek2[q];
      double2* o = part + (int64_t)blockIdx.x * total + (int64_t)s * n * n;
      const double vr = re[q].value(), vi = im[q].value();
      o[k1 * n + k2] = make_double2(vr, vi);
      if (a.pa[s] == a.pb[s] && k1 != k2) o[k2 * n + k1] = make_double2(vr, -vi);
    }
  }
}

// Real Gram X^T X of N x m rows (G_V of the stored [A | B]).
template <class AR>
__global__ void k_gram_real_lp(int64_t N, int m, const typename AR::V* __restrict__ X,
                               double* __restrict__ part) {
  using V = typename AR::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  V* sm = reinterpret_cast<V*>(smraw);
  // the upper triangle k1 <= k2 only (the Gram is symmetric), mirrored on output
  const int ldb = m + 1, total = m * m, tri = m * (m + 1) / 2;
  const int e0 = blockIdx.y * blockDim.x * GDF_EPT;
  typename AR::A acc[GDF_EPT];
  int ek1[GDF_EPT], ek2[GDF_EPT];
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) {
    acc[q].zero();
    const int e = e0 + q * blockDim.x + threadIdx.x;
    if (e < tri) tri_entry(m, e, ek1[q], ek2[q]);
    else ek1[q] = -1;
  }
  for (int64_t tile = blockIdx.x; tile * GDF_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * GDF_ROWS;
    const int rows = (int)((int64_t)GDF_ROWS < N - base ? (int64_t)GDF_ROWS : N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
      int r = e / m, k = e - r * m;
      sm[r * ldb + k] = X[(base + r) * m + k];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GDF_EPT; ++q) {
      if (ek1[q] >= 0) {
        const int k1 = ek1[q], k2 = ek2[q];
        for (int r = 0; r < rows; ++r) acc[q].fma2(sm[r * ldb + k1], sm[r * ldb + k2]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) {
    if (ek1[q] >= 0) {
      const int k1 = ek1[q], k2 = ek2[q];
      const double v = acc[q].value();
      part[(int64_t)blockIdx.x * total + k1 * m + k2] = v;
      if (k1 != k2) part[(int64_t)blockIdx.x * total + k2 * m + k1] = v;
    }
  }
}

// ------------------------------------------------------------------ affine
// out_l = sum_t X_t,l C_t (C_t n x n complex FP64, converted once per block);
// written as FP64 rows (out_d) and/or rows of the policy (out_v).  With
// a.base (FP64 rows of term 0), out_d = base + sum_t X_t C_t - X_0: the
// increment (C_0 less the identity) in the policy's arithmetic, the sum with
// the FP64 base in FP64, so out_d keeps FP64 accuracy where the increment
// is small (a retraction over one time step).
template <class AR>
__global__ void k_affine_lp(int64_t N, int n, AffineArgsLP a, const double2* __restrict__ C,
                            double* __restrict__ out_d, typename AR::V* __restrict__ out_v,
                            int* status, int TR) {
  using V = typename AR::V;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, nn = n * n;
  const uint32_t tbytes = (uint32_t)(sizeof(V) * TR * n2);  // one term's tile of TR rows
  const size_t sst = (size_t)tbytes * a.nterms;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smraw);
  unsigned char* S0 = smraw + 16;
  V* Cr = reinterpret_cast<V*>(S0 + 2 * sst);  // nterms x n x n
  V* Ci = Cr + a.nterms * nn;
  const int t = threadIdx.x;
  const int64_t ntiles = (N + TR - 1) / TR;
  for (int e = t; e < a.nterms * nn; e += blockDim.x) {
    double2 c = C[e];
    if (a.base && e < nn && e / n == e % n) c.x -= 1.0;  // term 0: C_0 - I
    Cr[e] = AR::from(c.x);
    Ci[e] = AR::from(c.y);
  }
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  auto issue = [&](int64_t tl, int st) {
    if (t != 0 || tl >= ntiles || (tl + 1) * TR > N) return;
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[st], (uint32_t)sst);
    for (int b = 0; b < a.nterms; ++b)
      bulk_g2s(S0 + st * sst + b * tbytes,
               reinterpret_cast<const V*>(a.X[b]) + tl * TR * n2, tbytes, &bar[st]);
  };
  int it = 0;
  issue(blockIdx.x, 0);
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
    const int stg = it & 1;
    const int64_t base = tile * TR;
    const int rows = (int)((int64_t)TR < N - base ? (int64_t)TR : N - base);
    V* Xs = reinterpret_cast<V*>(S0 + stg * sst);
    issue(tile + gridDim.x, stg ^ 1);
    if (rows == TR) {
      mbar_wait(&bar[stg], (it >> 1) & 1, status);
    } else {
      for (int b = 0; b < a.nterms; ++b) {
        const V* src = reinterpret_cast<const V*>(a.X[b]);
        for (int e = t; e < rows * n2; e += blockDim.x) Xs[b * TR * n2 + e] = src[base * n2 + e];
      }
      __syncthreads();
    }
    for (int e = t; e < rows * n; e += blockDim.x) {
      int r = e / n, k = e - r * n;
      typename AR::A re, im;
      re.zero();
      im.zero();
      for (int b = 0; b < a.nterms; ++b) {
        const V* x = Xs + (b * TR + r) * n2;
        const V* cr = Cr + b * nn;
        const V* ci = Ci + b * nn;
        for (int q = 0; q < n; ++q) {
          V xr = x[q], xi = x[n + q], c_r = cr[q * n + k], c_i = ci[q * n + k];
          // (xr + i xi)(cr + i ci) = (xr cr - xi ci) + i (xr ci + xi cr)
          re.fma2(xr, c_r);
          re.fma2(AR::neg(xi), c_i);
          im.fma2(xr, c_i);
          im.fma2(xi, c_r);
        }
      }
      const int64_t o = (base + r) * n2;
      if (out_d) {
        double vr = re.value(), vi = im.value();
        if (a.base) {
          vr += a.base[o + k];
          vi += a.base[o + n + k];
        }
        out_d[o + k] = vr;
        out_d[o + n + k] = vi;
      }
      if (out_v) {
        out_v[o + k] = re.out();
        out_v[o + n + k] = im.out();
      }
    }
    __syncthreads();
  }
}

// ============================================================ host wrappers
template <class AR>
static void launch_all(LpOp op, const LpArgs& A, cudaStream_t st) {
  using V = typename AR::V;
  const GridC& g = *A.g;
  const int n = A.n, p = A.p, n2 = 2 * n;
  const int64_t N = A.N;
  switch (op) {
    case LP_SPLIT:
      k_split<AR><<<ceil_div(A.m, 256), 256, 0, st>>>(A.m, A.dsrc, (V*)A.v0);
      break;
    case LP_PREP: {
      int64_t nz = A.dsrc ? (int64_t)n2 * p : 0, nf = A.F ? (int64_t)p * g.Nx : 0;
      if (nz + nf == 0) break;
      k_prep<AR><<<ceil_div(nz + nf, 256), 256, 0, st>>>(g, nz, A.dsrc, (V*)A.v0, (V*)A.v1, nf, A.F,
                                                          (V*)A.v2, A.skip);
      break;
    }
    case LP_DEPOSIT: {
      if constexpr (AR::kVec4) {  // FP32 rows: reconstruction on the tensor cores
        if ((A.tc & VP_TC_DEPOSIT) && deposit_tc_supported(n, p, g.Nx, g.Kp)) {
          const int ch = ceil_div(p, chunk_w(p, g.Nx));
          const int64_t tiles = ceil_div(N, 128);
          const int gx = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, A.num_sms / ch));
          deposit_tc(g, N, n, p, (const float*)A.v0, (const float*)A.v1, A.counts, A.j, gx,
                     A.skip, A.status, st);
          break;
        }
      }
      int PC = chunk_w(p, g.Nx);
      // double-float rows that store no cell indices (the energy check of the
      // FP32 form): 16-sample chunks, so that two blocks fit an SM (the 32-
      // sample counts and Q stages take 145 KB); the counts are exact sums, so
      // the chunking does not change them
      if (!AR::kVec4 && !A.j && PC > 16) PC = 16;
      const int ch = ceil_div(p, PC);
      const size_t qst = (sizeof(V) * TILE_ROWS * n2 + 15) & ~size_t(15);
      const bool vec = AR::kVec4 && (n & 3) == 0;
      const int nr = dep_nr<AR>(n);
      size_t smem = ((16 + 2 * qst + sizeof(V) * n2 * (PC + 1) + 15) & ~size_t(15)) +
                    ((vec && nr == 0) ? ((sizeof(float) * PC * (n2 + 4) + 15) & ~size_t(15)) : 0) +
                    sizeof(unsigned long long) * PC * g.Nx;
      int gx = grid_bps(ceil_div(N, TILE_ROWS), ch, (A.tune ? A.tune : kTuneDefault)[TUNE_DEPOSIT], A.num_sms);
      auto kern = k_deposit_lp<AR, 0>;
      if constexpr (AR::kVec4) {
        if (nr == kDepNrF32[0]) kern = k_deposit_lp<AR, kDepNrF32[0]>;
        if (nr == kDepNrF32[1]) kern = k_deposit_lp<AR, kDepNrF32[1]>;
        if (nr == kDepNrF32[2]) kern = k_deposit_lp<AR, kDepNrF32[2]>;
      } else {
        if (nr == kDepNrDF[0]) kern = k_deposit_lp<AR, kDepNrDF[0]>;
        if (nr == kDepNrDF[1]) kern = k_deposit_lp<AR, kDepNrDF[1]>;
      }
      kern<<<dim3(gx, ch), TILE_THREADS, smem, st>>>(
          g, N, n, p, PC, (const V*)A.v0, (const V*)A.v1, A.counts, A.j, A.skip, A.status);
      break;
    }
    case LP_PROJECT: {
      if constexpr (AR::kVec4) {  // FP32 rows: tensor cores where the shapes allow
        if ((A.tc & VP_TC_PROJECT) && project_tc_supported(n, p, g.Nx)) {
          project_tc(g, N, n, p, (const float*)A.v0, (const float*)A.v1, A.j, A.part, A.gridx,
                     A.skip, A.status, st);
          break;
        }
      }
      int PC = chunk_w(p, g.Nx);
      // double-float rows that store no cell indices (the energy check of the
      // FP32 form): 16-sample chunks, so that two blocks fit an SM (the 32-
      // sample counts and Q stages take 145 KB); the counts are exact sums, so
      // the chunking does not change them
      if (!AR::kVec4 && !A.j && PC > 16) PC = 16;
      const int ch = ceil_div(p, PC);
      const size_t qst = (sizeof(V) * TILE_ROWS * n2 + 15) & ~size_t(15);
      const size_t jst = (sizeof(uint16_t) * TILE_ROWS * PC + 15) & ~size_t(15);
      size_t smem = 16 + 2 * qst + 2 * jst + sizeof(V) * (PC * g.Nx + TILE_ROWS * (PC + 1));
      if (n2 <= 4 * (TILE_THREADS / PC))
        k_project_lp<AR, 4><<<dim3(A.gridx, ch), TILE_THREADS, smem, st>>>(
            g, N, n, p, PC, (const V*)A.v0, (const V*)A.v1, A.j, A.part, A.skip, A.status);
      else
        k_project_lp<AR, 16><<<dim3(A.gridx, ch), TILE_THREADS, smem, st>>>(
            g, N, n, p, PC, (const V*)A.v0, (const V*)A.v1, A.j, A.part, A.skip, A.status);
      break;
    }
    case LP_BASIS_M: {
      int PC = chunk_w(p, g.Nx);
      if constexpr (AR::kVec4) {
        if ((A.tc & VP_TC_BASIS_M) && A.bop && basis_tc_supported(n, p)) {
          basis_tc(g, N, n, p, PC, (const float*)A.v0, (const float*)A.v1, (const float*)A.v2,
                   A.j, (float*)A.v3, A.bop, A.num_sms, A.status, st);
          break;
        }
      }
      {
        const int nch = ceil_div(p, PC);
        const size_t qst = (sizeof(V) * TILE_ROWS * n2 + 15) & ~size_t(15);
        const size_t jst = (sizeof(uint16_t) * TILE_ROWS * nch * PC + 15) & ~size_t(15);
        const size_t smem2 = 16 + 2 * qst + 2 * jst +
                             sizeof(V) * ((size_t)n2 * (p + 1) + (size_t)n2 * n2 +
                                          (size_t)TILE_ROWS * (p + 1));
        // split form when two blocks fit an SM (with one block per SM the
        // double-float form measured slower than the chunked kernel below)
        if (smem2 <= 112 * 1024) {
          int gx = grid_bps(ceil_div(N, TILE_ROWS), 1,
                            (A.tune ? A.tune : kTuneDefault)[TUNE_BASIS_M], A.num_sms);
          if (n <= 12)
            k_basis_M2_lp<AR, 3><<<gx, TILE_THREADS, smem2, st>>>(
                g, N, n, p, PC, (const V*)A.v0, (const V*)A.v1, (const V*)A.v2, A.j, (V*)A.v3,
                A.status);
          else
            k_basis_M2_lp<AR, 10><<<gx, TILE_THREADS, smem2, st>>>(
                g, N, n, p, PC, (const V*)A.v0, (const V*)A.v1, (const V*)A.v2, A.j, (V*)A.v3,
                A.status);
          break;
        }
      }
      size_t smem = sizeof(V) * (TILE_ROWS * (n2 + 1) + n2 * (PC + 1) + 2 * TILE_ROWS * (PC + 1)) +
                    ((AR::kVec4 && (n & 3) == 0) ? 16 + sizeof(float) * PC * (n2 + 4) : 0);
      int gx = grid_bps(ceil_div(N, TILE_ROWS), 1, (A.tune ? A.tune : kTuneDefault)[TUNE_BASIS_M], A.num_sms);
      k_basis_M_lp<AR><<<gx, TILE_THREADS, smem, st>>>(g, N, n, p, PC, (const V*)A.v0,
                                                       (const V*)A.v1, (const V*)A.v2, A.j,
                                                       (V*)A.v3);
      break;
    }
    case LP_GRAM: {
      if constexpr (AR::kVec4) {
        if ((A.tc & VP_TC_GRAM) && gram_tc_supported(n, A.gram.nblk, A.gram.npairs) &&
            (int64_t)(A.gridx - 1) * 32 < N) {
          gram_tc(N, n, A.gram, 0, A.part, A.gridx, A.status, st);
          break;
        }
      }
      int gy = ceil_div(gram_entries(A.gram, n), TILE_THREADS * GDF_EPT);
      size_t smem = 16 + 2 * sizeof(V) * A.gram.nblk * GDF_ROWS * n2;
      k_gram_lp<AR><<<dim3(A.gridx, gy), TILE_THREADS, smem, st>>>(N, n, A.gram, (double2*)A.part,
                                                                   A.status);
      break;
    }
    case LP_GRAM_REAL: {
      if constexpr (AR::kVec4) {
        if ((A.tc & VP_TC_GRAM) && gram_tc_supported(n, 1, 1) && (int64_t)(A.gridx - 1) * 32 < N) {
          GramArgsLP gr{};
          gr.blk[0] = A.v0;
          gr.nblk = 1;
          gr.npairs = 1;
          gram_tc(N, n, gr, 1, A.part, A.gridx, A.status, st);
          break;
        }
      }
      int m = n2;
      int gy = ceil_div(m * (m + 1) / 2, TILE_THREADS * GDF_EPT);
      size_t smem = sizeof(V) * GDF_ROWS * (m + 1);
      k_gram_real_lp<AR><<<dim3(A.gridx, gy), TILE_THREADS, smem, st>>>(N, m, (const V*)A.v0, A.part);
      break;
    }
    case LP_AFFINE: {
      if constexpr (AR::kVec4) {
        if ((A.tc & VP_TC_AFFINE) && A.bop && affine_tc_supported(n, A.aff.nterms)) {
          affine_tc(g, N, n, A.aff, A.C, A.dout, (float*)A.v0, A.bop, A.num_sms, A.status, st);
          break;
        }
      }
      // rows per tile: 64, or fewer when two stages of every term would not fit
      int TR = TILE_ROWS;
      auto smem_for = [&](int tr) {
        return 16 + sizeof(V) * (2 * (size_t)A.aff.nterms * n * n + 2 * (size_t)A.aff.nterms * tr * n2);
      };
      while (TR > 16 && smem_for(TR) > 200 * 1024) TR /= 2;
      size_t smem = smem_for(TR);
      int gx = grid_bps(ceil_div(N, TR), 1, (A.tune ? A.tune : kTuneDefault)[TUNE_AFFINE], A.num_sms);
      k_affine_lp<AR><<<gx, TILE_THREADS, smem, st>>>(N, n, A.aff, A.C, A.dout, (V*)A.v0, A.status, TR);
      break;
    }
  }
}

void lp_launch(int arith, LpOp op, const LpArgs& a, cudaStream_t st) {
  if (arith == 2) launch_all<ArithF32>(op, a, st);
  else launch_all<ArithDF>(op, a, st);
}

template <class AR>
static void set_attrs() {
  const int big = 220 * 1024;
  cudaFuncSetAttribute(k_deposit_lp<AR, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  if constexpr (AR::kVec4) {
    cudaFuncSetAttribute(k_deposit_lp<AR, kDepNrF32[0]>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_deposit_lp<AR, kDepNrF32[1]>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_deposit_lp<AR, kDepNrF32[2]>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  } else {
    cudaFuncSetAttribute(k_deposit_lp<AR, kDepNrDF[0]>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_deposit_lp<AR, kDepNrDF[1]>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  }
  cudaFuncSetAttribute(k_project_lp<AR, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_project_lp<AR, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_basis_M_lp<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_basis_M2_lp<AR, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_basis_M2_lp<AR, 10>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gram_lp<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gram_real_lp<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_affine_lp<AR>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

void df_init() {
  set_attrs<ArithDF>();
  set_attrs<ArithF32>();
}

}  // namespace vpk
