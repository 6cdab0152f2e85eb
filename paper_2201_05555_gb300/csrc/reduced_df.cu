// Particle-loop kernels of the reduced model in double-float arithmetic.
//
// GB300 executes FP32 at 58x its FP64 rate (measured 68.8 vs 1.19 TFLOP/s),
// so the three particle loops (deposit of X_r = Re(Q zeta), projection
// U_X^T G, and Gamma zeta^H) represent every FP64 operand as an unevaluated
// sum hi + lo of two floats (|lo| <= ulp(hi)/2, about 48 significant bits)
// and form each dot product with the compensated algorithm "Dot2" of Ogita,
// Rump and Oishi (SIAM J. Sci. Comput. 26, 2005): an error-free product
// (FMA) and an error-free sum (TwoSum) per term, with the rounding errors
// accumulated separately, which gives the result as if computed in twice
// the working precision.  Storage stays FP64; results are FP64.  The cell
// index of every (particle, sample) is written by the deposit and reused by
// the projection and the basis kernel at the same (Q, zeta).
#include "vp_internal.cuh"

namespace vpk {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ float2 df_split(double d) {
  float h = __double2float_rn(d);
  float l = __double2float_rn(d - (double)h);
  return make_float2(h, l);
}

// Running compensated sum: value = s + c.
struct Acc {
  float s, c;
  __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
  // += a * b with a, b double-float
  __device__ __forceinline__ void fma2(float2 a, float2 b) {
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
  // += a * b with a double-float, b a plain float
  __device__ __forceinline__ void fma1(float2 a, float b) {
    float p = a.x * b;
    float e = fmaf(a.x, b, -p);
    e = fmaf(a.y, b, e);
    float t = s + p;
    float bp = t - s;
    float es = (s - (t - bp)) + (p - bp);
    s = t;
    c += es + e;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
  __device__ __forceinline__ float2 df() const {
    float h = s + c;
    return make_float2(h, c - (h - s));
  }
};

// Cell index and fixed-point fraction of t = th + tl (cell units,
// unwrapped): j in [0, Nx), w1 = round(frac * 2^S) in [0, 2^S].
__device__ __forceinline__ void cell_fixed(float th, float tl, int Nx, float inv_Nx, float scale,
                                           long long one, int& j, long long& w1) {
  float fl = floorf(th);
  // exact th - fl = a + e (TwoSum)
  float a = th - fl;
  float z = a - th;
  float e = (th - (a - z)) + (-fl - z);
  long long q = __float2ll_rn(a * scale) + __float2ll_rn(e * scale) + __float2ll_rn(tl * scale);
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

// Split Q (N x 2n doubles) into its double-float shadow (N x 2n float2).
__global__ void k_split(int64_t m, const double* __restrict__ x, float2* __restrict__ out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < m) out[e] = df_split(x[e]);
}

void split_df(int64_t m, const double* x, float2* out, cudaStream_t st) {
  k_split<<<ceil_div(m, 256), 256, 0, st>>>(m, x, out);
}

__device__ __forceinline__ void load_q2(float2* Qs, int ldq, const float2* __restrict__ Q2, int n2,
                                        int64_t base, int rows) {
  for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
    int r = e / n2, k = e - r * n2;
    Qs[r * ldq + k] = Q2[(base + r) * n2 + k];
  }
}

// z chunk as double-float, optionally scaled (1/h for positions in cells)
__device__ __forceinline__ void load_z2(float2* Zs, int ldz, const double* __restrict__ Z, int n2,
                                        int p, int c0, int PC, double scale) {
  for (int e = threadIdx.x; e < n2 * PC; e += blockDim.x) {
    int k = e / PC, ii = e - k * PC;
    Zs[k * ldz + ii] = df_split((c0 + ii < p) ? scale * Z[(int64_t)k * p + c0 + ii] : 0.0);
  }
}

// ------------------------------------------------ deposit (double-float)
__global__ void k_deposit_df(GridC g, int64_t N, int n, int p, int PC,
                             const float2* __restrict__ Q2, const double* __restrict__ Z,
                             unsigned long long* __restrict__ counts, uint16_t* __restrict__ jout,
                             const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, ldq = n2 + 1, ldz = PC + 1, Nx = g.Nx;
  float2* Qs = reinterpret_cast<float2*>(smraw);
  float2* Zs = Qs + TILE_ROWS * ldq;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(Zs + ((n2 * ldz + 1) & ~1));
  const int c0 = blockIdx.y * PC;
  load_z2(Zs, ldz, Z, n2, p, c0, PC, g.inv_h);
  for (int e = threadIdx.x; e < PC * Nx; e += blockDim.x) cnt[e] = 0ull;
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const bool active = c0 + ii < p;
  const long long one = 1ll << g.S;
  const float scale = (float)g.fp_scale, inv_Nx = (float)g.inv_Nx;
  unsigned long long* mycnt = cnt + ii * Nx;
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    __syncthreads();
    load_q2(Qs, ldq, Q2, n2, base, rows);
    __syncthreads();
    if (active) {
      for (int r = rsub; r < rows; r += RP) {
        const float2* q = Qs + r * ldq;
        Acc x;
        x.zero();
        for (int k = 0; k < n; ++k) {
          x.fma2(q[k], Zs[k * ldz + ii]);
          float2 mb = make_float2(-q[n + k].x, -q[n + k].y);
          x.fma2(mb, Zs[(n + k) * ldz + ii]);
        }
        float2 tt = x.df();
        int j;
        long long w1;
        cell_fixed(tt.x, tt.y, Nx, inv_Nx, scale, one, j, w1);
        int j1 = (j + 1 == Nx) ? 0 : j + 1;
        atomicAdd(mycnt + j, (unsigned long long)(one - w1));
        atomicAdd(mycnt + j1, (unsigned long long)w1);
        if (jout) jout[(base + r) * p + c0 + ii] = (uint16_t)j;
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < PC * Nx; e += blockDim.x) {
    int c = e / Nx;
    if (c0 + c < p && cnt[e]) atomicAdd(&counts[(int64_t)(c0 + c) * Nx + (e - c * Nx)], cnt[e]);
  }
}

static inline int chunk_w(int p, int Nx) {
  int pc = 1;
  while (pc < p && pc < 32) pc <<= 1;
  while (pc > 1 && (size_t)pc * Nx * 8 > 96 * 1024) pc >>= 1;
  return pc;
}

void deposit_df(const GridC& g, int64_t N, int n, int p, const float2* Q2, const double* Z,
                unsigned long long* counts, uint16_t* jout, const int* skip, int num_sms,
                cudaStream_t st) {
  int PC = chunk_w(p, g.Nx);
  int ch = ceil_div(p, PC);
  int n2 = 2 * n;
  size_t smem = sizeof(float2) * (TILE_ROWS * (n2 + 1) + ((n2 * (PC + 1) + 1) & ~1)) +
                sizeof(unsigned long long) * PC * g.Nx;
  int gx = tile_grid_x(N, ch, num_sms);
  k_deposit_df<<<dim3(gx, ch), TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, Z, counts, jout, skip);
}

// --------------------------------------- projection g_X = U_X^T G (double-float)
// G_li = (q/m) F_i[j_li] with j from the deposit at the same (Q, zeta).
#define PDF_MAXACC 16
__global__ void k_project_df(GridC g, int64_t N, int n, int p, int PC,
                             const float2* __restrict__ Q2, const double* __restrict__ F,
                             const uint16_t* __restrict__ jin, double* __restrict__ part,
                             const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, ldq = n2 + 1, Nx = g.Nx, ldG = PC + 1;
  float2* Qs = reinterpret_cast<float2*>(smraw);
  float2* Fs = Qs + TILE_ROWS * ldq;  // PC x Nx, q/m F split
  float2* Gs = Fs + PC * Nx;          // TILE_ROWS x ldG
  const int c0 = blockIdx.y * PC;
  const int t = threadIdx.x;
  for (int e = t; e < PC * Nx; e += blockDim.x) {
    int c = e / Nx;
    Fs[e] = df_split((c0 + c < p) ? g.qm * F[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : 0.0);
  }
  const int npairs = n2 * PC;
  Acc acc[PDF_MAXACC];
#pragma unroll
  for (int a = 0; a < PDF_MAXACC; ++a) acc[a].zero();
  const int pc_eff = min(PC, p - c0);
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    __syncthreads();
    load_q2(Qs, ldq, Q2, n2, base, rows);
    for (int e = t; e < rows * PC; e += blockDim.x) {
      int r = e / PC, c = e - r * PC;
      float2 G = make_float2(0.f, 0.f);
      if (c < pc_eff) G = Fs[c * Nx + jin[(base + r) * p + c0 + c]];
      Gs[r * ldG + c] = G;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < PDF_MAXACC; ++a) {
      int e = t + a * blockDim.x;
      if (e < npairs) {
        int k = e / PC, c = e - k * PC;
        for (int r = 0; r < rows; ++r) acc[a].fma2(Qs[r * ldq + k], Gs[r * ldG + c]);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < PDF_MAXACC; ++a) {
    int e = t + a * blockDim.x;
    if (e < npairs) {
      int k = e / PC, c = e - k * PC;
      double v = acc[a].value();
      if (c0 + c < p) part[(int64_t)blockIdx.x * n2 * p + (int64_t)k * p + c0 + c] = (k < n) ? v : -v;
    }
  }
}

void project_df(const GridC& g, int64_t N, int n, int p, const float2* Q2, const double* F,
                const uint16_t* jin, double* part, int gridx, const int* skip, cudaStream_t st) {
  int PC = chunk_w(p, g.Nx);
  int ch = ceil_div(p, PC);
  int n2 = 2 * n;
  size_t smem = sizeof(float2) * (TILE_ROWS * (n2 + 1) + PC * g.Nx + TILE_ROWS * (PC + 1));
  k_project_df<<<dim3(gridx, ch), TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, F, jin, part, skip);
}

// -------------------------------------- M = Gamma zeta^H (double-float)
// Gamma_li = (q/m) F_i[j_li] + i Im(Q_l zeta_i); M_lk = sum_i Gamma_li conj(zeta_ki).
#define BMDF_MAXACC 16
__global__ void k_basis_M_df(GridC g, int64_t N, int n, int p, int PC,
                             const float2* __restrict__ Q2, const double* __restrict__ Z,
                             const double* __restrict__ F, const uint16_t* __restrict__ jin,
                             double* __restrict__ M) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, ldq = n2 + 1, ldz = PC + 1, Nx = g.Nx, ldG = PC + 1;
  float2* Qs = reinterpret_cast<float2*>(smraw);
  float2* Zs = Qs + TILE_ROWS * ldq;
  float2* Fs = Zs + n2 * ldz;
  float2* Gr = Fs + PC * Nx;             // TILE_ROWS x ldG, real part of Gamma
  float2* Gi = Gr + TILE_ROWS * ldG;     // imaginary part
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const int npairs = TILE_ROWS * n;
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    Acc ar[BMDF_MAXACC], ai[BMDF_MAXACC];
#pragma unroll
    for (int a = 0; a < BMDF_MAXACC; ++a) { ar[a].zero(); ai[a].zero(); }
    __syncthreads();
    load_q2(Qs, ldq, Q2, n2, base, rows);
    for (int c0 = 0; c0 < p; c0 += PC) {
      __syncthreads();
      load_z2(Zs, ldz, Z, n2, p, c0, PC, 1.0);
      for (int e = t; e < PC * Nx; e += blockDim.x) {
        int c = e / Nx;
        Fs[e] = df_split((c0 + c < p) ? g.qm * F[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : 0.0);
      }
      __syncthreads();
      const bool active = c0 + ii < p;
      for (int r = rsub; r < rows; r += RP) {
        float2 gr = make_float2(0.f, 0.f), gi = make_float2(0.f, 0.f);
        if (active) {
          const float2* q = Qs + r * ldq;
          Acc v;
          v.zero();
          for (int k = 0; k < n; ++k) {
            v.fma2(q[n + k], Zs[k * ldz + ii]);   // B a
            v.fma2(q[k], Zs[(n + k) * ldz + ii]); // A b
          }
          gr = Fs[ii * Nx + jin[(base + r) * p + c0 + ii]];
          gi = v.df();
        }
        Gr[r * ldG + ii] = gr;
        Gi[r * ldG + ii] = gi;
      }
      __syncthreads();
      const int pc_eff = min(PC, p - c0);
#pragma unroll
      for (int a = 0; a < BMDF_MAXACC; ++a) {
        int e = t + a * blockDim.x;
        if (e < npairs) {
          int r = e / n, k = e - r * n;
          if (r < rows) {
            for (int c = 0; c < pc_eff; ++c) {
              float2 za = Zs[k * ldz + c], zb = Zs[(n + k) * ldz + c];
              float2 grc = Gr[r * ldG + c], gic = Gi[r * ldG + c];
              // Gamma conj(zeta) = (Gr a + Gi b) + i (Gi a - Gr b)
              ar[a].fma2(grc, za);
              ar[a].fma2(gic, zb);
              ai[a].fma2(gic, za);
              ai[a].fma2(make_float2(-grc.x, -grc.y), zb);
            }
          }
        }
      }
    }
#pragma unroll
    for (int a = 0; a < BMDF_MAXACC; ++a) {
      int e = t + a * blockDim.x;
      if (e < npairs) {
        int r = e / n, k = e - r * n;
        if (r < rows) {
          M[(base + r) * n2 + k] = ar[a].value();
          M[(base + r) * n2 + n + k] = ai[a].value();
        }
      }
    }
  }
}

void basis_M_df(const GridC& g, int64_t N, int n, int p, const float2* Q2, const double* Z,
                const double* F, const uint16_t* jin, double* M, int num_sms, cudaStream_t st) {
  int PC = chunk_w(p, g.Nx);
  int n2 = 2 * n;
  size_t smem = sizeof(float2) * (TILE_ROWS * (n2 + 1) + n2 * (PC + 1) + PC * g.Nx +
                                  2 * TILE_ROWS * (PC + 1));
  int gx = tile_grid_x(N, 1, num_sms);
  k_basis_M_df<<<gx, TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, Z, F, jin, M);
}

void df_init() {
  const int big = 220 * 1024;
  cudaFuncSetAttribute(k_deposit_df, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_project_df, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_basis_M_df, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace vpk
