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

// z chunk from a pre-split (2n x p) float2 array, zero padded
__device__ __forceinline__ void load_zc(float2* Zs, int ldz, const float2* __restrict__ Z2, int n2,
                                        int p, int c0, int PC) {
  for (int e = threadIdx.x; e < n2 * PC; e += blockDim.x) {
    int k = e / PC, ii = e - k * PC;
    Zs[k * ldz + ii] = (c0 + ii < p) ? Z2[(int64_t)k * p + c0 + ii] : make_float2(0.f, 0.f);
  }
}

// Split, once per field evaluation: Z2 = df(Z), Zh2 = df(Z / h) (2n x p) and
// F2 = df(q/m F) (p x Nx).
__global__ void k_prep_df(GridC g, int64_t nz, const double* __restrict__ Z, float2* Z2,
                          float2* Zh2, int64_t nf, const double* __restrict__ F, float2* F2,
                          const int* skip) {
  if (skip && *skip) return;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < nz) {
    double z = Z[e];
    if (Z2) Z2[e] = df_split(z);
    if (Zh2) Zh2[e] = df_split(z * g.inv_h);
  } else if (F && e - nz < nf) {
    F2[e - nz] = df_split(g.qm * F[e - nz]);
  }
}

void prep_df(const GridC& g, int n, int p, const double* Z, float2* Z2, float2* Zh2,
             const double* F, float2* F2, const int* skip, cudaStream_t st) {
  int64_t nz = Z ? (int64_t)2 * n * p : 0, nf = F ? (int64_t)p * g.Nx : 0;
  if (nz + nf == 0) return;
  k_prep_df<<<ceil_div(nz + nf, 256), 256, 0, st>>>(g, nz, Z, Z2, Zh2, nf, F, F2, skip);
}

// ------------------------------------------------ deposit (double-float)
__global__ void k_deposit_df(GridC g, int64_t N, int n, int p, int PC,
                             const float2* __restrict__ Q2, const float2* __restrict__ Zh2,
                             unsigned long long* __restrict__ counts, uint16_t* __restrict__ jout,
                             const int* skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, ldq = n2 + 1, ldz = PC + 1, Nx = g.Nx;
  float2* Qs = reinterpret_cast<float2*>(smraw);
  float2* Zs = Qs + TILE_ROWS * ldq;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(Zs + ((n2 * ldz + 1) & ~1));
  const int c0 = blockIdx.y * PC;
  load_zc(Zs, ldz, Zh2, n2, p, c0, PC);
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
        cell_fixed(tt.x, tt.y, Nx, inv_Nx, scale, g.S, one, j, w1);
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

void deposit_df(const GridC& g, int64_t N, int n, int p, const float2* Q2, const float2* Zh2,
                unsigned long long* counts, uint16_t* jout, const int* skip, int num_sms,
                cudaStream_t st) {
  int PC = chunk_w(p, g.Nx);
  int ch = ceil_div(p, PC);
  int n2 = 2 * n;
  size_t smem = sizeof(float2) * (TILE_ROWS * (n2 + 1) + ((n2 * (PC + 1) + 1) & ~1)) +
                sizeof(unsigned long long) * PC * g.Nx;
  int gx = tile_grid_x(N, ch, 2 * num_sms);  // 4 blocks per SM hide the atomic latency
  k_deposit_df<<<dim3(gx, ch), TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, Zh2, counts, jout, skip);
}

// --------------------------------------- projection g_X = U_X^T G (double-float)
// G_li = (q/m) F_i[j_li] with j from the deposit at the same (Q, zeta).
template <int PDF_MAXACC>
__global__ void __launch_bounds__(TILE_THREADS)
k_project_df(GridC g, int64_t N, int n, int p, int PC,
                             const float2* __restrict__ Q2, const float2* __restrict__ F2,
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
    Fs[e] = (c0 + c < p) ? F2[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : make_float2(0.f, 0.f);
  }
  const int npairs = n2 * PC;
  // thread t owns sample column c = t % PC and rows k = t / PC + a (blockDim / PC)
  const int cc = t % PC, kk0 = t / PC, kstep = blockDim.x / PC;
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
    // rows in groups of four: the loads of a group are issued together
    int r = 0;
    for (; r + 4 <= rows; r += 4) {
      const float2 G0 = Gs[r * ldG + cc], G1 = Gs[(r + 1) * ldG + cc];
      const float2 G2 = Gs[(r + 2) * ldG + cc], G3 = Gs[(r + 3) * ldG + cc];
#pragma unroll
      for (int a = 0; a < PDF_MAXACC; ++a) {
        int k = kk0 + a * kstep;
        if (k < n2) {
          const float2 q0 = Qs[r * ldq + k], q1 = Qs[(r + 1) * ldq + k];
          const float2 q2 = Qs[(r + 2) * ldq + k], q3 = Qs[(r + 3) * ldq + k];
          acc[a].fma2(q0, G0);
          acc[a].fma2(q1, G1);
          acc[a].fma2(q2, G2);
          acc[a].fma2(q3, G3);
        }
      }
    }
    for (; r < rows; ++r) {
      const float2 G = Gs[r * ldG + cc];
#pragma unroll
      for (int a = 0; a < PDF_MAXACC; ++a) {
        int k = kk0 + a * kstep;
        if (k < n2) acc[a].fma2(Qs[r * ldq + k], G);
      }
    }
  }
  (void)npairs;
#pragma unroll
  for (int a = 0; a < PDF_MAXACC; ++a) {
    int k = kk0 + a * kstep;
    if (k < n2 && c0 + cc < p) {
      double v = acc[a].value();
      part[(int64_t)blockIdx.x * n2 * p + (int64_t)k * p + c0 + cc] = (k < n) ? v : -v;
    }
  }
}

void project_df(const GridC& g, int64_t N, int n, int p, const float2* Q2, const float2* F2,
                const uint16_t* jin, double* part, int gridx, const int* skip, cudaStream_t st) {
  int PC = chunk_w(p, g.Nx);
  int ch = ceil_div(p, PC);
  int n2 = 2 * n;
  size_t smem = sizeof(float2) * (TILE_ROWS * (n2 + 1) + PC * g.Nx + TILE_ROWS * (PC + 1));
  if (n2 <= 4 * (TILE_THREADS / PC))
    k_project_df<4><<<dim3(gridx, ch), TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, F2, jin, part, skip);
  else
    k_project_df<16><<<dim3(gridx, ch), TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, F2, jin, part, skip);
}

// -------------------------------------- M = Gamma zeta^H (double-float)
// Gamma_li = (q/m) F_i[j_li] + i Im(Q_l zeta_i); M_lk = sum_i Gamma_li conj(zeta_ki).
// Z2, F2: pre-split zeta and q/m F; M written as double-float rows.
template <int MAXACC>
__global__ void __launch_bounds__(TILE_THREADS)
k_basis_M_df(GridC g, int64_t N, int n, int p, int PC, const float2* __restrict__ Q2,
             const float2* __restrict__ Z2, const float2* __restrict__ F2,
             const uint16_t* __restrict__ jin, float2* __restrict__ M) {
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
    Acc ar[MAXACC], ai[MAXACC];
#pragma unroll
    for (int a = 0; a < MAXACC; ++a) { ar[a].zero(); ai[a].zero(); }
    __syncthreads();
    load_q2(Qs, ldq, Q2, n2, base, rows);
    for (int c0 = 0; c0 < p; c0 += PC) {
      __syncthreads();
      load_zc(Zs, ldz, Z2, n2, p, c0, PC);
      for (int e = t; e < PC * Nx; e += blockDim.x) {
        int c = e / Nx;
        Fs[e] = (c0 + c < p) ? F2[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : make_float2(0.f, 0.f);
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
      for (int a = 0; a < MAXACC; ++a) {
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
    for (int a = 0; a < MAXACC; ++a) {
      int e = t + a * blockDim.x;
      if (e < npairs) {
        int r = e / n, k = e - r * n;
        if (r < rows) {
          M[(base + r) * n2 + k] = ar[a].df();
          M[(base + r) * n2 + n + k] = ai[a].df();
        }
      }
    }
  }
}

void basis_M_df(const GridC& g, int64_t N, int n, int p, const float2* Q2, const float2* Z2,
                const float2* F2, const uint16_t* jin, float2* M, int num_sms, cudaStream_t st) {
  int PC = chunk_w(p, g.Nx);
  int n2 = 2 * n;
  size_t smem = sizeof(float2) * (TILE_ROWS * (n2 + 1) + n2 * (PC + 1) + PC * g.Nx +
                                  2 * TILE_ROWS * (PC + 1));
  int gx = tile_grid_x(N, 1, num_sms);
  if (TILE_ROWS * n <= 4 * TILE_THREADS)
    k_basis_M_df<4><<<gx, TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, Z2, F2, jin, M);
  else
    k_basis_M_df<16><<<gx, TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q2, Z2, F2, jin, M);
}

// ------------------------------------------------------ Gram (double-float)
// out_s = blk[pa[s]]^H blk[pb[s]] (n x n complex) from double-float rows;
// part[blockIdx.x][s][k1][k2] as double2.
#define GDF_ROWS 32
#define GDF_EPT 4
__global__ void k_gram_df(int64_t N, int n, GramArgsDF a, double2* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int n2 = 2 * n, ldb = n2 + 1;
  const int total = a.npairs * n * n;
  const int e0 = blockIdx.y * blockDim.x * GDF_EPT;
  Acc re[GDF_EPT], im[GDF_EPT];
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) { re[q].zero(); im[q].zero(); }
  for (int64_t tile = blockIdx.x; tile * GDF_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * GDF_ROWS;
    const int rows = (int)((int64_t)GDF_ROWS < N - base ? (int64_t)GDF_ROWS : N - base);
    __syncthreads();
    for (int b = 0; b < a.nblk; ++b)
      for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
        int r = e / n2, k = e - r * n2;
        sm[(b * GDF_ROWS + r) * ldb + k] = a.blk[b][(base + r) * n2 + k];
      }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GDF_EPT; ++q) {
      int e = e0 + q * blockDim.x + threadIdx.x;
      if (e < total) {
        int s = e / (n * n), rem = e - s * n * n, k1 = rem / n, k2 = rem - k1 * n;
        const float2* X = sm + a.pa[s] * GDF_ROWS * ldb;
        const float2* Y = sm + a.pb[s] * GDF_ROWS * ldb;
        for (int r = 0; r < rows; ++r) {
          float2 xr = X[r * ldb + k1], xi = X[r * ldb + n + k1];
          float2 yr = Y[r * ldb + k2], yi = Y[r * ldb + n + k2];
          // conj(x) y = (xr yr + xi yi) + i (xr yi - xi yr)
          re[q].fma2(xr, yr);
          re[q].fma2(xi, yi);
          im[q].fma2(xr, yi);
          im[q].fma2(make_float2(-xi.x, -xi.y), yr);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) {
    int e = e0 + q * blockDim.x + threadIdx.x;
    if (e < total) part[(int64_t)blockIdx.x * total + e] = make_double2(re[q].value(), im[q].value());
  }
}

void gram_df(int64_t N, int n, const GramArgsDF& a, double2* part, int gridx, cudaStream_t st) {
  int total = a.npairs * n * n;
  int gy = ceil_div(total, TILE_THREADS * GDF_EPT);
  size_t smem = sizeof(float2) * a.nblk * GDF_ROWS * (2 * n + 1);
  k_gram_df<<<dim3(gridx, gy), TILE_THREADS, smem, st>>>(N, n, a, part);
}

// Real Gram X^T X of N x m double-float rows (G_V of the stored [A | B]).
__global__ void k_gram_real_df(int64_t N, int m, const float2* __restrict__ X,
                               double* __restrict__ part) {
  extern __shared__ __align__(16) unsigned char smraw[];
  float2* sm = reinterpret_cast<float2*>(smraw);
  const int ldb = m + 1, total = m * m;
  const int e0 = blockIdx.y * blockDim.x * GDF_EPT;
  Acc acc[GDF_EPT];
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) acc[q].zero();
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
      int e = e0 + q * blockDim.x + threadIdx.x;
      if (e < total) {
        int k1 = e / m, k2 = e - k1 * m;
        for (int r = 0; r < rows; ++r) acc[q].fma2(sm[r * ldb + k1], sm[r * ldb + k2]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < GDF_EPT; ++q) {
    int e = e0 + q * blockDim.x + threadIdx.x;
    if (e < total) part[(int64_t)blockIdx.x * total + e] = acc[q].value();
  }
}

void gram_real_df(int64_t N, int m, const float2* X, double* part, int gridx, cudaStream_t st) {
  int gy = ceil_div(m * m, TILE_THREADS * GDF_EPT);
  size_t smem = sizeof(float2) * GDF_ROWS * (m + 1);
  k_gram_real_df<<<dim3(gridx, gy), TILE_THREADS, smem, st>>>(N, m, X, part);
}

// --------------------------------------------------- affine (double-float)
// out_l = sum_t X_t,l C_t (C_t n x n complex FP64, converted once per block);
// written as FP64 rows (out_d) and/or double-float rows (out_f).
__global__ void k_affine_df(int64_t N, int n, AffineArgsDF a, const double2* __restrict__ C,
                            double* __restrict__ out_d, float2* __restrict__ out_f) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const int n2 = 2 * n, ldb = n2 + 1, nn = n * n;
  float2* Cr = reinterpret_cast<float2*>(smraw);  // nterms x n x n
  float2* Ci = Cr + a.nterms * nn;
  float2* Xs = Ci + a.nterms * nn;
  for (int e = threadIdx.x; e < a.nterms * nn; e += blockDim.x) {
    double2 c = C[e];
    Cr[e] = df_split(c.x);
    Ci[e] = df_split(c.y);
  }
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    __syncthreads();
    for (int b = 0; b < a.nterms; ++b)
      for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
        int r = e / n2, k = e - r * n2;
        Xs[(b * TILE_ROWS + r) * ldb + k] = a.X[b][(base + r) * n2 + k];
      }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * n; e += blockDim.x) {
      int r = e / n, k = e - r * n;
      Acc re, im;
      re.zero();
      im.zero();
      for (int b = 0; b < a.nterms; ++b) {
        const float2* x = Xs + (b * TILE_ROWS + r) * ldb;
        const float2* cr = Cr + b * nn;
        const float2* ci = Ci + b * nn;
        for (int q = 0; q < n; ++q) {
          float2 xr = x[q], xi = x[n + q], c_r = cr[q * n + k], c_i = ci[q * n + k];
          // (xr + i xi)(cr + i ci) = (xr cr - xi ci) + i (xr ci + xi cr)
          re.fma2(xr, c_r);
          re.fma2(make_float2(-xi.x, -xi.y), c_i);
          im.fma2(xr, c_i);
          im.fma2(xi, c_r);
        }
      }
      const int64_t o = (base + r) * n2;
      if (out_d) {
        out_d[o + k] = re.value();
        out_d[o + n + k] = im.value();
      }
      if (out_f) {
        out_f[o + k] = re.df();
        out_f[o + n + k] = im.df();
      }
    }
  }
}

void affine_df(int64_t N, int n, const AffineArgsDF& a, const double2* C, double* out_d,
               float2* out_f, int num_sms, cudaStream_t st) {
  size_t smem = sizeof(float2) * (2 * a.nterms * n * n + a.nterms * TILE_ROWS * (2 * n + 1));
  int gx = tile_grid_x(N, 1, num_sms);
  k_affine_df<<<gx, TILE_THREADS, smem, st>>>(N, n, a, C, out_d, out_f);
}

void df_init() {
  const int big = 220 * 1024;
  cudaFuncSetAttribute(k_deposit_df, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_project_df<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_project_df<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_basis_M_df<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_basis_M_df<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gram_df, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gram_real_df, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_affine_df, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

}  // namespace vpk
