// Kernels of the dynamical reduced model (Sec. 3.2 - 5) in complex storage:
// Q = A + iB (N x n) stored as rows [A_l | B_l] (2n doubles), zeta = a + ib
// stored as Z = [a; b] (2n x p).  X_r = Re(Q zeta) = A a - B b and
// V_r = Im(Q zeta) = B a + A b are the paper's U_X Z and U_V Z.
//
// Tile kernels: a block stages TILE_ROWS rows of Q in shared memory (row
// stride 2n+1 doubles, conflict-free) and works on (row, sample) pairs with
// lanes mapped to samples of a chunk of PC samples (PC a power of two <= 32),
// so reads of Q are broadcasts and per-sample grids are distinct addresses.
#include "vp_internal.cuh"

namespace vpk {

static inline int chunk_width(int p, int Nx) {
  int pc = 1;
  while (pc < p && pc < 32) pc <<= 1;
  while (pc > 1 && (size_t)pc * Nx * 8 > 96 * 1024) pc >>= 1;
  return pc;
}

int tile_grid_x(int64_t N, int chunks, int num_sms) {
  int tiles = ceil_div(N, TILE_ROWS);
  int want = (2 * num_sms + chunks - 1) / chunks;
  int gx = tiles < want ? tiles : want;
  return gx < 1 ? 1 : gx;
}

// Load rows [base, base+rows) of Q (or rows idx[base..]) into Qs (stride ldq).
// Rows named by idx outside [0, nrows) load as zeros and set VP_EINVAL.
__device__ __forceinline__ void load_q_tile(double* Qs, int ldq, const double* __restrict__ Q,
                                            int n2, int64_t base, int rows,
                                            const int32_t* __restrict__ idx, int64_t nrows = 0,
                                            int* status = nullptr) {
  for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
    int r = e / n2, k = e - r * n2;
    int64_t row = idx ? (int64_t)idx[base + r] : base + r;
    if (idx && (row < 0 || row >= nrows)) {
      vp_set_status(status, VP_EINVAL);
      Qs[r * ldq + k] = 0.0;
      continue;
    }
    Qs[r * ldq + k] = __ldg(Q + row * n2 + k);
  }
}

// Z chunk [c0, c0+PC) into Zs (n2 x ldz), zero padded.
__device__ __forceinline__ void load_z_chunk(double* Zs, int ldz, const double* __restrict__ Z,
                                             int n2, int p, int c0, int PC) {
  for (int e = threadIdx.x; e < n2 * PC; e += blockDim.x) {
    int k = e / PC, ii = e - k * PC;
    Zs[k * ldz + ii] = (c0 + ii < p) ? Z[(int64_t)k * p + c0 + ii] : 0.0;
  }
}

__device__ __forceinline__ double recon_x(const double* q, const double* Zs, int ldz, int n,
                                          int ii) {
  double x = 0.0;
  for (int k = 0; k < n; ++k) {
    x = fma(q[k], Zs[k * ldz + ii], x);
    x = fma(-q[n + k], Zs[(n + k) * ldz + ii], x);
  }
  return x;
}

__device__ __forceinline__ void recon_xv(const double* q, const double* Zs, int ldz, int n, int ii,
                                         double& x, double& v) {
  x = 0.0;
  v = 0.0;
  for (int k = 0; k < n; ++k) {
    double a = Zs[k * ldz + ii], b = Zs[(n + k) * ldz + ii];
    double A = q[k], B = q[n + k];
    x = fma(A, a, x);
    x = fma(-B, b, x);
    v = fma(B, a, v);
    v = fma(A, b, v);
  }
}

// ------------------------------------------------------------ reconstruct
__global__ void k_reconstruct(int64_t N, int n, int p, int PC, const double* __restrict__ Q,
                              const double* __restrict__ Z, double* __restrict__ X,
                              double* __restrict__ V) {
  extern __shared__ double sm[];
  const int n2 = 2 * n, ldq = n2 + 1, ldz = PC + 1, ldo = TILE_ROWS + 1;
  double* Qs = sm;
  double* Zs = Qs + TILE_ROWS * ldq;
  double* Xs = Zs + n2 * ldz;
  double* Vs = Xs + PC * ldo;
  const int c0 = blockIdx.y * PC;
  load_z_chunk(Zs, ldz, Z, n2, p, c0, PC);
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const int pc_eff = min(PC, p - c0);
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    __syncthreads();
    load_q_tile(Qs, ldq, Q, n2, base, rows, nullptr);
    __syncthreads();
    for (int r = rsub; r < rows; r += RP) {
      double x, v;
      recon_xv(Qs + r * ldq, Zs, ldz, n, ii, x, v);
      Xs[ii * ldo + r] = x;
      Vs[ii * ldo + r] = v;
    }
    __syncthreads();
    for (int e = t; e < pc_eff * rows; e += blockDim.x) {
      int c = e / rows, r = e - c * rows;
      int64_t o = (int64_t)(c0 + c) * N + base + r;
      X[o] = Xs[c * ldo + r];
      if (V) V[o] = Vs[c * ldo + r];
    }
  }
}

void reconstruct(int64_t N, int n, int p, const double* Q, const double* Z, double* X, double* V,
                 cudaStream_t st) {
  int PC = chunk_width(p, 1);
  int ch = ceil_div(p, PC);
  int n2 = 2 * n;
  size_t smem = sizeof(double) * (TILE_ROWS * (n2 + 1) + n2 * (PC + 1) + 2 * PC * (TILE_ROWS + 1));
  int gx = tile_grid_x(N, ch, VP_NSM_DEFAULT);
  k_reconstruct<<<dim3(gx, ch), TILE_THREADS, smem, st>>>(N, n, p, PC, Q, Z, X, V);
}

// ---------------------------------------------------- deposit of X_r = U_X Z
__global__ void k_deposit_reduced(GridC g, int64_t N, int n, int p, int PC,
                                  const double* __restrict__ Q, const double* __restrict__ Z,
                                  unsigned long long* __restrict__ counts, const int* skip) {
  if (skip && *skip) return;
  extern __shared__ double sm[];
  const int n2 = 2 * n, ldq = n2 + 1, ldz = PC + 1, Nx = g.Nx;
  double* Qs = sm;
  double* Zs = Qs + TILE_ROWS * ldq;
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(Zs + n2 * ldz);
  const int c0 = blockIdx.y * PC;
  load_z_chunk(Zs, ldz, Z, n2, p, c0, PC);
  for (int e = threadIdx.x; e < PC * Nx; e += blockDim.x) cnt[e] = 0ull;
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const bool active = c0 + ii < p;
  const unsigned long long one = 1ull << g.S;
  unsigned long long* mycnt = cnt + ii * Nx;
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    __syncthreads();
    load_q_tile(Qs, ldq, Q, n2, base, rows, nullptr);
    __syncthreads();
    if (active) {
      for (int r = rsub; r < rows; r += RP) {
        double x = recon_x(Qs + r * ldq, Zs, ldz, n, ii);
        int j;
        double s;
        cell_of(x, g.inv_h, Nx, g.dNx, g.inv_Nx, j, s);
        unsigned long long w1 = (unsigned long long)__double2ll_rn(s * g.fp_scale);
        int j1 = (j + 1 == Nx) ? 0 : j + 1;
        atomicAdd(mycnt + j, one - w1);
        atomicAdd(mycnt + j1, w1);
      }
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < PC * Nx; e += blockDim.x) {
    int c = e / Nx;
    if (c0 + c < p && cnt[e]) atomicAdd(&counts[(int64_t)(c0 + c) * Nx + (e - c * Nx)], cnt[e]);
  }
}

void deposit_reduced(const GridC& g, int64_t N, int n, int p, const double* Q, const double* Z,
                     unsigned long long* counts, const int* skip, int num_sms, cudaStream_t st) {
  int PC = chunk_width(p, g.Nx);
  int ch = ceil_div(p, PC);
  int n2 = 2 * n;
  size_t smem = sizeof(double) * (TILE_ROWS * (n2 + 1) + n2 * (PC + 1)) +
                sizeof(unsigned long long) * PC * g.Nx;
  int gx = tile_grid_x(N, ch, num_sms);
  k_deposit_reduced<<<dim3(gx, ch), TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q, Z, counts, skip);
}

// ------------------------------------------------- projection g_X = U_X^T G
// part[blockIdx.x][k][i] (2n x p per block): sum over the block's rows of
//   k < n :  A_lk G_li,   k >= n : -B_l(k-n) G_li
// G_li from GX (p x N) if given, else (scale_l) * F_i[cell(X_r,li)] with
// scale_l = q/m, or c_l / m_p for DEIM rows (idx != null).
#define PROJ_MAXACC 16
__global__ void k_project(GridC g, int64_t count, int n, int p, int PC,
                          const double* __restrict__ Q, const double* __restrict__ Z,
                          const double* __restrict__ F, const double* __restrict__ GX, int64_t ldg,
                          const int32_t* __restrict__ idx, const double* __restrict__ cw,
                          int64_t nrows, double* __restrict__ part, const int* skip, int* status) {
  if (skip && *skip) return;
  extern __shared__ double sm[];
  const int n2 = 2 * n, ldq = n2 + 1, ldz = PC + 1, Nx = g.Nx, ldG = PC + 1;
  double* Qs = sm;
  double* Zs = Qs + TILE_ROWS * ldq;
  double* Fs = Zs + n2 * ldz;   // PC x Nx
  double* Gs = Fs + PC * Nx;    // TILE_ROWS x ldG
  const int c0 = blockIdx.y * PC;
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const bool active = c0 + ii < p;
  if (!GX) {
    load_z_chunk(Zs, ldz, Z, n2, p, c0, PC);
    for (int e = t; e < PC * Nx; e += blockDim.x) {
      int c = e / Nx;
      Fs[e] = (c0 + c < p) ? F[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : 0.0;
    }
  }
  const int npairs = n2 * PC;
  double acc[PROJ_MAXACC];
#pragma unroll
  for (int a = 0; a < PROJ_MAXACC; ++a) acc[a] = 0.0;
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < count; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < count - base ? (int64_t)TILE_ROWS : count - base);
    __syncthreads();
    load_q_tile(Qs, ldq, Q, n2, base, rows, idx, nrows, status);
    if (GX) {
      for (int e = t; e < PC * rows; e += blockDim.x) {
        int c = e / rows, r = e - c * rows;
        Gs[r * ldG + c] = (c0 + c < p) ? GX[(int64_t)(c0 + c) * ldg + base + r] : 0.0;
      }
    }
    __syncthreads();
    if (!GX) {
      for (int r = rsub; r < rows; r += RP) {
        double G = 0.0;
        if (active) {
          double x = recon_x(Qs + r * ldq, Zs, ldz, n, ii);
          int j;
          double s;
          cell_of(x, g.inv_h, Nx, g.dNx, g.inv_Nx, j, s);
          double sc = cw ? cw[base + r] / g.mp : g.qm;
          G = sc * Fs[ii * Nx + j];
        }
        Gs[r * ldG + ii] = G;
      }
      __syncthreads();
    }
    for (int a = 0, e = t; e < npairs; ++a, e += blockDim.x) {
      int k = e / PC, c = e - k * PC;
      double s = 0.0;
      for (int r = 0; r < rows; ++r) s = fma(Qs[r * ldq + k], Gs[r * ldG + c], s);
      acc[a] += s;
    }
  }
  for (int a = 0, e = t; e < npairs; ++a, e += blockDim.x) {
    int k = e / PC, c = e - k * PC;
    if (c0 + c < p) part[(int64_t)blockIdx.x * n2 * p + (int64_t)k * p + c0 + c] = (k < n) ? acc[a] : -acc[a];
  }
}

void project(const GridC& g, int64_t count, int n, int p, const double* Q, const double* Z,
             const double* F, const double* GX, int64_t ldg, const int32_t* idx, const double* cw,
             int64_t nrows, double* part, int gridx, const int* skip, int* status,
             cudaStream_t st) {
  int PC = chunk_width(p, g.Nx);
  int ch = ceil_div(p, PC);
  int n2 = 2 * n;
  size_t smem = sizeof(double) * (TILE_ROWS * (n2 + 1) + n2 * (PC + 1) + PC * g.Nx +
                                  TILE_ROWS * (PC + 1));
  k_project<<<dim3(gridx, ch), TILE_THREADS, smem, st>>>(g, count, n, p, PC, Q, Z, F, GX, ldg, idx,
                                                         cw, nrows, part, skip, status);
}

int project_chunks(int p, int Nx) { return ceil_div(p, chunk_width(p, Nx)); }
int chunk_pc(int p, int Nx) { return chunk_width(p, Nx); }

// ------------------------------------------------ M = Gamma zeta^H (N x n)
// Gamma_li = GX_li + i V_r,li at R = Q zeta; M_lk = sum_i Gamma_li conj(zeta_ki).
#define BM_MAXACC 16
__global__ void k_basis_M(GridC g, int64_t N, int n, int p, int PC, const double* __restrict__ Q,
                          const double* __restrict__ Z, const double* __restrict__ F,
                          double* __restrict__ M) {
  extern __shared__ double sm[];
  const int n2 = 2 * n, ldq = n2 + 1, ldz = PC + 1, Nx = g.Nx, ldG = PC + 1;
  double* Qs = sm;
  double* Zs = Qs + TILE_ROWS * ldq;
  double* Fs = Zs + n2 * ldz;
  // Fs region rounded up to an even number of doubles: Gam needs 16-byte alignment
  double2* Gam = reinterpret_cast<double2*>(Fs + ((PC * Nx + 1) & ~1));  // TILE_ROWS x ldG
  const int t = threadIdx.x, ii = t & (PC - 1), rsub = t / PC, RP = blockDim.x / PC;
  const int npairs = TILE_ROWS * n;
  for (int64_t tile = blockIdx.x; tile * TILE_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * TILE_ROWS;
    const int rows = (int)((int64_t)TILE_ROWS < N - base ? (int64_t)TILE_ROWS : N - base);
    double2 acc[BM_MAXACC];
#pragma unroll
    for (int a = 0; a < BM_MAXACC; ++a) acc[a] = make_double2(0.0, 0.0);
    __syncthreads();
    load_q_tile(Qs, ldq, Q, n2, base, rows, nullptr);
    for (int c0 = 0; c0 < p; c0 += PC) {
      __syncthreads();
      load_z_chunk(Zs, ldz, Z, n2, p, c0, PC);
      for (int e = t; e < PC * Nx; e += blockDim.x) {
        int c = e / Nx;
        Fs[e] = (c0 + c < p) ? g.qm * F[(int64_t)(c0 + c) * Nx + (e - c * Nx)] : 0.0;
      }
      __syncthreads();
      const bool active = c0 + ii < p;
      for (int r = rsub; r < rows; r += RP) {
        double2 gm = make_double2(0.0, 0.0);
        if (active) {
          double x, v;
          recon_xv(Qs + r * ldq, Zs, ldz, n, ii, x, v);
          int j;
          double s;
          cell_of(x, g.inv_h, Nx, g.dNx, g.inv_Nx, j, s);
          gm = make_double2(Fs[ii * Nx + j], v);
        }
        Gam[r * ldG + ii] = gm;
      }
      __syncthreads();
      const int pc_eff = min(PC, p - c0);
      for (int a = 0, e = t; e < npairs; ++a, e += blockDim.x) {
        int r = e / n, k = e - r * n;
        if (r < rows) {
          double2 s = acc[a];
          for (int c = 0; c < pc_eff; ++c) {
            double2 G = Gam[r * ldG + c];
            double za = Zs[k * ldz + c], zb = Zs[(n + k) * ldz + c];
            // G * conj(a + ib) = (Gr a + Gi b) + i (Gi a - Gr b)
            s.x = fma(G.x, za, fma(G.y, zb, s.x));
            s.y = fma(G.y, za, fma(-G.x, zb, s.y));
          }
          acc[a] = s;
        }
      }
    }
    for (int a = 0, e = t; e < npairs; ++a, e += blockDim.x) {
      int r = e / n, k = e - r * n;
      if (r < rows) {
        M[(base + r) * n2 + k] = acc[a].x;
        M[(base + r) * n2 + n + k] = acc[a].y;
      }
    }
  }
}

void basis_M(const GridC& g, int64_t N, int n, int p, const double* Q, const double* Z,
             const double* F, double* M, int num_sms, cudaStream_t st) {
  int PC = chunk_width(p, g.Nx);
  int n2 = 2 * n;
  size_t smem = sizeof(double) * (TILE_ROWS * (n2 + 1) + n2 * (PC + 1) + ((PC * g.Nx + 1) & ~1)) +
                sizeof(double2) * TILE_ROWS * (PC + 1);
  int gx = tile_grid_x(N, 1, num_sms);
  k_basis_M<<<gx, TILE_THREADS, smem, st>>>(g, N, n, p, PC, Q, Z, F, M);
}

// ------------------------------------------------------------ Gram matrices
// out_s = B_{pa[s]}^H B_{pb[s]} (n x n complex) for each pair s; rows tiled
// by GRAM_ROWS; part[blockIdx.x][s][k1][k2] (double2); blockIdx.y slices the
// entry list so that each thread keeps at most GRAM_EPT accumulators.
#define GRAM_ROWS 32
#define GRAM_EPT 8
__global__ void k_gram(int64_t N, int n, GramArgs a, double2* __restrict__ part) {
  extern __shared__ double sm[];
  const int n2 = 2 * n, ldb = n2 + 1;
  const int total = a.npairs * n * n;
  const int e0 = blockIdx.y * blockDim.x * GRAM_EPT;
  double2 acc[GRAM_EPT];
#pragma unroll
  for (int q = 0; q < GRAM_EPT; ++q) acc[q] = make_double2(0.0, 0.0);
  for (int64_t tile = blockIdx.x; tile * GRAM_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * GRAM_ROWS;
    const int rows = (int)((int64_t)GRAM_ROWS < N - base ? (int64_t)GRAM_ROWS : N - base);
    __syncthreads();
    for (int b = 0; b < a.nblk; ++b)
      for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
        int r = e / n2, k = e - r * n2;
        sm[(b * GRAM_ROWS + r) * ldb + k] = __ldg(a.blk[b] + (base + r) * n2 + k);
      }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GRAM_EPT; ++q) {
      int e = e0 + q * blockDim.x + threadIdx.x;
      if (e < total) {
        int s = e / (n * n), rem = e - s * n * n, k1 = rem / n, k2 = rem - k1 * n;
        const double* X = sm + a.pa[s] * GRAM_ROWS * ldb;
        const double* Y = sm + a.pb[s] * GRAM_ROWS * ldb;
        double2 c = acc[q];
        for (int r = 0; r < rows; ++r) {
          double xr = X[r * ldb + k1], xi = X[r * ldb + n + k1];
          double yr = Y[r * ldb + k2], yi = Y[r * ldb + n + k2];
          // conj(x) * y
          c.x = fma(xr, yr, fma(xi, yi, c.x));
          c.y = fma(xr, yi, fma(-xi, yr, c.y));
        }
        acc[q] = c;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < GRAM_EPT; ++q) {
    int e = e0 + q * blockDim.x + threadIdx.x;
    if (e < total) part[(int64_t)blockIdx.x * total + e] = acc[q];
  }
}

void gram(int64_t N, int n, const GramArgs& a, double2* part, int gridx, cudaStream_t st) {
  int total = a.npairs * n * n;
  int gy = ceil_div(total, TILE_THREADS * GRAM_EPT);
  size_t smem = sizeof(double) * a.nblk * GRAM_ROWS * (2 * n + 1);
  k_gram<<<dim3(gridx, gy), TILE_THREADS, smem, st>>>(N, n, a, part);
}

// Real Gram X^T X of an N x m row-major matrix (m <= 128).
__global__ void k_gram_real(int64_t N, int m, const double* __restrict__ X,
                            double* __restrict__ part) {
  extern __shared__ double sm[];
  const int ldb = m + 1;
  const int total = m * m;
  const int e0 = blockIdx.y * blockDim.x * GRAM_EPT;
  double acc[GRAM_EPT];
#pragma unroll
  for (int q = 0; q < GRAM_EPT; ++q) acc[q] = 0.0;
  for (int64_t tile = blockIdx.x; tile * GRAM_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * GRAM_ROWS;
    const int rows = (int)((int64_t)GRAM_ROWS < N - base ? (int64_t)GRAM_ROWS : N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
      int r = e / m, k = e - r * m;
      sm[r * ldb + k] = __ldg(X + (base + r) * m + k);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < GRAM_EPT; ++q) {
      int e = e0 + q * blockDim.x + threadIdx.x;
      if (e < total) {
        int k1 = e / m, k2 = e - k1 * m;
        double c = acc[q];
        for (int r = 0; r < rows; ++r) c = fma(sm[r * ldb + k1], sm[r * ldb + k2], c);
        acc[q] = c;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < GRAM_EPT; ++q) {
    int e = e0 + q * blockDim.x + threadIdx.x;
    if (e < total) part[(int64_t)blockIdx.x * total + e] = acc[q];
  }
}

void gram_real(int64_t N, int m, const double* X, double* part, int gridx, cudaStream_t st) {
  int gy = ceil_div(m * m, TILE_THREADS * GRAM_EPT);
  size_t smem = sizeof(double) * GRAM_ROWS * (m + 1);
  k_gram_real<<<dim3(gridx, gy), TILE_THREADS, smem, st>>>(N, m, X, part);
}

int gram_grid_x(int64_t N, int num_sms) {
  int tiles = ceil_div(N, GRAM_ROWS);
  int want = 2 * num_sms;
  return tiles < want ? tiles : want;
}

// ----------------------------------------------------- partial reductions
// out[e] = sum_b part[b * elems + e] in a fixed order (deterministic): one
// block per element, thread t sums parts t, t+256, ..., then a fixed tree.
__global__ void k_reduce_partials(int nparts, int64_t elems, const double* __restrict__ part,
                                  double* __restrict__ out, const int* skip) {
  if (skip && *skip) return;
  __shared__ double red[256];
  const int64_t e = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) s += part[(int64_t)b * elems + e];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = red[0];
}

void reduce_partials(int nparts, int64_t elems, const double* part, double* out, const int* skip,
                     cudaStream_t st) {
  k_reduce_partials<<<(unsigned)elems, 256, 0, st>>>(nparts, elems, part, out, skip);
}

// ---------------------------------------------------- affine combinations
// out_l = sum_t X_t,l C_t with C_t (n x n complex, row-major double2).
// out may alias an input: each block reads its rows before writing them.
__global__ void k_affine(int64_t N, int n, AffineArgs a, const double2* __restrict__ C,
                         double* out) {
  extern __shared__ double sm[];
  const int n2 = 2 * n, ldb = n2 + 1;
  double2* Cs = reinterpret_cast<double2*>(sm);
  double* Xs = sm + 2 * a.nterms * n * n;
  for (int e = threadIdx.x; e < a.nterms * n * n; e += blockDim.x) Cs[e] = C[e];
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
      double2 s = make_double2(0.0, 0.0);
      for (int b = 0; b < a.nterms; ++b) {
        const double* x = Xs + (b * TILE_ROWS + r) * ldb;
        const double2* c = Cs + b * n * n;
        for (int q = 0; q < n; ++q) {
          double2 cq = c[q * n + k];
          double xr = x[q], xi = x[n + q];
          s.x = fma(xr, cq.x, fma(-xi, cq.y, s.x));
          s.y = fma(xr, cq.y, fma(xi, cq.x, s.y));
        }
      }
      out[(base + r) * n2 + k] = s.x;
      out[(base + r) * n2 + n + k] = s.y;
    }
  }
}

void affine(int64_t N, int n, const AffineArgs& a, const double2* C, double* out, int num_sms,
            cudaStream_t st) {
  size_t smem = sizeof(double2) * a.nterms * n * n + sizeof(double) * a.nterms * TILE_ROWS * (2 * n + 1);
  int gx = tile_grid_x(N, 1, num_sms);
  k_affine<<<gx, TILE_THREADS, smem, st>>>(N, n, a, C, out);
}

// F of potentials phi (p x Nx): F_j = (phi_{j+1} - phi_j) / h.
__global__ void k_cell_gradient(GridC g, int p, const double* __restrict__ phi, double* __restrict__ F) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)p * g.Nx) return;
  int64_t i = e / g.Nx;
  int j = (int)(e - i * g.Nx);
  int j1 = (j + 1 == g.Nx) ? 0 : j + 1;
  F[e] = (phi[i * g.Nx + j1] - phi[e]) * g.inv_h;
}

void cell_gradient(const GridC& g, int p, const double* phi, double* F, cudaStream_t st) {
  int64_t n = (int64_t)p * g.Nx;
  k_cell_gradient<<<ceil_div(n, 256), 256, 0, st>>>(g, p, phi, F);
}

}  // namespace vpk

namespace vpk {
void reduced_init() {
  const int big = 220 * 1024;
  cudaFuncSetAttribute(k_reconstruct, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_deposit_reduced, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_project, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_basis_M, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_gram_real, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
  cudaFuncSetAttribute(k_affine, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}
}  // namespace vpk
