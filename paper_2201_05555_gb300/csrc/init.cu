// Truncated complex SVD start of the reduced model (Sec. 3.2, Algorithm 2):
// R0 = X0 + i V0 (N x p), Q = n leading left singular vectors, zeta = Q^H R0.
//
// Computed through the p x p Hermitian Gram matrix A = R0^H R0 = W S^2 W^H:
// Q = R0 W_n S_n^-1.  A is diagonalised by a cyclic Jacobi method in one
// thread block (round-robin ordering: p/2 disjoint rotations per round).
// Forming A squares the condition number, so Q is re-orthonormalised with
// Q <- Q G^{-1/2}, G = Q^H Q (the same Jacobi routine), which keeps the span.
// The phase of each column of Q is left as it comes (it is free).
#include "vp_internal.cuh"

namespace vpk {

__device__ __forceinline__ double2 d2conj(double2 a) { return make_double2(a.x, -a.y); }

// ------------------------------------------------------------- Gram R0^H R0
// part[blockIdx.x][i][j] (double2), rows of R0 = particles.
#define IG_ROWS 32
__global__ void k_rgram(int64_t N, int p, const double* __restrict__ X, const double* __restrict__ V,
                        double2* __restrict__ part) {
  extern __shared__ double ism[];
  double* xs = ism;                 // p x IG_ROWS
  double* vs = ism + p * IG_ROWS;   // p x IG_ROWS
  const int tot = p * p;
  const int e0 = blockIdx.y * blockDim.x * 16;
  double2 acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = make_double2(0.0, 0.0);
  for (int64_t tile = blockIdx.x; tile * IG_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * IG_ROWS;
    const int rows = (int)((int64_t)IG_ROWS < N - base ? (int64_t)IG_ROWS : N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < p * IG_ROWS; e += blockDim.x) {
      int i = e / IG_ROWS, r = e - i * IG_ROWS;
      xs[e] = r < rows ? X[(int64_t)i * N + base + r] : 0.0;
      vs[e] = r < rows ? V[(int64_t)i * N + base + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      int e = e0 + threadIdx.x + q * blockDim.x;
      if (e < tot) {
        int i = e / p, j = e - i * p;
        double2 s = acc[q];
        for (int r = 0; r < IG_ROWS; ++r) {
          double xi = xs[i * IG_ROWS + r], vi = vs[i * IG_ROWS + r];
          double xj = xs[j * IG_ROWS + r], vj = vs[j * IG_ROWS + r];
          // conj(x_i + i v_i)(x_j + i v_j)
          s.x = fma(xi, xj, fma(vi, vj, s.x));
          s.y = fma(xi, vj, fma(-vi, xj, s.y));
        }
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    int e = e0 + threadIdx.x + q * blockDim.x;
    if (e < tot) part[(int64_t)blockIdx.x * tot + e] = acc[q];
  }
}

// ------------------------------------------------------- Hermitian Jacobi
#define JACOBI_SMEM_M 76
// Diagonalise the Hermitian m x m matrix A (global, overwritten) and
// accumulate the unitary W (global, m x m): A_in = W diag(lambda) W^H.
// Writes lambda (descending) and the matching columns of W sorted into Wout
// (m x m).  m <= 256 (even m uses all slots; odd m adds an idle slot).
// With in_smem (m <= JACOBI_SMEM_M) A and W are copied to shared memory and
// rotated there.  A pair is rotated unless |a_jk| <= 1e-15 sqrt|a_jj a_kk| or
// both diagonal entries are below 1e-14 of the largest one (a pair inside the
// rounding-level null space of a rank-deficient matrix, whose rotations would
// go on forever and change no eigenpair above it).
__global__ void k_jacobi(int m, double2* A_g, double2* W_g, double* lambda, double2* Wout,
                         int max_sweeps, int* status, int in_smem) {
  extern __shared__ double2 jac_sm[];
  __shared__ double2 rot_c[128], rot_s[128];
  __shared__ int pj[128], pk[128];
  __shared__ double off_s, tot_s, nu_s;
  __shared__ int nrot;
  __shared__ int order[256];
  const int t = threadIdx.x, nt = blockDim.x;
  double2* A = in_smem ? jac_sm : A_g;
  double2* W = in_smem ? jac_sm + m * m : W_g;
  if (in_smem)
    for (int e = t; e < m * m; e += nt) A[e] = A_g[e];
  for (int e = t; e < m * m; e += nt) W[e] = make_double2((e / m) == (e % m) ? 1.0 : 0.0, 0.0);
  __syncthreads();
  const int slots = (m + 1) & ~1;  // round-robin slots (one idle when m is odd)
  const int npair = slots / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence: off-diagonal mass against the whole
    if (t == 0) {
      off_s = 0.0;
      tot_s = 0.0;
      nrot = 0;
      double dm = 0.0;
      for (int j = 0; j < m; ++j) dm = fmax(dm, fabs(A[j * m + j].x));
      nu_s = 1e-14 * dm;
    }
    __syncthreads();
    double off = 0.0, tot = 0.0;
    for (int e = t; e < m * m; e += nt) {
      double2 a = A[e];
      double v = a.x * a.x + a.y * a.y;
      tot += v;
      if ((e / m) != (e % m)) off += v;
    }
    atomicAdd(&off_s, off);
    atomicAdd(&tot_s, tot);
    __syncthreads();
    const bool conv = !(off_s > 1e-30 * tot_s);
    __syncthreads();
    if (conv) break;
    for (int round = 0; round < slots - 1; ++round) {
      // slot s pairs (s, slots-1-s) in the rotated arrangement; slot 0 stays fixed
      for (int q = t; q < npair; q += nt) {
        int a = q, b = slots - 1 - q;
        int ia = (a == 0) ? 0 : 1 + (a - 1 + round) % (slots - 1);
        int ib = (b == 0) ? 0 : 1 + (b - 1 + round) % (slots - 1);
        int j = ia < ib ? ia : ib, k = ia < ib ? ib : ia;
        pj[q] = j;
        pk[q] = k;
        double2 c = make_double2(1.0, 0.0), s = make_double2(0.0, 0.0);
        if (k < m) {
          double2 ajk = A[j * m + k];
          double mag = sqrt(ajk.x * ajk.x + ajk.y * ajk.y);
          double ajj = A[j * m + j].x, akk = A[k * m + k].x;
          // rotate unless a_jk is below rounding of the diagonal pair (the
          // classical threshold |a_jk| <= eps sqrt|a_jj a_kk|)
          if (mag > 1e-15 * sqrt(fabs(ajj * akk)) && mag > 1e-300 &&
              fmax(fabs(ajj), fabs(akk)) > nu_s) {
            atomicAdd(&nrot, 1);
            double tau = (akk - ajj) / (2.0 * mag);
            double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            double cs = 1.0 / sqrt(1.0 + tt * tt), sn = tt * cs;
            // unitary [[cs, sn e^{i phi}], [-sn e^{-i phi}, cs]] with e^{i phi} = ajk / |ajk|
            c = make_double2(cs, 0.0);
            s = make_double2(sn * ajk.x / mag, sn * ajk.y / mag);
          }
        }
        rot_c[q] = c;
        rot_s[q] = s;
      }
      __syncthreads();
      // A <- A G (columns j, k), W <- W G
      for (int e = t; e < npair * m; e += nt) {
        int q = e / m, r = e - q * m;
        int j = pj[q], k = pk[q];
        if (k >= m) continue;
        double cs = rot_c[q].x;
        double2 s = rot_s[q];
        double2 arj = A[r * m + j], ark = A[r * m + k];
        // new_j = cs a_j - conj(s) a_k ; new_k = s a_j + cs a_k
        double2 nj = make_double2(cs * arj.x - (s.x * ark.x + s.y * ark.y),
                                  cs * arj.y - (s.x * ark.y - s.y * ark.x));
        double2 nk = make_double2(s.x * arj.x - s.y * arj.y + cs * ark.x,
                                  s.x * arj.y + s.y * arj.x + cs * ark.y);
        A[r * m + j] = nj;
        A[r * m + k] = nk;
        double2 wrj = W[r * m + j], wrk = W[r * m + k];
        W[r * m + j] = make_double2(cs * wrj.x - (s.x * wrk.x + s.y * wrk.y),
                                    cs * wrj.y - (s.x * wrk.y - s.y * wrk.x));
        W[r * m + k] = make_double2(s.x * wrj.x - s.y * wrj.y + cs * wrk.x,
                                    s.x * wrj.y + s.y * wrj.x + cs * wrk.y);
      }
      __syncthreads();
      // A <- G^H A (rows j, k)
      for (int e = t; e < npair * m; e += nt) {
        int q = e / m, c = e - q * m;
        int j = pj[q], k = pk[q];
        if (k >= m) continue;
        double cs = rot_c[q].x;
        double2 s = rot_s[q];
        double2 ajc = A[j * m + c], akc = A[k * m + c];
        // row_j = cs a_j - s a_k ; row_k = conj(s) a_j + cs a_k
        double2 nj = make_double2(cs * ajc.x - (s.x * akc.x - s.y * akc.y),
                                  cs * ajc.y - (s.x * akc.y + s.y * akc.x));
        double2 nk = make_double2(s.x * ajc.x + s.y * ajc.y + cs * akc.x,
                                  s.x * ajc.y - s.y * ajc.x + cs * akc.y);
        A[j * m + c] = nj;
        A[k * m + c] = nk;
      }
      __syncthreads();
    }
    // a sweep without rotations: every pair is below the threshold
    const int nr = nrot;
    __syncthreads();
    if (nr == 0) break;
    if (sweep == max_sweeps - 1 && t == 0) vp_set_status(status, VP_ENOCONV);
  }
  // sort eigenvalues descending (m <= 256, one thread: selection order)
  if (t == 0) {
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 0; i < m; ++i) {
      int best = i;
      for (int j = i + 1; j < m; ++j)
        if (A[order[j] * m + order[j]].x > A[order[best] * m + order[best]].x) best = j;
      int tmp = order[i];
      order[i] = order[best];
      order[best] = tmp;
    }
  }
  __syncthreads();
  for (int i = t; i < m; i += nt) lambda[i] = A[order[i] * m + order[i]].x;
  for (int e = t; e < m * m; e += nt) {
    int r = e / m, c = e - r * m;
    Wout[e] = W[r * m + order[c]];
  }
}

// Coefficients of Q = R0 W_n S_n^-1: C[i][k] = W[i][k] / sqrt(lambda_k) (p x n).
__global__ void k_init_coeff(int p, int n, const double2* W, const double* lambda, double2* C,
                             int* status) {
  for (int e = threadIdx.x; e < p * n; e += blockDim.x) {
    int i = e / n, k = e - i * n;
    double l = lambda[k];
    if (!(l > 0.0)) {
      vp_set_status(status, VP_ENUMERIC);
      C[e] = make_double2(0.0, 0.0);
      continue;
    }
    double w = 1.0 / sqrt(l);
    double2 v = W[i * p + k];
    C[e] = make_double2(v.x * w, v.y * w);
  }
}

// Q_lk = sum_i R0_li C_ik, R0_li = X[i][l] + i V[i][l] (Q stored as [Re | Im]).
__global__ void k_r_times(int64_t N, int p, int n, const double* __restrict__ X,
                          const double* __restrict__ V, const double2* __restrict__ C,
                          double* __restrict__ Q) {
  extern __shared__ double2 csm[];  // p x n
  for (int e = threadIdx.x; e < p * n; e += blockDim.x) csm[e] = C[e];
  __syncthreads();
  const int n2 = 2 * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N * n;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t l = e / n;
    int k = (int)(e - l * n);
    double2 s = make_double2(0.0, 0.0);
    for (int i = 0; i < p; ++i) {
      double x = X[(int64_t)i * N + l], v = V[(int64_t)i * N + l];
      double2 c = csm[i * n + k];
      s.x = fma(x, c.x, fma(-v, c.y, s.x));
      s.y = fma(x, c.y, fma(v, c.x, s.y));
    }
    Q[l * n2 + k] = s.x;
    Q[l * n2 + n + k] = s.y;
  }
}

// G^{-1/2} = W diag(lambda^-1/2) W^H (n x n) from the eigen-decomposition of G.
__global__ void k_inv_sqrt(int n, const double2* W, const double* lambda, double2* out, int* status) {
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e - r * n;
    double2 s = make_double2(0.0, 0.0);
    for (int k = 0; k < n; ++k) {
      double l = lambda[k];
      if (!(l > 0.0)) {
        vp_set_status(status, VP_ENUMERIC);
        continue;
      }
      double w = 1.0 / sqrt(l);
      double2 a = W[r * n + k], b = d2conj(W[c * n + k]);
      s.x += w * (a.x * b.x - a.y * b.y);
      s.y += w * (a.x * b.y + a.y * b.x);
    }
    out[e] = s;
  }
}

// zeta_ki = sum_l conj(Q_lk) R0_li; part[blockIdx.x][k][i] (double2).
__global__ void k_zeta(int64_t N, int p, int n, const double* __restrict__ Q,
                       const double* __restrict__ X, const double* __restrict__ V,
                       double2* __restrict__ part) {
  extern __shared__ double ism[];
  const int n2 = 2 * n;
  double* qs = ism;                    // IG_ROWS x n2
  double* xs = ism + IG_ROWS * n2;     // p x IG_ROWS
  double* vs = xs + p * IG_ROWS;
  const int tot = n * p;
  const int e0 = blockIdx.y * blockDim.x * 16;
  double2 acc[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) acc[q] = make_double2(0.0, 0.0);
  for (int64_t tile = blockIdx.x; tile * IG_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * IG_ROWS;
    const int rows = (int)((int64_t)IG_ROWS < N - base ? (int64_t)IG_ROWS : N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < IG_ROWS * n2; e += blockDim.x) {
      int r = e / n2, k = e - r * n2;
      qs[e] = r < rows ? Q[(base + r) * n2 + k] : 0.0;
    }
    for (int e = threadIdx.x; e < p * IG_ROWS; e += blockDim.x) {
      int i = e / IG_ROWS, r = e - i * IG_ROWS;
      xs[e] = r < rows ? X[(int64_t)i * N + base + r] : 0.0;
      vs[e] = r < rows ? V[(int64_t)i * N + base + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      int e = e0 + threadIdx.x + q * blockDim.x;
      if (e < tot) {
        int k = e / p, i = e - k * p;
        double2 s = acc[q];
        for (int r = 0; r < IG_ROWS; ++r) {
          double a = qs[r * n2 + k], b = qs[r * n2 + n + k];
          double x = xs[i * IG_ROWS + r], v = vs[i * IG_ROWS + r];
          // (a - i b)(x + i v)
          s.x = fma(a, x, fma(b, v, s.x));
          s.y = fma(a, v, fma(-b, x, s.y));
        }
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    int e = e0 + threadIdx.x + q * blockDim.x;
    if (e < tot) part[(int64_t)blockIdx.x * tot + e] = acc[q];
  }
}

// Z = [Re zeta; Im zeta] from zeta (n x p double2).
__global__ void k_zeta_to_Z(int n, int p, const double2* zeta, double* Z) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * p; e += gridDim.x * blockDim.x) {
    int k = e / p, i = e - k * p;
    Z[(int64_t)k * p + i] = zeta[e].x;
    Z[(int64_t)(n + k) * p + i] = zeta[e].y;
  }
}

// Dynamic shared memory above 48 KB (p up to 256: 2 p IG_ROWS doubles = 128 KB).
void init_kernels_init() {
  const int lim = 227 * 1024;
  cudaFuncSetAttribute(k_rgram, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_r_times, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_zeta, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void init_launch_rgram(int64_t N, int p, const double* X, const double* V, double2* part, int gx,
                       cudaStream_t st) {
  dim3 grid(gx, ceil_div((int64_t)p * p, 256 * 16));
  k_rgram<<<grid, 256, sizeof(double) * 2 * p * IG_ROWS, st>>>(N, p, X, V, part);
}
void init_launch_jacobi(int m, double2* A, double2* W, double* lambda, double2* Wout, int* status,
                        cudaStream_t st) {
  const int in_smem = m <= JACOBI_SMEM_M;
  const size_t smem = in_smem ? sizeof(double2) * 2 * m * m : 0;
  k_jacobi<<<1, 512, smem, st>>>(m, A, W, lambda, Wout, 60, status, in_smem);
}
void init_launch_coeff(int p, int n, const double2* W, const double* lambda, double2* C, int* status,
                       cudaStream_t st) {
  k_init_coeff<<<1, 256, 0, st>>>(p, n, W, lambda, C, status);
}
void init_launch_r_times(int64_t N, int p, int n, const double* X, const double* V, const double2* C,
                         double* Q, int num_sms, cudaStream_t st) {
  int gx = ceil_div(N * n, 256);
  if (gx > 4 * num_sms) gx = 4 * num_sms;
  k_r_times<<<gx, 256, sizeof(double2) * p * n, st>>>(N, p, n, X, V, C, Q);
}
void init_launch_inv_sqrt(int n, const double2* W, const double* lambda, double2* out, int* status,
                          cudaStream_t st) {
  k_inv_sqrt<<<1, 256, 0, st>>>(n, W, lambda, out, status);
}
void init_launch_zeta(int64_t N, int p, int n, const double* Q, const double* X, const double* V,
                      double2* part, int gx, cudaStream_t st) {
  dim3 grid(gx, ceil_div((int64_t)n * p, 256 * 16));
  k_zeta<<<grid, 256, sizeof(double) * (IG_ROWS * 2 * n + 2 * p * IG_ROWS), st>>>(N, p, n, Q, X, V, part);
}
void init_launch_zeta_to_Z(int n, int p, const double2* zeta, double* Z, cudaStream_t st) {
  k_zeta_to_Z<<<ceil_div((int64_t)n * p, 256), 256, 0, st>>>(n, p, zeta, Z);
}

}  // namespace vpk
