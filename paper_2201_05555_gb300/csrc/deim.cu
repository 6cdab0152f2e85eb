// Hyper-reduction on the device (Sec. 4.2).
// DEIM construction: snapshot columns Lambda^0(X_r) Phi (eq. Ydeim), the
// basis of the first d left singular vectors of the snapshot matrix, the
// greedy interpolation indices and the weights c = (P^T Psi)^-T Psi^T M_q of
// the DEIM-indexed gradient.
// DMD of the potential (Algorithm 1): with the truncated SVD Y = U S V^T of
// the window data, B = Y' V S^-1 and A = U^T B, the exact-DMD prediction
// Theta (Pi (.) lambda^(s/dt)) with Theta = B W, A W = W Lambda, equals
// B A^(s/dt) B^+ Phi (Theta^+ = W^-1 B^+), so whole and half steps need only
// real powers of A and its principal square root (Denman-Beavers iteration),
// no complex eigen-decomposition.
//
// Layouts: snapshot matrix Y stored column by column (m x N, leading
// dimension ldy >= N); basis Psi column by column (d x N).  FP64 throughout.
// The singular vectors come from the Gram matrix Y^T Y (cyclic Jacobi of
// init.cu), so directions of singular values below ~1e-8 sigma_1 are not
// resolved; the interpolation indices need only the leading ones.
#include "vp_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace vpk {
void init_launch_jacobi(int m, double2* A, double2* W, double* lambda, double2* Wout, int* status,
                        cudaStream_t st);
}

namespace {
using namespace vpk;

__global__ void k_phi_at(GridC g, int64_t N, int p, const double* __restrict__ X, int64_t ldx,
                         const double* __restrict__ phi, double* __restrict__ Y, int64_t ldy) {
  const int i = blockIdx.y;
  const double* x = X + (int64_t)i * ldx;
  const double* ph = phi + (int64_t)i * g.Nx;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
       l += (int64_t)gridDim.x * blockDim.x) {
    int j;
    double s;
    cell_of(x[l], g.inv_h, g.Nx, g.dNx, g.inv_Nx, j, s);
    const int j1 = (j + 1 == g.Nx) ? 0 : j + 1;
    Y[(int64_t)i * ldy + l] = fma(s, ph[j1], (1.0 - s) * ph[j]);
  }
}

// part[blockIdx.x][a][b] = sum over this block's rows of Y_a Y_b (m x m, m <= 256)
#define YG_ROWS 32
__global__ void k_ygram(int64_t N, int m, const double* __restrict__ Y, int64_t ldy,
                        double* __restrict__ part) {
  extern __shared__ double ys[];  // m x YG_ROWS
  const int tot = m * m;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  const int e0 = blockIdx.y * blockDim.x * 8;
  for (int64_t tile = blockIdx.x; tile * YG_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * YG_ROWS;
    const int rows = (int)((int64_t)YG_ROWS < N - base ? (int64_t)YG_ROWS : N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < m * YG_ROWS; e += blockDim.x) {
      const int a = e / YG_ROWS, r = e - a * YG_ROWS;
      ys[e] = r < rows ? Y[(int64_t)a * ldy + base + r] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * blockDim.x + threadIdx.x;
      if (e < tot) {
        const int a = e / m, b = e - a * m;
        double s = acc[q];
        for (int r = 0; r < YG_ROWS; ++r) s = fma(ys[a * YG_ROWS + r], ys[b * YG_ROWS + r], s);
        acc[q] = s;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int e = e0 + q * blockDim.x + threadIdx.x;
    if (e < tot) part[(int64_t)blockIdx.x * tot + e] = acc[q];
  }
}

__global__ void k_to_complex(int m, const double* __restrict__ a, double2* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
    out[e] = make_double2(a[e], 0.0);
}

// psi_k = Y w_k / sqrt(lambda_k), k < d; sigma = sqrt(max(lambda, 0)) (m values)
__global__ void k_psi(int64_t N, int m, int d, const double* __restrict__ Y, int64_t ldy,
                      const double2* __restrict__ W, const double* __restrict__ lam,
                      double* __restrict__ Psi, double* __restrict__ sigma, int* status) {
  extern __shared__ double cs[];  // m x d coefficients
  for (int e = threadIdx.x; e < m * d; e += blockDim.x) {
    const int a = e / d, k = e - a * d;
    const double l = lam[k];
    if (!(l > 0.0)) {
      vp_set_status(status, VP_ENUMERIC);
      cs[e] = 0.0;
    } else {
      cs[e] = W[a * m + k].x / sqrt(l);
    }
  }
  if (sigma && blockIdx.x == 0)
    for (int a = threadIdx.x; a < m; a += blockDim.x) sigma[a] = lam[a] > 0.0 ? sqrt(lam[a]) : 0.0;
  __syncthreads();
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
       l += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < d; ++k) {
      double s = 0.0;
      for (int a = 0; a < m; ++a) s = fma(Y[(int64_t)a * ldy + l], cs[a * d + k], s);
      Psi[(int64_t)k * N + l] = s;
    }
  }
}

// Solve A c = b for the k x k system A_ij = Psi_j[idx_i], b_i = Psi_k[idx_i]
// (Gauss-Jordan with partial pivoting, one block, k <= 128): c -> cvec.
__global__ void k_deim_small(int64_t N, int k, const double* __restrict__ Psi,
                             const int32_t* __restrict__ idx, double* __restrict__ cvec,
                             int* status) {
  extern __shared__ double ab[];  // k x (k + 1)
  __shared__ int piv, ok;
  const int w = k + 1;
  for (int e = threadIdx.x; e < k * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    ab[e] = Psi[(int64_t)j * N + idx[i]];  // column j < k of the basis, j = k the right side
  }
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int c = 0; c < k; ++c) {
    if (threadIdx.x == 0) {
      int b = c;
      double best = fabs(ab[c * w + c]);
      for (int r = c + 1; r < k; ++r)
        if (fabs(ab[r * w + c]) > best) {
          best = fabs(ab[r * w + c]);
          b = r;
        }
      piv = b;
      if (!(best > 0.0) || !isfinite(best)) ok = 0;
    }
    __syncthreads();
    if (!ok) break;
    if (piv != c)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double t = ab[c * w + j];
        ab[c * w + j] = ab[piv * w + j];
        ab[piv * w + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / ab[c * w + c];
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) ab[c * w + j] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < k * w; e += blockDim.x) {
      const int r = e / w, j = e - r * w;
      if (r != c && j != c) ab[e] -= ab[r * w + c] * ab[c * w + j];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < k; r += blockDim.x)
      if (r != c) ab[r * w + c] = 0.0;
    __syncthreads();
  }
  if (!ok) {
    if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
    for (int i = threadIdx.x; i < k; i += blockDim.x) cvec[i] = 0.0;
    return;
  }
  for (int i = threadIdx.x; i < k; i += blockDim.x) cvec[i] = ab[i * w + k];
}

// |psi_k - sum_{j<k} c_j psi_j| per row; block partial arg-max (lowest row on ties)
__global__ void k_deim_resid(int64_t N, int k, const double* __restrict__ Psi,
                             const double* __restrict__ cvec, double* __restrict__ pval,
                             int64_t* __restrict__ pidx) {
  __shared__ double cs[128];
  __shared__ double bv[32];
  __shared__ int64_t bi[32];
  for (int j = threadIdx.x; j < k; j += blockDim.x) cs[j] = cvec[j];
  __syncthreads();
  double best = -1.0;
  int64_t bidx = INT64_MAX;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
       l += (int64_t)gridDim.x * blockDim.x) {
    double r = Psi[(int64_t)k * N + l];
    for (int j = 0; j < k; ++j) r = fma(-cs[j], Psi[(int64_t)j * N + l], r);
    const double a = fabs(r);
    if (a > best || (a == best && l < bidx)) {
      best = a;
      bidx = l;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (ob > best || (ob == best && oi < bidx)) {
      best = ob;
      bidx = oi;
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    bv[wid] = best;
    bi[wid] = bidx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > best || (bv[w] == best && bi[w] < bidx)) {
        best = bv[w];
        bidx = bi[w];
      }
    // warp 0's own result is already in best/bidx only for lane 0; fold it in
    if (bv[0] > best || (bv[0] == best && bi[0] < bidx)) {
      best = bv[0];
      bidx = bi[0];
    }
    pval[blockIdx.x] = best;
    pidx[blockIdx.x] = bidx;
  }
}

__global__ void k_deim_pick(int nb, const double* __restrict__ pval,
                            const int64_t* __restrict__ pidx, int32_t* __restrict__ idx, int k) {
  if (threadIdx.x != 0) return;
  double best = -1.0;
  int64_t b = INT64_MAX;
  for (int i = 0; i < nb; ++i)
    if (pval[i] > best || (pval[i] == best && pidx[i] < b)) {
      best = pval[i];
      b = pidx[i];
    }
  idx[k] = (int32_t)b;
}

// block partial column sums of Psi (d x N): part[blockIdx.x][k]
__global__ void k_colsum(int64_t N, int d, const double* __restrict__ Psi, double* __restrict__ part) {
  __shared__ double red[32];
  for (int k = 0; k < d; ++k) {
    double s = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
         l += (int64_t)gridDim.x * blockDim.x)
      s += Psi[(int64_t)k * N + l];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      part[(int64_t)blockIdx.x * d + k] = t;
    }
    __syncthreads();
  }
}

// c = (P^T Psi)^-T (Mq * colsum): solve A^T c = b with A_ij = Psi_j[idx_i]
__global__ void k_deim_weights(int64_t N, int d, const double* __restrict__ Psi,
                               const int32_t* __restrict__ idx, const double* __restrict__ colsum,
                               double Mq, double* __restrict__ c, int* status) {
  extern __shared__ double ab[];  // d x (d + 1): rows of A^T
  __shared__ int piv, ok;
  const int w = d + 1;
  for (int e = threadIdx.x; e < d * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;  // (A^T)_ij = A_ji = Psi_i[idx_j]
    ab[e] = j < d ? Psi[(int64_t)i * N + idx[j]] : Mq * colsum[i];
  }
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int cc = 0; cc < d; ++cc) {
    if (threadIdx.x == 0) {
      int b = cc;
      double best = fabs(ab[cc * w + cc]);
      for (int r = cc + 1; r < d; ++r)
        if (fabs(ab[r * w + cc]) > best) {
          best = fabs(ab[r * w + cc]);
          b = r;
        }
      piv = b;
      if (!(best > 0.0) || !isfinite(best)) ok = 0;
    }
    __syncthreads();
    if (!ok) break;
    if (piv != cc)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double t = ab[cc * w + j];
        ab[cc * w + j] = ab[piv * w + j];
        ab[piv * w + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / ab[cc * w + cc];
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) ab[cc * w + j] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < d * w; e += blockDim.x) {
      const int r = e / w, j = e - r * w;
      if (r != cc && j != cc) ab[e] -= ab[r * w + cc] * ab[cc * w + j];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < d; r += blockDim.x)
      if (r != cc) ab[r * w + cc] = 0.0;
    __syncthreads();
  }
  if (!ok) {
    if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
    return;
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) c[i] = ab[i * w + d];
}

// ------------------------------------------------------------------- DMD
// out (r columns of length n) = sum_a Y_a C[a][k] (Y: m columns of length n)
__global__ void k_cols_times(int n, int m, int r, const double* __restrict__ Y,
                             const double* __restrict__ C, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * r; e += gridDim.x * blockDim.x) {
    const int k = e / n, x = e - k * n;
    double s = 0.0;
    for (int a = 0; a < m; ++a) s = fma(Y[(int64_t)a * n + x], C[a * r + k], s);
    out[e] = s;
  }
}

// G[k1][k2] = <U_k1, B_k2> over length n (columns)
__global__ void k_cols_dot(int n, int r1, int r2, const double* __restrict__ U,
                           const double* __restrict__ B, double* __restrict__ G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r1 * r2; e += gridDim.x * blockDim.x) {
    const int k1 = e / r2, k2 = e - k1 * r2;
    double s = 0.0;
    for (int x = 0; x < n; ++x) s = fma(U[(int64_t)k1 * n + x], B[(int64_t)k2 * n + x], s);
    G[e] = s;
  }
}

// C[a][k] = W[a][k] / sigma_k (m x r) from the Jacobi eigenvectors (real parts)
__global__ void k_dmd_coeff(int m, int r, const double2* __restrict__ W, const double* __restrict__ lam,
                            double* __restrict__ C, int* status) {
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int a = e / r, k = e - a * r;
    const double l = lam[k];
    if (!(l > 0.0)) {
      vp_set_status(status, VP_ENUMERIC);
      C[e] = 0.0;
    } else {
      C[e] = W[a * m + k].x / sqrt(l);
    }
  }
}

// In-place inverse of an r x r matrix in shared memory (Gauss-Jordan with
// partial pivoting on [M | I]); aug is r x 2r.  Returns false if singular.
__device__ bool small_inverse(double* aug, int r) {
  __shared__ int piv, ok;
  const int w = 2 * r;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int c = 0; c < r; ++c) {
    if (threadIdx.x == 0) {
      int b = c;
      double best = fabs(aug[c * w + c]);
      for (int i = c + 1; i < r; ++i)
        if (fabs(aug[i * w + c]) > best) {
          best = fabs(aug[i * w + c]);
          b = i;
        }
      piv = b;
      if (!(best > 0.0) || !isfinite(best)) ok = 0;
    }
    __syncthreads();
    if (!ok) return false;
    if (piv != c)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double t = aug[c * w + j];
        aug[c * w + j] = aug[piv * w + j];
        aug[piv * w + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / aug[c * w + c];
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) aug[c * w + j] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < r * w; e += blockDim.x) {
      const int i = e / w, j = e - i * w;
      if (i != c && j != c) aug[e] -= aug[i * w + c] * aug[c * w + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < r; i += blockDim.x)
      if (i != c) aug[i * w + c] = 0.0;
    __syncthreads();
  }
  return true;
}

// Inv = G^-1 (r x r, one block)
__global__ void k_inverse(int r, const double* __restrict__ G, double* __restrict__ Inv, int* status) {
  extern __shared__ double aug[];
  const int w = 2 * r;
  for (int e = threadIdx.x; e < r * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    aug[e] = j < r ? G[i * r + j] : (j - r == i ? 1.0 : 0.0);
  }
  __syncthreads();
  if (!small_inverse(aug, r)) {
    if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
    return;
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) Inv[e] = aug[(e / r) * w + r + e % r];
}

// Principal square root S of A (r x r) by the Denman-Beavers iteration
// Y <- (Y + Z^-1) / 2, Z <- (Z + Y^-1) / 2 from Y = A, Z = I (Y -> A^1/2); at
// most 60 iterations, stop when |dY|_F <= 1e-15 |Y|_F.  Needs no eigenvalue of
// A on the closed negative real axis; otherwise VP_ENUMERIC.
__global__ void k_sqrtm(int r, const double* __restrict__ A, double* __restrict__ S, int* status) {
  extern __shared__ double sm[];
  const int rr = r * r, w = 2 * r;
  double* Yk = sm;
  double* Zk = Yk + rr;
  double* aug = Zk + rr;  // r x 2r
  double* Yi = aug + r * w;
  __shared__ double red[2];
  __shared__ int done;
  for (int e = threadIdx.x; e < rr; e += blockDim.x) {
    Yk[e] = A[e];
    Zk[e] = (e / r == e % r) ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0) done = 0;
  __syncthreads();
  int it = 0;
  for (; it < 60 && !done; ++it) {
    // Yi = Y^-1
    for (int e = threadIdx.x; e < r * w; e += blockDim.x) {
      const int i = e / w, j = e - i * w;
      aug[e] = j < r ? Yk[i * r + j] : (j - r == i ? 1.0 : 0.0);
    }
    __syncthreads();
    if (!small_inverse(aug, r)) break;
    for (int e = threadIdx.x; e < rr; e += blockDim.x) Yi[e] = aug[(e / r) * w + r + e % r];
    __syncthreads();
    // aug <- Z^-1
    for (int e = threadIdx.x; e < r * w; e += blockDim.x) {
      const int i = e / w, j = e - i * w;
      aug[e] = j < r ? Zk[i * r + j] : (j - r == i ? 1.0 : 0.0);
    }
    __syncthreads();
    if (!small_inverse(aug, r)) break;
    if (threadIdx.x == 0) {
      red[0] = 0.0;
      red[1] = 0.0;
    }
    __syncthreads();
    double dn = 0.0, yn = 0.0;
    for (int e = threadIdx.x; e < rr; e += blockDim.x) {
      const double yn_e = 0.5 * (Yk[e] + aug[(e / r) * w + r + e % r]);
      const double zn_e = 0.5 * (Zk[e] + Yi[e]);
      dn += (yn_e - Yk[e]) * (yn_e - Yk[e]);
      yn += yn_e * yn_e;
      Yk[e] = yn_e;
      Zk[e] = zn_e;
    }
    atomicAdd(&red[0], dn);
    atomicAdd(&red[1], yn);
    __syncthreads();
    if (threadIdx.x == 0 && red[0] <= 1e-30 * red[1]) done = 1;
    __syncthreads();
  }
  __syncthreads();
  if (!done) {
    if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
    return;
  }
  for (int e = threadIdx.x; e < rr; e += blockDim.x) S[e] = Yk[e];
}

// out (q x cols) = A (q x K) B (K x cols), row-major
__global__ void k_mm(int q, int K, int cols, const double* __restrict__ A,
                     const double* __restrict__ B, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < q * cols; e += gridDim.x * blockDim.x) {
    const int i = e / cols, j = e - i * cols;
    double s = 0.0;
    for (int k = 0; k < K; ++k) s = fma(A[i * K + k], B[(int64_t)k * cols + j], s);
    out[e] = s;
  }
}

// Gaussian RBF through (eta_s, values) evaluated at eta, one block:
// out (p x K) = E (K_ss^-1 values), K_ss = exp(-(eps |eta_i - eta_j|)^2).
__global__ void k_rbf(int dim, int q, const double* __restrict__ eta_s, int K,
                      const double* __restrict__ values, int p, const double* __restrict__ eta,
                      double eps, double* __restrict__ out, int* status) {
  extern __shared__ double aug[];  // q x (q + K)
  __shared__ int piv, ok;
  const int w = q + K;
  for (int e = threadIdx.x; e < q * w; e += blockDim.x) {
    const int i = e / w, j = e - i * w;
    if (j < q) {
      double d2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double d = eta_s[i * dim + a] - eta_s[j * dim + a];
        d2 = fma(d, d, d2);
      }
      aug[e] = exp(-eps * eps * d2);
    } else {
      aug[e] = values[i * K + (j - q)];
    }
  }
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int c = 0; c < q; ++c) {  // Gauss-Jordan with partial pivoting
    if (threadIdx.x == 0) {
      int b = c;
      double best = fabs(aug[c * w + c]);
      for (int i = c + 1; i < q; ++i)
        if (fabs(aug[i * w + c]) > best) {
          best = fabs(aug[i * w + c]);
          b = i;
        }
      piv = b;
      if (!(best > 0.0) || !isfinite(best)) ok = 0;
    }
    __syncthreads();
    if (!ok) break;
    if (piv != c)
      for (int j = threadIdx.x; j < w; j += blockDim.x) {
        const double t = aug[c * w + j];
        aug[c * w + j] = aug[piv * w + j];
        aug[piv * w + j] = t;
      }
    __syncthreads();
    const double inv = 1.0 / aug[c * w + c];
    __syncthreads();
    for (int j = threadIdx.x; j < w; j += blockDim.x) aug[c * w + j] *= inv;
    __syncthreads();
    for (int e = threadIdx.x; e < q * w; e += blockDim.x) {
      const int i = e / w, j = e - i * w;
      if (i != c && j != c) aug[e] -= aug[i * w + c] * aug[c * w + j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < q; i += blockDim.x)
      if (i != c) aug[i * w + c] = 0.0;
    __syncthreads();
  }
  if (!ok) {
    if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
    return;
  }
  for (int e = threadIdx.x; e < p * K; e += blockDim.x) {
    const int i = e / K, k = e - i * K;
    double s = 0.0;
    for (int j = 0; j < q; ++j) {
      double d2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double d = eta[i * dim + a] - eta_s[j * dim + a];
        d2 = fma(d, d, d2);
      }
      s = fma(exp(-eps * eps * d2), aug[j * w + q + k], s);
    }
    out[e] = s;
  }
}

// Phi_i = B (A^k S^h beta_i): one block per sample
__global__ void k_dmd_eval(int nx, int r, const double* __restrict__ B, const double* __restrict__ A,
                           const double* __restrict__ S, const double* __restrict__ beta, int ksteps,
                           int half, double* __restrict__ Phi) {
  extern __shared__ double g[];  // 2 r
  const int i = blockIdx.x;
  double* ga = g;
  double* gb = g + r;
  for (int k = threadIdx.x; k < r; k += blockDim.x) ga[k] = beta[i * r + k];
  __syncthreads();
  auto apply = [&](const double* M) {
    for (int k = threadIdx.x; k < r; k += blockDim.x) {
      double s = 0.0;
      for (int j = 0; j < r; ++j) s = fma(M[k * r + j], ga[j], s);
      gb[k] = s;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < r; k += blockDim.x) ga[k] = gb[k];
    __syncthreads();
  };
  if (half) apply(S);
  for (int st = 0; st < ksteps; ++st) apply(A);
  for (int x = threadIdx.x; x < nx; x += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < r; ++k) s = fma(B[(int64_t)k * nx + x], ga[k], s);
    Phi[(int64_t)i * nx + x] = s;
  }
}

}  // namespace

namespace vpk {
void deim_init() {
  const int lim = 200 * 1024;
  cudaFuncSetAttribute(k_ygram, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_psi, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_deim_small, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_deim_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_rbf, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_sqrtm, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}
}  // namespace vpk

extern "C" {

vp_status vp_potential_at_particles(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p,
                                    const double* X, int64_t ldx, const double* phi, double* Y,
                                    int64_t ldy, void* stream) {
  if (!ctx || !grid || !X || !phi || !Y || N < 1 || p < 1 || p > 65535 || ldx < N || ldy < N ||
      grid->Nx < 3 || grid->Nx > VP_MAX_NX || !(grid->L > 0.0))
    return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  GridC g = make_gridc(*grid, N);
  int bx = ceil_div(N, 256);
  const int want = (4 * ctx->num_sms + p - 1) / p;
  if (bx > want) bx = want;
  VP_K(VP_K_SUBSET, (k_phi_at<<<dim3(bx, p), 256, 0, st>>>(g, N, p, X, ldx, phi, Y, ldy)));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_deim_basis(vp_ctx* ctx, int64_t N, int32_t m, const double* Y, int64_t ldy, int32_t d,
                        double* Psi, double* sigma, void* stream) {
  if (!ctx || !Y || !Psi || N < 1 || m < 1 || m > 256 || d < 1 || d > m || d > 128 || ldy < N ||
      (int64_t)m * d > 25600)
    return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int tot = m * m;
  int gx = std::min<int64_t>(ceil_div(N, YG_ROWS), 2 * ctx->num_sms);
  const int gy = ceil_div(tot, 256 * 8);
  size_t bytes = arena_bytes((size_t)gx * tot, 8) + arena_bytes(tot, 8) + 3 * arena_bytes(tot, 16) +
                 arena_bytes(m, 8);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, bytes, &base));
  Arena a{(char*)base, 0, bytes};
  double* part = a.take<double>((size_t)gx * tot);
  double* G = a.take<double>(tot);
  double2* Gc = a.take<double2>(tot);
  double2* Wj = a.take<double2>(tot);
  double2* Ws = a.take<double2>(tot);
  double* lam = a.take<double>(m);
  VP_K(VP_K_SUBSET, (k_ygram<<<dim3(gx, gy), 256, sizeof(double) * m * YG_ROWS, st>>>(N, m, Y, ldy,
                                                                                      part)));
  VP_K(VP_K_REDUCE, reduce_partials(gx, tot, part, G, nullptr, st));
  VP_K(VP_K_SUBSET, (k_to_complex<<<ceil_div(tot, 256), 256, 0, st>>>(tot, G, Gc)));
  VP_K(VP_K_INIT, init_launch_jacobi(m, Gc, Wj, lam, Ws, ctx->d_status, st));
  int bx = std::min<int64_t>(ceil_div(N, 256), 4 * ctx->num_sms);
  VP_K(VP_K_SUBSET, (k_psi<<<bx, 256, sizeof(double) * m * d, st>>>(N, m, d, Y, ldy, Ws, lam, Psi,
                                                                    sigma, ctx->d_status)));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_deim_indices(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi, int32_t* idx,
                          void* stream) {
  if (!ctx || !Psi || !idx || N < 1 || d < 1 || d > 128 || d > N) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nb = std::min<int64_t>(ceil_div(N, 256), 2 * ctx->num_sms);
  size_t bytes = arena_bytes(nb, 8) + arena_bytes(nb, 8) + arena_bytes(128, 8);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, bytes, &base));
  Arena a{(char*)base, 0, bytes};
  double* pval = a.take<double>(nb);
  int64_t* pidx = a.take<int64_t>(nb);
  double* cvec = a.take<double>(128);
  for (int k = 0; k < d; ++k) {
    if (k > 0)
      VP_K(VP_K_SUBSET, (k_deim_small<<<1, 256, sizeof(double) * k * (k + 1), st>>>(
                            N, k, Psi, idx, cvec, ctx->d_status)));
    VP_K(VP_K_SUBSET, (k_deim_resid<<<nb, 256, 0, st>>>(N, k, Psi, cvec, pval, pidx)));
    VP_K(VP_K_SUBSET, (k_deim_pick<<<1, 32, 0, st>>>(nb, pval, pidx, idx, k)));
  }
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_deim_weights(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi, const int32_t* idx,
                          double Mq, double* c, void* stream) {
  if (!ctx || !Psi || !idx || !c || N < 1 || d < 1 || d > 128) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int nb = std::min<int64_t>(ceil_div(N, 256), 2 * ctx->num_sms);
  size_t bytes = arena_bytes((size_t)nb * d, 8) + arena_bytes(d, 8);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, bytes, &base));
  Arena a{(char*)base, 0, bytes};
  double* part = a.take<double>((size_t)nb * d);
  double* colsum = a.take<double>(d);
  VP_K(VP_K_SUBSET, (k_colsum<<<nb, 256, 0, st>>>(N, d, Psi, part)));
  VP_K(VP_K_REDUCE, reduce_partials(nb, d, part, colsum, nullptr, st));
  VP_K(VP_K_SUBSET, (k_deim_weights<<<1, 256, sizeof(double) * d * (d + 1), st>>>(
                        N, d, Psi, idx, colsum, Mq, c, ctx->d_status)));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_dmd_fit(vp_ctx* ctx, int32_t nx, int32_t m, const double* Y, const double* Yp,
                     double tol, int32_t r_max, int32_t* r_out, double* B, double* Bpinv,
                     double* A, double* S, double* sigma, void* stream) {
  if (!ctx || !Y || !Yp || !r_out || !B || !Bpinv || !A || !S || nx < 1 || nx > 4096 || m < 1 ||
      m > 256 || r_max < 1 || r_max > 64 || !(tol >= 0.0))
    return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int tot = m * m;
  const int gx = std::max(1, std::min(ceil_div(nx, YG_ROWS), 64));
  const int gy = ceil_div(tot, 256 * 8);
  size_t bytes = arena_bytes((size_t)gx * tot, 8) + arena_bytes(tot, 8) + 3 * arena_bytes(tot, 16) +
                 arena_bytes(m, 8) + arena_bytes((size_t)m * r_max, 8) +
                 arena_bytes((size_t)r_max * nx, 8) + 2 * arena_bytes((size_t)r_max * r_max, 8);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, bytes, &base));
  Arena a{(char*)base, 0, bytes};
  double* part = a.take<double>((size_t)gx * tot);
  double* G = a.take<double>(tot);
  double2* Gc = a.take<double2>(tot);
  double2* Wj = a.take<double2>(tot);
  double2* Ws = a.take<double2>(tot);
  double* lam = a.take<double>(m);
  double* C = a.take<double>((size_t)m * r_max);
  double* U = a.take<double>((size_t)r_max * nx);
  double* BtB = a.take<double>((size_t)r_max * r_max);
  double* BtBi = a.take<double>((size_t)r_max * r_max);
  // 1. Y^T Y and its eigen-decomposition (singular values and right vectors of Y)
  VP_K(VP_K_SUBSET, (k_ygram<<<dim3(gx, gy), 256, sizeof(double) * m * YG_ROWS, st>>>(nx, m, Y, nx,
                                                                                       part)));
  VP_K(VP_K_REDUCE, reduce_partials(gx, tot, part, G, nullptr, st));
  VP_K(VP_K_SUBSET, (k_to_complex<<<ceil_div(tot, 256), 256, 0, st>>>(tot, G, Gc)));
  VP_K(VP_K_INIT, init_launch_jacobi(m, Gc, Wj, lam, Ws, ctx->d_status, st));
  std::vector<double> lh(m);
  VP_CUDA(cudaMemcpyAsync(lh.data(), lam, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
  VP_CUDA(cudaStreamSynchronize(st));
  // 2. rank: singular values above tol sigma_1, and above 1e-7 sigma_1 (the
  // Gram matrix resolves singular values down to ~1e-8 sigma_1 only)
  const double s1 = lh[0] > 0.0 ? std::sqrt(lh[0]) : 0.0;
  const double tol_eff = std::max(tol, 1e-7);
  int r = 0;
  for (int k = 0; k < m && r < r_max; ++k)
    if (lh[k] > 0.0 && std::sqrt(lh[k]) > tol_eff * s1) ++r;
  if (r < 1) return vp_fail(ctx, VP_ENUMERIC, "DMD data matrix is zero");
  *r_out = r;
  if (sigma) VP_K(VP_K_INIT, sqrt_nonneg(m, lam, sigma, st));
  // 3. C = V_r S_r^-1; U_r = Y C, B = Y' C; A = U_r^T B; B^+ = (B^T B)^-1 B^T
  VP_K(VP_K_SUBSET, (k_dmd_coeff<<<1, 256, 0, st>>>(m, r, Ws, lam, C, ctx->d_status)));
  const int gcols = std::max(1, std::min(ceil_div((int64_t)nx * r, 256), 4 * ctx->num_sms));
  VP_K(VP_K_SUBSET, (k_cols_times<<<gcols, 256, 0, st>>>(nx, m, r, Y, C, U)));
  VP_K(VP_K_SUBSET, (k_cols_times<<<gcols, 256, 0, st>>>(nx, m, r, Yp, C, B)));
  VP_K(VP_K_SUBSET, (k_cols_dot<<<ceil_div(r * r, 256), 256, 0, st>>>(nx, r, r, U, B, A)));
  VP_K(VP_K_SUBSET, (k_cols_dot<<<ceil_div(r * r, 256), 256, 0, st>>>(nx, r, r, B, B, BtB)));
  VP_K(VP_K_SUBSET, (k_inverse<<<1, 256, sizeof(double) * 2 * r * r, st>>>(r, BtB, BtBi,
                                                                           ctx->d_status)));
  // B^+ (r x nx) = BtBi (r x r) * B^T; B is stored as r columns of length nx,
  // i.e. the row-major r x nx matrix B^T
  VP_K(VP_K_SUBSET, (k_mm<<<gcols, 256, 0, st>>>(r, r, nx, BtBi, B, Bpinv)));
  // 4. principal square root of A for half steps
  VP_K(VP_K_SUBSET, (k_sqrtm<<<1, 256, sizeof(double) * (4 * r * r + 2 * r * r), st>>>(
                        r, A, S, ctx->d_status)));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_dmd_coords(vp_ctx* ctx, int32_t nx, int32_t r, const double* Bpinv, int32_t q,
                        const double* Phi, double* beta, void* stream) {
  if (!ctx || !Bpinv || !Phi || !beta || nx < 1 || r < 1 || r > 64 || q < 1) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // beta (q x r) = Phi (q x nx) Bpinv^T: entry (i, k) = sum_x Phi[i][x] Bpinv[k][x]
  VP_K(VP_K_SUBSET, (k_cols_dot<<<ceil_div(q * r, 256), 256, 0, st>>>(nx, q, r, Phi, Bpinv, beta)));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_rbf_interpolate(vp_ctx* ctx, int32_t dim, int32_t q, const double* eta_s, int32_t K,
                             const double* values, int32_t p, const double* eta, double eps,
                             double* out, void* stream) {
  if (!ctx || !eta_s || !values || !eta || !out || dim < 1 || q < 1 || K < 1 || p < 1 ||
      (int64_t)q * (q + K) * 8 > 200 * 1024 || !(eps > 0.0))
    return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  VP_K(VP_K_SUBSET, (k_rbf<<<1, 256, sizeof(double) * q * (q + K), st>>>(
                        dim, q, eta_s, K, values, p, eta, eps, out, ctx->d_status)));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_dmd_potential(vp_ctx* ctx, int32_t nx, int32_t r, const double* B, const double* A,
                           const double* S, int32_t p, const double* beta, int32_t ksteps,
                           int32_t half, double* Phi, void* stream) {
  if (!ctx || !B || !A || !S || !beta || !Phi || nx < 1 || r < 1 || r > 64 || p < 1 ||
      ksteps < 0 || half < 0 || half > 1)
    return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  VP_K(VP_K_SUBSET, (k_dmd_eval<<<p, 128, sizeof(double) * 2 * r, st>>>(nx, r, B, A, S, beta, ksteps,
                                                                        half, Phi)));
  VP_LAUNCHED();
  return VP_OK;
}

}  // extern "C"
