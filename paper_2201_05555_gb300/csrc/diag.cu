// Accuracy diagnostics of the reduced model (Sec. 6.1, eqs. relative_errors,
// relative_errors_complex_SVD; Sec. 6.2, eq. error_ham_tot) and the
// adaptive-rank indicator |(I - U U^T) G|_F / |G|_F.  FP64; block partial
// sums are reduced in a fixed order, so results repeat bit for bit.
#include "vp_internal.cuh"

namespace {
using namespace vpk;

#define DG_ROWS 32

__device__ __forceinline__ void block_sum_n(double* acc, int k, double* red) {
  // sums acc[0..k) over the block into red[0..k) (thread 0 holds the result)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q = 0; q < k; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[q * 32 + wid] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int q = 0; q < k; ++q) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[q * 32 + w];
      red[q * 32] = t;
    }
  __syncthreads();
}

// Positions and velocities of a tile of particles under sample i from the
// rows [A | B] of Q (U_X = [A, -B], U_V = [B, A]) and the coefficients
// c = [a; b] (2n x p, column i).
__device__ __forceinline__ void xv_of(const double* qr, int n, const double* __restrict__ c, int p,
                                      int i, double& x, double& v) {
  double sx = 0.0, sv = 0.0;
  for (int m = 0; m < n; ++m) {
    const double a = __ldg(c + (int64_t)m * p + i), b = __ldg(c + (int64_t)(n + m) * p + i);
    sx = fma(qr[m], a, fma(-qr[n + m], b, sx));
    sv = fma(qr[n + m], a, fma(qr[m], b, sv));
  }
  x = sx;
  v = sv;
}

// part[block][0..4) = sums of (X - X_r)^2, X^2, (V - V_r)^2, V^2 over the
// block's particle-samples; X, V full-order (p x N, sample by sample)
__global__ void k_rel_err(int64_t N, int n, int p, const double* __restrict__ Q,
                          const double* __restrict__ Z, const double* __restrict__ X,
                          const double* __restrict__ V, double* __restrict__ part) {
  extern __shared__ double qt[];  // DG_ROWS x 2n
  __shared__ double red[4 * 32];
  const int n2 = 2 * n;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t tile = blockIdx.x; tile * DG_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * DG_ROWS;
    const int rows = (int)min((int64_t)DG_ROWS, N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) qt[e] = Q[base * n2 + e];
    __syncthreads();
    for (int e = threadIdx.x; e < p * DG_ROWS; e += blockDim.x) {
      const int i = e / DG_ROWS, r = e - i * DG_ROWS;
      if (r >= rows) continue;
      double x, v;
      xv_of(qt + r * n2, n, Z, p, i, x, v);
      const double xf = X[(int64_t)i * N + base + r], vf = V[(int64_t)i * N + base + r];
      acc[0] = fma(xf - x, xf - x, acc[0]);
      acc[1] = fma(xf, xf, acc[1]);
      acc[2] = fma(vf - v, vf - v, acc[2]);
      acc[3] = fma(vf, vf, acc[3]);
    }
  }
  block_sum_n(acc, 4, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) part[(int64_t)blockIdx.x * 4 + q] = red[q * 32];
}

// part[block][0..2) = sums of |G - U g|^2 and |G|^2 over the block's
// particle-samples, with G = [(q/m) F(cell of x); v] at R = U Z and g = U^T G
__global__ void k_normal_part(GridC gc, int64_t N, int n, int p, const double* __restrict__ Q,
                              const double* __restrict__ Z, const double* __restrict__ F,
                              const double* __restrict__ g, double* __restrict__ part) {
  extern __shared__ double qt[];
  __shared__ double red[2 * 32];
  const int n2 = 2 * n;
  double acc[2] = {0.0, 0.0};
  for (int64_t tile = blockIdx.x; tile * DG_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * DG_ROWS;
    const int rows = (int)min((int64_t)DG_ROWS, N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) qt[e] = Q[base * n2 + e];
    __syncthreads();
    for (int e = threadIdx.x; e < p * DG_ROWS; e += blockDim.x) {
      const int i = e / DG_ROWS, r = e - i * DG_ROWS;
      if (r >= rows) continue;
      double x, v, ux, uv;
      xv_of(qt + r * n2, n, Z, p, i, x, v);
      xv_of(qt + r * n2, n, g, p, i, ux, uv);
      int j;
      double s;
      cell_of(x, gc.inv_h, gc.Nx, gc.dNx, gc.inv_Nx, j, s);
      const double gx = gc.qm * __ldg(F + (int64_t)i * gc.Nx + j);
      acc[0] = fma(gx - ux, gx - ux, fma(v - uv, v - uv, acc[0]));
      acc[1] = fma(gx, gx, fma(v, v, acc[1]));
    }
  }
  block_sum_n(acc, 2, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 2; ++q) part[(int64_t)blockIdx.x * 2 + q] = red[q * 32];
}

// out[k] = sqrt(s[2k] / s[2k + 1]) for k < pairs
__global__ void k_ratio_sqrt(int pairs, const double* __restrict__ s, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k < pairs) out[k] = s[2 * k + 1] > 0.0 ? sqrt(s[2 * k] / s[2 * k + 1]) : 0.0;
}

// Delta H and its three bounding terms (2-norms over the p parameters)
__global__ void k_ham_terms(int p, const double* __restrict__ h00, const double* __restrict__ h11,
                            const double* __restrict__ hh0, const double* __restrict__ hh1,
                            double* __restrict__ out) {
  __shared__ double red[4 * 32];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double a = h11[i] - h00[i], b = h11[i] - hh1[i], c = hh0[i] - h00[i], d = hh1[i] - hh0[i];
    acc[0] = fma(a, a, acc[0]);
    acc[1] = fma(b, b, acc[1]);
    acc[2] = fma(c, c, acc[2]);
    acc[3] = fma(d, d, acc[3]);
  }
  block_sum_n(acc, 4, red);
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) out[q] = sqrt(red[q * 32]);
}
}  // namespace

namespace vpk {
int diag_blocks(int64_t N, int sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, DG_ROWS), 2 * sms));
}

void rel_err_parts(int64_t N, int n, int p, const double* Q, const double* Z, const double* X,
                   const double* V, double* part, int nb, cudaStream_t st) {
  k_rel_err<<<nb, 256, sizeof(double) * DG_ROWS * 2 * n, st>>>(N, n, p, Q, Z, X, V, part);
}

void normal_parts(const GridC& g, int64_t N, int n, int p, const double* Q, const double* Z,
                  const double* F, const double* gproj, double* part, int nb, cudaStream_t st) {
  k_normal_part<<<nb, 256, sizeof(double) * DG_ROWS * 2 * n, st>>>(g, N, n, p, Q, Z, F, gproj, part);
}

void ratio_sqrt(int pairs, const double* s, double* out, cudaStream_t st) {
  k_ratio_sqrt<<<1, 32, 0, st>>>(pairs, s, out);
}

void ham_terms(int p, const double* h00, const double* h11, const double* hh0, const double* hh1,
               double* out, cudaStream_t st) {
  k_ham_terms<<<1, 256, 0, st>>>(p, h00, h11, hh0, hh1, out);
}
}  // namespace vpk
