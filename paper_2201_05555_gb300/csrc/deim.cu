// Hyper-reduction on the device (Sec. 4.2).
// DEIM construction: snapshot columns Lambda^0(X_r) Phi (eq. Ydeim), the
// basis of the first d left singular vectors of the snapshot matrix, the
// greedy interpolation indices and the weights c = (P^T Psi)^-T Psi^T M_q of
// the DEIM-indexed gradient.
// DMD of the potential (Algorithm 1): with the truncated SVD Y = U S V^T of
// the window data, B = Y' V S^-1 and A = U^T B, the exact-DMD prediction
// Theta (Pi (.) lambda^(s/dt)) with Theta = B W, A W = W Lambda, equals
// B A^(s/dt) B^+ Phi (Theta^+ = W^-1 B^+), so whole steps need only real
// powers of A and half steps the real part of its principal square root
// (from the complex Schur form of the small r x r matrix A).
//
// Layouts: snapshot matrix Y stored column by column (m x N, leading
// dimension ldy >= N); basis Psi column by column (d x N).  FP64 throughout.
// The singular vectors come from the Gram matrix Y^T Y (cyclic Jacobi of
// init.cu), so directions of singular values below ~1e-8 sigma_1 are not
// resolved; the interpolation indices need only the leading ones.
#include "vp_internal.cuh"
#include "dfloat.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

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

// part[blockIdx.x][e] = sum over this block's rows of Y_a Y_b for the packed
// lower triangle e = a (a + 1) / 2 + b, b <= a (m (m + 1) / 2 entries, m <= 256)
#define YG_ROWS 32
__device__ __forceinline__ void tri_ab(int e, int& a, int& b) {
  int aa = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (aa * (aa + 1) / 2 > e) --aa;
  while ((aa + 1) * (aa + 2) / 2 <= e) ++aa;
  a = aa;
  b = e - aa * (aa + 1) / 2;
}
__global__ void k_ygram(int64_t N, int m, const double* __restrict__ Y, int64_t ldy,
                        double* __restrict__ part) {
  extern __shared__ double ys[];  // m x YG_ROWS
  const int tot = m * (m + 1) / 2;
  double acc[8];
  int ea[8], eb[8];
  const int e0 = blockIdx.y * blockDim.x * 8;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    acc[q] = 0.0;
    const int e = e0 + q * blockDim.x + threadIdx.x;
    ea[q] = -1;
    eb[q] = 0;
    if (e < tot) tri_ab(e, ea[q], eb[q]);
  }
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
      if (ea[q] >= 0) {
        const double* ya = ys + ea[q] * YG_ROWS;
        const double* yb = ys + eb[q] * YG_ROWS;
        double s = acc[q];
        for (int r = 0; r < YG_ROWS; ++r) s = fma(ya[r], yb[r], s);
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

// Round-robin sweeps of the cyclic Jacobi method on a symmetric m x m matrix A
// (shared memory, row-major) with the rotations accumulated into W (A <- J^T A J,
// W <- W J).  The m/2 disjoint pairs of a round rotate together; a pair
// (j, k) rotates unless |a_jk| <= rel sqrt|a_jj a_kk|, |a_jk| <= floor_rel
// max_i |a_ii|, or both diagonal entries are below null_rel max_i |a_ii| (a
// pair inside the rounding-level null space, whose rotations would go on
// forever and change no eigenpair above it).  Returns after a sweep without
// rotations (true) or after max_sweeps (false).  The rotation angle comes from
// an FP32 tangent (FP64 division and square roots are slow on this part),
// normalised in the working precision R so that the rotation stays orthogonal
// to R's rounding.  All threads of the block call it.
template <class R>
__device__ bool jacobi_sweeps(int m, int ld, R* A, R* W, int max_sweeps, R rel, R floor_rel, R null_rel,
                              R* rc, R* rs, int* pj, int* pk, int* nrot, R* nu_fl) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int slots = (m + 1) & ~1, npair = slots / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (t == 0) {
      *nrot = 0;
      R dm = 0;
      for (int j = 0; j < m; ++j) dm = fmax(dm, fabs(A[j * ld + j]));
      nu_fl[0] = null_rel * dm;
      nu_fl[1] = floor_rel * dm;
    }
    __syncthreads();
    const R nu = nu_fl[0], fl = nu_fl[1];
    for (int round = 0; round < slots - 1; ++round) {
      for (int q = t; q < npair; q += nt) {
        const int a = q, b = slots - 1 - q;
        const int ia = (a == 0) ? 0 : 1 + (a - 1 + round) % (slots - 1);
        const int ib = (b == 0) ? 0 : 1 + (b - 1 + round) % (slots - 1);
        const int j = min(ia, ib), k = max(ia, ib);
        pj[q] = j;
        pk[q] = k;
        R c = 1, sn = 0;
        if (k < m) {
          const R ajk = A[j * ld + k], ajj = A[j * ld + j], akk = A[k * ld + k];
          if (fabs(ajk) > rel * sqrt(fabs(ajj * akk)) && fabs(ajk) > fl &&
              (float)fabs(ajk) > 0.0f && fmax(fabs(ajj), fabs(akk)) > nu) {
            *nrot = 1;  // any rotation this sweep (the same value from every writer)
            const R dd = akk - ajj;
            R tt;
            if (fabs(dd) > (R)1e18 * fabs(ajk)) {  // tiny angle, beyond FP32 range: t = a_jk / dd
              tt = ajk / dd;
            } else {
              const float tau = (float)dd / (2.0f * (float)ajk);
              tt = (R)((tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f))));
            }
            c = rsqrt(fma(tt, tt, (R)1));
            sn = tt * c;
          }
        }
        rc[q] = c;
        rs[q] = sn;
      }
      __syncthreads();
      for (int e = t; e < npair * m; e += nt) {  // columns j, k of A and W
        const int q = e / m, r = e - q * m;
        const int j = pj[q], k = pk[q];
        if (k >= m || rs[q] == (R)0) continue;
        const R c = rc[q], sn = rs[q];
        const R aj = A[r * ld + j], ak = A[r * ld + k];
        A[r * ld + j] = c * aj - sn * ak;
        A[r * ld + k] = sn * aj + c * ak;
        const R wj = W[r * ld + j], wk = W[r * ld + k];
        W[r * ld + j] = c * wj - sn * wk;
        W[r * ld + k] = sn * wj + c * wk;
      }
      __syncthreads();
      for (int e = t; e < npair * m; e += nt) {  // rows j, k of A
        const int q = e / m, cidx = e - q * m;
        const int j = pj[q], k = pk[q];
        if (k >= m || rs[q] == (R)0) continue;
        const R c = rc[q], sn = rs[q];
        const R aj = A[j * ld + cidx], ak = A[k * ld + cidx];
        A[j * ld + cidx] = c * aj - sn * ak;
        A[k * ld + cidx] = sn * aj + c * ak;
      }
      __syncthreads();
    }
    const bool conv = *nrot == 0;
    __syncthreads();
    if (conv) return true;
  }
  return false;
}

// lambda (descending) and the columns of W in the same order (Wout, m x m
// row-major) from the diagonal of the converged A
__device__ void jacobi_output(int m, int ld, const double* A, const double* W, double* lambda,
                              double* Wout, int* order) {
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) {  // eigenvalues descending (selection order)
    for (int i = 0; i < m; ++i) order[i] = i;
    for (int i = 0; i < m; ++i) {
      int best = i;
      for (int j = i + 1; j < m; ++j)
        if (A[order[j] * ld + order[j]] > A[order[best] * ld + order[best]]) best = j;
      const int tmp = order[i];
      order[i] = order[best];
      order[best] = tmp;
    }
  }
  __syncthreads();
  for (int i = t; i < m; i += nt) lambda[i] = A[order[i] * ld + order[i]];
  for (int e = t; e < m * m; e += nt) {
    const int r = e / m, c = e - r * m;
    Wout[e] = W[r * ld + order[c]];
  }
}

// G (packed lower triangle) into the full m x m A and W = I
__device__ void jacobi_load(int m, int ld, const double* Gin, double* A, double* W) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    const int hi = max(i, j), lo = min(i, j);
    A[i * ld + j] = Gin[hi * (hi + 1) / 2 + lo];
    W[i * ld + j] = i == j ? 1.0 : 0.0;
  }
}

// Real symmetric cyclic Jacobi in FP64 (m <= 256; one block; G given as its
// packed lower triangle): G = W diag(lambda) W^T with lambda descending and
// the columns of W (Wout, m x m row-major) in the same order.  Pairs rotate
// unless |g_jk| <= 1e-15 sqrt|g_jj g_kk| or both diagonal entries are below
// 1e-14 of the largest one; stops after a sweep without rotations (at most
// max_sweeps, else VP_ENOCONV).  With m <= JS_SMEM_M, A and W live in shared
// memory.
#define JS_SMEM_M 111
__global__ void k_jacobi_sym(int m, const double* __restrict__ Gin, double* __restrict__ Ag,
                             double* __restrict__ Wg, double* __restrict__ lambda,
                             double* __restrict__ Wout, int max_sweeps, int* status) {
  extern __shared__ double js[];
  __shared__ double rc[128], rs[128], nu[2];
  __shared__ int pj[128], pk[128], nrot, order[256];
  const bool sm = m <= JS_SMEM_M;
  // rows padded to m + 1 in shared memory: the column updates of a round
  // walk down a column, which a stride of m would put in one bank
  const int ld = sm ? m + 1 : m;
  double* A = sm ? js : Ag;
  double* W = sm ? js + m * ld : Wg;
  jacobi_load(m, ld, Gin, A, W);
  __syncthreads();
  const bool conv = jacobi_sweeps<double>(m, ld, A, W, max_sweeps, 1e-15, 0.0, 1e-14, rc, rs, pj,
                                          pk, &nrot, nu);
  if (!conv && threadIdx.x == 0) vp_set_status(status, VP_ENOCONV);
  jacobi_output(m, ld, A, W, lambda, Wout, order);
}

// ------------------------------------------- double-float symmetric Jacobi
// c a - s b
__device__ __forceinline__ DFv dfv_rot(DFv c, DFv a, DFv s, DFv b) {
  return dfv_add(dfv_mul(c, a), dfv_neg(dfv_mul(s, b)));
}

// ------------------------ cyclic Jacobi with one block barrier per round
// The sweeps of the double-float kernel and of its FP64 finish (m <= 64).
// The same rotations as jacobi_sweeps (round-robin pairs, the same
// thresholds, the column update of a round before its row update), laid out
// so that a round needs one barrier instead of three:
// - A is double-buffered: a thread owns a 2 x 2 block (the rows of pair q1,
//   the columns of pair q2), reads it from the current copy, applies the
//   column rotation of q2 and then the row rotation of q1, and writes the
//   other copy; W's columns are rotated in place (each entry by one task);
// - the rotations of the next round are computed in the same phase by the
//   first warp, from the three entries of each next pair that this round
//   produces, evaluated by the same operations as the block update.
// At the start of a sweep the null-space threshold is taken from the
// diagonal and the first round's rotations from A itself (two more
// barriers).  Element operations of a rotation: c a - s b and s a + c b.
__device__ __forceinline__ double jrot(double c, double a, double s, double b) {
  return fma(c, a, -(s * b));
}
__device__ __forceinline__ double jrotp(double s, double a, double c, double b) {
  return fma(s, a, c * b);
}
__device__ __forceinline__ DFv jrot(DFv c, DFv a, DFv s, DFv b) { return dfv_rot(c, a, s, b); }
__device__ __forceinline__ DFv jrotp(DFv s, DFv a, DFv c, DFv b) {
  return dfv_rot(s, a, dfv_neg(c), b);
}
__device__ __forceinline__ bool jmoving(double s) { return s != 0.0; }
__device__ __forceinline__ bool jmoving(DFv s) { return s.h != 0.f; }
__device__ __forceinline__ void jident(double& c, double& sn) {
  c = 1.0;
  sn = 0.0;
}
__device__ __forceinline__ void jident(DFv& c, DFv& sn) {
  c = dfv(1.f, 0.f);
  sn = dfv(0.f, 0.f);
}
__device__ __forceinline__ double jlead(double a) { return a; }
__device__ __forceinline__ double jlead(DFv a) { return (double)a.h; }

// The rotation (c, s) of a pair from a_jj, a_kk, a_jk, or false (c = 1,
// s = 0) below the thresholds of jacobi_sweeps: |a_jk| <= rel sqrt|a_jj a_kk|,
// |a_jk| <= fl, or both diagonal entries at most nu.  FP64: an FP32 tangent,
// c = (1 + t^2)^-1/2 in FP64.
__device__ bool jparams(double ajj, double akk, double ajk, double rel, double fl, double nu,
                        double& c, double& sn) {
  c = 1.0;
  sn = 0.0;
  if (!(fabs(ajk) > rel * sqrt(fabs(ajj * akk)) && fabs(ajk) > fl && (float)fabs(ajk) > 0.0f &&
        fmax(fabs(ajj), fabs(akk)) > nu))
    return false;
  const double dd = akk - ajj;
  double tt;
  if (fabs(dd) > 1e18 * fabs(ajk)) {  // tiny angle, beyond FP32 range: t = a_jk / dd
    tt = ajk / dd;
  } else {
    const float tau = (float)dd / (2.0f * (float)ajk);
    tt = (double)((tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f))));
  }
  c = rsqrt(fma(tt, tt, 1.0));
  sn = tt * c;
  return true;
}
// Double-float: the thresholds on the leading parts (rel must stay well above
// the double-float rounding of ~4e-15 per operation, which the entries
// accumulate over the sweeps); the tangent in FP32 from the leading parts,
// c = (1 + t^2)^-1/2 by an FP32 reciprocal square root and one Newton step
// in double-float, s = t c, so that the rotation is orthogonal to
// double-float rounding.
__device__ bool jparams(DFv ajj, DFv akk, DFv ajk, double rel_d, double fl, double nu_d, DFv& c,
                        DFv& sn) {
  (void)fl;
  const float rel = (float)rel_d, nu = (float)nu_d;
  c = dfv(1.f, 0.f);
  sn = dfv(0.f, 0.f);
  const float x = fabsf(ajk.h);
  if (!(x > rel * sqrtf(fabsf(ajj.h) * fabsf(akk.h)) && x > 0.f &&
        fmaxf(fabsf(ajj.h), fabsf(akk.h)) > nu))
    return false;
  const DFv dd = dfv_add(akk, dfv_neg(ajj));
  float tt;
  if (fabsf(dd.h) > 1e18f * x) {  // tiny angle: t = a_jk / dd
    tt = ajk.h / dd.h;
  } else {
    const float tau = dd.h / (2.0f * ajk.h);
    tt = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(fmaf(tau, tau, 1.0f)));
  }
  // u = 1 + t^2 exactly as a double-float (t^2 by an FMA), y ~ u^-1/2
  const float t2 = tt * tt;
  const DFv u = fast_two_sum(1.0f, t2);
  const DFv uu = dfv_add(u, dfv(fmaf(tt, tt, -t2), 0.f));
  const float y0 = rsqrtf(uu.h);
  // y = y0 + y0 (1 - u y0^2) / 2
  const DFv y0sq = dfv_mul(dfv(y0, 0.f), dfv(y0, 0.f));
  const DFv r = dfv_add(dfv(1.f, 0.f), dfv_neg(dfv_mul(uu, y0sq)));
  c = dfv_add(dfv(y0, 0.f), dfv_mul(dfv(0.5f * y0, 0.f), r));
  sn = dfv_mul(dfv(tt, 0.f), c);
  return true;
}

// Pair q of round r of the round-robin schedule over `slots` (even) indices:
// slot 0 stays, the others turn; j < k (k == m is the padding of odd m).
__device__ __forceinline__ void rr_pair(int slots, int r, int q, int& j, int& k) {
  const int a = q, b = slots - 1 - q;
  const int ia = (a == 0) ? 0 : 1 + (a - 1 + r) % (slots - 1);
  const int ib = (b == 0) ? 0 : 1 + (b - 1 + r) % (slots - 1);
  j = min(ia, ib);
  k = max(ia, ib);
}
// The entry (x, y) of A after a round, by the operations of the block
// update: the column pass of y's pair (moving my, rotation cy, sy) on rows x
// and, if x's pair moves, its partner; then the row pass of x's pair.
template <class T>
__device__ __forceinline__ T jnew(const T* A, int ld, int x, int xp, bool xk, bool mx, T cx, T sx,
                                  int y, int yp, bool yk, bool my, T cy, T sy) {
  auto col = [&](int i) -> T {
    if (!my) return A[i * ld + y];
    const T aj = A[i * ld + (yk ? yp : y)], ak = A[i * ld + (yk ? y : yp)];
    return yk ? jrotp(sy, aj, cy, ak) : jrot(cy, aj, sy, ak);
  };
  const T tx = col(x);
  if (!mx) return tx;
  const T tp = col(xp);
  const T tj = xk ? tp : tx, tk = xk ? tx : tp;
  return xk ? jrotp(sx, tj, cx, tk) : jrot(cx, tj, sx, tk);
}

// The schedule of every round (the same in each sweep), in shared memory:
// pair q of round r is (pj, pk)[r * 32 + q]; index x of round r belongs to
// pair pq[r * 64 + x] >> 1, as its larger index when the low bit is set.
// Task tables: block e = (q1, q2) and W task e = (q, row), one byte each.
struct JacTabs {
  uint8_t pj[63 * 32], pk[63 * 32], pq[63 * 64];
  uint16_t blk[32 * 32], wt[64 * 32];
};
__device__ void jacobi_tabs(int m, JacTabs* tb) {
  const int slots = (m + 1) & ~1, npair = slots / 2, R = slots - 1;
  for (int e = threadIdx.x; e < R * npair; e += blockDim.x) {
    const int r = e / npair, q = e - r * npair;
    int j, k;
    rr_pair(slots, r, q, j, k);
    tb->pj[r * 32 + q] = (uint8_t)j;
    tb->pk[r * 32 + q] = (uint8_t)k;
    tb->pq[r * 64 + j] = (uint8_t)(2 * q);
    if (k < m) tb->pq[r * 64 + k] = (uint8_t)(2 * q + 1);
  }
  for (int e = threadIdx.x; e < npair * npair; e += blockDim.x)
    tb->blk[e] = (uint16_t)(((e / npair) << 8) | (e % npair));
  for (int e = threadIdx.x; e < m * npair; e += blockDim.x)
    tb->wt[e] = (uint16_t)(((e / m) << 8) | (e % m));
}

// Sweeps as jacobi_sweeps for m <= 64 with blockDim.x >= 64: A (rows ld
// apart) and its second copy A2, W, all in shared memory; tb from
// jacobi_tabs; rc, rs hold 2 x 32 rotations, flag 2 ints, thr 2 doubles
// (shared).  On return A points to the copy that holds the result.  Returns
// after a sweep without rotations (true) or after max_sweeps (false).
template <class T>
__device__ bool jacobi_sweeps_1b(int m, int ld, T*& A, T* A2, T* W, int max_sweeps, double rel,
                                 double floor_rel, double null_rel, const JacTabs* tb, T* rc, T* rs,
                                 int* flag, double* thr) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int slots = (m + 1) & ~1, npair = slots / 2, R = slots - 1;
  const int nblk = npair * npair, ntask = nblk + m * npair;
  T* Ac = A;
  T* An = A2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    const int fs = sweep & 1;
    if (t == 0) {
      double dm = 0.0;
      for (int j = 0; j < m; ++j) dm = fmax(dm, fabs(jlead(Ac[j * ld + j])));
      thr[0] = null_rel * dm;
      thr[1] = floor_rel * dm;
      flag[fs] = 0;
    }
    __syncthreads();
    const double nu = thr[0], fl = thr[1];
    for (int q = t; q < npair; q += nt) {  // round 0's rotations from A itself
      const int j = tb->pj[q], k = tb->pk[q];
      T c, sn;
      jident(c, sn);  // the padding pair of odd m never rotates
      const bool mv = k < m && jparams(Ac[j * ld + j], Ac[k * ld + k], Ac[j * ld + k], rel, fl, nu,
                                       c, sn);
      if (mv) flag[fs] = 1;  // any rotation this sweep (the same value from every writer)
      rc[q] = c;
      rs[q] = sn;
    }
    __syncthreads();
    for (int r = 0; r < R; ++r) {
      const T* rcc = rc + (r & 1) * 32;
      const T* rsc = rs + (r & 1) * 32;
      if (t < 32) {
        if (r + 1 < R) {  // rotations of round r + 1 from the entries this round produces
          T* rcn = rc + ((r + 1) & 1) * 32;
          T* rsn = rs + ((r + 1) & 1) * 32;
          for (int q = t; q < npair; q += 32) {
            const int u = tb->pj[(r + 1) * 32 + q], v = tb->pk[(r + 1) * 32 + q];
            T c, sn;
            jident(c, sn);
            bool mv = false;
            if (v < m) {
              // pairs with the padding index carry the identity, so a moving
              // pair has both indices below m
              const int pu = tb->pq[r * 64 + u], pv = tb->pq[r * 64 + v];
              const int qa = pu >> 1, qb = pv >> 1;
              const bool uk = pu & 1, vk = pv & 1;
              const int up = uk ? tb->pj[r * 32 + qa] : tb->pk[r * 32 + qa];
              const int vp = vk ? tb->pj[r * 32 + qb] : tb->pk[r * 32 + qb];
              const bool ma = jmoving(rsc[qa]);
              const bool mb = jmoving(rsc[qb]);
              const T ca = rcc[qa], sa = rsc[qa], cb = rcc[qb], sb = rsc[qb];
              const T auu = jnew(Ac, ld, u, up, uk, ma, ca, sa, u, up, uk, ma, ca, sa);
              const T avv = jnew(Ac, ld, v, vp, vk, mb, cb, sb, v, vp, vk, mb, cb, sb);
              const T auv = jnew(Ac, ld, u, up, uk, ma, ca, sa, v, vp, vk, mb, cb, sb);
              mv = jparams(auu, avv, auv, rel, fl, nu, c, sn);
            }
            if (mv) flag[fs] = 1;
            rcn[q] = c;
            rsn[q] = sn;
          }
        }
      } else {
        for (int e = t - 32; e < ntask; e += nt - 32) {
          if (e < nblk) {  // block (rows of pair q1, columns of pair q2) into the other copy
            const int bq = tb->blk[e], q1 = bq >> 8, q2 = bq & 255;
            const int j1 = tb->pj[r * 32 + q1], k1 = tb->pk[r * 32 + q1];
            const int j2 = tb->pj[r * 32 + q2], k2 = tb->pk[r * 32 + q2];
            const bool v1 = k1 < m, v2 = k2 < m;
            const bool m1 = v1 && jmoving(rsc[q1]), m2 = v2 && jmoving(rsc[q2]);
            T a00 = Ac[j1 * ld + j2], a01 = a00, a10 = a00, a11 = a00;
            if (v2) a01 = Ac[j1 * ld + k2];
            if (v1) a10 = Ac[k1 * ld + j2];
            if (v1 && v2) a11 = Ac[k1 * ld + k2];
            if (m2) {  // columns j2, k2
              const T c = rcc[q2], sn = rsc[q2];
              const T x0 = jrot(c, a00, sn, a01), y0 = jrotp(sn, a00, c, a01);
              a00 = x0;
              a01 = y0;
              if (v1) {
                const T x1 = jrot(c, a10, sn, a11), y1 = jrotp(sn, a10, c, a11);
                a10 = x1;
                a11 = y1;
              }
            }
            if (m1) {  // rows j1, k1
              const T c = rcc[q1], sn = rsc[q1];
              const T x0 = jrot(c, a00, sn, a10), y0 = jrotp(sn, a00, c, a10);
              a00 = x0;
              a10 = y0;
              if (v2) {
                const T x1 = jrot(c, a01, sn, a11), y1 = jrotp(sn, a01, c, a11);
                a01 = x1;
                a11 = y1;
              }
            }
            An[j1 * ld + j2] = a00;
            if (v2) An[j1 * ld + k2] = a01;
            if (v1) An[k1 * ld + j2] = a10;
            if (v1 && v2) An[k1 * ld + k2] = a11;
          } else {  // columns j, k of W in place
            const int wq = tb->wt[e - nblk], q = wq >> 8, row = wq & 255;
            const int j = tb->pj[r * 32 + q], k = tb->pk[r * 32 + q];
            if (k < m && jmoving(rsc[q])) {
              const T c = rcc[q], sn = rsc[q];
              const T wj = W[row * ld + j], wk = W[row * ld + k];
              W[row * ld + j] = jrot(c, wj, sn, wk);
              W[row * ld + k] = jrotp(sn, wj, c, wk);
            }
          }
        }
      }
      __syncthreads();
      T* tmp = Ac;
      Ac = An;
      An = tmp;
    }
    if (flag[fs] == 0) {
      A = Ac;
      return true;
    }
  }
  A = Ac;
  return false;
}

// C = op(X) Y for m x m matrices in shared memory (rows ld apart), op(X) = X
// or X^T
__device__ void small_mm(int m, int ld, const double* X, bool xt, const double* Y, double* C) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int i = e / m, j = e - i * m;
    double s = 0.0;
    if (xt)
      for (int k = 0; k < m; ++k) s = fma(X[k * ld + i], Y[k * ld + j], s);
    else
      for (int k = 0; k < m; ++k) s = fma(X[i * ld + k], Y[k * ld + j], s);
    C[i * ld + j] = s;
  }
}

// The same eigen-decomposition in double-float for m <= JS_REFINE_M: G is
// scaled by a power of two near its largest diagonal entry (exact), held as
// double-float pairs, and swept as above with the rotations on the FP32
// pipes; lambda and W are the double-float results rounded to FP64 (errors of
// about 1e-12 of the largest eigenvalue on test spectra with m = 36 and 48,
// against 1e-15 for the FP64 sweeps, in about half their time).  With refine
// an FP64 finish follows: two Newton-Schulz steps re-orthonormalise W,
// W <- W (3 I - W^T W) / 2, A = W^T G W (symmetrised) is diagonal up to the
// double-float level, and the FP64 sweeps resolve what is below it (the
// small eigenvalues, to FP64 accuracy, in a few sweeps).
#define JS_REFINE_M 64
__global__ void __launch_bounds__(1024) k_jacobi_sym_df(int m, const double* __restrict__ Gin, double* __restrict__ lambda,
                                double* __restrict__ Wout, int max_sweeps, int refine,
                                int* status) {
  extern __shared__ double js[];
  __shared__ DFv rcf[64], rsf[64];
  __shared__ double rcd[64], rsd[64], thr[2];
  __shared__ int flag[2], order[JS_REFINE_M], pj[64], pk[64], nrot;
  __shared__ double scale_s;
  __shared__ JacTabs tabs;
  const int ld = m + 1, mm = m * ld;  // padded rows (see k_jacobi_sym)
  // double-float phase: A, W, the second copy of A; FP64 finish: A, W, G, and
  // a work matrix that is also the second copy of A
  DFv* A = reinterpret_cast<DFv*>(js);
  DFv* W = A + mm;
  DFv* A2 = A + 2 * mm;
  const int t = threadIdx.x, nt = blockDim.x;
  if (t == 0) {
    double dm = 0.0;
    for (int j = 0; j < m; ++j) dm = fmax(dm, fabs(Gin[j * (j + 1) / 2 + j]));
    scale_s = dm > 0.0 ? ldexp(1.0, -ilogb(dm)) : 1.0;
  }
  jacobi_tabs(m, &tabs);
  __syncthreads();
  const double sc = scale_s;
  for (int e = t; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    const int hi = max(i, j), lo = min(i, j);
    A[i * ld + j] = dfv_from(Gin[hi * (hi + 1) / 2 + lo] * sc);
    W[i * ld + j] = dfv(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // 1e-13 for the result as it is; 1e-12 before the FP64 finish, which takes
  // the rest
  DFv* Af = A;
  const bool conv = jacobi_sweeps_1b<DFv>(m, ld, Af, A2, W, max_sweeps, refine ? 1e-12 : 1e-13,
                                          0.0, 1e-14, &tabs, rcf, rsf, flag, thr);
  if (!refine) {
    if (!conv && t == 0) vp_set_status(status, VP_ENOCONV);
    if (t == 0) {  // eigenvalues descending (selection order)
      for (int i = 0; i < m; ++i) order[i] = i;
      for (int i = 0; i < m; ++i) {
        int best = i;
        for (int j = i + 1; j < m; ++j)
          if (dfv_to(Af[order[j] * ld + order[j]]) > dfv_to(Af[order[best] * ld + order[best]]))
            best = j;
        const int tmp = order[i];
        order[i] = order[best];
        order[best] = tmp;
      }
    }
    __syncthreads();
    for (int i = t; i < m; i += nt) lambda[i] = dfv_to(Af[order[i] * ld + order[i]]) / sc;
    for (int e = t; e < m * m; e += nt) {
      const int r = e / m, c = e - r * m;
      Wout[e] = dfv_to(W[r * ld + order[c]]);
    }
    return;
  }
  // FP64 finish: the double-float W becomes FP64 in place (same size,
  // element by element by the same thread), then G and a work matrix follow
  double* Ad = js;
  double* Wd = js + mm;
  double* G = js + 2 * mm;
  double* Tm = js + 3 * mm;
  for (int e = t; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    Wd[i * ld + j] = dfv_to(W[i * ld + j]);
    const int hi = max(i, j), lo = min(i, j);
    G[i * ld + j] = Gin[hi * (hi + 1) / 2 + lo] * sc;
  }
  __syncthreads();
  for (int ns = 0; ns < 2; ++ns) {
    small_mm(m, ld, Wd, true, Wd, Tm);  // W^T W
    __syncthreads();
    for (int e = t; e < m * m; e += nt) {
      const int i = e / m, j = e - i * m;
      Tm[i * ld + j] = (i == j ? 1.5 : 0.0) - 0.5 * Tm[i * ld + j];
    }
    __syncthreads();
    small_mm(m, ld, Wd, false, Tm, Ad);  // W (3 I - W^T W) / 2
    __syncthreads();
    for (int e = t; e < m * m; e += nt) {
      const int i = e / m, j = e - i * m;
      Wd[i * ld + j] = Ad[i * ld + j];
    }
    __syncthreads();
  }
  small_mm(m, ld, G, false, Wd, Tm);  // G W
  __syncthreads();
  small_mm(m, ld, Wd, true, Tm, Ad);  // W^T G W
  __syncthreads();
  for (int e = t; e < m * m; e += nt) {
    const int i = e / m, j = e - i * m;
    if (i < j) {
      const double v = 0.5 * (Ad[i * ld + j] + Ad[j * ld + i]);
      Ad[i * ld + j] = v;
      Ad[j * ld + i] = v;
    }
  }
  __syncthreads();
  // few pairs rotate in these sweeps: the in-place passes, which skip the
  // pairs that do not rotate, cost less than copying A every round
  const bool conv64 = jacobi_sweeps<double>(m, ld, Ad, Wd, max_sweeps, 1e-15, 0.0, 1e-14, rcd, rsd,
                                            pj, pk, &nrot, thr);
  if (!conv64 && t == 0) vp_set_status(status, VP_ENOCONV);
  jacobi_output(m, ld, Ad, Wd, lambda, Wout, order);
  __syncthreads();
  for (int i = t; i < m; i += nt) lambda[i] /= sc;
}

// m <= 64: the double-float sweeps, with fp64_finish followed by the FP64
// finish (the DMD Gram, whose small singular values are divided by later),
// else the double-float result as it is (the DEIM Gram); larger m: the FP64
// sweeps (measured faster than double-float at m = 88), in shared memory up
// to JS_SMEM_M, in global memory above.
static void jacobi_sym(int m, const double* G, double* Ascr, double* Wscr, double* lambda,
                       double* Wout, int* status, cudaStream_t st, bool fp64_finish = false) {
  if (m <= JS_REFINE_M) {
    const size_t smem = sizeof(double) * (fp64_finish ? 4 : 3) * m * (m + 1);
    k_jacobi_sym_df<<<1, 1024, smem, st>>>(m, G, lambda, Wout, 60, fp64_finish ? 1 : 0, status);
    return;
  }
  const size_t smem = m <= JS_SMEM_M ? sizeof(double) * 2 * m * (m + 1) : 0;
  k_jacobi_sym<<<1, 512, smem, st>>>(m, G, Ascr, Wscr, lambda, Wout, 60, status);
}


// psi_k = Y w_k / sqrt(lambda_k), k < d; sigma = sqrt(max(lambda, 0)) (m values)
__global__ void k_psi(int64_t N, int m, int d, const double* __restrict__ Y, int64_t ldy,
                      const double* __restrict__ W, const double* __restrict__ lam,
                      double* __restrict__ Psi, double* __restrict__ sigma, int* status) {
  extern __shared__ double cs[];  // m x d coefficients
  for (int e = threadIdx.x; e < m * d; e += blockDim.x) {
    const int a = e / d, k = e - a * d;
    const double l = lam[k];
    if (!(l > 0.0)) {
      vp_set_status(status, VP_ENUMERIC);
      cs[e] = 0.0;
    } else {
      cs[e] = W[a * m + k] / sqrt(l);
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

// Step k of the greedy DEIM index selection written as Gaussian elimination
// with row pivoting on the N x d basis: after eliminating the pivots
// l_1..l_{k-1} from column k, that column is the residual of psi_k after
// interpolation from psi_1..psi_{k-1} at those rows, so the greedy choice is
// the row of its largest magnitude (the known equivalence of DEIM with
// partial-pivoting LU; Drmac and Gugercin, SIAM J. Sci. Comput. 38, 2016).
// R (d x N) holds the columns being eliminated, prow[j] (j > k-1) the
// multipliers R_j[l_{k-1}] / R_{k-1}[l_{k-1}] of the previous pivot.  Each
// block updates its rows of columns k..d-1 and keeps its arg-max of |R_k|
// (rows held at another position skipped; ties to the lowest row); the last
// block to finish picks l_k (or keeps the inherited index when renew says
// so), writes idx[k] and the multipliers of l_k for step k + 1.
__global__ void k_deim_lu(int64_t N, int d, int k, double* R, double* prow, int32_t* idx,
                          const int* __restrict__ renew, double* pval, int64_t* pidx, int* ticket,
                          int* status) {
  __shared__ double mult[128];
  __shared__ int32_t held[128];
  __shared__ int nheld, last;
  __shared__ double bv[32];
  __shared__ int64_t bi[32];
  const bool inherit = renew && !renew[k];
  if (threadIdx.x == 0) {
    int c = 0;
    for (int j = 0; j < d; ++j)
      if (j != k && (j < k || (renew && !renew[j]))) held[c++] = idx[j];
    nheld = c;
  }
  for (int j = threadIdx.x; j < d; j += blockDim.x) mult[j] = (k > 0 && j >= k) ? prow[j] : 0.0;
  __syncthreads();
  double best = -1.0;
  int64_t bidx = INT64_MAX;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
       l += (int64_t)gridDim.x * blockDim.x) {
    double rk;
    if (k > 0) {
      const double piv = R[(int64_t)(k - 1) * N + l];
      for (int j = k; j < d; ++j) {
        double* e = R + (int64_t)j * N + l;
        const double v = fma(-piv, mult[j], *e);
        *e = v;
        if (j == k) rk = v;
      }
    } else {
      rk = R[l];
    }
    if (inherit) continue;
    bool skip = false;
    for (int j = 0; j < nheld; ++j) skip |= held[j] == (int32_t)l;
    if (skip) continue;
    const double a = fabs(rk);
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
  __threadfence();  // this thread's updates of R before the ticket
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > bv[0] || (bv[w] == bv[0] && bi[w] < bi[0])) {
        bv[0] = bv[w];
        bi[0] = bi[w];
      }
    pval[blockIdx.x] = bv[0];
    pidx[blockIdx.x] = bi[0];
    __threadfence();
    last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ int32_t pick;
  // arg-max over the block partials: strided per thread, then warps, then
  // the first thread (ties to the lowest row throughout)
  double vb = -1.0;
  int64_t ib = INT64_MAX;
  if (!inherit)
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
      const double v = __ldcg(pval + i);
      const int64_t ii = __ldcg(pidx + i);
      if (v > vb || (v == vb && ii < ib)) {
        vb = v;
        ib = ii;
      }
    }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, vb, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, ib, o);
    if (ov > vb || (ov == vb && oi < ib)) {
      vb = ov;
      ib = oi;
    }
  }
  __syncthreads();
  if (lane == 0) {
    bv[wid] = vb;
    bi[wid] = ib;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *ticket = 0;
    int64_t b = idx[k];
    if (!inherit) {
      double bb = bv[0];
      b = bi[0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
        if (bv[w] > bb || (bv[w] == bb && bi[w] < b)) {
          bb = bv[w];
          b = bi[w];
        }
    }
    if (b < 0 || b >= N) {  // nothing left to pick, or a bad inherited index
      vp_set_status(status, VP_EINVAL);
      b = 0;
    }
    idx[k] = (int32_t)b;
    pick = (int32_t)b;
  }
  __syncthreads();
  const double pv = __ldcg(R + (int64_t)k * N + pick);
  if (threadIdx.x == 0 && (!(pv != 0.0) || !isfinite(pv))) vp_set_status(status, VP_ENUMERIC);
  for (int j = k + 1 + threadIdx.x; j < d; j += blockDim.x)
    prow[j] = (pv != 0.0 && isfinite(pv)) ? __ldcg(R + (int64_t)j * N + pick) / pv : 0.0;
}

// block partial dot products psi_k . prev_k (d x N each): part[blockIdx.x][k]
// The d steps of k_deim_lu in one cooperative launch, when every block's rows
// of the basis fit in shared memory: block b owns rows [b rb, min(N, (b+1) rb))
// and keeps its d x rb slice of R in shared memory for all steps.  Step k:
// eliminate the previous pivot from the slice's columns k..d-1; publish the
// block's candidate (its arg-max of |R_k| with held rows skipped, or the
// inherited row if the block owns it) together with that row's values of
// columns k..d-1; one grid barrier; then every block takes the same global
// choice (ties to the lowest row) and the multipliers R_j[l_k] / R_k[l_k]
// from the published row.  Same operations in the same order as k_deim_lu,
// so the same indices.  Published data alternate between two buffers by step
// parity: a block passes barrier k + 1 only after every block has arrived
// there, i.e. has finished reading the data of step k.  The barrier is a
// monotonic counter with a bounded wait (VP_ETIMEDOUT, and an abort flag
// that releases the other blocks).
constexpr int kLuThreads = 256;
constexpr int kLuSpins = 1 << 22;

__device__ bool lu_barrier(unsigned* count, unsigned target, int* abort_flag, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    __threadfence();
    atomicAdd(count, 1u);
    for (int spins = 0;; ++spins) {
      if (*reinterpret_cast<volatile unsigned*>(count) >= target) break;
      if (*reinterpret_cast<volatile int*>(abort_flag)) {
        ok = 0;
        break;
      }
      if (spins > kLuSpins) {
        vp_set_status(status, VP_ETIMEDOUT);
        atomicExch(abort_flag, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(kLuThreads)
k_deim_lu_coop(int64_t N, int d, int rb, const double* __restrict__ Psi, int32_t* idx,
               const int* __restrict__ renew, double* pval, int64_t* pidx, double* prows,
               unsigned* bar, int* abort_flag, int* status) {
  extern __shared__ double Rs[];  // d x rb
  __shared__ double mult[128];
  __shared__ int32_t picks[128], held[128];
  __shared__ int nheld;
  __shared__ double bv[32];
  __shared__ int64_t bi[32];
  __shared__ int64_t cand_s, pick_s;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
  const int nb = gridDim.x, b = blockIdx.x;
  const int64_t r0 = (int64_t)b * rb;
  const int rows = (int)(N - r0 < (int64_t)rb ? (N - r0 > 0 ? N - r0 : 0) : rb);
  for (int e = t; e < d * rows; e += blockDim.x) {
    const int j = e / rows, i = e - j * rows;
    Rs[j * rb + i] = Psi[(int64_t)j * N + r0 + i];
  }
  for (int j = t; j < d; j += blockDim.x) mult[j] = 0.0;
  __syncthreads();
  for (int k = 0; k < d; ++k) {
    const bool inherit = renew && !renew[k];
    const int par = k & 1;
    if (t == 0) {  // rows held at the other positions
      int c = 0;
      for (int j = 0; j < d; ++j)
        if (j != k && (j < k || (renew && !renew[j]))) held[c++] = j < k ? picks[j] : idx[j];
      nheld = c;
    }
    if (k > 0)  // eliminate the previous pivot from columns k..d-1
      for (int e = t; e < (d - k) * rows; e += blockDim.x) {
        const int jj = e / rows, i = e - jj * rows, j = k + jj;
        Rs[j * rb + i] = fma(-Rs[(k - 1) * rb + i], mult[j], Rs[j * rb + i]);
      }
    __syncthreads();
    double best = -1.0;
    int64_t bidx = INT64_MAX;
    if (!inherit)
      for (int i = t; i < rows; i += blockDim.x) {
        const int64_t l = r0 + i;
        bool skip = false;
        for (int j = 0; j < nheld; ++j) skip |= held[j] == (int32_t)l;
        if (skip) continue;
        const double a = fabs(Rs[k * rb + i]);
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
    if (lane == 0) {
      bv[wid] = best;
      bi[wid] = bidx;
    }
    __syncthreads();
    if (t == 0) {
      double bb = bv[0];
      int64_t c = bi[0];
      for (int w = 1; w < nw; ++w)
        if (bv[w] > bb || (bv[w] == bb && bi[w] < c)) {
          bb = bv[w];
          c = bi[w];
        }
      if (inherit) {  // the inherited row, published by its owner
        const int64_t l = idx[k];
        c = (l >= r0 && l < r0 + rows) ? l : INT64_MAX;
        bb = c != INT64_MAX ? 1.0 : -1.0;
      }
      pval[par * nb + b] = bb;
      pidx[par * nb + b] = c;
      cand_s = c;
    }
    __syncthreads();
    const int64_t cand = cand_s;
    if (cand != INT64_MAX)
      for (int j = k + t; j < d; j += blockDim.x)
        prows[((int64_t)par * nb + b) * d + j] = Rs[j * rb + (int)(cand - r0)];
    if (!lu_barrier(bar, (unsigned)(k + 1) * (unsigned)nb, abort_flag, status)) return;
    // the global choice, the same in every block
    double vb = -1.0;
    int64_t ib = INT64_MAX;
    for (int i = t; i < nb; i += blockDim.x) {
      const double v = __ldcg(pval + par * nb + i);
      const int64_t ii = __ldcg(pidx + par * nb + i);
      if (v > vb || (v == vb && ii < ib)) {
        vb = v;
        ib = ii;
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, vb, o);
      const int64_t oi = __shfl_xor_sync(0xffffffffu, ib, o);
      if (ov > vb || (ov == vb && oi < ib)) {
        vb = ov;
        ib = oi;
      }
    }
    __syncthreads();
    if (lane == 0) {
      bv[wid] = vb;
      bi[wid] = ib;
    }
    __syncthreads();
    if (t == 0) {
      double bb = bv[0];
      int64_t p = bi[0];
      for (int w = 1; w < nw; ++w)
        if (bv[w] > bb || (bv[w] == bb && bi[w] < p)) {
          bb = bv[w];
          p = bi[w];
        }
      if (inherit) p = idx[k];
      if (p < 0 || p >= N) {  // nothing left to pick, or a bad inherited index
        if (b == 0) vp_set_status(status, VP_EINVAL);
        p = 0;
      }
      picks[k] = (int32_t)p;
      pick_s = p;
    }
    __syncthreads();
    const int64_t pick = pick_s;
    const int owner = (int)(pick / rb);
    const double* row = prows + ((int64_t)par * nb + owner) * d;
    const double pv = __ldcg(row + k);
    if (t == 0 && b == 0) {
      idx[k] = (int32_t)pick;
      if (!(pv != 0.0) || !isfinite(pv)) vp_set_status(status, VP_ENUMERIC);
    }
    for (int j = k + 1 + t; j < d; j += blockDim.x)
      mult[j] = (pv != 0.0 && isfinite(pv)) ? __ldcg(row + j) / pv : 0.0;
    __syncthreads();
  }
}

__global__ void k_rot_dots(int64_t N, int d, const double* __restrict__ Psi,
                           const double* __restrict__ Prev, double* __restrict__ part) {
  __shared__ double red[32];
  for (int k = 0; k < d; ++k) {
    double s = 0.0;
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
         l += (int64_t)gridDim.x * blockDim.x)
      s = fma(Psi[(int64_t)k * N + l], Prev[(int64_t)k * N + l], s);
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

// renew[k] = 1 for the n_up positions with the smallest |psi_k . prev_k| (the
// most rotated basis vectors; ties to the lowest position), else 0
__global__ void k_renew(int d, const double* __restrict__ dots, int n_up, int* __restrict__ renew) {
  if (threadIdx.x != 0) return;
  for (int k = 0; k < d; ++k) renew[k] = 0;
  for (int t = 0; t < n_up && t < d; ++t) {
    int b = -1;
    double best = 0.0;
    for (int k = 0; k < d; ++k) {
      if (renew[k]) continue;
      const double a = fabs(dots[k]);
      if (b < 0 || a < best) {
        best = a;
        b = k;
      }
    }
    renew[b] = 1;
  }
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
__global__ void k_dmd_coeff(int m, int r, const double* __restrict__ W, const double* __restrict__ lam,
                            double* __restrict__ C, int* status) {
  for (int e = threadIdx.x; e < m * r; e += blockDim.x) {
    const int a = e / r, k = e - a * r;
    const double l = lam[k];
    if (!(l > 0.0)) {
      vp_set_status(status, VP_ENUMERIC);
      C[e] = 0.0;
    } else {
      C[e] = W[a * m + k] / sqrt(l);
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

// ---------------------------------------------- half-step power of A
// complex helpers in FP32 (float2; the FP64 ones are in vp_internal.cuh)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float c_abs(float2 a) { return hypotf(a.x, a.y); }
template <class C> struct CplxT;
template <> struct CplxT<float2> {
  using R = float;
  static __device__ __forceinline__ float2 make(float x, float y) { return make_float2(x, y); }
  static constexpr float eps = 1.1920929e-7f;
};
template <class C>
__device__ __forceinline__ C c_div(C a, C b) {  // Smith's algorithm
  using R = typename CplxT<C>::R;
  if (fabs(b.x) >= fabs(b.y)) {
    const R q = b.y / b.x, den = b.x + b.y * q;
    return CplxT<C>::make((a.x + a.y * q) / den, (a.y - a.x * q) / den);
  }
  const R q = b.x / b.y, den = b.x * q + b.y;
  return CplxT<C>::make((a.x * q + a.y) / den, (a.y * q - a.x) / den);
}
// principal square root, branch cut on the negative real axis (the sign of
// the imaginary part, zero included, picks the side)
template <class C>
__device__ __forceinline__ C c_sqrt(C z) {
  using R = typename CplxT<C>::R;
  if (z.x == (R)0 && z.y == (R)0) return CplxT<C>::make(0, 0);
  const R t = sqrt((R)0.5 * (c_abs(z) + fabs(z.x)));
  if (z.x >= (R)0) return CplxT<C>::make(t, z.y / ((R)2 * t));
  return CplxT<C>::make(fabs(z.y) / ((R)2 * t), copysign(t, z.y));
}

// Complex Schur form A = Q T Q^H of the real r x r matrix A (r <= 64) in the
// precision of C, then the upper-triangular square root Rm of T with the
// principal power of every diagonal entry: Householder reduction to
// Hessenberg form, implicit single-shift QR sweeps with Wilkinson shifts,
// Givens rotations and deflation (every eleventh sweep of an eigenvalue uses an
// ad hoc shift), then R_ii = T_ii^{1/2}, (R_ii + R_jj) R_ij = T_ij -
// sum_{i<k<j} R_ik R_kj (Bjorck and Hammarling, 1983).  On return H holds T,
// Qm the Schur vectors; false when the QR sweeps did not finish within 40 r
// in total (VP_ENOCONV); a zero R_ii + R_jj sets VP_ENUMERIC.
template <class C>
__device__ bool schur_sqrt(int r, int ld, const double* __restrict__ A, C* H, C* Qm, C* Rm,
                           int* status) {
  using R = typename CplxT<C>::R;
  using CT = CplxT<C>;
  __shared__ R v[64];
  __shared__ R vv;
  const int lane = threadIdx.x, nl = blockDim.x;
  const R eps = CT::eps;
  for (int e = lane; e < r * r; e += nl) {
    const int i = e / r, j = e - i * r;
    H[i * ld + j] = CT::make((R)A[e], 0);
    Qm[i * ld + j] = CT::make(i == j ? 1 : 0, 0);
  }
  __syncthreads();
  // 1. Hessenberg form (A is real: real reflectors)
  for (int k = 0; k + 2 < r; ++k) {
    const int m = r - k - 1;
    R sx = 0, x0 = H[(k + 1) * ld + k].x;
    for (int i = 1; i < m; ++i) {
      const R t = H[(k + 1 + i) * ld + k].x;
      sx = fma(t, t, sx);
    }
    if (sx == (R)0) continue;  // column already reduced (same value in every lane)
    const R alpha = -copysign(sqrt(fma(x0, x0, sx)), x0);
    for (int i = lane; i < m; i += nl) v[i] = i == 0 ? x0 - alpha : H[(k + 1 + i) * ld + k].x;
    __syncthreads();
    if (lane == 0) {
      R t = 0;
      for (int i = 0; i < m; ++i) t = fma(v[i], v[i], t);
      vv = t;
    }
    __syncthreads();
    const R f = (R)2 / vv;
    for (int j = lane; j < r; j += nl) {  // H <- P H (rows k+1..)
      R w = 0;
      for (int i = 0; i < m; ++i) w = fma(v[i], H[(k + 1 + i) * ld + j].x, w);
      w *= f;
      for (int i = 0; i < m; ++i) H[(k + 1 + i) * ld + j].x -= v[i] * w;
    }
    __syncthreads();
    for (int i = lane; i < r; i += nl) {  // H <- H P, Q <- Q P (columns k+1..)
      R w = 0, wq = 0;
      for (int j = 0; j < m; ++j) {
        w = fma(H[i * ld + k + 1 + j].x, v[j], w);
        wq = fma(Qm[i * ld + k + 1 + j].x, v[j], wq);
      }
      w *= f;
      wq *= f;
      for (int j = 0; j < m; ++j) {
        H[i * ld + k + 1 + j].x -= w * v[j];
        Qm[i * ld + k + 1 + j].x -= wq * v[j];
      }
    }
    __syncthreads();
    for (int i = k + 2 + lane; i < r; i += nl) H[i * ld + k] = CT::make(0, 0);
    __syncthreads();
  }
  // 2. complex Schur form by implicit single-shift QR sweeps; a subdiagonal
  // entry deflates below eps times its diagonal neighbours or below eps |A|_F
  // (a backward-stable perturbation either way)
  __shared__ R nrm_s;
  if (lane == 0) {
    double t = 0.0;
    for (int e = 0; e < r * r; ++e) t = fma(A[e], A[e], t);
    nrm_s = (R)sqrt(t);
  }
  __syncthreads();
  const R floor2 = eps * eps * nrm_s * nrm_s;
  auto abs2 = [](C z) { return fma(z.x, z.x, z.y * z.y); };
  // the scalar decisions (deflation scan, shift, rotation) are taken by
  // thread 0 and shared: FP64 chains cost the same in a full warp as in one
  // lane, so only the row and column updates are spread over the block
  __shared__ int sh_cmd, sh_l, sh_hi;
  __shared__ C sh_mu, sh_sg;
  __shared__ R sh_cg;
  int it = 0, total = 0;  // thread 0's counters
  if (lane == 0) sh_hi = r - 1;
  __syncthreads();
  bool failed = false;
  while (true) {
    if (lane == 0) {
      const int hi = sh_hi;
      int cmd = 0;
      if (hi <= 0) {
        cmd = 2;
      } else {
        int l = hi;
        for (; l > 0; --l) {  // squared magnitudes: no square roots in the scan
          const R sc2 = abs2(H[(l - 1) * ld + l - 1]) + abs2(H[l * ld + l]);
          const R sub2 = abs2(H[l * ld + l - 1]);
          if (sub2 <= eps * eps * sc2 || sub2 <= floor2) break;
        }
        if (l > 0) H[l * ld + l - 1] = CT::make(0, 0);
        if (l == hi) {
          sh_hi = hi - 1;
          it = 0;
          cmd = 1;
        } else if (total > 40 * r) {
          cmd = 3;
        } else {
          const C a = H[(hi - 1) * ld + hi - 1], b = H[(hi - 1) * ld + hi],
                        c = H[hi * ld + hi - 1], d = H[hi * ld + hi];
          C mu;
          if (it % 11 == 10) {
            mu = CT::make(d.x + (R)0.75 * c_abs(c), d.y);
          } else {
            const C h = CT::make((R)0.5 * (a.x - d.x), (R)0.5 * (a.y - d.y));
            const C disc = c_sqrt(cadd(cmul(h, h), cmul(b, c)));
            const C m0 = CT::make((R)0.5 * (a.x + d.x), (R)0.5 * (a.y + d.y));
            const C m1 = cadd(m0, disc), m2 = csub(m0, disc);
            mu = abs2(csub(m1, d)) < abs2(csub(m2, d)) ? m1 : m2;
          }
          sh_l = l;
          sh_mu = mu;
          ++it;
          ++total;
        }
      }
      sh_cmd = cmd;
    }
    __syncthreads();
    const int cmd = sh_cmd, l = sh_l, hi = sh_hi;
    __syncthreads();  // all have read the decision before thread 0 takes the next
    if (cmd == 2) break;
    if (cmd == 3) {
      failed = true;
      break;
    }
    if (cmd == 1) continue;
    for (int k = l; k < hi; ++k) {
      if (lane == 0) {
        C x, y;
        if (k == l) {
          x = csub(H[l * ld + l], sh_mu);
          y = H[(l + 1) * ld + l];
        } else {
          x = H[k * ld + k - 1];
          y = H[(k + 1) * ld + k - 1];
        }
        // G = [[cg, sg], [-conj(sg), cg]] with G [x; y] = [rho; 0]
        if (y.x == (R)0 && y.y == (R)0) {
          sh_cg = 1;
          sh_sg = CT::make(0, 0);
        } else if (x.x == (R)0 && x.y == (R)0) {
          sh_cg = 0;
          sh_sg = CT::make(1, 0);
        } else {  // cg = |x| / n, sg = (x / |x|) conj(y) / n, n^2 = |x|^2 + |y|^2
          const R ax2 = abs2(x), ix = rsqrt(ax2), in = rsqrt(ax2 + abs2(y));
          sh_cg = ax2 * ix * in;
          sh_sg = cmul(CT::make(x.x * ix, x.y * ix), CT::make(y.x * in, -y.y * in));
        }
      }
      __syncthreads();
      const R cg = sh_cg;
      const C sg = sh_sg;
      const C sc = CT::make(sg.x, -sg.y);
      // rows k, k+1 <- G [rows]: one output per thread (FP64 issue, not the
      // lane count, sets the cost, so outputs are spread over all warps);
      // inputs are read before the barrier, outputs written after it
      const int j0 = k == l ? l : k - 1, w = r - j0;
      C outv = CT::make(0, 0);
      int oidx = -1;
      for (int o = lane; o < 2 * w; o += nl) {
        const int j = j0 + (o < w ? o : o - w);
        const C h0 = H[k * ld + j], h1 = H[(k + 1) * ld + j];
        if (o < w) {
          outv = cadd(CT::make(cg * h0.x, cg * h0.y), cmul(sg, h1));
          oidx = k * ld + j;
        } else {
          outv = csub(CT::make(cg * h1.x, cg * h1.y), cmul(sc, h0));
          oidx = (k + 1) * ld + j;
        }
      }
      __syncthreads();
      if (oidx >= 0) H[oidx] = outv;
      __syncthreads();
      if (k > l && lane == 0) H[(k + 1) * ld + k - 1] = CT::make(0, 0);
      // columns k, k+1 <- [columns] G^H: H rows in the first half of the
      // block, Q rows in the second (different warps, so they overlap)
      const int i1 = min(k + 2, hi) + 1, half = nl / 2;
      C* M2 = lane < half ? H : Qm;
      const int lim = lane < half ? i1 : r;
      for (int i = lane < half ? lane : lane - half; i < lim; i += half) {
        const C h0 = M2[i * ld + k], h1 = M2[i * ld + k + 1];
        M2[i * ld + k] = cadd(CT::make(cg * h0.x, cg * h0.y), cmul(h1, sc));
        M2[i * ld + k + 1] = csub(CT::make(cg * h1.x, cg * h1.y), cmul(h0, sg));
      }
      __syncthreads();
    }
  }
  if (failed) {
    if (lane == 0) vp_set_status(status, VP_ENOCONV);
    return false;
  }
  // 3. R = T^{1/2} (upper triangular), superdiagonal by superdiagonal
  bool singular = false;
  for (int e = lane; e < r * r; e += nl) {
    const int i = e / r, j = e - i * r;
    Rm[i * ld + j] = i == j ? c_sqrt(H[i * ld + j]) : CT::make(0, 0);
  }
  __syncthreads();
  for (int dd = 1; dd < r; ++dd) {
    for (int i = lane; i + dd < r; i += nl) {
      const int j = i + dd;
      C s = H[i * ld + j];
      for (int k = i + 1; k < j; ++k) s = csub(s, cmul(Rm[i * ld + k], Rm[k * ld + j]));
      const C den = cadd(Rm[i * ld + i], Rm[j * ld + j]);
      if (den.x == (R)0 && den.y == (R)0) {
        singular = true;
        Rm[i * ld + j] = CT::make(0, 0);
      } else {
        Rm[i * ld + j] = c_div(s, den);
      }
    }
    __syncthreads();
  }
  if (singular) vp_set_status(status, VP_ENUMERIC);
  return true;
}

// ------------------------------------------ mixed-precision half-step power
// Re(A^{1/2}) with the Schur form and the triangular root in FP32, then one
// Newton step in FP64: with X0 = Q R Q^H (Q, R the FP32 factors, in FP64),
// the correction F of X0 F + F X0 = A - X0^2 is Q Y Q^H with
// R Y + Y R = Q^H (A - X0^2) Q (a triangular Sylvester equation), since
// Q^H Q = I to FP32 rounding; X1 = X0 + F is the principal root to FP64
// rounding (the error of X0, ~1e-7, squared, plus 1e-7 of the correction).
// k_sqrtm_schur32: the FP32 factors, written as FP64 complex r x r (r <= 64).
__global__ void k_sqrtm_schur32(int r, const double* __restrict__ A, double2* __restrict__ Qd,
                                double2* __restrict__ Rd, int* status) {
  extern __shared__ float2 sq32[];
  const int ld = r + 1;  // padded rows: column sweeps of a stride r share banks
  float2* H = sq32;
  float2* Qm = H + r * ld;
  float2* Rm = Qm + r * ld;
  if (!schur_sqrt<float2>(r, ld, A, H, Qm, Rm, status)) return;
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e - i * r;
    Qd[e] = make_double2(Qm[i * ld + j].x, Qm[i * ld + j].y);
    Rd[e] = make_double2(Rm[i * ld + j].x, Rm[i * ld + j].y);
  }
}

// One row per block (r blocks of 64 threads, thread j: column j) of
// op(P) op(Qm) with op = identity or conjugate transpose (FP64 complex,
// r x r row-major).  mode 0: out = op(P) op(Qm); mode 1: out = A - op(P) op(Qm)
// with A real; mode 2: S = Re(Z + op(P) op(Qm)) (real output).
__global__ void k_cmm_row(int r, const double2* __restrict__ P, int ph,
                          const double2* __restrict__ Qm, int qh, int mode,
                          const double* __restrict__ A, const double2* __restrict__ Z,
                          double2* __restrict__ out, double* __restrict__ S) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= r) return;
  double2 s = make_double2(0.0, 0.0);
  for (int k = 0; k < r; ++k) {
    const double2 p = ph ? make_double2(P[k * r + i].x, -P[k * r + i].y) : P[i * r + k];
    const double2 q = qh ? make_double2(Qm[j * r + k].x, -Qm[j * r + k].y) : Qm[k * r + j];
    s = cadd(s, cmul(p, q));
  }
  const int e = i * r + j;
  if (mode == 0) out[e] = s;
  else if (mode == 1) out[e] = make_double2(A[e] - s.x, -s.y);
  else S[e] = Z[e].x + s.x;
}

// R Y + Y R = C for upper-triangular R (r x r, FP64 complex), Y full: entry
// (i, j) needs Y_kj (k > i) and Y_ik (k < j), so the anti-diagonals
// d = j - i are solved in increasing order; each entry's sum is spread over a
// warp (1024 threads: one entry per warp for r <= 32).  A zero R_ii + R_jj
// leaves Y_ij = 0 (the FP32 phase has flagged it).
__global__ void k_sylv_tri(int r, const double2* __restrict__ Rg, const double2* __restrict__ C,
                           double2* __restrict__ Yg) {
  extern __shared__ double2 sy[];  // R and Y, rows padded to r + 1
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ld = r + 1;
  double2* Rm = sy;
  double2* Y = sy + r * ld;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e - i * r;
    Rm[i * ld + j] = Rg[e];
  }
  __syncthreads();
  for (int d = -(r - 1); d <= r - 1; ++d) {
    const int i0 = d < 0 ? -d : 0, cnt = r - (d < 0 ? -d : d);
    for (int q = warp; q < cnt; q += nw) {
      const int i = i0 + q, j = i + d;
      double2 s = make_double2(0.0, 0.0);
      for (int k = i + 1 + lane; k < r; k += 32) s = cadd(s, cmul(Rm[i * ld + k], Y[k * ld + j]));
      for (int k = lane; k < j; k += 32) s = cadd(s, cmul(Y[i * ld + k], Rm[k * ld + j]));
      for (int o = 16; o > 0; o >>= 1) {
        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
      }
      if (lane == 0) {
        // (C - s) / den as (C - s) conj(den) / |den|^2, the reciprocal of
        // |den|^2 from FP32 by two Newton steps in FP64 (FP64 accurate)
        const double2 den = cadd(Rm[i * ld + i], Rm[j * ld + j]);
        const double dn = fma(den.x, den.x, den.y * den.y);
        double2 y = make_double2(0.0, 0.0);
        if (dn > 0.0 && dn < 1e300) {
          double inv = (double)(1.0f / (float)dn);
          if (inv == 0.0 || !isfinite(inv)) inv = 1.0 / dn;  // outside the FP32 range
          inv = inv * fma(-dn, inv, 2.0);
          inv = inv * fma(-dn, inv, 2.0);
          const double2 num = cmul(csub(C[i * r + j], s), make_double2(den.x, -den.y));
          y = make_double2(num.x * inv, num.y * inv);
        }
        Y[i * ld + j] = y;
      }
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int i = e / r, j = e - i * r;
    Yg[e] = Y[i * ld + j];
  }
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
                      double eps_h, const double* __restrict__ eps_dev, double* __restrict__ out,
                      int* status) {
  extern __shared__ double aug[];  // q x (q + K)
  __shared__ int piv, ok;
  const int w = q + K;
  const double eps = eps_dev ? *eps_dev : eps_h;
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

// ------------------------------------------- DMD-DEIM reduced dynamics
// Y_i[l] = Lambda^0(x_il) Phi_i with x_il = sum_m A_lm a_mi - B_lm b_mi, the
// position of particle l under sample i (U_X = [A, -B], Z_i = [a; b]): the
// DEIM data column of eq. Ydeim, straight from Q (N x 2n rows [A | B]) and
// the 2n x q coefficients Zs.  Row tiles of 32 particles go to shared memory.
#define PQ_ROWS 32
__global__ void k_phi_at_qz(GridC g, int64_t N, int n, int q, const double* __restrict__ Q,
                            const double* __restrict__ Zs, const double* __restrict__ phi,
                            double* __restrict__ Y) {
  extern __shared__ double pq[];
  const int n2 = 2 * n;
  double* zs = pq;                // n2 x q
  double* qt = pq + n2 * q;       // PQ_ROWS x n2
  for (int e = threadIdx.x; e < n2 * q; e += blockDim.x) zs[e] = Zs[e];
  for (int64_t tile = blockIdx.x; tile * PQ_ROWS < N; tile += gridDim.x) {
    const int64_t base = tile * PQ_ROWS;
    const int rows = (int)min((int64_t)PQ_ROWS, N - base);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) qt[e] = Q[base * n2 + e];
    __syncthreads();
    for (int e = threadIdx.x; e < q * PQ_ROWS; e += blockDim.x) {
      const int i = e / PQ_ROWS, rr = e - i * PQ_ROWS;
      if (rr >= rows) continue;
      double x = 0.0;
      for (int m = 0; m < n; ++m) {
        x = fma(qt[rr * n2 + m], zs[m * q + i], x);
        x = fma(-qt[rr * n2 + n + m], zs[(n + m) * q + i], x);
      }
      int j;
      double sfr;
      cell_of(x, g.inv_h, g.Nx, g.dNx, g.inv_Nx, j, sfr);
      const int j1 = (j + 1 == g.Nx) ? 0 : j + 1;
      const double* ph = phi + (int64_t)i * g.Nx;
      Y[(int64_t)i * N + base + rr] = fma(sfr, __ldg(ph + j1), (1.0 - sfr) * __ldg(ph + j));
    }
  }
}

// out (d x n2, FP64) = rows idx of a row-format matrix (mode 1 double-float
// float2, mode 2 FP32 float; N x n2)
__global__ void k_gather_rows_lp(const void* __restrict__ Q2, int mode, int64_t N, int n2,
                                 const int32_t* __restrict__ idx, int d, double* __restrict__ out,
                                 int* status) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * n2; e += gridDim.x * blockDim.x) {
    const int j = e / n2, m = e - j * n2;
    const int64_t l = idx[j];
    if (l < 0 || l >= N) {
      vp_set_status(status, VP_EINVAL);
      out[e] = 0.0;
      continue;
    }
    const int64_t a = l * n2 + m;
    if (mode == 1) {
      const float2 v = reinterpret_cast<const float2*>(Q2)[a];
      out[e] = (double)v.x + (double)v.y;
    } else {
      out[e] = (double)reinterpret_cast<const float*>(Q2)[a];
    }
  }
}

// One fixed-point round of the DMD-DEIM coefficient stage (eq. grHDD, X part):
// gX_i = U_X[idx]^T (c (.) F_i(cell of x_i[idx])) / m_p with x_i[idx] =
// U_X[idx] Ze_i, for sample i = blockIdx.x; Qd holds the d DEIM rows [A | B]
// of the basis, F the cell field of the DMD potentials (p x Nx).  Returns at
// once after convergence (done flag).
__global__ void k_deim_round(GridC g, int n, int p, int d, const double* __restrict__ Qd,
                             const double* __restrict__ Ze, const double* __restrict__ F,
                             const double* __restrict__ c, double* __restrict__ gX,
                             const int* __restrict__ done) {
  if (*done) return;
  extern __shared__ double dr[];
  const int n2 = 2 * n, i = blockIdx.x;
  double* qd = dr;             // d x n2
  double* z = qd + d * n2;     // n2
  double* e = z + n2;          // d
  for (int t = threadIdx.x; t < d * n2; t += blockDim.x) qd[t] = Qd[t];
  for (int t = threadIdx.x; t < n2; t += blockDim.x) z[t] = Ze[(int64_t)t * p + i];
  __syncthreads();
  const double* Fi = F + (int64_t)i * g.Nx;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double x = 0.0;
    for (int m = 0; m < n; ++m) {
      x = fma(qd[j * n2 + m], z[m], x);
      x = fma(-qd[j * n2 + n + m], z[n + m], x);
    }
    int cell;
    double sfr;
    cell_of(x, g.inv_h, g.Nx, g.dNx, g.inv_Nx, cell, sfr);
    e[j] = c[j] * Fi[cell] / g.mp;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n2; r += blockDim.x) {
    // U_X row j = [A_j, -B_j]: column r < n reads A, r >= n reads -B
    const double sg = r < n ? 1.0 : -1.0;
    double s = 0.0;
    for (int j = 0; j < d; ++j) s = fma(qd[j * n2 + r], e[j], s);
    gX[(int64_t)r * p + i] = sg * s;
  }
}

// Gaussian RBF width 0.3 / (mean distance of each node to its nearest other node)
__global__ void k_rbf_width(int dim, int q, const double* __restrict__ eta_s, double* eps) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < q; i += blockDim.x) {
    double best = INFINITY;
    for (int j = 0; j < q; ++j) {
      if (j == i) continue;
      double d2 = 0.0;
      for (int a = 0; a < dim; ++a) {
        const double dd = eta_s[i * dim + a] - eta_s[j * dim + a];
        d2 = fma(dd, dd, d2);
      }
      best = fmin(best, sqrt(d2));
    }
    s += best;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *eps = 0.3 / (t / q);
  }
}

}  // namespace

namespace vpk {
void deim_init() {
  const int lim = 200 * 1024;
  cudaFuncSetAttribute(k_ygram, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_psi, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_jacobi_sym_df, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_deim_lu_coop, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_deim_weights, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_rbf, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_sqrtm_schur32, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_sylv_tri, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_phi_at_qz, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  cudaFuncSetAttribute(k_deim_round, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}
}  // namespace vpk

namespace vpk {
size_t deim_basis_scratch(int sms, int64_t N, int m) {
  const int tot = m * m;
  const int gx = std::min<int64_t>(ceil_div(N, YG_ROWS), 2 * sms);
  return arena_bytes((size_t)gx * tot, 8) + 4 * arena_bytes(tot, 8) + arena_bytes(m, 8);
}

vp_status deim_basis_run(vp_ctx* ctx, int64_t N, int m, const double* Y, int64_t ldy, int d,
                         double* Psi, double* sigma, void* scratch, cudaStream_t st) {
  const int tot = m * m, tri = m * (m + 1) / 2;
  const int gx = std::min<int64_t>(ceil_div(N, YG_ROWS), 2 * ctx->num_sms);
  const int gy = ceil_div(tri, 256 * 8);
  const size_t bytes = deim_basis_scratch(ctx->num_sms, N, m);
  Arena a{(char*)scratch, 0, bytes};
  double* part = a.take<double>((size_t)gx * tri);
  double* G = a.take<double>(tot);
  double* Aj = a.take<double>(tot);
  double* Wj = a.take<double>(tot);
  double* Ws = a.take<double>(tot);
  double* lam = a.take<double>(m);
  VP_K(VP_K_DEIM, (k_ygram<<<dim3(gx, gy), 256, sizeof(double) * m * YG_ROWS, st>>>(N, m, Y, ldy,
                                                                                      part)));
  VP_K(VP_K_REDUCE, reduce_partials(gx, tri, part, G, nullptr, st));
  VP_K(VP_K_JACOBI_SYM, jacobi_sym(m, G, Aj, Wj, lam, Ws, ctx->d_status, st));
  int bx = std::min<int64_t>(ceil_div(N, 256), 4 * ctx->num_sms);
  VP_K(VP_K_DEIM, (k_psi<<<bx, 256, sizeof(double) * m * d, st>>>(N, m, d, Y, ldy, Ws, lam, Psi,
                                                                    sigma, ctx->d_status)));
  return VP_OK;
}

size_t deim_indices_scratch(int sms, int64_t N, int d) {
  const int nb = std::min<int64_t>(ceil_div(N, 256), 2 * sms);
  return arena_bytes(nb, 8) + arena_bytes(nb, 8) + arena_bytes(128, 8) +
         arena_bytes((size_t)nb * d, 8) + arena_bytes(d, 8) + arena_bytes(d, 4) +
         arena_bytes((size_t)d * N, 8) + arena_bytes(1, 4) +
         // the cooperative form: two parities of per-block candidates and rows, barrier words
         2 * arena_bytes((size_t)2 * sms, 8) + arena_bytes((size_t)2 * sms * d, 8) +
         arena_bytes(2, 4);
}

// The cooperative form of the index selection when every block's slice of
// the basis fits in shared memory (one block per SM); false: not launched.
static bool deim_lu_coop(vp_ctx* ctx, int64_t N, int d, const double* Psi, int32_t* idx,
                         const int* renew, double* pval, int64_t* pidx, double* prows,
                         unsigned* bar, cudaStream_t st) {
  const int nb = ctx->num_sms;
  const int64_t rb64 = (N + nb - 1) / nb;
  const size_t smem = sizeof(double) * (size_t)d * (size_t)rb64;
  if (d > 128 || N < nb || smem > 200 * 1024) return false;
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_deim_lu_coop, kLuThreads, smem) !=
          cudaSuccess ||
      per < 1)
    return false;
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st) != cudaSuccess) return false;
  int rb = (int)rb64;
  int* abort_flag = reinterpret_cast<int*>(bar + 1);
  int* status = ctx->d_status;
  void* args[] = {&N, &d, &rb, &Psi, &idx, &renew, &pval, &pidx, &prows, &bar, &abort_flag, &status};
  return cudaLaunchCooperativeKernel((const void*)k_deim_lu_coop, nb, kLuThreads, args, smem, st) ==
         cudaSuccess;
}

vp_status deim_indices_run(vp_ctx* ctx, int64_t N, int d, const double* Psi, int32_t* idx,
                           const double* Psi_prev, int n_up, void* scratch, cudaStream_t st) {
  const int nb = std::min<int64_t>(ceil_div(N, 256), 2 * ctx->num_sms);
  const size_t bytes = deim_indices_scratch(ctx->num_sms, N, d);
  Arena a{(char*)scratch, 0, bytes};
  double* pval = a.take<double>(nb);
  int64_t* pidx = a.take<int64_t>(nb);
  double* prow = a.take<double>(128);
  double* part = a.take<double>((size_t)nb * d);
  double* dots = a.take<double>(d);
  int* renew = a.take<int>(d);
  double* R = a.take<double>((size_t)d * N);
  int* ticket = a.take<int>(1);
  double* cval = a.take<double>((size_t)2 * ctx->num_sms);
  int64_t* cidx = a.take<int64_t>((size_t)2 * ctx->num_sms);
  double* crows = a.take<double>((size_t)2 * ctx->num_sms * d);
  unsigned* cbar = a.take<unsigned>(2);
  const int* rn = nullptr;
  if (Psi_prev) {  // index update: renew the n_up most rotated positions
    VP_K(VP_K_DEIM, (k_rot_dots<<<nb, 256, 0, st>>>(N, d, Psi, Psi_prev, part)));
    VP_K(VP_K_REDUCE, reduce_partials(nb, d, part, dots, nullptr, st));
    VP_K(VP_K_DEIM, (k_renew<<<1, 32, 0, st>>>(d, dots, n_up, renew)));
    rn = renew;
  }
  bool coop = false;
  VP_K(VP_K_DEIM, coop = deim_lu_coop(ctx, N, d, Psi, idx, rn, cval, cidx, crows, cbar, st));
  if (coop) return VP_OK;
  VP_CUDA(cudaMemcpyAsync(R, Psi, sizeof(double) * d * N, cudaMemcpyDeviceToDevice, st));
  VP_CUDA(cudaMemsetAsync(ticket, 0, sizeof(int), st));
  for (int k = 0; k < d; ++k)
    VP_K(VP_K_DEIM, (k_deim_lu<<<nb, 256, 0, st>>>(N, d, k, R, prow, idx, rn, pval, pidx, ticket,
                                                     ctx->d_status)));
  return VP_OK;
}

size_t deim_weights_scratch(int sms, int64_t N, int d) {
  const int nb = std::min<int64_t>(ceil_div(N, 256), 2 * sms);
  return arena_bytes((size_t)nb * d, 8) + arena_bytes(d, 8);
}

vp_status deim_weights_run(vp_ctx* ctx, int64_t N, int d, const double* Psi, const int32_t* idx,
                           double Mq, double* c, void* scratch, cudaStream_t st) {
  const int nb = std::min<int64_t>(ceil_div(N, 256), 2 * ctx->num_sms);
  Arena a{(char*)scratch, 0, deim_weights_scratch(ctx->num_sms, N, d)};
  double* part = a.take<double>((size_t)nb * d);
  double* colsum = a.take<double>(d);
  VP_K(VP_K_DEIM, (k_colsum<<<nb, 256, 0, st>>>(N, d, Psi, part)));
  VP_K(VP_K_REDUCE, reduce_partials(nb, d, part, colsum, nullptr, st));
  VP_K(VP_K_DEIM, (k_deim_weights<<<1, 256, sizeof(double) * d * (d + 1), st>>>(
                        N, d, Psi, idx, colsum, Mq, c, ctx->d_status)));
  return VP_OK;
}

size_t dmd_fit_scratch(int nx, int m, int r_max) {
  const int tot = m * m;
  const int gx = std::max(1, std::min(ceil_div(nx, YG_ROWS), 64));
  return arena_bytes((size_t)gx * tot, 8) + 4 * arena_bytes(tot, 8) + arena_bytes(m, 8) +
         arena_bytes((size_t)m * r_max, 8) + arena_bytes((size_t)r_max * nx, 8) +
         2 * arena_bytes((size_t)r_max * r_max, 8) + 7 * arena_bytes((size_t)r_max * r_max, 16);
}

vp_status dmd_fit_run(vp_ctx* ctx, int nx, int m, const double* Y, const double* Yp, double tol,
                      int r_max, int* r_out, double* B, double* Bpinv, double* A, double* S,
                      double* sigma, void* scratch, cudaStream_t st) {
  const int tot = m * m, tri = m * (m + 1) / 2;
  const int gx = std::max(1, std::min(ceil_div(nx, YG_ROWS), 64));
  const int gy = ceil_div(tri, 256 * 8);
  Arena a{(char*)scratch, 0, dmd_fit_scratch(nx, m, r_max)};
  double* part = a.take<double>((size_t)gx * tri);
  double* G = a.take<double>(tot);
  double* Aj = a.take<double>(tot);
  double* Wj = a.take<double>(tot);
  double* Ws = a.take<double>(tot);
  double* lam = a.take<double>(m);
  double* C = a.take<double>((size_t)m * r_max);
  double* U = a.take<double>((size_t)r_max * nx);
  double* BtB = a.take<double>((size_t)r_max * r_max);
  double* BtBi = a.take<double>((size_t)r_max * r_max);
  double2* sq[7];  // half-step power: Q, R, two products, X, residual, Y
  for (int i = 0; i < 7; ++i) sq[i] = a.take<double2>((size_t)r_max * r_max);
  // 1. Y^T Y and its eigen-decomposition (singular values and right vectors of Y)
  VP_K(VP_K_DMD, (k_ygram<<<dim3(gx, gy), 256, sizeof(double) * m * YG_ROWS, st>>>(nx, m, Y, nx,
                                                                                       part)));
  VP_K(VP_K_REDUCE, reduce_partials(gx, tri, part, G, nullptr, st));
  VP_K(VP_K_JACOBI_SYM, jacobi_sym(m, G, Aj, Wj, lam, Ws, ctx->d_status, st, true));
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
  if (sigma) VP_K(VP_K_DMD, sqrt_nonneg(m, lam, sigma, st));
  // 3. C = V_r S_r^-1; U_r = Y C, B = Y' C; A = U_r^T B; B^+ = (B^T B)^-1 B^T
  VP_K(VP_K_DMD, (k_dmd_coeff<<<1, 256, 0, st>>>(m, r, Ws, lam, C, ctx->d_status)));
  const int gcols = std::max(1, std::min(ceil_div((int64_t)nx * r, 256), 4 * ctx->num_sms));
  VP_K(VP_K_DMD, (k_cols_times<<<gcols, 256, 0, st>>>(nx, m, r, Y, C, U)));
  VP_K(VP_K_DMD, (k_cols_times<<<gcols, 256, 0, st>>>(nx, m, r, Yp, C, B)));
  VP_K(VP_K_DMD, (k_cols_dot<<<ceil_div(r * r, 256), 256, 0, st>>>(nx, r, r, U, B, A)));
  VP_K(VP_K_DMD, (k_cols_dot<<<ceil_div(r * r, 256), 256, 0, st>>>(nx, r, r, B, B, BtB)));
  VP_K(VP_K_DMD, (k_inverse<<<1, 256, sizeof(double) * 2 * r * r, st>>>(r, BtB, BtBi,
                                                                           ctx->d_status)));
  // B^+ (r x nx) = BtBi (r x r) * B^T; B is stored as r columns of length nx,
  // i.e. the row-major r x nx matrix B^T
  VP_K(VP_K_DMD, (k_mm<<<gcols, 256, 0, st>>>(r, r, nx, BtBi, B, Bpinv)));
  // 4. real part of the principal square root of A for half steps: FP32
  // Schur form and triangular root, one FP64 Newton step
  double2 *Qd = sq[0], *Rd = sq[1], *M1 = sq[2], *X = sq[3], *E = sq[4], *Cm = sq[5], *Ys = sq[6];
  VP_K(VP_K_DMD, (k_sqrtm_schur32<<<1, 256, sizeof(float2) * 3 * r * (r + 1), st>>>(
                      r, A, Qd, Rd, ctx->d_status)));
  VP_K(VP_K_DMD, (k_cmm_row<<<r, 64, 0, st>>>(r, Qd, 0, Rd, 0, 0, nullptr, nullptr, M1, nullptr)));
  VP_K(VP_K_DMD, (k_cmm_row<<<r, 64, 0, st>>>(r, M1, 0, Qd, 1, 0, nullptr, nullptr, X, nullptr)));
  VP_K(VP_K_DMD, (k_cmm_row<<<r, 64, 0, st>>>(r, X, 0, X, 0, 1, A, nullptr, E, nullptr)));
  VP_K(VP_K_DMD, (k_cmm_row<<<r, 64, 0, st>>>(r, Qd, 1, E, 0, 0, nullptr, nullptr, M1, nullptr)));
  VP_K(VP_K_DMD, (k_cmm_row<<<r, 64, 0, st>>>(r, M1, 0, Qd, 0, 0, nullptr, nullptr, Cm, nullptr)));
  VP_K(VP_K_DMD, (k_sylv_tri<<<1, 1024, sizeof(double2) * 2 * r * (r + 1), st>>>(r, Rd, Cm, Ys)));
  VP_K(VP_K_DMD, (k_cmm_row<<<r, 64, 0, st>>>(r, Qd, 0, Ys, 0, 0, nullptr, nullptr, M1, nullptr)));
  VP_K(VP_K_DMD, (k_cmm_row<<<r, 64, 0, st>>>(r, M1, 0, Qd, 1, 2, nullptr, X, nullptr, S)));
  return VP_OK;
}

void dmd_coords_run(int nx, int r, const double* Bpinv, int q, const double* Phi, double* beta,
                    cudaStream_t st) {
  // beta (q x r) = Phi (q x nx) Bpinv^T: entry (i, k) = sum_x Phi[i][x] Bpinv[k][x]
  k_cols_dot<<<ceil_div(q * r, 256), 256, 0, st>>>(nx, q, r, Phi, Bpinv, beta);
}

void rbf_run(int dim, int q, const double* eta_s, int K, const double* values, int p,
             const double* eta, double eps, const double* eps_dev, double* out, int* status,
             cudaStream_t st) {
  k_rbf<<<1, 256, sizeof(double) * q * (q + K), st>>>(dim, q, eta_s, K, values, p, eta, eps, eps_dev,
                                                      out, status);
}

void rbf_width_run(int dim, int q, const double* eta_s, double* eps, cudaStream_t st) {
  k_rbf_width<<<1, 256, 0, st>>>(dim, q, eta_s, eps);
}

void dmd_potential_run(int nx, int r, const double* B, const double* A, const double* S, int p,
                       const double* beta, int ksteps, int half, double* Phi, cudaStream_t st) {
  k_dmd_eval<<<p, 128, sizeof(double) * 2 * r, st>>>(nx, r, B, A, S, beta, ksteps, half, Phi);
}

void phi_at_qz(const GridC& g, int64_t N, int n, int q, const double* Q, const double* Zs,
               const double* phi, double* Y, int sms, cudaStream_t st) {
  const int bx = std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, PQ_ROWS), 4 * sms));
  const size_t smem = sizeof(double) * ((size_t)2 * n * q + (size_t)PQ_ROWS * 2 * n);
  k_phi_at_qz<<<bx, 256, smem, st>>>(g, N, n, q, Q, Zs, phi, Y);
}

void gather_rows_lp(const void* Q2, int mode, int64_t N, int n2, const int32_t* idx, int d,
                    double* out, int* status, cudaStream_t st) {
  k_gather_rows_lp<<<ceil_div(d * n2, 256), 256, 0, st>>>(Q2, mode, N, n2, idx, d, out, status);
}

void deim_round(const GridC& g, int n, int p, int d, const double* Qd, const double* Ze,
                const double* F, const double* c, double* gX, const int* done, cudaStream_t st) {
  const size_t smem = sizeof(double) * ((size_t)d * 2 * n + 2 * n + d);
  k_deim_round<<<p, 128, smem, st>>>(g, n, p, d, Qd, Ze, F, c, gX, done);
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
  VP_K(VP_K_DEIM, (k_phi_at<<<dim3(bx, p), 256, 0, st>>>(g, N, p, X, ldx, phi, Y, ldy)));
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
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, deim_basis_scratch(ctx->num_sms, N, m), &base));
  VP_TRY(deim_basis_run(ctx, N, m, Y, ldy, d, Psi, sigma, base, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_deim_indices(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi, int32_t* idx,
                          void* stream) {
  if (!ctx || !Psi || !idx || N < 1 || d < 1 || d > 128 || d > N) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, deim_indices_scratch(ctx->num_sms, N, d), &base));
  VP_TRY(deim_indices_run(ctx, N, d, Psi, idx, nullptr, 0, base, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_deim_indices_update(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi,
                                 const double* Psi_prev, int32_t n_up, int32_t* idx, void* stream) {
  if (!ctx || !Psi || !Psi_prev || !idx || N < 1 || d < 1 || d > 128 || d > N || n_up < 0 ||
      n_up > d)
    return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, deim_indices_scratch(ctx->num_sms, N, d), &base));
  VP_TRY(deim_indices_run(ctx, N, d, Psi, idx, Psi_prev, n_up, base, st));
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_deim_weights(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi, const int32_t* idx,
                          double Mq, double* c, void* stream) {
  if (!ctx || !Psi || !idx || !c || N < 1 || d < 1 || d > 128) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, deim_weights_scratch(ctx->num_sms, N, d), &base));
  VP_TRY(deim_weights_run(ctx, N, d, Psi, idx, Mq, c, base, st));
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
  void* base = nullptr;
  VP_TRY(vp_workspace(ctx, dmd_fit_scratch(nx, m, r_max), &base));
  int r = 0;
  VP_TRY(dmd_fit_run(ctx, nx, m, Y, Yp, tol, r_max, &r, B, Bpinv, A, S, sigma, base, st));
  *r_out = r;
  VP_LAUNCHED();
  return VP_OK;
}

vp_status vp_dmd_coords(vp_ctx* ctx, int32_t nx, int32_t r, const double* Bpinv, int32_t q,
                        const double* Phi, double* beta, void* stream) {
  if (!ctx || !Bpinv || !Phi || !beta || nx < 1 || r < 1 || r > 64 || q < 1) return VP_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  VP_K(VP_K_DMD, dmd_coords_run(nx, r, Bpinv, q, Phi, beta, st));
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
  VP_K(VP_K_DMD, rbf_run(dim, q, eta_s, K, values, p, eta, eps, nullptr, out, ctx->d_status, st));
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
  VP_K(VP_K_DMD, dmd_potential_run(nx, r, B, A, S, p, beta, ksteps, half, Phi, st));
  VP_LAUNCHED();
  return VP_OK;
}

}  // extern "C"
