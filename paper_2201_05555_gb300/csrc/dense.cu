// Single-block FP64 kernels for the small dense algebra of the reduced model:
// n x n complex matrices (n <= 40) built from Gram matrices over the N rows,
// Gauss-Jordan solves with partial pivoting, and the per-step coefficient
// updates.  Complex n x n matrices are row-major double2 in global memory.
#include "vp_internal.cuh"
#include "dfloat.cuh"

#include <cstddef>
#include <type_traits>

namespace vpk {

__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

// ---------------------------------------------- element types of the kernels
// The small dense kernels run on a complex element type CT: double2 (FP64),
// or DC, real and imaginary parts as double-float pairs (16 bytes like
// double2, so the shared-memory layouts are the same).  This part issues
// FP64 at 1/64 of the FP32 rate, and one block of these kernels is bound by
// it; the double-float operations run on the FP32 pipes at about five times
// the FP64 throughput, with ~1e-14 relative rounding per operation instead
// of ~1e-16, and run on 1024 threads (the FP64 ones on 256: more warps do
// not raise the FP64 rate).  Inputs and outputs in global memory stay double2.
struct DC {
  DFv re, im;
};
__device__ __forceinline__ DC cadd(DC a, DC b) { return DC{dfv_add(a.re, b.re), dfv_add(a.im, b.im)}; }
__device__ __forceinline__ DC csub(DC a, DC b) {
  return DC{dfv_add(a.re, dfv_neg(b.re)), dfv_add(a.im, dfv_neg(b.im))};
}
__device__ __forceinline__ DC cmul(DC a, DC b) {
  return DC{dfv_add(dfv_mul(a.re, b.re), dfv_neg(dfv_mul(a.im, b.im))),
            dfv_add(dfv_mul(a.re, b.im), dfv_mul(a.im, b.re))};
}
__device__ __forceinline__ DC cconj(DC a) { return DC{a.re, dfv_neg(a.im)}; }
__device__ __forceinline__ DC cscale(DC a, double s) {
  const DFv f = dfv_from(s);
  return DC{dfv_mul(a.re, f), dfv_mul(a.im, f)};
}
// a real factor in the working precision, converted once outside the loops
// (a conversion from FP64 runs on the FP64 pipe)
__device__ __forceinline__ double cfac(double2*, double s) { return s; }
__device__ __forceinline__ DFv cfac(DC*, double s) { return dfv_from(s); }
__device__ __forceinline__ DC cscale(DC a, DFv f) { return DC{dfv_mul(a.re, f), dfv_mul(a.im, f)}; }
// conversions from and to the global double2 layout
template <class CT>
__device__ __forceinline__ CT cload(double2 a);
template <>
__device__ __forceinline__ double2 cload<double2>(double2 a) { return a; }
template <>
__device__ __forceinline__ DC cload<DC>(double2 a) { return DC{dfv_from(a.x), dfv_from(a.y)}; }
template <class CT>
__device__ __forceinline__ CT cload(DC a);
template <>
__device__ __forceinline__ DC cload<DC>(DC a) { return a; }
__device__ __forceinline__ double2 cto(double2 a) { return a; }
__device__ __forceinline__ double2 cto(DC a) { return make_double2(dfv_to(a.re), dfv_to(a.im)); }
template <class CT>
__device__ __forceinline__ CT cval(double re, double im) {
  return cload<CT>(make_double2(re, im));
}
__device__ __forceinline__ double cabs2(DC a) { return cabs2(cto(a)); }
// a + d (real d)
__device__ __forceinline__ double2 cadd_re(double2 a, double d) {
  a.x += d;
  return a;
}
__device__ __forceinline__ DC cadd_re(DC a, double d) { return DC{dfv_add(a.re, dfv_from(d)), a.im}; }
// conj(p) / |p|^2 with |p|^2 = a2, formed in FP64
__device__ __forceinline__ double2 cinv_a2(double2 pv, double a2) { return cscale(cconj(pv), 1.0 / a2); }
__device__ __forceinline__ DC cinv_a2(DC pv, double a2) {
  return cload<DC>(cscale(cconj(cto(pv)), 1.0 / a2));
}

// out = alpha * op(A) op(B) + beta * out (all n x n); op = 0 plain, 1 conj-transpose.
// out must not alias A or B.  Ends with __syncthreads().
template <class CT, class TA, class TB>
__device__ void cmm(CT* out, const TA* A, int opA, const TB* B, int opB, CT alpha, double beta,
                    int n) {
  const CT zero = cval<CT>(0.0, 0.0);
  const auto fb = cfac(out, beta);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e - r * n;
    CT s = zero;
    for (int k = 0; k < n; ++k) {
      CT a = opA ? cconj(cload<CT>(A[k * n + r])) : cload<CT>(A[r * n + k]);
      CT b = opB ? cconj(cload<CT>(B[c * n + k])) : cload<CT>(B[k * n + c]);
      s = cadd(s, cmul(a, b));
    }
    CT v = cmul(alpha, s);
    out[e] = beta == 0.0 ? v : cadd(v, cscale(out[e], fb));
  }
  __syncthreads();
}

// out = a*A + b*op(B) + d*I (elementwise), n x n.  out may alias A.
template <class CT, class TA, class TB>
__device__ void cadd_mat(CT* out, double a, const TA* A, double b, const TB* B, int opB, double d,
                         int n) {
  const CT zero = cval<CT>(0.0, 0.0);
  const auto fa = cfac(out, a), fb = cfac(out, b);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e - r * n;
    CT x = A ? cscale(cload<CT>(A[e]), fa) : zero;
    if (B) x = cadd(x, cscale(opB ? cconj(cload<CT>(B[c * n + r])) : cload<CT>(B[e]), fb));
    if (r == c) x = cadd_re(x, d);
    out[e] = x;
  }
  __syncthreads();
}
template <class CT, class TA>
__device__ void cadd_mat(CT* out, double a, const TA* A, double b, std::nullptr_t, int opB,
                         double d, int n) {
  cadd_mat(out, a, A, b, static_cast<const CT*>(nullptr), opB, d, n);
}

// Solve A X = B in place (A: n x n, lda; B: n x m, ldb; both in shared
// memory) by Gauss-Jordan with partial pivoting.  Returns false if a pivot
// vanishes.  Pivot ties resolve to the lowest row (deterministic).
template <class CT>
__device__ bool gj_solve(CT* A, int lda, CT* B, int ldb, int n, int m, CT* col) {
  __shared__ int piv;
  __shared__ int ok;
  __shared__ CT inv_s;
  if (threadIdx.x == 0) ok = 1;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = c;
      for (int r = c + threadIdx.x; r < n; r += 32) {
        double v = cabs2(A[r * lda + c]);
        if (v > best) { best = v; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        double ob = __shfl_xor_sync(0xffffffffu, best, o);
        int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        piv = bi;
        if (!(best > 0.0) || !isfinite(best)) ok = 0;
      }
    }
    __syncthreads();
    if (!ok) return false;
    const int pr = piv;
    if (pr != c) {
      for (int j = threadIdx.x; j < n + m; j += blockDim.x) {
        CT* a = j < n ? &A[c * lda + j] : &B[c * ldb + j - n];
        CT* b = j < n ? &A[pr * lda + j] : &B[pr * ldb + j - n];
        CT t = *a;
        *a = *b;
        *b = t;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {  // the inverse of the pivot, once (FP64)
      const CT pv = A[c * lda + c];
      inv_s = cinv_a2(pv, cabs2(pv));
    }
    __syncthreads();
    const CT inv = inv_s;
    for (int j = threadIdx.x; j < n + m; j += blockDim.x) {
      CT* a = j < n ? &A[c * lda + j] : &B[c * ldb + j - n];
      *a = cmul(*a, inv);
    }
    for (int r = threadIdx.x; r < n; r += blockDim.x) col[r] = A[r * lda + c];
    __syncthreads();
    for (int e = threadIdx.x; e < n * (n + m); e += blockDim.x) {
      int r = e / (n + m), j = e - r * (n + m);
      if (r == c) continue;
      CT f = col[r];
      if (j < n) A[r * lda + j] = csub(A[r * lda + j], cmul(f, A[c * lda + j]));
      else B[r * ldb + j - n] = csub(B[r * ldb + j - n], cmul(f, B[c * ldb + j - n]));
    }
    __syncthreads();
  }
  return true;
}

// Solve in place M = [A | B] (n x w, leading dimension ld; A is n x n) by
// Gauss-Jordan elimination without pivoting, for the systems of this file:
// Hermitian positive definite (zeta zeta^H) or close to the identity
// (Cayley and tangent factors with small steps), where elimination in the
// natural order is stable.  Per pivot c: the scaled pivot row (columns > c)
// goes to shared memory, then every row is updated from `src` into `dst`
// (ping-pong with `work`, n x w), two barriers per pivot.  Only columns > c
// are kept current, so on return the B part of M holds A^-1 B and the A part
// is undefined.  Returns false (M undefined) when a pivot falls below 1e-14
// times the largest initial diagonal entry or is not finite; callers then
// rebuild M and use gj_solve.
template <class CT>
__device__ bool gj_np(CT* M, int ld, int n, int w, CT* work, CT* rowc) {
  __shared__ int bad;
  __shared__ double dscale;
  if (threadIdx.x == 0) {
    double d = 0.0;
    for (int r = 0; r < n; ++r) d = fmax(d, cabs2(M[r * ld + r]));
    dscale = d;
    bad = !(d > 0.0) || !isfinite(d);
  }
  __syncthreads();
  CT* src = M;
  CT* dst = work;
  int lds = ld, ldd = w;
  for (int c = 0; c < n; ++c) {
    const int w1 = w - c - 1;  // columns c+1 .. w-1
    if (threadIdx.x < w1 || threadIdx.x == 0) {  // the threads that scale the pivot row
      const CT pv = src[c * lds + c];
      const double a2 = cabs2(pv);
      if (threadIdx.x == 0 && (!(a2 > 1e-28 * dscale) || !isfinite(a2))) bad = 1;
      const CT inv = cinv_a2(pv, a2);
      for (int j = threadIdx.x; j < w1; j += blockDim.x) rowc[j] = cmul(src[c * lds + c + 1 + j], inv);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n * w1; e += blockDim.x) {
      const int r = e / w1, jj = e - r * w1, j = c + 1 + jj;
      dst[r * ldd + j] = (r == c) ? rowc[jj] : csub(src[r * lds + j], cmul(src[r * lds + c], rowc[jj]));
    }
    __syncthreads();
    CT* t = src;
    src = dst;
    dst = t;
    const int tl = lds;
    lds = ldd;
    ldd = tl;
  }
  if (src != M) {  // result of an odd number of pivots sits in work: copy the B part
    for (int e = threadIdx.x; e < n * (w - n); e += blockDim.x) {
      const int r = e / (w - n), j = n + e - r * (w - n);
      M[r * ld + j] = src[r * lds + j];
    }
    __syncthreads();
  }
  return !bad;
}

// Hermitian H = zeta zeta^H (n x n) from Z = [a; b] (2n x p).  In
// double-float, Z is converted once, in chunks of ZG_CHUNK columns staged in
// zs (2n x ZG_CHUNK double-float pairs of shared memory), since a conversion
// from FP64 runs on the FP64 pipe.
#define ZG_CHUNK 32
template <class CT>
__device__ void zeta_gram(CT* H, const double* Z, int n, int p, DFv* zs = nullptr) {
  if constexpr (!std::is_same<CT, double2>::value) {
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) H[e] = cval<CT>(0.0, 0.0);
    for (int i0 = 0; i0 < p; i0 += ZG_CHUNK) {
      const int w = min(ZG_CHUNK, p - i0);
      __syncthreads();  // the previous chunk is used up
      for (int e = threadIdx.x; e < 2 * n * w; e += blockDim.x) {
        const int r = e / w, i = e - r * w;
        zs[r * ZG_CHUNK + i] = dfv_from(Z[(int64_t)r * p + i0 + i]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int r = e / n, c = e - r * n;
        CT s = H[e];
        for (int i = 0; i < w; ++i) {
          const CT zr = CT{zs[r * ZG_CHUNK + i], zs[(n + r) * ZG_CHUNK + i]};
          const CT zc = CT{zs[c * ZG_CHUNK + i], zs[(n + c) * ZG_CHUNK + i]};
          s = cadd(s, cmul(zr, cconj(zc)));
        }
        H[e] = s;
      }
    }
    __syncthreads();
    return;
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e - r * n;
    CT s = cval<CT>(0.0, 0.0);
    for (int i = 0; i < p; ++i) {
      CT zr = cval<CT>(Z[(int64_t)r * p + i], Z[(int64_t)(n + r) * p + i]);
      CT zc = cval<CT>(Z[(int64_t)c * p + i], Z[(int64_t)(n + c) * p + i]);
      s = cadd(s, cmul(zr, cconj(zc)));
    }
    H[e] = s;
  }
  __syncthreads();
}

// ----------------------------------------------------------- basis velocity
// X(Q, zeta) = -i (M - Q (Q^H M)) H^-1 = M C0 + Q C1 (times scale), with
// H = zeta zeta^H, C0 = -i scale H^-1, C1 = i scale (Q^H M) H^-1.
// Shared: aug n x 3n.  Output C (2 x n x n).
template <class CT>
__global__ void k_small_basis_coeffs(int n, int p, const double2* __restrict__ QhM,
                                     const double* __restrict__ Z, double scale, double2* C,
                                     double2* tmp, int* status, int in_smem) {
  extern __shared__ double2 aug_raw[];
  CT* aug = reinterpret_cast<CT*>(aug_raw);
  const int ld = 3 * n;
  CT* H = in_smem ? aug + n * ld : reinterpret_cast<CT*>(tmp);  // n x n
  CT* work = aug + n * ld + n * n;                               // n x 3n (in_smem)
  __shared__ CT rowc[128];
  // double-float: the staging of Z follows the work matrix in shared memory
  zeta_gram(H, Z, n, p, reinterpret_cast<DFv*>(work + n * ld));
  const CT one = cval<CT>(1.0, 0.0), zero = cval<CT>(0.0, 0.0);
  auto build = [&]() {
    for (int e = threadIdx.x; e < n * ld; e += blockDim.x) {
      int r = e / ld, c = e - r * ld;
      CT v;
      if (c < n) v = H[r * n + c];
      else if (c < 2 * n) v = c - n == r ? one : zero;
      else v = cconj(cload<CT>(QhM[(c - 2 * n) * n + r]));  // (Q^H M)^H
      aug[e] = v;
    }
    __syncthreads();
  };
  build();
  __shared__ CT col[64];
  bool ok = in_smem && gj_np(aug, ld, n, ld, work, rowc);
  if (!ok) {
    build();
    if (!gj_solve(aug, ld, aug + n, ld, n, 2 * n, col)) {
      if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
      return;
    }
  }
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    int r = e / n, c = e - r * n;
    double2 hinv = cto(aug[r * ld + n + c]);          // H^-1
    double2 y = cconj(cto(aug[c * ld + 2 * n + r]));  // ((H^-1 (Q^H M)^H)^H)[r][c] = (Q^H M H^-1)[r][c]
    C[e] = make_double2(scale * hinv.y, -scale * hinv.x);          // -i s H^-1
    C[n * n + e] = make_double2(-scale * y.y, scale * y.x);        // +i s (Q^H M) H^-1
  }
}

void small_basis_coeffs(int n, int p, const double2* QhM, const double* Z, double scale,
                        double2* C, double2* tmp, int* status, cudaStream_t st, bool df) {
  size_t smem = sizeof(double2) * n * 7 * n;
  if (df) smem += sizeof(DFv) * 2 * n * ZG_CHUNK;
  if (df)
    k_small_basis_coeffs<DC><<<1, 1024, smem, st>>>(n, p, QhM, Z, scale, C, tmp, status, 1);
  else
    k_small_basis_coeffs<double2><<<1, 256, smem, st>>>(n, p, QhM, Z, scale, C, tmp, status, 1);
}

// ------------------------------------------------------- Cayley retraction
// Inputs G0 = Q0^H Q0, P = Q0^H xi, XX = xi^H xi.  With W = xi - Q0 P / 2,
// C = [W, -Q0], D = [Q0, W]:  R = Q0 + C (I - D^H C / 2)^-1 D^H Q0
//   = Q0 (I - P Yt / 2 - Yb) + xi Yt,   [Yt; Yb] = (I - K/2)^-1 [G0; W^H Q0],
// K = D^H C = [[Q0^H W, -G0], [W^H W, -W^H Q0]],
// Q0^H W = P - G0 P / 2,  W^H W = XX - P^H P + P^H G0 P / 4.
// Output C (2 x n x n): coefficient of Q0, coefficient of xi.
template <class CT>
__global__ void k_small_cayley(int n, const double2* __restrict__ G0g, const double2* __restrict__ Pg,
                               const double2* __restrict__ XXg, double2* C, double2* tmp,
                               int* status, int in_smem, int fast) {
  extern __shared__ double2 aug_raw[];  // 2n x 3n, then (in_smem) G0, P, XX, T, QW, WW
  CT* aug = reinterpret_cast<CT*>(aug_raw);
  const int nn = n * n, ld = 3 * n;
  CT* sb = aug + 6 * nn;
  CT* tb = reinterpret_cast<CT*>(tmp);
  // inputs in the working type: shared memory, or after the temporaries in tmp
  CT* ib = in_smem ? sb : tb + 3 * nn;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    ib[e] = cload<CT>(G0g[e]);
    ib[nn + e] = cload<CT>(Pg[e]);
    ib[2 * nn + e] = cload<CT>(XXg[e]);
  }
  __syncthreads();
  const CT* G0 = ib;
  const CT* P = ib + nn;
  const CT* XX = ib + 2 * nn;
  CT* T = in_smem ? sb + 3 * nn : tb;            // G0 P
  CT* QW = in_smem ? sb + 4 * nn : tb + nn;      // Q0^H W
  CT* WW = in_smem ? sb + 5 * nn : tb + 2 * nn;  // W^H W
  const CT one = cval<CT>(1.0, 0.0);
  cmm(T, G0, 0, P, 0, one, 0.0, n);
  cadd_mat(QW, 1.0, P, -0.5, T, 0, 0.0, n);
  cmm(WW, P, 1, P, 0, cval<CT>(-1.0, 0.0), 0.0, n);
  cmm(WW, P, 1, T, 0, cval<CT>(0.25, 0.0), 1.0, n);
  cadd_mat(WW, 1.0, WW, 1.0, XX, 0, 0.0, n);
  const auto fhalf = cfac(aug, 0.5), fmhalf = cfac(aug, -0.5);
  auto build = [&]() {
    for (int e = threadIdx.x; e < 2 * n * ld; e += blockDim.x) {
      int r = e / ld, c = e - r * ld;
      int rb = r >= n, cb = c / n, rr = r - rb * n, cc = c - cb * n;
      CT v;
      const bool dg = rr == cc;
      if (!rb && cb == 0) {
        v = cscale(QW[rr * n + cc], fmhalf);
        if (dg) v = cadd_re(v, 1.0);
      } else if (!rb && cb == 1) {
        v = cscale(G0[rr * n + cc], fhalf);
      } else if (!rb && cb == 2) {
        v = G0[rr * n + cc];
      } else if (rb && cb == 0) {
        v = cscale(WW[rr * n + cc], fmhalf);
      } else {  // W^H Q0 = (Q0^H W)^H
        CT wq = cconj(QW[cc * n + rr]);
        if (cb == 1) {
          v = cscale(wq, fhalf);
          if (dg) v = cadd_re(v, 1.0);
        } else {
          v = wq;
        }
      }
      aug[e] = v;
    }
    __syncthreads();
  };
  build();
  __shared__ CT col[128];
  __shared__ CT rowc[256];
  bool ok = fast && gj_np(aug, ld, 2 * n, ld, aug + 12 * nn, rowc);
  if (!ok) {
    build();
    if (!gj_solve(aug, ld, aug + 2 * n, ld, 2 * n, n, col)) {
      if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
      return;
    }
  }
  // copy Yt, Yb out of the system (reuse T, QW)
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    int r = e / n, c = e - r * n;
    T[e] = aug[r * ld + 2 * n + c];         // Yt
    QW[e] = aug[(n + r) * ld + 2 * n + c];  // Yb
  }
  __syncthreads();
  // alpha = I - P Yt / 2 - Yb ; beta = Yt
  CT* alpha = WW;
  cmm(alpha, P, 0, T, 0, cval<CT>(-0.5, 0.0), 0.0, n);
  cadd_mat(alpha, 1.0, alpha, -1.0, QW, 0, 1.0, n);
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    C[e] = cto(alpha[e]);
    C[nn + e] = cto(T[e]);
  }
}

void small_cayley_coeffs(int n, const double2* G0, const double2* P, const double2* XX, double2* C,
                         double2* tmp, int* status, cudaStream_t st, bool df) {
  size_t full = sizeof(double2) * 12 * n * n;
  int in_smem = full <= 200 * 1024;
  int fast = in_smem && sizeof(double2) * 18 * n * n <= 200 * 1024;  // + work for gj_np
  size_t smem = fast ? sizeof(double2) * 18 * n * n : in_smem ? full : sizeof(double2) * 6 * n * n;
  if (df)
    k_small_cayley<DC><<<1, 1024, smem, st>>>(n, G0, P, XX, C, tmp, status, in_smem, fast);
  else
    k_small_cayley<double2><<<1, 256, smem, st>>>(n, G0, P, XX, C, tmp, status, in_smem, fast);
}

// ------------------------------------------------------- tangent velocity
// Y(xi, Z) (Sec. 5) with R = R_Q0(xi), Xp = X(R, Z), W = xi - Q0 P / 2:
//   Ups = (2 Xp - W (Q0^H Xp) + Q0 (W^H Xp)) T1,   T1 = (Q0^H R + I)^-1
//   Y   = -Q0 T2 (R + Q0)^H Ups + Ups - Q0 (Ups^H Q0),   T2 = (R^H Q0 + I)^-1 = T1^H
// Written as Ups = Xp u1 + xi u2 + Q0 u3 and Y = Xp u1 + xi u2 + Q0 c with
//   u1 = 2 T1, u2 = -A1 T1, u3 = (P A1 / 2 + A2 - P^H A1 / 2) T1,
//   Q0^H Ups = A1 u1 + P u2 + G0 u3,  R^H Ups = A4 u1 + A5 u2 + A3^H u3,
//   c = u3 - T2 (R^H Ups + Q0^H Ups) - (Q0^H Ups)^H,
// where A1 = Q0^H Xp, A2 = xi^H Xp, A3 = Q0^H R, A4 = R^H Xp, A5 = R^H xi.
// grams: [A1, A2, A3, A4, A5] (5 x n x n); output C = scale * [u1, u2, c]
// (coefficients of Xp, xi, Q0).  Inputs are read in place (global) unless
// they fit in shared memory.
template <class CT>
__global__ void k_small_tangent(int n, const double2* __restrict__ grams_g,
                                const double2* __restrict__ G0g, const double2* __restrict__ Pg,
                                double scale, double2* C, double2* tmp, int* status, int in_smem,
                                int fast) {
  extern __shared__ double2 aug_raw[];  // n x 2n, then (in_smem) 7 inputs and 8 temporaries
  CT* aug = reinterpret_cast<CT*>(aug_raw);
  const int nn = n * n, ld = 2 * n;
  const CT one = cval<CT>(1.0, 0.0), mone = cval<CT>(-1.0, 0.0), zero = cval<CT>(0.0, 0.0);
  CT* sb = aug + 2 * nn;
  CT* tb = in_smem ? sb + 7 * nn : reinterpret_cast<CT*>(tmp);
  if (in_smem) {
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      for (int q = 0; q < 5; ++q) sb[q * nn + e] = cload<CT>(grams_g[q * nn + e]);
      sb[5 * nn + e] = cload<CT>(G0g[e]);
      sb[6 * nn + e] = cload<CT>(Pg[e]);
    }
    __syncthreads();
  }
  CT *T1 = tb, *u1 = tb + nn, *u2 = tb + 2 * nn, *u3 = tb + 3 * nn, *W1 = tb + 4 * nn,
     *QU = tb + 5 * nn, *RU = tb + 6 * nn, *W2 = tb + 7 * nn;
  __shared__ CT col[64];
  __shared__ CT rowc[128];
  // the rest, on inputs of type TI (CT in shared memory, or double2 in global)
  auto body = [&](auto grams, auto G0, auto P) {
    auto A1 = grams, A2 = grams + nn, A3 = grams + 2 * nn, A4 = grams + 3 * nn, A5 = grams + 4 * nn;
    auto build = [&]() {
      for (int e = threadIdx.x; e < n * ld; e += blockDim.x) {
        int r = e / ld, c = e - r * ld;
        CT v;
        if (c < n) { v = cload<CT>(A3[r * n + c]); if (r == c) v = cadd_re(v, 1.0); }
        else v = c - n == r ? one : zero;
        aug[e] = v;
      }
      __syncthreads();
    };
    build();
    bool ok = fast && gj_np(aug, ld, n, ld, aug + 17 * nn, rowc);
    if (!ok) {
      build();
      if (!gj_solve(aug, ld, aug + n, ld, n, n, col)) {
        if (threadIdx.x == 0) vp_set_status(status, VP_ENUMERIC);
        return;
      }
    }
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      int r = e / n, c = e - r * n;
      T1[e] = aug[r * ld + n + c];
    }
    __syncthreads();
    cadd_mat(u1, 2.0, T1, 0.0, nullptr, 0, 0.0, n);
    cmm(u2, A1, 0, T1, 0, mone, 0.0, n);
    // W1 = P A1 / 2 + A2 - P^H A1 / 2
    cmm(W1, P, 0, A1, 0, cval<CT>(0.5, 0.0), 0.0, n);
    cmm(W1, P, 1, A1, 0, cval<CT>(-0.5, 0.0), 1.0, n);
    cadd_mat(W1, 1.0, W1, 1.0, A2, 0, 0.0, n);
    cmm(u3, W1, 0, T1, 0, one, 0.0, n);
    // QU = A1 u1 + P u2 + G0 u3
    cmm(QU, A1, 0, u1, 0, one, 0.0, n);
    cmm(QU, P, 0, u2, 0, one, 1.0, n);
    cmm(QU, G0, 0, u3, 0, one, 1.0, n);
    // RU = A4 u1 + A5 u2 + A3^H u3
    cmm(RU, A4, 0, u1, 0, one, 0.0, n);
    cmm(RU, A5, 0, u2, 0, one, 1.0, n);
    cmm(RU, A3, 1, u3, 0, one, 1.0, n);
    // c = u3 - T1^H (RU + QU) - QU^H
    cadd_mat(W2, 1.0, RU, 1.0, QU, 0, 0.0, n);
    cmm(W1, T1, 1, W2, 0, one, 0.0, n);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      int r = e / n, c = e - r * n;
      CT cc = csub(csub(u3[e], W1[e]), cconj(QU[c * n + r]));
      C[e] = cscale(cto(u1[e]), scale);
      C[nn + e] = cscale(cto(u2[e]), scale);
      C[2 * nn + e] = cscale(cto(cc), scale);
    }
  };
  if (in_smem) {
    body(static_cast<const CT*>(sb), static_cast<const CT*>(sb + 5 * nn),
         static_cast<const CT*>(sb + 6 * nn));
  } else if constexpr (std::is_same<CT, double2>::value) {
    body(grams_g, G0g, Pg);
  } else {  // double-float: the inputs converted once, after the temporaries in tmp
    CT* ib = tb + 8 * nn;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      for (int q = 0; q < 5; ++q) ib[q * nn + e] = cload<CT>(grams_g[q * nn + e]);
      ib[5 * nn + e] = cload<CT>(G0g[e]);
      ib[6 * nn + e] = cload<CT>(Pg[e]);
    }
    __syncthreads();
    body(static_cast<const CT*>(ib), static_cast<const CT*>(ib + 5 * nn),
         static_cast<const CT*>(ib + 6 * nn));
  }
}

void small_tangent_coeffs(int n, const double2* grams, const double2* G0, const double2* P,
                          double scale, double2* C, double2* tmp, int* status, cudaStream_t st,
                          bool df) {
  size_t full = sizeof(double2) * 17 * n * n;
  int in_smem = full <= 200 * 1024;
  int fast = in_smem && sizeof(double2) * 19 * n * n <= 200 * 1024;  // + work for gj_np
  size_t smem = fast ? sizeof(double2) * 19 * n * n : in_smem ? full : sizeof(double2) * 2 * n * n;
  if (df)
    k_small_tangent<DC><<<1, 1024, smem, st>>>(n, grams, G0, P, scale, C, tmp, status, in_smem, fast);
  else
    k_small_tangent<double2><<<1, 256, smem, st>>>(n, grams, G0, P, scale, C, tmp, status, in_smem,
                                                   fast);
}

// ------------------------------------------------- fixed-point iteration
// g = gX + G_V Ze, G_V = U_V^T U_V from the raw Gram of the stored rows
// [A | B] (U_V = [B, A]); k_new = J_2n g; |k_new - k| <= tol |k_new| stops.
__device__ __forceinline__ int vperm(int k, int n) { return k < n ? n + k : k - n; }

__device__ double block_sum2(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  __syncthreads();
  return s;
}

// Fixed-point update of the coefficient stage, spread over blocks of
// sample columns: block b owns columns [b CW, (b+1) CW) and writes
// k_new = J (gX + G_V Ze) and Ze = Z0 + dt/2 k_new for them (a column depends
// only on its own column of Ze).  kr is a ring of the iterates two to
// CU_QMAX iterations back (iterate j in slot j mod (CU_QMAX - 1)).  Each
// block leaves its sums |k_new - k|^2, |k_new|^2 and |k_new - k_{m-q}|^2
// (q = 2 .. CU_QMAX) in `partials`; the last block to finish (ticket counter)
// adds them in block order (deterministic), counts the iteration and decides:
// converged (relative update <= tol), on a q-cycle or a plateau (see
// vp_step_opts; rhist keeps the last CU_PW relative updates), non-finite
// (VP_ENUMERIC) or out of iterations (VP_ENOCONV).  Every later launch of the
// step returns at once through `done`.
#define CU_CW 1
#define CU_QMAX 4                 // longest cycle the stop rule recognises
#define CU_NP (2 + CU_QMAX - 1)   // partial sums per block
#define CU_PW 8                   // plateau window (iterations)
__global__ void k_coeff_update(int n, int p, const double* __restrict__ gX,
                               const double* __restrict__ GVraw, const double* __restrict__ Z0,
                               double* k, double* kr, double* Ze, double dt, double tol,
                               int maxit, double cycle_max, double cycle_ratio, int* done,
                               int* iters, int* ticket, double* partials, double* rhist,
                               int* status,
                               const double* __restrict__ part, int nparts, void* Z2, void* Zh2,
                               double inv_h, int zmode) {
  if (*done) return;
  // iteration number of this launch; iterate m - q exists for q <= m
  const int m_it = *iters + 1;
  const int64_t zsz = (int64_t)2 * n * p;
  extern __shared__ double cu_sm[];
  __shared__ double red[32];
  __shared__ int last;
  const int n2 = 2 * n;
  const int i0 = blockIdx.x * CU_CW, cw = min(CU_CW, p - i0);
  double* GV = cu_sm;                 // n2 x n2, G_V = U_V^T U_V
  double* Zs = cu_sm + n2 * n2;       // n2 x CU_CW, this block's columns of Ze
  double* Gs = Zs + n2 * CU_CW;       // n2 x CU_CW, projection of this block's columns
  double* Sl = Gs + n2 * CU_CW;       // slice sums of the partials
  for (int e = threadIdx.x; e < n2 * n2; e += blockDim.x) {
    int a = e / n2, b = e - a * n2;
    GV[e] = GVraw[vperm(a, n) * n2 + vperm(b, n)];
  }
  for (int e = threadIdx.x; e < n2 * cw; e += blockDim.x) {
    int r = e / cw, c = e - r * cw;
    Zs[r * CU_CW + c] = Ze[(int64_t)r * p + i0 + c];
  }
  if (part) {
    // slice sl of output o sums partials sl, sl + S, ... with eight
    // independent accumulators (many loads in flight); the slices are then
    // added in slice order (deterministic)
    const int64_t tot = (int64_t)n2 * p;
    const int nout = n2 * cw;
    const int S = max(1, (int)blockDim.x / nout);
    for (int e = threadIdx.x; e < nout * S; e += blockDim.x) {
      const int o = e % nout, sl = e / nout;
      const int r = o / cw, c = o - r * cw;
      const double* src = part + (int64_t)r * p + i0 + c;
      double a[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = 0.0;
      int b = sl;
      for (; b + 7 * S < nparts; b += 8 * S) {
#pragma unroll
        for (int u = 0; u < 8; ++u) a[u] += __ldcg(src + (int64_t)(b + u * S) * tot);
      }
      for (; b < nparts; b += S) a[0] += __ldcg(src + (int64_t)b * tot);
      Sl[o * S + sl] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    __syncthreads();
    for (int o = threadIdx.x; o < nout; o += blockDim.x) {
      const int r = o / cw, c = o - r * cw;
      double g = 0.0;
      for (int sl = 0; sl < S; ++sl) g += Sl[o * S + sl];
      Gs[r * CU_CW + c] = g;
    }
  } else {
    for (int e = threadIdx.x; e < n2 * cw; e += blockDim.x) {
      int r = e / cw, c = e - r * cw;
      Gs[r * CU_CW + c] = gX[(int64_t)r * p + i0 + c];
    }
  }
  __syncthreads();
  double d2 = 0.0, k2 = 0.0, c2[CU_QMAX - 1];
#pragma unroll
  for (int q = 0; q < CU_QMAX - 1; ++q) c2[q] = 0.0;
  // k_new[r] = g[n + r] (r < n), k_new[n + r] = -g[r], g = gX + G_V Ze
  for (int e = threadIdx.x; e < n2 * cw; e += blockDim.x) {
    int r = e / cw, c = e - r * cw;
    const int64_t o = (int64_t)r * p + i0 + c;
    int gr = r < n ? n + r : r - n;
    double sgn = r < n ? 1.0 : -1.0;
    double g = Gs[gr * CU_CW + c];
    for (int m = 0; m < n2; ++m) g = fma(GV[gr * n2 + m], Zs[m * CU_CW + c], g);
    double kn = sgn * g;
    const double kold = k[o];
    double dk = kn - kold;
    d2 = fma(dk, dk, d2);
    k2 = fma(kn, kn, k2);
#pragma unroll
    for (int q = 2; q <= CU_QMAX; ++q)
      if (q <= m_it) {
        const double dc = kn - kr[(int64_t)((m_it - q) % (CU_QMAX - 1)) * zsz + o];
        c2[q - 2] = fma(dc, dc, c2[q - 2]);
      }
    // iterate m - 1 takes the slot of iterate m - CU_QMAX, read just above
    kr[(int64_t)((m_it - 1) % (CU_QMAX - 1)) * zsz + o] = kold;
    k[o] = kn;
    const double ze = fma(0.5 * dt, kn, Z0[o]);
    Ze[o] = ze;
    if (Z2) store_lp(Z2, o, ze, zmode);
    if (Zh2) store_lp(Zh2, o, ze * inv_h, zmode);
  }
  double D2 = block_sum2(d2, red), K2 = block_sum2(k2, red), C2[CU_QMAX - 1];
#pragma unroll
  for (int q = 0; q < CU_QMAX - 1; ++q) C2[q] = block_sum2(c2[q], red);
  if (threadIdx.x == 0) {
    partials[CU_NP * blockIdx.x] = D2;
    partials[CU_NP * blockIdx.x + 1] = K2;
#pragma unroll
    for (int q = 0; q < CU_QMAX - 1; ++q) partials[CU_NP * blockIdx.x + 2 + q] = C2[q];
    __threadfence();
    last = (atomicAdd(ticket, 1) == (int)gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x >= 32) return;
  __threadfence();
  // warp 0 of the last block: lane l adds blocks l, l + 32, ...; lane 0 then
  // adds the lanes by a fixed butterfly (its order does not depend on timing)
  D2 = 0.0;
  K2 = 0.0;
#pragma unroll
  for (int q = 0; q < CU_QMAX - 1; ++q) C2[q] = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) {
    D2 += __ldcg(partials + CU_NP * b);
    K2 += __ldcg(partials + CU_NP * b + 1);
#pragma unroll
    for (int q = 0; q < CU_QMAX - 1; ++q) C2[q] += __ldcg(partials + CU_NP * b + 2 + q);
  }
  for (int o = 16; o > 0; o >>= 1) {
    D2 += __shfl_xor_sync(0xffffffffu, D2, o);
    K2 += __shfl_xor_sync(0xffffffffu, K2, o);
#pragma unroll
    for (int q = 0; q < CU_QMAX - 1; ++q) C2[q] += __shfl_xor_sync(0xffffffffu, C2[q], o);
  }
  if (threadIdx.x != 0) return;
  *ticket = 0;
  int it = *iters + 1;
  *iters = it;
  const double diff = sqrt(D2), nk = sqrt(K2);
  bool conv = diff <= tol * nk;
  // q-cycle: the iterate is back where it was q iterations ago (to tol), the
  // return distance is small against the update (a converging iteration
  // returns only to a sizeable fraction of its update), and the cycle's
  // relative amplitude is at most cycle_max; the shortest such q
  int cycle = 0;
  bool finite = isfinite(D2) && isfinite(K2);
  for (int q = 2; q <= CU_QMAX; ++q) {
    const double ret = sqrt(C2[q - 2]);
    finite = finite && isfinite(C2[q - 2]);
    if (!cycle && q <= it && cycle_max > 0.0 && ret <= tol * nk && ret <= cycle_ratio * diff &&
        diff <= cycle_max * nk)
      cycle = q;
  }
  // plateau: the relative update has not halved over CU_PW iterations
  // (r_m >= r_{m-CU_PW} / 2; r_j lives in rhist[j % CU_PW])
  const double r = nk > 0.0 ? diff / nk : 0.0;
  const bool plateau = !conv && !cycle && cycle_max > 0.0 && r <= cycle_max && it > CU_PW &&
                       r >= 0.5 * rhist[it % CU_PW];
  rhist[it % CU_PW] = r;
  if (!finite) {
    vp_set_status(status, VP_ENUMERIC);
    *done = 1;
  } else if (conv || cycle || plateau) {
    done[3] = conv ? 0 : (cycle ? cycle : 1);
    *done = 1;
  } else if (it >= maxit) {
    vp_set_status(status, VP_ENOCONV);
    *done = 1;
  }
}

// flags: [0] done, [1] iterations, [2] ticket (zero between launches),
// [3] how it stopped: 0 converged, 1 plateau, q >= 2 a q-cycle;
// kr: (CU_QMAX - 1) x 2n x p ring of earlier iterates; partials: CU_NP
// doubles per block (p blocks), then the CU_PW relative updates.
void coeff_update(int n, int p, const double* gX, const double* GVraw, const double* Z0, double* k,
                  double* kr, double* Ze, double dt, double tol, int maxit, double cycle_max,
                  double cycle_ratio, double* partials, int* done, int* iters, int* status,
                  cudaStream_t st, const double* part, int nparts, void* Z2, void* Zh2,
                  double inv_h, int zmode) {
  const int nb = (p + CU_CW - 1) / CU_CW;
  // GV, Zs, Gs and the slice sums (at most max(blockDim, 2n CU_CW) of them)
  size_t smem = sizeof(double) * (4 * n * n + 4 * (size_t)n * CU_CW + 256 + 2 * (size_t)n * CU_CW);
  k_coeff_update<<<nb, 256, smem, st>>>(n, p, gX, GVraw, Z0, k, kr, Ze, dt, tol, maxit, cycle_max,
                                        cycle_ratio, done, iters, done + 2, partials,
                                        partials + (size_t)CU_NP * nb, status, part,
                                        nparts, Z2, Zh2, inv_h, zmode);
}

// Loewdin factor G^{-1/2} of a Hermitian positive definite G close to I
// (G = Q^H Q of a basis that left the manifold by rounding only), by the
// coupled Newton-Schulz iteration Y <- Y T / 2, Zm <- T Zm / 2 with
// T = 3 I - Zm Y, from Y = G, Zm = I (Higham, Functions of Matrices, 2008,
// Sec. 6.3): Zm -> G^{-1/2} quadratically while |I - G| < 1.  Stops when
// |Zm Y - I|_F <= 1e-15 sqrt(n) (two or three iterations at a deviation of
// 1e-7).  |G - I|_F >= 0.9 sets VP_EDRIFT and returns C = I.
__global__ void k_lowdin(int n, const double2* __restrict__ G, double2* __restrict__ C,
                         int* status) {
  extern __shared__ double2 lw[];
  __shared__ double red[32];
  __shared__ int stop;
  const int nn = n * n;
  double2 *Y = lw, *Zm = lw + nn, *T = lw + 2 * nn, *U = lw + 3 * nn;
  double e2 = 0.0;
  for (int e = threadIdx.x; e < nn; e += blockDim.x) {
    const bool d = (e / n) == (e % n);
    Y[e] = G[e];
    Zm[e] = make_double2(d ? 1.0 : 0.0, 0.0);
    const double2 dv = make_double2(G[e].x - (d ? 1.0 : 0.0), G[e].y);
    e2 += cabs2(dv);
  }
  const double dev = sqrt(block_sum2(e2, red));
  if (!(dev < 0.9)) {
    if (threadIdx.x == 0) vp_set_status(status, VP_EDRIFT);
    for (int e = threadIdx.x; e < nn; e += blockDim.x) C[e] = Zm[e];
    return;
  }
  const double2 one = make_double2(1.0, 0.0), half = make_double2(0.5, 0.0);
  for (int it = 0; it < 12; ++it) {
    cmm(T, Zm, 0, Y, 0, one, 0.0, n);  // T = Zm Y
    double r2 = 0.0;
    for (int e = threadIdx.x; e < nn; e += blockDim.x) {
      const bool d = (e / n) == (e % n);
      r2 += cabs2(make_double2(T[e].x - (d ? 1.0 : 0.0), T[e].y));
    }
    const double res = sqrt(block_sum2(r2, red));
    if (threadIdx.x == 0) stop = !(res > 1e-15 * sqrt((double)n));
    __syncthreads();
    if (stop) break;
    cadd_mat(T, -1.0, T, 0.0, nullptr, 0, 3.0, n);  // T = 3 I - Zm Y
    cmm(U, Y, 0, T, 0, half, 0.0, n);               // Y T / 2
    double2* t = Y;
    Y = U;
    U = t;
    cmm(U, T, 0, Zm, 0, half, 0.0, n);  // T Zm / 2
    t = Zm;
    Zm = U;
    U = t;
  }
  for (int e = threadIdx.x; e < nn; e += blockDim.x) C[e] = Zm[e];
}

void lowdin(int n, const double2* G, double2* C, int* status, cudaStream_t st) {
  k_lowdin<<<1, 256, sizeof(double2) * 4 * n * n, st>>>(n, G, C, status);
}

// Zs (rows x nsub) = columns idx of Z (rows x p); an index outside [0, p)
// records VP_EINVAL and gives a zero column.
__global__ void k_gather_cols(int rows, int p, const double* __restrict__ Z,
                              const int32_t* __restrict__ idx, int nsub, double* __restrict__ Zs,
                              int* status) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)rows * nsub) return;
  const int r = (int)(e / nsub), j = (int)(e - (int64_t)r * nsub);
  const int c = idx[j];
  if (c < 0 || c >= p) {
    vp_set_status(status, VP_EINVAL);
    Zs[e] = 0.0;
    return;
  }
  Zs[e] = Z[(int64_t)r * p + c];
}

void gather_cols(int rows, int p, const double* Z, const int32_t* idx, int nsub, double* Zs,
                 int* status, cudaStream_t st) {
  k_gather_cols<<<ceil_div((int64_t)rows * nsub, 256), 256, 0, st>>>(rows, p, Z, idx, nsub, Zs,
                                                                     status);
}

// Greedy parameter subsample (Sec. 4.1, eq. pSampl), one block: dmin holds
// each column's distance to the chosen set; the chosen column and ties are
// resolved by a block arg-max that prefers the lowest index.
__global__ void k_param_subsample(int rows, int p, const double* __restrict__ Z, int p_max,
                                  double tol, int32_t* __restrict__ idx, int32_t* count) {
  extern __shared__ double ps_sm[];
  double* dmin = ps_sm;  // p
  __shared__ double bv[32];
  __shared__ int bi[32];
  __shared__ int pick;
  __shared__ double dfirst;
  __shared__ int stop;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5, nw = (blockDim.x + 31) >> 5;
  auto argmax = [&](const double* v) {  // largest v, lowest index on ties
    double best = -1.0;
    int bidx = 0x7fffffff;
    for (int i = t; i < p; i += blockDim.x)
      if (v[i] > best) { best = v[i]; bidx = i; }
    for (int o = 16; o > 0; o >>= 1) {
      double ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
    }
    if (lane == 0) { bv[wid] = best; bi[wid] = bidx; }
    __syncthreads();
    if (t == 0) {
      double b = -1.0;
      int k = 0x7fffffff;
      for (int w = 0; w < nw; ++w)
        if (bv[w] > b || (bv[w] == b && bi[w] < k)) { b = bv[w]; k = bi[w]; }
      pick = k;
      bv[0] = b;
    }
    __syncthreads();
  };
  auto dist = [&](int i, int j) {
    double s = 0.0;
    for (int r = 0; r < rows; ++r) {
      const double d = Z[(int64_t)r * p + i] - Z[(int64_t)r * p + j];
      s = fma(d, d, s);
    }
    return sqrt(s);
  };
  for (int i = t; i < p; i += blockDim.x) {  // norms first
    double s = 0.0;
    for (int r = 0; r < rows; ++r) s = fma(Z[(int64_t)r * p + i], Z[(int64_t)r * p + i], s);
    dmin[i] = sqrt(s);
  }
  __syncthreads();
  argmax(dmin);
  int k = pick;
  if (t == 0) { idx[0] = k; stop = 0; dfirst = -1.0; }
  for (int i = t; i < p; i += blockDim.x) dmin[i] = (i == k) ? -1.0 : dist(i, k);
  __syncthreads();
  int chosen = 1;
  while (chosen < p_max) {
    argmax(dmin);
    if (t == 0) {
      const double d = bv[0];
      if (dfirst < 0.0) dfirst = d;
      else if (d <= tol * dfirst) stop = 1;
      if (!stop) idx[chosen] = pick;
    }
    __syncthreads();
    if (stop) break;
    k = pick;
    for (int i = t; i < p; i += blockDim.x)
      if (dmin[i] >= 0.0) dmin[i] = (i == k) ? -1.0 : fmin(dmin[i], dist(i, k));
    ++chosen;
    __syncthreads();
  }
  if (t == 0) *count = chosen;
}

void param_subsample(int rows, int p, const double* Z, int p_max, double tol, int32_t* idx,
                     int32_t* count, cudaStream_t st) {
  k_param_subsample<<<1, 256, sizeof(double) * p, st>>>(rows, p, Z, p_max, tol, idx, count);
}

// Z1 = Z0 + dt k
__global__ void k_axpy(int64_t m, double a, const double* x, const double* y, double* out) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < m) out[e] = fma(a, x[e], y[e]);
}
void axpy(int64_t m, double a, const double* x, const double* y, double* out, cudaStream_t st) {
  k_axpy<<<ceil_div(m, 256), 256, 0, st>>>(m, a, x, y, out);
}

// g = gX + G_V Z (2n x p), G_V = U_V^T U_V from the raw Gram; gX may be null.
__global__ void k_add_linear(int n, int p, const double* __restrict__ gX,
                             const double* __restrict__ GVraw, const double* __restrict__ Z,
                             double* __restrict__ g) {
  const int n2 = 2 * n;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n2 * p) return;
  int r = (int)(e / p), i = (int)(e - (int64_t)r * p);
  double s = gX ? gX[e] : 0.0;
  const int pr = vperm(r, n);
  for (int c = 0; c < n2; ++c) s = fma(GVraw[pr * n2 + vperm(c, n)], Z[(int64_t)c * p + i], s);
  g[e] = s;
}
void add_linear(int n, int p, const double* gX, const double* GVraw, const double* Z, double* g,
                cudaStream_t st) {
  int64_t m = (int64_t)2 * n * p;
  k_add_linear<<<ceil_div(m, 256), 256, 0, st>>>(n, p, gX, GVraw, Z, g);
}

__global__ void k_sqrt_nonneg(int m, const double* x, double* out) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < m) out[e] = sqrt(fmax(x[e], 0.0));
}
void sqrt_nonneg(int m, const double* x, double* out, cudaStream_t st) {
  k_sqrt_nonneg<<<ceil_div(m, 256), 256, 0, st>>>(m, x, out);
}

// --------------------------------------------------------------- energies
// E_out[i] = Efield[i], H_out[i] = 1/2 Z_i^T G_V Z_i + Efield[i];
// resid = |Q^H Q - I|_F from the complex Gram QhQ (nullable).  Block i takes
// sample i (the FP64 work spread over the SMs): thread a forms
// s_a = sum_b G_V[a][b] z_b in order, and the block adds z_a s_a in a fixed
// tree (deterministic).  Block 0 also forms the residual.
#define EN_THREADS 128
__global__ void __launch_bounds__(EN_THREADS)
k_energies(int n, int p, const double* __restrict__ GVraw, const double* __restrict__ Z,
           const double* __restrict__ Efield, double* E_out, double* H_out, int64_t stride,
           const double2* __restrict__ QhQ, double* resid, int* status) {
  __shared__ double red[32];
  const int n2 = 2 * n, i = blockIdx.x;
  double part = 0.0;
  for (int a = threadIdx.x; a < n2 && i < p; a += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < n2; ++b) s = fma(GVraw[vperm(a, n) * n2 + vperm(b, n)], Z[(int64_t)b * p + i], s);
    part = fma(Z[(int64_t)a * p + i], s, part);
  }
  const double kin = block_sum2(part, red);
  if (threadIdx.x == 0 && i < p) {
    const double E = Efield[i];
    const double H = 0.5 * kin + E;
    if (E_out) E_out[i * stride] = E;
    if (H_out) H_out[i * stride] = H;
    if (!isfinite(H)) vp_set_status(status, VP_ENUMERIC);
  }
  if (QhQ && resid && blockIdx.x == 0) {
    double s = 0.0;
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
      int r = e / n, c = e - r * n;
      double2 v = QhQ[e];
      if (r == c) v.x -= 1.0;
      s += cabs2(v);
    }
    double tot = block_sum2(s, red);
    if (threadIdx.x == 0) *resid = sqrt(tot);
  }
}

void energies(int n, int p, const double* GVraw, const double* Z, const double* Efield,
              double* E_out, double* H_out, int64_t stride, const double2* QhQ, double* resid,
              int* status, cudaStream_t st) {
  k_energies<<<p > 0 ? p : 1, EN_THREADS, 0, st>>>(n, p, GVraw, Z, Efield, E_out, H_out, stride, QhQ, resid,
                                       status);
}

void dense_init() {
  cudaFuncSetAttribute(k_small_basis_coeffs<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_small_cayley<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_small_tangent<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_small_basis_coeffs<DC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_small_cayley<DC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_small_tangent<DC>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_coeff_update, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_lowdin, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

}  // namespace vpk
