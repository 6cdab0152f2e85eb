// Per-step calls on N-row inputs of a stated element type (vp_dtype): the
// charge deposit (Sec. 2.1, eq. PoissonSystem), the gather of the field
// gradient (eq. VPHamEqn), the reconstruction X_r = U_X Z, V_r = U_V Z and
// the projection g = U^T [G_X; V_r] (Sec. 3.2, eq. grads) with positions,
// basis rows and gradients in FP64, FP32 or BF16.
//
// Element types and arithmetic:
// - the deposit and the gather convert each position to FP64 and then take
//   the same cell and fixed-point weight as the FP64 calls, so their results
//   are those of the FP64 calls on the rounded positions (the deposit
//   exactly, the gather up to the rounding of its output to the type);
// - the reconstruction and the projection multiply and accumulate in FP64
//   for FP64 inputs and in FP32 for FP32 and BF16 inputs (BF16 products are
//   exact in FP32); the projection's per-block partial sums are added in
//   FP64 in block order, and its V part goes through the Gram matrix
//   U_V^T U_V, accumulated the same way.
#include <cuda_bf16.h>

#include "vp_internal.cuh"

#include <algorithm>

namespace vpk {
namespace {

template <class T>
__device__ __forceinline__ double to_f64(T v) { return (double)v; }
template <>
__device__ __forceinline__ double to_f64<__nv_bfloat16>(__nv_bfloat16 v) {
  return (double)__bfloat162float(v);
}
template <class T, class A>
__device__ __forceinline__ A to_acc(T v) { return (A)v; }
template <>
__device__ __forceinline__ float to_acc<__nv_bfloat16, float>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <class T>
__device__ __forceinline__ T from_f64(double v) { return (T)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 from_f64<__nv_bfloat16>(double v) {
  return __double2bfloat16(v);
}
// accumulation type: FP64 for FP64 inputs, FP32 otherwise
template <class T> struct Acc { using type = float; };
template <> struct Acc<double> { using type = double; };

// ---------------------------------------------------------------- deposit
template <class T>
__global__ void k_deposit_t(GridC g, int64_t N, const T* __restrict__ X, int64_t ldx,
                            unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned long long sc[];
  const int i = blockIdx.y;
  for (int c = threadIdx.x; c < g.Nx; c += blockDim.x) sc[c] = 0ull;
  __syncthreads();
  const T* x = X + (int64_t)i * ldx;
  const unsigned long long one = 1ull << g.S;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
       l += (int64_t)gridDim.x * blockDim.x) {
    int j;
    double s;
    cell_of(to_f64(x[l]), g.inv_h, g.Nx, g.dNx, g.inv_Nx, j, s);
    const unsigned long long w1 = (unsigned long long)__double2ll_rn(s * g.fp_scale);
    const int j1 = (j + 1 == g.Nx) ? 0 : j + 1;
    atomicAdd(&sc[j], one - w1);
    atomicAdd(&sc[j1], w1);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < g.Nx; c += blockDim.x)
    if (sc[c]) atomicAdd(&counts[(int64_t)i * g.Nx + c], sc[c]);
}

// ----------------------------------------------------------------- gather
template <class T>
__global__ void k_gather_t(GridC g, int64_t N, const T* __restrict__ X, int64_t ldx,
                           const double* __restrict__ F, const int32_t* __restrict__ idx,
                           int64_t d, T* __restrict__ GX, int* status) {
  extern __shared__ double sF[];
  const int i = blockIdx.y;
  for (int c = threadIdx.x; c < g.Nx; c += blockDim.x) sF[c] = g.qm * F[(int64_t)i * g.Nx + c];
  __syncthreads();
  const T* x = X + (int64_t)i * ldx;
  const int64_t cnt = idx ? d : N;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < cnt;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t l = idx ? (int64_t)idx[r] : r;
    if (l < 0 || l >= N) {  // a DEIM index outside the particle range
      vp_set_status(status, VP_EINVAL);
      GX[(int64_t)i * cnt + r] = from_f64<T>(0.0);
      continue;
    }
    int j;
    double s;
    cell_of(to_f64(x[l]), g.inv_h, g.Nx, g.dNx, g.inv_Nx, j, s);
    GX[(int64_t)i * cnt + r] = from_f64<T>(sF[j]);
  }
}

// ------------------------------------------------------------ reconstruct
// X_li = sum_k A_lk a_ki - B_lk b_ki, V_li = sum_k B_lk a_ki + A_lk b_ki:
// one thread per (row, sample), rows of Q (ld ldq) staged per tile.
constexpr int kTRows = 64;
template <class T>
__global__ void k_reconstruct_t(int64_t N, int n, int p, const T* __restrict__ Q, int64_t ldq,
                                const double* __restrict__ Z, T* __restrict__ X,
                                T* __restrict__ V, int64_t ldx) {
  using A = typename Acc<T>::type;
  extern __shared__ __align__(16) unsigned char smt[];
  const int n2 = 2 * n;
  A* Zs = reinterpret_cast<A*>(smt);  // n2 x 32 (this block's samples)
  A* Qs = Zs + n2 * 32;               // kTRows x (n2 + 1)
  const int c0 = blockIdx.y * 32, ii = threadIdx.x & 31, rsub = threadIdx.x >> 5;
  const int RP = blockDim.x >> 5;
  for (int e = threadIdx.x; e < n2 * 32; e += blockDim.x) {
    const int k = e >> 5, c = e & 31;
    Zs[e] = (c0 + c < p) ? (A)Z[(int64_t)k * p + c0 + c] : (A)0;
  }
  for (int64_t base = (int64_t)blockIdx.x * kTRows; base < N; base += (int64_t)gridDim.x * kTRows) {
    const int rows = (int)(N - base < (int64_t)kTRows ? N - base : (int64_t)kTRows);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
      const int r = e / n2, k = e - r * n2;
      Qs[r * (n2 + 1) + k] = to_acc<T, A>(Q[(base + r) * ldq + k]);
    }
    __syncthreads();
    if (c0 + ii >= p) continue;
    for (int r = rsub; r < rows; r += RP) {
      const A* q = Qs + r * (n2 + 1);
      A x = 0, v = 0;
      for (int k = 0; k < n; ++k) {
        const A a = Zs[k * 32 + ii], b = Zs[(n + k) * 32 + ii];
        x = fma(q[k], a, x);
        x = fma(-q[n + k], b, x);
        v = fma(q[n + k], a, v);
        v = fma(q[k], b, v);
      }
      const int64_t o = (int64_t)(c0 + ii) * ldx + base + r;
      X[o] = from_f64<T>((double)x);
      if (V) V[o] = from_f64<T>((double)v);
    }
  }
}

// ------------------------------------------------- projection (X part)
// part[bx][k][i] = sum over the block's rows l of U_X,lk GX_il with
// U_X,l = [A_l, -B_l]: per tile of kTRows rows the Q rows and the GX values
// of this block's 32 samples are staged, thread (k, c) pairs accumulate.
template <class T>
__global__ void k_project_t(int64_t N, int n, int p, const T* __restrict__ Q, int64_t ldq,
                            const T* __restrict__ GX, int64_t ldg, double* __restrict__ part) {
  using A = typename Acc<T>::type;
  extern __shared__ __align__(16) unsigned char smt[];
  const int n2 = 2 * n;
  A* Qs = reinterpret_cast<A*>(smt);  // kTRows x (n2 + 1)
  A* Gs = Qs + kTRows * (n2 + 1);     // kTRows x 33
  const int c0 = blockIdx.y * 32;
  const int npairs = n2 * 32;
  constexpr int kMaxAcc = 20;  // n2 * 32 <= 80 * 32 = kMaxAcc * 128
  A acc[kMaxAcc];
#pragma unroll
  for (int a = 0; a < kMaxAcc; ++a) acc[a] = 0;
  for (int64_t base = (int64_t)blockIdx.x * kTRows; base < N; base += (int64_t)gridDim.x * kTRows) {
    const int rows = (int)(N - base < (int64_t)kTRows ? N - base : (int64_t)kTRows);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * n2; e += blockDim.x) {
      const int r = e / n2, k = e - r * n2;
      Qs[r * (n2 + 1) + k] = to_acc<T, A>(Q[(base + r) * ldq + k]);
    }
    for (int e = threadIdx.x; e < rows * 32; e += blockDim.x) {
      const int c = e / rows, r = e - c * rows;
      Gs[r * 33 + c] = (c0 + c < p) ? to_acc<T, A>(GX[(int64_t)(c0 + c) * ldg + base + r]) : (A)0;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < kMaxAcc; ++a) {
      const int e = threadIdx.x + a * blockDim.x;
      if (e < npairs) {
        const int k = e >> 5, c = e & 31;
        A s = 0;
        for (int r = 0; r < rows; ++r) s = fma(Qs[r * (n2 + 1) + k], Gs[r * 33 + c], s);
        acc[a] += s;
      }
    }
  }
#pragma unroll
  for (int a = 0; a < kMaxAcc; ++a) {
    const int e = threadIdx.x + a * blockDim.x;
    if (e < npairs) {
      const int k = e >> 5, c = e & 31;
      if (c0 + c < p) {
        const double v = (double)acc[a];
        part[(int64_t)blockIdx.x * n2 * p + (int64_t)k * p + c0 + c] = (k < n) ? v : -v;
      }
    }
  }
}

// Real Gram [A B]^T [A B] of the N x 2n rows (ld ldq), per-block partials.
template <class T>
__global__ void k_gram_real_t(int64_t N, int m, const T* __restrict__ Q, int64_t ldq,
                              double* __restrict__ part) {
  using A = typename Acc<T>::type;
  extern __shared__ __align__(16) unsigned char smt[];
  A* sm = reinterpret_cast<A*>(smt);  // kTRows x (m + 1)
  const int total = m * m;
  constexpr int kMaxAcc = 50;  // m * m <= 6400 = kMaxAcc * 128
  A acc[kMaxAcc];
#pragma unroll
  for (int a = 0; a < kMaxAcc; ++a) acc[a] = 0;
  for (int64_t base = (int64_t)blockIdx.x * kTRows; base < N; base += (int64_t)gridDim.x * kTRows) {
    const int rows = (int)(N - base < (int64_t)kTRows ? N - base : (int64_t)kTRows);
    __syncthreads();
    for (int e = threadIdx.x; e < rows * m; e += blockDim.x) {
      const int r = e / m, k = e - r * m;
      sm[r * (m + 1) + k] = to_acc<T, A>(Q[(base + r) * ldq + k]);
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < kMaxAcc; ++a) {
      const int e = threadIdx.x + a * blockDim.x;
      if (e < total) {
        const int k1 = e / m, k2 = e - k1 * m;
        A s = 0;
        for (int r = 0; r < rows; ++r) s = fma(sm[r * (m + 1) + k1], sm[r * (m + 1) + k2], s);
        acc[a] += s;
      }
    }
  }
#pragma unroll
  for (int a = 0; a < kMaxAcc; ++a) {
    const int e = threadIdx.x + a * blockDim.x;
    if (e < total) part[(int64_t)blockIdx.x * total + e] = (double)acc[a];
  }
}

}  // namespace

static int typed_size(int dtype) { return dtype == 0 ? 8 : dtype == 1 ? 4 : 2; }
int vp_dtype_size(int dtype) { return typed_size(dtype); }

#define VP_TYPED_DISPATCH(dtype, ...)                          \
  do {                                                          \
    if ((dtype) == 0) { using T = double; __VA_ARGS__; }        \
    else if ((dtype) == 1) { using T = float; __VA_ARGS__; }    \
    else { using T = __nv_bfloat16; __VA_ARGS__; }              \
  } while (0)

void deposit_typed(const GridC& g, int64_t N, int p, const void* X, int64_t ldx, int dtype,
                   unsigned long long* counts, int num_sms, cudaStream_t st) {
  int bx = (int)std::min<int64_t>(ceil_div(N, 256 * 8), (2 * num_sms + p - 1) / p);
  if (bx < 1) bx = 1;
  VP_TYPED_DISPATCH(dtype, (k_deposit_t<T><<<dim3(bx, p), 256, g.Nx * sizeof(unsigned long long), st>>>(
                                g, N, static_cast<const T*>(X), ldx, counts)));
}

void gather_typed(const GridC& g, int64_t N, int p, const void* X, int64_t ldx, int dtype,
                  const double* F, const int32_t* idx, int64_t d, void* GX, int num_sms,
                  int* status, cudaStream_t st) {
  const int64_t cnt = idx ? d : N;
  int bx = (int)std::min<int64_t>(ceil_div(cnt, 256 * 4), (4 * num_sms + p - 1) / p);
  if (bx < 1) bx = 1;
  VP_TYPED_DISPATCH(dtype, (k_gather_t<T><<<dim3(bx, p), 256, g.Nx * sizeof(double), st>>>(
                                g, N, static_cast<const T*>(X), ldx, F, idx, d, static_cast<T*>(GX),
                                status)));
}

void reconstruct_typed(int64_t N, int n, int p, const void* Q, int64_t ldq, int dtype,
                       const double* Z, void* X, void* V, int64_t ldx, int num_sms,
                       cudaStream_t st) {
  const int ch = ceil_div(p, 32), n2 = 2 * n;
  int gx = (int)std::min<int64_t>(ceil_div(N, kTRows), std::max(1, 4 * num_sms / ch));
  if (gx < 1) gx = 1;
  VP_TYPED_DISPATCH(dtype, {
    using A = typename Acc<T>::type;
    const size_t smem = sizeof(A) * ((size_t)n2 * 32 + (size_t)kTRows * (n2 + 1));
    k_reconstruct_t<T><<<dim3(gx, ch), 256, smem, st>>>(N, n, p, static_cast<const T*>(Q), ldq, Z,
                                                         static_cast<T*>(X), static_cast<T*>(V), ldx);
  });
}

void project_typed(int64_t N, int n, int p, const void* Q, int64_t ldq, int dtype, const void* GX,
                   int64_t ldg, double* part, int gridx, cudaStream_t st) {
  const int ch = ceil_div(p, 32), n2 = 2 * n;
  VP_TYPED_DISPATCH(dtype, {
    using A = typename Acc<T>::type;
    const size_t smem = sizeof(A) * ((size_t)kTRows * (n2 + 1) + (size_t)kTRows * 33);
    k_project_t<T><<<dim3(gridx, ch), 128, smem, st>>>(N, n, p, static_cast<const T*>(Q), ldq,
                                                        static_cast<const T*>(GX), ldg, part);
  });
}

void gram_real_typed(int64_t N, int m, const void* Q, int64_t ldq, int dtype, double* part,
                     int gridx, cudaStream_t st) {
  VP_TYPED_DISPATCH(dtype, {
    using A = typename Acc<T>::type;
    const size_t smem = sizeof(A) * (size_t)kTRows * (m + 1);
    k_gram_real_t<T><<<gridx, 128, smem, st>>>(N, m, static_cast<const T*>(Q), ldq, part);
  });
}

// grid of the typed projection and Gram: about two blocks per SM over the row tiles
int typed_grid_x(int64_t N, int chunks, int num_sms) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(N, kTRows),
                                                      std::max(1, 2 * num_sms / chunks)));
}

}  // namespace vpk
