// Loading of macro-particles on the device (Sec. 6.1, eq.
// initial_distribution): particle l of sample i takes x = F_x^-1(u_x) and
// v = F_v^-1(u_v), with F_x the CDF of (1 + alpha cos kx)/L on [0, L) and F_v
// the CDF of a Gaussian mixture truncated to [-10, 10].  Quiet start: u_x =
// phi_2(l) (base-2 radical inverse), u_v = (l + 1/2)/N (the 2-D Hammersley
// set).  Seeded: one Philox4x32-10 block per particle (Salmon et al., SC 2011),
// counter (l mod 2^32, l div 2^32, i, 0), key (seed mod 2^32, seed div 2^32);
// u_x from words 0-1 and u_v from words 2-3 as 53-bit doubles.  Inverses by
// bisection on the bracket, finished by safeguarded Newton steps.
#include "vp_internal.cuh"

namespace vpk {

struct Mix {
  double w[2], m[2], s[2];
  int nc;
  double lo_mass, norm;
};

__device__ double mix_cdf_raw(const Mix& M, double v) {
  double c = 0.0;
  for (int q = 0; q < M.nc; ++q) c += M.w[q] * 0.5 * erfc(-(v - M.m[q]) / (M.s[q] * 1.4142135623730951));
  return c;
}
__device__ double mix_pdf(const Mix& M, double v) {
  double d = 0.0;
  for (int q = 0; q < M.nc; ++q) {
    double z = (v - M.m[q]) / M.s[q];
    d += M.w[q] * exp(-0.5 * z * z) / (2.5066282746310002 * M.s[q]);
  }
  return d / M.norm;
}

// family: 0 Landau (alpha, sigma), 1 two-stream (v0, sigma, alpha),
// 2 bump-on-tail (vb, alpha, sigma_b); eta: p x 3.
__device__ void family_params(int family, const double* eta, double& alpha, Mix& M) {
  M.nc = 1;
  if (family == 0) {
    alpha = eta[0];
    M.w[0] = 1.0; M.m[0] = 0.0; M.s[0] = eta[1];
  } else if (family == 1) {
    alpha = eta[2];
    M.nc = 2;
    M.w[0] = 0.5; M.m[0] = eta[0]; M.s[0] = eta[1];
    M.w[1] = 0.5; M.m[1] = -eta[0]; M.s[1] = eta[1];
  } else {
    alpha = eta[1];
    M.nc = 2;
    M.w[0] = 0.9; M.m[0] = 0.0; M.s[0] = 1.0;
    M.w[1] = 0.1; M.m[1] = eta[0]; M.s[1] = eta[2];
  }
  M.lo_mass = 0.0;
  M.norm = 1.0;
  double lo = mix_cdf_raw(M, -10.0), hi = mix_cdf_raw(M, 10.0);
  M.lo_mass = lo;
  M.norm = hi - lo;
}

// Philox4x32 with 10 rounds: round constants 0xD2511F53, 0xCD9E8D57, key
// increments 0x9E3779B9, 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
  return ((double)(a >> 5) * 67108864.0 + (double)(b >> 6)) * (1.0 / 9007199254740992.0);
}

// mode 0: quiet start; mode 1: Philox with key `seed`.
__global__ void k_load(int family, int mode, unsigned long long seed, double k, int64_t N,
                       const double* __restrict__ eta, double* __restrict__ X,
                       double* __restrict__ V) {
  const int i = blockIdx.y;
  double alpha;
  Mix M;
  family_params(family, eta + 3 * i, alpha, M);
  const double L = 2.0 * 3.141592653589793 / k;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
       l += (int64_t)gridDim.x * blockDim.x) {
    double ux, uv;
    if (mode == 0) {
      // radical inverse base 2 of l
      unsigned long long b = (unsigned long long)l;
      double f = 0.5;
      ux = 0.0;
      while (b) {
        if (b & 1ull) ux += f;
        b >>= 1;
        f *= 0.5;
      }
      uv = ((double)l + 0.5) / (double)N;
    } else {
      const unsigned long long ul = (unsigned long long)l;
      const uint4 w = philox4x32_10(make_uint4((uint32_t)ul, (uint32_t)(ul >> 32), (uint32_t)i, 0u),
                                    make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
      ux = u53(w.x, w.y);
      uv = u53(w.z, w.w);
    }
    // x: solve x + (alpha/k) sin(kx) = ux L on [0, L]
    double a = 0.0, c = L, x = ux * L;
    for (int it = 0; it < 60; ++it) {
      double g = x + alpha / k * sin(k * x) - ux * L;
      if (g < 0.0) a = x; else c = x;
      double d = 1.0 + alpha * cos(k * x);
      double xn = x - g / d;
      if (!(xn > a && xn < c)) xn = 0.5 * (a + c);
      if (fabs(xn - x) <= 1e-15 * fmax(1.0, fabs(x))) { x = xn; break; }
      x = xn;
    }
    if (x >= L) x = nextafter(L, 0.0);
    if (x < 0.0) x = 0.0;
    // v: solve F_v(v) = uv on [-10, 10]
    double va = -10.0, vc = 10.0;
    for (int it = 0; it < 36; ++it) {  // bisection to a bracket of ~3e-10
      const double m = 0.5 * (va + vc);
      if ((mix_cdf_raw(M, m) - M.lo_mass) / M.norm < uv) va = m; else vc = m;
    }
    // Newton polish from the bracket's midpoint; a step may leave the bracket
    // by at most its width (the root can sit on an end point)
    const double w = vc - va;
    double v = 0.5 * (va + vc);
    for (int it = 0; it < 4; ++it) {
      double g = (mix_cdf_raw(M, v) - M.lo_mass) / M.norm - uv;
      double d = mix_pdf(M, v);
      if (!(d > 0.0)) break;
      double vn = v - g / d;
      if (vn < va - w || vn > vc + w) break;
      v = vn;
    }
    X[(int64_t)i * N + l] = x;
    V[(int64_t)i * N + l] = v;
  }
}

void load_particles(int family, int mode, unsigned long long seed, double k, int64_t N, int p,
                    const double* eta, double* X, double* V, int num_sms, cudaStream_t st) {
  int bx = ceil_div(N, 256);
  int want = (4 * num_sms + p - 1) / p;
  if (bx > want) bx = want;
  if (bx < 1) bx = 1;
  k_load<<<dim3(bx, p), 256, 0, st>>>(family, mode, seed, k, N, eta, X, V);
}

}  // namespace vpk
