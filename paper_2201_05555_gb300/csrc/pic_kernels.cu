// Particle <-> grid kernels of the geometric PIC discretisation (Sec. 2.1)
// and the full-order Stormer-Verlet step (Sec. 5, eq. sv_full_order).
#include "vp_internal.cuh"

#include <cooperative_groups.h>

namespace cg = cooperative_groups;

namespace vpk {

GridC make_gridc(const vp_grid& gr, int64_t N) {
  GridC g;
  g.Nx = gr.Nx;
  g.L = gr.L;
  g.h = gr.L / gr.Nx;
  g.inv_h = 1.0 / g.h;
  g.dNx = (double)gr.Nx;
  g.inv_Nx = 1.0 / g.dNx;
  g.Mq = gr.Mq;
  g.mp = gr.mp;
  g.qm = gr.Mq / gr.mp;
  g.bg_load = gr.background * g.h;
  g.S = fixed_point_bits(N);
  g.fp_scale = ldexp(1.0, g.S);
  g.fp_inv = ldexp(1.0, -g.S);
  // packed FP32 deposit: the weight sums of a cell stay below 2^(Sp + bl)
  // and the count below 2^bl (bl = bit length of N), so Sp + 2 bl <= 63
  int bl = 0;
  while (bl < 62 && (int64_t(1) << bl) <= N) ++bl;
  g.Sp = std::min(24, 63 - 2 * bl);
  if (g.Sp < 8) {
    g.Sp = 0;
    g.Kp = 0;
  } else {
    g.Kp = g.Sp + bl;
  }
  return g;
}

// ------------------------------------------------------------------ scans
// Block-wide inclusive prefix sum of a[0..n) in shared memory (blockDim.x a
// multiple of 32, n <= VP_MAX_NX).  Thread t owns a contiguous segment; the
// summation order is fixed, so results are deterministic.
__device__ void block_inclusive_scan(double* a, int n, double* warp_tot) {
  const int nt = blockDim.x, t = threadIdx.x;
  const int seg = (n + nt - 1) / nt;
  const int b = t * seg, e = min(n, b + seg);
  double run = 0.0;
  for (int c = b; c < e; ++c) { run += a[c]; a[c] = run; }
  // exclusive scan of segment totals
  const int lane = t & 31, w = t >> 5;
  double x = run;
  for (int o = 1; o < 32; o <<= 1) {
    double y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  if (w == 0) {
    double y = lane < (nt >> 5) ? warp_tot[lane] : 0.0;
    for (int o = 1; o < 32; o <<= 1) {
      double z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    if (lane < (nt >> 5)) warp_tot[lane] = y;  // inclusive warp prefix
  }
  __syncthreads();
  double off = (x - run) + (w > 0 ? warp_tot[w - 1] : 0.0);
  for (int c = b; c < e; ++c) a[c] += off;
  __syncthreads();
}

// Deterministic block sum of a[0..n).
__device__ double block_sum(const double* a, int n, double* red) {
  const int t = threadIdx.x, nt = blockDim.x;
  const int seg = (n + nt - 1) / nt;
  double s = 0.0;
  for (int c = t * seg; c < min(n, t * seg + seg); ++c) s += a[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((t & 31) == 0) red[t >> 5] = s;
  __syncthreads();
  double tot = 0.0;
  for (int w = 0; w < (nt >> 5); ++w) tot += red[w];
  __syncthreads();
  return tot;
}

// Periodic P1 Poisson by prefix sums.  On entry a[0..Nx) = rho.  On exit
// a = F (cell derivative of phi); returns the electric energy.  If phi is
// non-null it receives the nodal potential with zero mean.
// -(F_j - F_{j-1}) = rho_j  =>  F_j = mean(S) - S_j,  S_j = sum_{k<=j} rho_k,
// and the mean of F vanishes because phi is periodic.
__device__ double poisson_inplace(const GridC& g, double* a, double* tmp, double* red,
                                  double* phi_out) {
  const int Nx = g.Nx;
  block_inclusive_scan(a, Nx, red);
  double meanS = block_sum(a, Nx, red) / Nx;
  for (int c = threadIdx.x; c < Nx; c += blockDim.x) a[c] = meanS - a[c];
  __syncthreads();
  // energy = (h / (2 mp)) sum F^2
  for (int c = threadIdx.x; c < Nx; c += blockDim.x) tmp[c] = a[c] * a[c];
  __syncthreads();
  double e = 0.5 * g.h / g.mp * block_sum(tmp, Nx, red);
  if (phi_out) {
    // phi_j = phi_0 + h sum_{k<j} F_k, then remove the mean
    for (int c = threadIdx.x; c < Nx; c += blockDim.x) tmp[c] = (c == 0) ? 0.0 : g.h * a[c - 1];
    __syncthreads();
    block_inclusive_scan(tmp, Nx, red);
    double m = block_sum(tmp, Nx, red) / Nx;
    for (int c = threadIdx.x; c < Nx; c += blockDim.x) phi_out[c] = tmp[c] - m;
    __syncthreads();
  }
  return e;
}

// ---------------------------------------------------------------- deposit
__global__ void k_deposit(GridC g, int64_t N, const double* __restrict__ X, int64_t ldx,
                          unsigned long long* __restrict__ counts) {
  extern __shared__ unsigned long long sc[];
  const int i = blockIdx.y;
  for (int c = threadIdx.x; c < g.Nx; c += blockDim.x) sc[c] = 0ull;
  __syncthreads();
  const double* x = X + (int64_t)i * ldx;
  const unsigned long long one = 1ull << g.S;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < N;
       l += (int64_t)gridDim.x * blockDim.x) {
    int j;
    double s;
    cell_of(__ldg(x + l), g.inv_h, g.Nx, g.dNx, g.inv_Nx, j, s);
    unsigned long long w1 = (unsigned long long)__double2ll_rn(s * g.fp_scale);
    int j1 = (j + 1 == g.Nx) ? 0 : j + 1;
    atomicAdd(&sc[j], one - w1);
    atomicAdd(&sc[j1], w1);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < g.Nx; c += blockDim.x)
    if (sc[c]) atomicAdd(&counts[(int64_t)i * g.Nx + c], sc[c]);
}

void deposit_samples(const GridC& g, int64_t N, int p, const double* X, int64_t ldx,
                     unsigned long long* counts, int num_sms, cudaStream_t st) {
  const int bs = 256;
  int bx = ceil_div(N, bs * 8);
  int want = (2 * num_sms + p - 1) / p;
  if (bx > want) bx = want;
  if (bx < 1) bx = 1;
  k_deposit<<<dim3(bx, p), bs, g.Nx * sizeof(unsigned long long), st>>>(g, N, X, ldx, counts);
}

__global__ void k_counts_to_rho(GridC g, int p, const unsigned long long* counts, double* rho) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < (int64_t)p * g.Nx) rho[e] = g.Mq * ((double)counts[e] * g.fp_inv) + g.bg_load;
}

void counts_to_rho(const GridC& g, int p, const unsigned long long* counts, double* rho,
                   cudaStream_t st) {
  int64_t n = (int64_t)p * g.Nx;
  k_counts_to_rho<<<ceil_div(n, 256), 256, 0, st>>>(g, p, counts, rho);
}

// The same two launches through cudaLaunchKernel, whose return value is the
// launch's own error (the allocation-free deposit reports it without reading
// an error that earlier, unrelated work left pending on the thread).
cudaError_t deposit_samples_launch(const GridC& g, int64_t N, int p, const double* X, int64_t ldx,
                                   unsigned long long* counts, int num_sms, cudaStream_t st) {
  const int bs = 256;
  int bx = ceil_div(N, bs * 8);
  int want = (2 * num_sms + p - 1) / p;
  if (bx > want) bx = want;
  if (bx < 1) bx = 1;
  GridC ga = g;
  int64_t Na = N, lda = ldx;
  const double* Xa = X;
  unsigned long long* ca = counts;
  void* args[] = {&ga, &Na, &Xa, &lda, &ca};
  return cudaLaunchKernel((const void*)k_deposit, dim3(bx, p), dim3(bs),
                          args, g.Nx * sizeof(unsigned long long), st);
}

cudaError_t counts_to_rho_launch(const GridC& g, int p, const unsigned long long* counts,
                                 double* rho, cudaStream_t st) {
  const int64_t n = (int64_t)p * g.Nx;
  GridC ga = g;
  int pa = p;
  const unsigned long long* ca = counts;
  double* ra = rho;
  void* args[] = {&ga, &pa, &ca, &ra};
  return cudaLaunchKernel((const void*)k_counts_to_rho, dim3((unsigned)ceil_div(n, 256)), dim3(256),
                          args, 0, st);
}

// ---------------------------------------------------------------- Poisson
// One block per sample.  Input either rho (double) or fixed-point counts.
// F2 (nullable): (q/m) F also in the row format f2mode of the FP32-based
// forms (1 double-float, 2 FP32), for their projection and basis kernels.
__global__ void k_poisson(GridC g, const double* __restrict__ rho,
                          const unsigned long long* __restrict__ counts, double* phi, double* F,
                          double* energy, unsigned long long* zero_counts, const int* skip,
                          int* status, void* F2, int f2mode) {
  if (skip && *skip) return;
  __shared__ double a[VP_MAX_NX];
  __shared__ double tmp[VP_MAX_NX];
  __shared__ double red[32];
  const int i = blockIdx.x, Nx = g.Nx;
  const int64_t base = (int64_t)i * Nx;
  if (!rho && f2mode == 2 && g.Kp > 0) {
    // packed FP32 counts: node count_c = n_c 2^Sp - W_c + W_{c-1} (periodic)
    const unsigned long long mask = (1ull << g.Kp) - 1ull;
    for (int c = threadIdx.x; c < Nx; c += blockDim.x) {
      const unsigned long long P = counts[base + c];
      a[c] = (double)(P >> g.Kp);
      tmp[c] = (double)(P & mask);
    }
    __syncthreads();
    const double one = ldexp(1.0, g.Sp), inv = ldexp(1.0, -g.Sp);
    double nc[VP_MAX_NX / 256 + 1];
    int q = 0;
    for (int c = threadIdx.x; c < Nx; c += blockDim.x, ++q)
      nc[q] = fma(a[c], one, tmp[c == 0 ? Nx - 1 : c - 1] - tmp[c]);  // exact integers
    __syncthreads();
    q = 0;
    for (int c = threadIdx.x; c < Nx; c += blockDim.x, ++q) a[c] = g.Mq * (nc[q] * inv) + g.bg_load;
  } else {
    for (int c = threadIdx.x; c < Nx; c += blockDim.x) {
      double r = rho ? rho[base + c] : g.Mq * ((double)counts[base + c] * g.fp_inv) + g.bg_load;
      a[c] = r;
    }
  }
  __syncthreads();
  if (zero_counts)
    for (int c = threadIdx.x; c < Nx; c += blockDim.x) zero_counts[base + c] = 0ull;
  double e = poisson_inplace(g, a, tmp, red, phi ? phi + base : nullptr);
  for (int c = threadIdx.x; c < Nx; c += blockDim.x) F[base + c] = a[c];
  if (F2)
    for (int c = threadIdx.x; c < Nx; c += blockDim.x) store_lp(F2, base + c, g.qm * a[c], f2mode);
  if (threadIdx.x == 0) {
    if (energy) energy[i] = e;
    if (!isfinite(e)) vp_set_status(status, VP_ENUMERIC);
  }
}

void poisson(const GridC& g, int p, const double* rho, const unsigned long long* counts,
             double* phi, double* F, double* energy, unsigned long long* zero_counts,
             const int* skip, int* status, cudaStream_t st, void* F2, int f2mode) {
  k_poisson<<<p, 256, 0, st>>>(g, rho, counts, phi, F, energy, zero_counts, skip, status, F2,
                               f2mode);
}

// ----------------------------------------------------------------- gather
__global__ void k_gather(GridC g, int64_t N, const double* __restrict__ X, int64_t ldx,
                         const double* __restrict__ F, const int32_t* __restrict__ idx, int64_t d,
                         double* __restrict__ GX, int* status) {
  extern __shared__ double sF[];
  const int i = blockIdx.y;
  for (int c = threadIdx.x; c < g.Nx; c += blockDim.x) sF[c] = g.qm * F[(int64_t)i * g.Nx + c];
  __syncthreads();
  const double* x = X + (int64_t)i * ldx;
  const int64_t cnt = idx ? d : N;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < cnt;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t l = idx ? (int64_t)idx[r] : r;
    if (l < 0 || l >= N) {  // a DEIM index outside the particle range
      vp_set_status(status, VP_EINVAL);
      GX[(int64_t)i * cnt + r] = 0.0;
      continue;
    }
    int j;
    double s;
    cell_of(__ldg(x + l), g.inv_h, g.Nx, g.dNx, g.inv_Nx, j, s);
    GX[(int64_t)i * cnt + r] = sF[j];
  }
}

void gather(const GridC& g, int64_t N, int p, const double* X, int64_t ldx, const double* F,
            const int32_t* idx, int64_t d, double* GX, int num_sms, int* status, cudaStream_t st) {
  const int bs = 256;
  int64_t cnt = idx ? d : N;
  int bx = ceil_div(cnt, bs * 4);
  int want = (4 * num_sms + p - 1) / p;
  if (bx > want) bx = want;
  if (bx < 1) bx = 1;
  k_gather<<<dim3(bx, p), bs, g.Nx * sizeof(double), st>>>(g, N, X, ldx, F, idx, d, GX, status);
}

// ------------------------------------------------------- full-order step
// One cluster of CS blocks per sample; block r owns particles
// [r*chunk, min(N, (r+1)*chunk)).  Per step: one sweep (gather with the
// previous field, kick, drift, deposit into a double-buffered fixed-point
// grid in shared memory), one hardware cluster barrier, and a redundant
// Poisson solve in every block from the summed grids of all blocks read
// through distributed shared memory.  Kick-drift-kick ordering with the
// full-step velocity formed explicitly each step:
//   V_{t-1} = Vh + dt/2 a(X_{t-1});  Vh = V_{t-1} + dt/2 a(X_{t-1});
//   X_t = X_{t-1} + dt Vh,
// which is eq. sv_full_order with E_h = a = -GX.
struct FullSmem {
  unsigned long long counts[2][VP_MAX_NX];
  double acc[VP_MAX_NX];  // -qm F_j: acceleration on cell j
  double a[VP_MAX_NX];
  double tmp[VP_MAX_NX];
  double kin[2];
  double red[32];
};

__global__ void k_full_step(GridC g, int64_t N, double* __restrict__ X, double* __restrict__ V,
                            double dt, int nsteps, double* __restrict__ trace, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FullSmem& sm = *reinterpret_cast<FullSmem*>(smem_raw);
  cg::cluster_group cl = cg::this_cluster();
  const int CS = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int i = blockIdx.y;
  const int p = gridDim.y;
  const int Nx = g.Nx, t = threadIdx.x, nt = blockDim.x;
  const int64_t chunk = (N + CS - 1) / CS;
  const int64_t l0 = rank * chunk;
  const int64_t l1 = min(N, l0 + chunk);
  double* x = X + (int64_t)i * N;
  double* v = V + (int64_t)i * N;
  const double hdt = 0.5 * dt;
  const unsigned long long one = 1ull << g.S;

  auto deposit_one = [&](double xl, unsigned long long* cnt) {
    int j;
    double s;
    cell_of(xl, g.inv_h, Nx, g.dNx, g.inv_Nx, j, s);
    unsigned long long w1 = (unsigned long long)__double2ll_rn(s * g.fp_scale);
    int j1 = (j + 1 == Nx) ? 0 : j + 1;
    atomicAdd(&cnt[j], one - w1);
    atomicAdd(&cnt[j1], w1);
  };
  auto accel_at = [&](double xl) {
    int j;
    double s;
    cell_of(xl, g.inv_h, Nx, g.dNx, g.inv_Nx, j, s);
    return sm.acc[j];
  };
  // Sum the cluster's grids of buffer b, solve, set acc; returns the energy.
  auto solve = [&](int b) {
    for (int c = t; c < Nx; c += nt) {
      unsigned long long s = 0ull;
      for (int r = 0; r < CS; ++r) s += cl.map_shared_rank(&sm.counts[b][0], r)[c];
      sm.a[c] = g.Mq * ((double)s * g.fp_inv) + g.bg_load;
    }
    __syncthreads();
    double e = poisson_inplace(g, sm.a, sm.tmp, sm.red, nullptr);
    for (int c = t; c < Nx; c += nt) sm.acc[c] = -g.qm * sm.a[c];
    __syncthreads();
    return e;
  };
  auto cluster_kin = [&](int b) {
    double s = 0.0;
    for (int r = 0; r < CS; ++r) s += *cl.map_shared_rank(&sm.kin[b], r);
    return 0.5 * s;
  };
  auto block_kin = [&](double k, int b) {
    for (int o = 16; o > 0; o >>= 1) k += __shfl_xor_sync(0xffffffffu, k, o);
    if ((t & 31) == 0) sm.red[t >> 5] = k;
    __syncthreads();
    if (t == 0) {
      double s = 0.0;
      for (int w = 0; w < (nt >> 5); ++w) s += sm.red[w];
      sm.kin[b] = s;
    }
  };

  // phase 0: grid of X_0
  for (int c = t; c < Nx; c += nt) sm.counts[0][c] = 0ull;
  __syncthreads();
  for (int64_t l = l0 + t; l < l1; l += nt) deposit_one(x[l], sm.counts[0]);
  __syncthreads();
  cl.sync();
  solve(0);
  double E_prev = 0.0;

  for (int step = 1; step <= nsteps; ++step) {
    const int b = step & 1;
    for (int c = t; c < Nx; c += nt) sm.counts[b][c] = 0ull;
    __syncthreads();
    double kin = 0.0;
    for (int64_t l = l0 + t; l < l1; l += nt) {
      double xl = x[l], vl = v[l];
      double a = accel_at(xl);
      double vfull = (step == 1) ? vl : fma(hdt, a, vl);  // V_{step-1}
      kin = fma(vfull, vfull, kin);
      double vh = fma(hdt, a, vfull);
      double xn = fma(dt, vh, xl);
      x[l] = xn;
      v[l] = vh;
      deposit_one(xn, sm.counts[b]);
    }
    block_kin(kin, b);
    __syncthreads();
    cl.sync();
    double E = solve(b);
    if (rank == 0 && t == 0) {
      if (trace) {
        trace[((int64_t)(step - 1) * p + i) * 2 + 0] = E;
        if (step >= 2) trace[((int64_t)(step - 2) * p + i) * 2 + 1] = E_prev + cluster_kin(b);
      }
      if (!isfinite(E)) vp_set_status(status, VP_ENUMERIC);
    }
    E_prev = E;
  }
  // final half kick: V_n = Vh + dt/2 a(X_n), kinetic energy of V_n
  const int bf = (nsteps + 1) & 1;
  double kin = 0.0;
  for (int64_t l = l0 + t; l < l1; l += nt) {
    double vfull = fma(hdt, accel_at(x[l]), v[l]);
    v[l] = vfull;
    kin = fma(vfull, vfull, kin);
  }
  block_kin(kin, bf);
  __syncthreads();
  cl.sync();
  if (rank == 0 && t == 0 && trace && nsteps >= 1)
    trace[((int64_t)(nsteps - 1) * p + i) * 2 + 1] = E_prev + cluster_kin(bf);
  cl.sync();  // peers keep their shared memory alive until rank 0 has read it
}

void pic_init() {
  cudaFuncSetAttribute(k_full_step, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaFuncSetAttribute(k_full_step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)sizeof(FullSmem));
}

cudaError_t full_step(const GridC& g, int64_t N, int p, double* X, double* V, double dt,
                      int nsteps, double* trace, int* status, cudaStream_t st) {
  int cs = 16;
  while (cs > 1 && (int64_t)cs * 128 > N) cs >>= 1;  // at least ~128 particles per block
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.blockDim = dim3(256, 1, 1);
  cfg.dynamicSmemBytes = sizeof(FullSmem);
  cfg.stream = st;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  for (;; cs >>= 1) {
    cfg.gridDim = dim3(cs, p, 1);
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    int nclusters = 0;
    cudaError_t e = cudaOccupancyMaxActiveClusters(&nclusters, (void*)k_full_step, &cfg);
    if ((e == cudaSuccess && nclusters > 0) || cs == 1) {
      (void)cudaGetLastError();
      break;
    }
    (void)cudaGetLastError();
  }
  return cudaLaunchKernelEx(&cfg, k_full_step, g, N, X, V, dt, nsteps, trace, status);
}

}  // namespace vpk
