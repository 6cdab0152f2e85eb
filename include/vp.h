/*
 * vp.h -- C ABI of the GB300 library for the data-parallel hot path of the
 * adaptive symplectic dynamical reduced model of the parametric particle-based
 * 1D1V Vlasov-Poisson system (Hesthaven, Pagliantini, Ripamonti,
 * arXiv 2201.05555).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns a vp_status.  No call aborts, prints or exits.  The
 *   message of the last failure on a context is vp_last_error(ctx).
 * - Pointers named *_dev are device pointers owned by the caller; the library
 *   never frees them.  Host pointers are named *_host.  The library owns only
 *   its context and the workspace it allocates (on demand, within the byte
 *   budget given to vp_ctx_create).
 * - Device work is asynchronous on the caller's CUDA stream (`stream`, a
 *   cudaStream_t passed as void*; NULL = legacy default stream).  Arguments
 *   are validated on the host before any launch (VP_EINVAL).  Errors found on
 *   the device (non-convergence, non-finite energies, a singular small
 *   system) are written to a device status word and reported by
 *   vp_ctx_sync_status.
 * - Floating point: every entry point below computes in FP64 (dtype "f64").
 *   Fixed-point int64 charge accumulation makes deposits independent of the
 *   order of particles: repeated calls give bit-identical results.
 *
 * Data layouts (row-major, C order)
 * ---------------------------------
 * - Particles of p samples: X, V, GX are p x N arrays (sample i occupies
 *   elements [i*ld, i*ld + N)).  Positions are unwrapped (they are reduced
 *   modulo L only inside the particle-to-grid maps).
 * - The ortho-symplectic basis U = [[A, -B], [B, A]] (2N x 2n, Sec. 3.2,
 *   eq. dynManifold) is stored as the complex N x n matrix Q = A + iB,
 *   row l = [A_l0 .. A_l(n-1), B_l0 .. B_l(n-1)] (N x 2n doubles).  Tangent
 *   vectors xi, X(U,Z), Y(xi,Z) (2N x 2n) use the same storage.
 * - Coefficients Z = [a; b] (2n x p) exactly as in the paper (zeta = a + ib).
 * - Grid arrays rho, phi, F are p x Nx.  F_j = (phi_{j+1} - phi_j)/h is the
 *   derivative of the P1 potential on cell j = [x_j, x_{j+1}).
 *
 * Mesh conventions: nodes x_j = j h, h = L/Nx, periodic P1 hats; a particle
 * at wrapped position x lies in cell floor(x/h); the Poisson gauge is
 * sum_j phi_j = 0.
 */
#ifndef VP_H
#define VP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vp_status {
  VP_OK = 0,
  VP_EINVAL = 1,       /* invalid argument (checked on the host) */
  VP_ENOMEM = 2,       /* workspace over the context budget or cudaMalloc failed */
  VP_EBUSY = 3,        /* server full / admission refused */
  VP_EAGAIN = 4,       /* result not ready yet */
  VP_ETIMEDOUT = 5,    /* a bounded wait ran out */
  VP_ENOCONV = 6,      /* fixed-point iteration did not converge */
  VP_ENUMERIC = 7,     /* non-finite value or singular small system */
  VP_EDRIFT = 8,       /* basis left the ortho-symplectic manifold */
  VP_ECUDA = 9,        /* a CUDA runtime call failed */
  VP_EUNSUPPORTED = 10, /* size outside the compiled limits, or a call not available */
  VP_ECOMM = 11         /* a sum of the attached communicator (vp_ctx_set_comm) failed */
} vp_status;

typedef struct vp_ctx vp_ctx;

/* Mesh and particle constants (Sec. 2.1).  With q = -1, m = 1 and weights
 * omega = L/N (mean density 1): Mq = -L/N, mp = L/N, background = 1. */
typedef struct vp_grid {
  int32_t Nx;        /* nodes of the periodic P1 mesh, 3 <= Nx <= 1024 */
  double L;          /* domain length */
  double Mq;         /* charge of one macro-particle, q*omega (eq. PoissonSystem) */
  double mp;         /* mass of one macro-particle, m*omega (eq. HamEEfull) */
  double background; /* neutralising background density; P1 load background*h */
} vp_grid;

/* Options of the partitioned RK2 step (Sec. 5). */
typedef struct vp_step_opts {
  double tol;      /* fixed-point stop: |k_{m+1} - k_m|_F <= tol |k_{m+1}|_F (Sec. 6.1: 1e-9).
                    * With arith = 2 (FP32 rows) a tol below 1e-6 is raised to 1e-6: the
                    * map is then evaluated in FP32, whose updates stop shrinking near the
                    * FP32 rounding level (~1e-7 relative). */
  int32_t maxit;   /* iteration cap; exceeding it gives VP_ENOCONV */
  int32_t freeze_basis; /* 1: keep U fixed (global symplectic reduced basis, Sec. 3.1) */
  /* Stops for a discontinuous map.  The PIC force is piecewise constant in
   * each particle position (it jumps at the nodes), so the fixed-point map is
   * discontinuous and its updates need not fall to tol.  While the relative
   * update r_m = |k_m - k_{m-1}|_F / |k_m|_F is at most cycle_max, the
   * iteration also stops at iteration m
   * - on a short cycle, for the shortest period q in 2..4 with q <= m and
   *     |k_m - k_{m-q}|_F <= tol |k_m|_F                (back where it was),
   *     |k_m - k_{m-q}|_F <= cycle_ratio |k_m - k_{m-1}|_F (not a converging
   *     iteration, which returns only to a sizeable fraction of its update);
   * - on a plateau, when m > 8 and r_m >= r_{m-8} / 2: the update has not
   *   halved over 8 iterations (iterates wandering among configurations that
   *   differ by a few cell flips; a linear contraction triggers this only
   *   with a factor above 0.917).
   * k_m is the result.  cycle_max = 0 disables both.  Defaults 1e-3, 1e-2. */
  double cycle_max;
  double cycle_ratio;
  /* Arithmetic of the N-row work (deposit, projection, Gamma zeta^H, Gram
   * matrices, affine row updates):
   * 0 = FP64;
   * 1 = double-float (each FP64 operand as a sum of two floats, compensated
   *     dot products, about 48 significant bits);
   * 2 = FP32 (the precision form: FP32 row storage and accumulation).
   * Q and Z stay FP64 in memory; reductions across blocks, the small dense
   * algebra and the energies are FP64 in every mode.  Default 0. */
  int32_t arith;
  /* 1: after every step re-orthonormalise Q <- Q (Q^H Q)^-1/2 (the block
   * form keeps U symplectic): Gram and update in double-float, the factor by
   * a coupled Newton-Schulz iteration in FP64 (|Q^H Q - I|_F >= 0.9 reports
   * VP_EDRIFT).  Not in the paper; a safeguard against the drift of
   * U^T U = I in the precision form.  Default 0. */
  int32_t reortho;
  /* Parameter subsample of the basis evolution (Sec. 4.1): 0 = all samples;
   * otherwise the basis velocities use only the nsub columns sub_idx (device,
   * int32, from vp_param_subsample; n <= nsub <= p) of Z and of the gradient,
   * while every coefficient column is advanced.  arith 1 or 2 only. */
  int32_t nsub;
  const int32_t* sub_idx;
} vp_step_opts;

/* ------------------------------------------------------------------ context */
/* Create a context on `device`.  scratch_bytes bounds the workspace the
 * library may allocate for itself (0 = 16 GiB). */
vp_status vp_ctx_create(vp_ctx** ctx_out, int device, size_t scratch_bytes);
vp_status vp_ctx_destroy(vp_ctx* ctx);
const char* vp_last_error(const vp_ctx* ctx);
const char* vp_status_string(vp_status s);
/* Synchronise `stream`, then return and clear the device status word. */
vp_status vp_ctx_sync_status(vp_ctx* ctx, void* stream);
/* Bytes of workspace currently held by the context. */
size_t vp_ctx_workspace_bytes(const vp_ctx* ctx);
int32_t vp_version(void);

/* --------------------------------------------------- particle sharding */
/* The reduced model shards over particles (Sec. 3.2: every N-row quantity
 * of the reduced vector field -- X_r = U_X Z, the deposit, the gather, the
 * projection U^T G, Gamma zeta^H and the row updates of the Cayley
 * retraction -- is a sum or a map over the rows of U).  A rank holds the rows
 * of its own particles; the sums over rows are the only exchange:
 * the p x Nx charge counts (int64 fixed point, exact in any order), the
 * 2n x p projection and the small Gram matrices of the basis stages, of the
 * retraction and of the tangent velocity (FP64).  Poisson, the small dense
 * algebra, the fixed-point decision and the coefficient update then run
 * redundantly and identically on every rank. */
typedef struct vp_comm {
  /* In-place sum over the ranks of `count` values at the device pointer buf
   * (FP64, or the unsigned 64-bit charge counts), ordered on `stream` (a
   * cudaStream_t as void*): the library's earlier work on stream has written
   * buf, and its later work reads the sum.  Called on the host thread that
   * called the library, the same number of times and with the same counts on
   * every rank.  Returns 0 on success. */
  int (*sum_f64)(void* user, double* buf, int64_t count, void* stream);
  int (*sum_u64)(void* user, uint64_t* buf, int64_t count, void* stream);
  void* user;        /* passed back to both */
  int64_t n_global;  /* particles per sample over all ranks (fixed-point scales) */
} vp_comm;

/* Attach a communicator to ctx (copied; comm = NULL detaches).  With one
 * attached, vp_basis_update and vp_reduced_energy take Q_dev as this rank's
 * N rows and Z as the full (replicated) coefficients, and give on every rank
 * the results of the whole problem (n_global particles per sample): Q_dev
 * this rank's rows of the new basis, Z, traces, energies and iteration counts
 * identical on every rank.  The parameter subsample (nsub) is supported; the
 * other reduced-model and hyper-reduction calls return VP_EUNSUPPORTED while a
 * communicator is attached.  A failed sum makes the call return VP_ECOMM. */
vp_status vp_ctx_set_comm(vp_ctx* ctx, const vp_comm* comm);

/* ------------------------------------------------------ particle-grid maps */
/* a2. rho = Lambda^0(X)^T M_q + b for each of p samples (Sec. 2.1,
 * eq. PoissonSystem): cloud-in-cell (P1 hat) deposit plus the background
 * load background*h per node.  X_dev: p x N with leading dimension ldx >= N.
 * rho_dev: p x Nx.  1 <= N < 2^31, 1 <= p <= 65535. */
vp_status vp_deposit_cic(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p,
                         const double* X_dev, int64_t ldx, double* rho_dev, void* stream);

/* a3. Solve L phi = rho with sum(phi) = 0 for each sample, L = (1/h)
 * circ(-1, 2, -1) the periodic P1 stiffness matrix (eq. PoissonSystem), by
 * two prefix sums.  Writes the cell derivative F (p x Nx), optionally phi
 * (p x Nx) and the electric energy E = (1/(2 mp)) phi^T L phi = (h/(2 mp))
 * sum_j F_j^2 (p, eq. HamEEfull).  Null outputs are skipped.  Requires
 * sum_j rho_j = 0 (neutral system); the solve uses the consistent part. */
vp_status vp_poisson_periodic(vp_ctx* ctx, const vp_grid* grid, int32_t p, const double* rho_dev,
                              double* phi_dev, double* F_dev, double* energy_dev, void* stream);

/* a4. Gradient of the electric energy at the particles,
 * GX = m_p^-1 diag(M_q) grad Lambda^0(X) phi = (Mq/mp) F_{cell(X)} (eq. VPHamEqn);
 * the accelerations of eq. sv_full_order are -GX.  idx_dev == NULL: all N
 * particles, GX_dev p x N.  Otherwise only the d particles idx_dev[0..d)
 * (DEIM rows, Sec. 4.2), GX_dev p x d.  F_dev: p x Nx from vp_poisson_periodic. */
vp_status vp_gather_E(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, const double* X_dev,
                      int64_t ldx, const double* F_dev, const int32_t* idx_dev, int64_t d,
                      double* GX_dev, void* stream);

/* ------------------------------------------- typed per-step calls (vp_dtype)
 * The calls a2, a4, a1 and a5 above on N-row inputs of a stated element type
 * (positions, gradients and basis rows; grids, Z and g stay FP64), with
 * explicit leading dimensions.  FP64 inputs give the results of the calls
 * above.  Positions are converted to FP64 before their cell and weight are
 * taken, so the deposit and the gather equal the FP64 calls on the rounded
 * positions (the deposit exactly; the gather up to the rounding of its
 * output to the type).  The reconstruction and the projection multiply and
 * accumulate in FP32 for FP32 and BF16 inputs (FP64 for FP64), per-block
 * partial sums added in FP64.  Pointers must be aligned to their element
 * type; a bad dtype, flag or alignment returns VP_EINVAL. */
typedef enum vp_dtype { VP_F64 = 0, VP_F32 = 1, VP_BF16 = 2 } vp_dtype;
/* Deposit flag: charge accumulated as int64 fixed point (order-independent,
 * bit-identical on repetition).  It is the only accumulation the library
 * implements, so flags = 0 means the same. */
#define VP_DEPOSIT_FIXEDPOINT 1
/* a2 (Sec. 2.1, eq. PoissonSystem): rho = Lambda^0(X)^T M_q + b. */
vp_status vp_deposit_cic_t(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, const void* X_dev,
                           int64_t ldx, int32_t dtype, double* rho_dev, int32_t flags, void* stream);
/* a4 (eq. VPHamEqn): GX_dev (p x N, or p x d with idx_dev) in dtype. */
vp_status vp_gather_E_t(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, const void* X_dev,
                        int64_t ldx, int32_t dtype, const double* F_dev, const int32_t* idx_dev,
                        int64_t d, void* GX_dev, void* stream);
/* a1 (Sec. 3.2): Q_dev N rows of ldq >= 2n elements; X_dev, V_dev (nullable)
 * p x N with leading dimension ldx >= N, in dtype. */
vp_status vp_reconstruct_t(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const void* Q_dev,
                           int64_t ldq, int32_t dtype, const double* Z_dev, void* X_dev,
                           void* V_dev, int64_t ldx, void* stream);
/* a5 (eq. grads): g_dev (2n x p, FP64) = U^T [GX; V_r], GX_dev p x N with
 * leading dimension ldg >= N (nullable: the V part alone). */
vp_status vp_project_grad_t(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const void* Q_dev,
                            int64_t ldq, int32_t dtype, const void* GX_dev, int64_t ldg,
                            const double* Z_dev, double* g_dev, void* stream);

/* a10. nsteps Stormer-Verlet steps of the full-order model for each sample
 * (Sec. 5, eq. sv_full_order), in place on X_dev, V_dev (p x N, ld N).
 * trace_dev (nullable): (nsteps x p x 2) electric energy and Hamiltonian
 * H = 1/2 V^T V + E after each step (eq. high_fidelity_Hamiltonian).
 * One thread-block cluster per sample runs all steps in one launch. */
vp_status vp_full_step(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p, double* X_dev,
                       double* V_dev, double dt, int32_t nsteps, double* trace_dev, void* stream);

/* -------------------------------------------------------- reduced model */
/* a1. X_r = U_X Z, V_r = U_V Z (Sec. 3.2): X_dev, V_dev p x N (V_dev nullable).
 * Q_dev N x 2n, Z_dev 2n x p.  1 <= n <= 40 for every reduced-model call. */
vp_status vp_reconstruct(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q_dev,
                         const double* Z_dev, double* X_dev, double* V_dev, void* stream);

/* a5. g = U^T [GX; V_r] with V_r = U_V Z (eq. grads): the X part by a
 * projection of GX (p x N) onto the basis, the V part through the Gram
 * matrix U_V^T U_V (Sec. 4.3, cost item 1).  g_dev: 2n x p.  GX_dev == NULL
 * gives the V part alone. */
vp_status vp_project_grad(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q_dev,
                          const double* GX_dev, const double* Z_dev, double* g_dev, void* stream);

/* a6. Basis velocity X(U, Z) = (I - UU^T)(J G Z^T - G Z^T J^T) S(Z)^-1
 * (eq. UZred_basis), with G = [GX; V_r] evaluated at R = UZ (deposit,
 * Poisson, gather inside).  Xi_dev: N x 2n (complex storage). */
vp_status vp_basis_velocity(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                            const double* Q_dev, const double* Z_dev, double* Xi_dev, void* stream);

/* a7. Cayley retraction R_U0(xi) = cay(W U0^T - U0 W^T) U0, 2W = (2I -
 * U0 U0^T) xi (Sec. 5), evaluated in O(N n^2) with the Woodbury identity.
 * Qout_dev may alias Q0_dev. */
vp_status vp_cayley_retract(vp_ctx* ctx, int64_t N, int32_t n, const double* Q0_dev,
                            const double* xi_dev, double* Qout_dev, void* stream);

/* a8. Tangent velocity Y(xi, Z) of the local flow at U0 (Sec. 5), with the
 * basis velocity evaluated at R_U0(xi).  Y_dev: N x 2n. */
vp_status vp_tangent_velocity(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                              const double* Q0_dev, const double* xi_dev, const double* Z_dev,
                              double* Y_dev, void* stream);

/* a9. nsteps partitioned RK2 steps (Sec. 5, eqs. pRK_Z .. pRK_U_ktilde):
 * explicit midpoint + Cayley retraction for U, implicit midpoint (fixed point
 * from k = 0) for Z, in place on Q_dev (N x 2n) and Z_dev (2n x p).
 * opts NULL = {1e-9, 100, 0, 1e-3, 1e-2, 0, 0, 0, NULL}.  trace_dev (nullable): (nsteps x p x 2)
 * electric energy and reduced Hamiltonian 1/2|V_r|^2 + E (eq.
 * nonlinear_hamiltonian) of the state entering each step, taken from the
 * step's first field evaluation (no extra work; with arith = 2 from an extra
 * double-float evaluation, so the diagnostic keeps FP64 accuracy);
 * vp_reduced_energy gives the same diagnostics for the final state.
 * iters_dev (nullable): fixed-point iterations of each step (int32, nsteps).
 * kstate_dev (nullable, 2n x p, in/out): initial guess of the fixed point
 * (the paper leaves it unstated); on return it holds the last step's k2, so
 * passing it back warm-starts the next call.  NULL: start from k = 0 each step.
 * Synchronises `stream` once per step to steer the fixed point. */
vp_status vp_basis_update(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                          double* Q_dev, double* Z_dev, double dt, int32_t nsteps,
                          const vp_step_opts* opts, double* trace_dev, int32_t* iters_dev,
                          double* kstate_dev, void* stream);

/* Start of the reduced model (Sec. 3.2, Algorithm 2): truncated complex SVD
 * of R0 = X0 + i V0 (N x p), through the Gram matrix R0^H R0 = W S^2 W^H
 * (cyclic Jacobi on the device): Q = R0 W_n S_n^-1 re-orthonormalised as
 * Q (Q^H Q)^-1/2, zeta = Q^H R0.  X0_dev, V0_dev: p x N (ld N).  Outputs
 * Q_dev (N x 2n), Z_dev (2n x p), sigma_dev (p singular values, descending;
 * nullable).  The phase of each column of Q is free and not normalised.
 * 1 <= n <= min(p, 40), p <= 256.  Singular values below 1e-14 sigma_1 in the
 * first n give VP_ENUMERIC through the status word (S(Z) would be singular). */
vp_status vp_init_csvd(vp_ctx* ctx, int64_t N, int32_t p, int32_t n, const double* X0_dev,
                       const double* V0_dev, double* Q_dev, double* Z_dev, double* sigma_dev,
                       void* stream);

/* Greedy parameter subsample (Sec. 4.1, eq. pSampl) on the columns of Z0
 * (2n x p, device): the first index is the column of largest norm, then each
 * step adds the column whose distance min_j |Z0_i - Z0_j|_2 to the chosen set
 * is largest (ties to the lowest index), until p_max columns or until that
 * distance falls to tol times the one of the second choice.  idx_dev (device,
 * int32, p_max entries) receives the indices in order of choice, *count the
 * number chosen.  p <= 1024.  Synchronises `stream`. */
vp_status vp_param_subsample(vp_ctx* ctx, int32_t n, int32_t p, const double* Z0_dev,
                             int32_t p_max, double tol, int32_t* idx_dev, int32_t* count,
                             void* stream);

/* The same start with the rank chosen at t = 0 from the singular values (the
 * paper observes that a constant rank suffices; the rule is a reading): n =
 * the smallest k in [n_min, n_max] whose relative tail energy
 * sum_{j>k} sigma_j^2 / sum_j sigma_j^2 < tail_tol (n_max if none), lowered
 * while sigma_n < 1e-6 sigma_1, even below n_min (cond S(Z) <= 1e12; singular
 * values from the Gram matrix resolve ~1e-8 sigma_1).  Q_dev must hold N x 2 n_max; Q (N x 2n) and
 * Z (2n x p) are written densely for the chosen n, returned in *n_out.
 * Synchronises `stream` once (the eigenvalues go to the host for the rule). */
vp_status vp_init_csvd_rank(vp_ctx* ctx, int64_t N, int32_t p, int32_t n_min, int32_t n_max,
                            double tail_tol, const double* X0_dev, const double* V0_dev,
                            double* Q_dev, double* Z_dev, double* sigma_dev, int32_t* n_out,
                            void* stream);

/* a11. FP64 diagnostics of a reduced state: electric energy E_i and
 * Hamiltonian H_i = 1/2 |U_V Z_i|^2 + E_i (p each, eq. nonlinear_hamiltonian),
 * and the manifold residual |Q^H Q - I|_F (= |U^T U - I|_F / sqrt 2; U^T J U = J
 * holds exactly for the block form).  Any output may be NULL. */
vp_status vp_reduced_energy(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                            const double* Q_dev, const double* Z_dev, double* E_dev, double* H_dev,
                            double* resid_dev, void* stream);

/* Accuracy diagnostics (Sec. 6.1-6.2); FP64, deterministic.
 * vp_rel_errors: eq. relative_errors, eps_dev[0] = |S_X - X_r|_F / |S_X|_F,
 *   eps_dev[1] = |S_V - V_r|_F / |S_V|_F, with the full-order snapshots
 *   X_dev, V_dev (p x N, sample by sample) and X_r, V_r = U Z.
 * vp_target_errors: eq. relative_errors_complex_SVD, the same errors for the
 *   projection onto the ortho-symplectic basis of size 2n from the complex SVD
 *   of S_X + i S_V (Gram route: tails below ~1e-8 of |S| are not resolved).
 * vp_rank_indicator: out_dev[0] = |(I - U U^T) G|_F / |G|_F, G the Hamiltonian
 *   gradient of the full model at R = U Z: the share of the force outside the
 *   basis (an indicator for rank adaptivity, which the paper leaves open).
 * vp_half_basis: Qh_dev = R_{Q0}(dt/2 X(Q0, Z0)), the basis at the first
 *   stage of the step (Sec. 5).
 * vp_hamiltonian_error_terms: eq. error_ham_tot, out_dev[0..4) =
 *   |H(U1 Z1) - H(U0 Z0)|, |H(U1 Z1) - H(Uh Z1)|, |H(Uh Z0) - H(U0 Z0)|,
 *   |H(Uh Z1) - H(Uh Z0)| (2-norms over the p parameters). */
vp_status vp_rel_errors(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q_dev,
                        const double* Z_dev, const double* X_dev, const double* V_dev,
                        double* eps_dev, void* stream);
vp_status vp_target_errors(vp_ctx* ctx, int64_t N, int32_t p, int32_t n, const double* X_dev,
                           const double* V_dev, double* eps_dev, void* stream);
vp_status vp_rank_indicator(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                            const double* Q_dev, const double* Z_dev, double* out_dev, void* stream);
/* Re-initialisation at a larger rank (Sec. 6.4, two-stream instability in the
 * nonlinear regime: the reduced model restarts from the complex SVD of the
 * full-order solutions of all samples at the restart time, with a larger
 * basis).  The trigger is a reading: the rank indicator of the current state
 * (Q_dev N x 2n, Z_dev 2n x p, as vp_rank_indicator) above `threshold`
 * (threshold < 0 always restarts, +inf never does, a NaN indicator restarts).
 * On a restart, Q_new_dev (N x 2 n_new) and Z_new_dev (2 n_new x p) receive
 * the start of vp_init_csvd from the full-order states X_dev, V_dev (p x N,
 * ld N, unwrapped positions), 1 <= n_new <= min(p, N, 40); otherwise they are
 * not written.  *indicator (host, nullable) receives the indicator,
 * *restarted (host) 1 or 0.  Synchronises `stream` once: the decision is
 * taken on the host.  The caller owns every buffer; a NaN threshold, a null
 * pointer or an n_new out of range is VP_EINVAL. */
vp_status vp_restart_csvd(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                          const double* Q_dev, const double* Z_dev, const double* X_dev,
                          const double* V_dev, double threshold, int32_t n_new, double* Q_new_dev,
                          double* Z_new_dev, double* indicator, int32_t* restarted, void* stream);
vp_status vp_half_basis(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                        const double* Q0_dev, const double* Z0_dev, double dt, double* Qh_dev,
                        void* stream);
vp_status vp_hamiltonian_error_terms(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n,
                                     int32_t p, const double* Q0_dev, const double* Z0_dev,
                                     const double* Qh_dev, const double* Q1_dev, const double* Z1_dev,
                                     double* out_dev, void* stream);

/* a12. DEIM-indexed nonlinear gradient (Sec. 4.3, eq. grHDD):
 * gX = m_p^-1 U_X^T diag(grad Lambda^0(X_r) Phi_DMD) P c, evaluated at the d
 * rows idx_dev of X_r = U_X Z only.  c_dev: the d DEIM weights
 * c = (P^T Psi)^-T Psi^T M_q.  phi_dev: p x Nx potentials Phi_DMD.
 * gX_dev: 2n x p.  Add the linear part U_V^T V_r (vp_project_grad with GX = 0)
 * for the full g^DD. */
vp_status vp_deim_gather_project(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                                 const double* Q_dev, const double* Z_dev, int64_t d,
                                 const int32_t* idx_dev, const double* c_dev,
                                 const double* phi_dev, double* gX_dev, void* stream);

/* ------------------------------------------------------ DEIM construction */
/* Sec. 4.2, eq. Ydeim: the snapshot columns Lambda^0(X) Phi, i.e. the P1
 * interpolant of each sample's nodal potential at its particles.
 * X_dev: p x N (ld ldx) positions (unwrapped), phi_dev: p x Nx potentials,
 * Y_dev: p columns of length N (ld ldy). */
vp_status vp_potential_at_particles(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t p,
                                    const double* X_dev, int64_t ldx, const double* phi_dev,
                                    double* Y_dev, int64_t ldy, void* stream);
/* DEIM basis: the first d left singular vectors of the snapshot matrix
 * Y (N x m, stored as m columns of length N, ld ldy), written as d columns of
 * length N (Psi_dev, d x N), from the Gram matrix Y^T Y (Jacobi): directions
 * with singular values below ~1e-8 sigma_1 are not resolved.  sigma_dev
 * (nullable): the m singular values, descending.  m <= 256, d <= min(m, 128),
 * m d <= 25600.  A vanishing singular value among the first d gives
 * VP_ENUMERIC through the status word. */
vp_status vp_deim_basis(vp_ctx* ctx, int64_t N, int32_t m, const double* Y_dev, int64_t ldy,
                        int32_t d, double* Psi_dev, double* sigma_dev, void* stream);
/* Greedy DEIM interpolation indices for the ordered basis Psi (d x N): the
 * first is the row where |psi_1| is largest, the k-th where the residual of
 * psi_k interpolated from the first k-1 vectors at the first k-1 indices is
 * largest (ties to the lowest row).  idx_dev: d int32.  d <= 128. */
vp_status vp_deim_indices(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi_dev,
                          int32_t* idx_dev, void* stream);
/* Adaptive update of the DEIM indices (Sec. 4.2, eq. indices_adaptive_DEIM).
 * On entry idx_dev holds the indices of the previous basis Psi_prev (d x N);
 * the n_up positions k whose vectors rotated most, i.e. with the smallest
 * |psi_k . psi_prev_k| (absolute value: singular vectors carry an arbitrary
 * sign; ties to the lowest k), are renewed in increasing k by the greedy rule
 * of vp_deim_indices (interpolation residual of psi_k from psi_1..psi_{k-1}
 * at the indices then held), never taking a row held at another position;
 * the other positions keep their rows.  The printed arg-max of the inner
 * products would pick the least-rotated vectors while the paper's text asks
 * for the most-rotated; this reading follows the text.  n_up = d is the
 * greedy procedure, n_up = 0 keeps the indices.  0 <= n_up <= d <= 128. */
vp_status vp_deim_indices_update(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi_dev,
                                 const double* Psi_prev_dev, int32_t n_up, int32_t* idx_dev,
                                 void* stream);
/* Weights of the DEIM-indexed gradient (eq. grHDD): c = (P^T Psi)^-T Psi^T M_q
 * with equal particle charges M_q (all entries Mq).  c_dev: d doubles. */
vp_status vp_deim_weights(vp_ctx* ctx, int64_t N, int32_t d, const double* Psi_dev,
                          const int32_t* idx_dev, double Mq, double* c_dev, void* stream);

/* ------------------------------------------------------------------- DMD */
/* DMD of the electric potential (Sec. 4.2, Algorithm 1) on window data of
 * the sampled parameters: Y, Y' (nx x m, stored as m columns of length nx;
 * eq. DMD_potential_Y_time_parameter).  Truncated SVD Y = U S V^T with the
 * singular values above max(tol, 1e-7) sigma_1 (at most r_max <= 64; *r_out
 * receives r), from the Gram matrix Y^T Y (Jacobi), which resolves singular
 * values down to ~1e-8 sigma_1 only.  Outputs (device, sized for r_max):
 *   B = Y' V S^-1 (r columns of length nx) - the exact-DMD modes are B W;
 *   Bpinv = (B^T B)^-1 B^T (r x nx, row-major);
 *   A = U^T B (r x r), whose eigenvalues are the DMD eigenvalues;
 *   S = Re(A^1/2) with the principal power of every eigenvalue (complex
 *     Schur form of A, triangular square root), for half steps;
 *   sigma (nullable): the m singular values of Y.
 * Since Theta^+ = W^-1 Bpinv, the real part of the DMD potential
 * Theta (Pi (.) lambda^(s/dt)) with Pi = Theta^+ Phi equals
 * B Re(A^(s/dt)) Bpinv Phi: whole steps use real powers of A, half steps S.
 * An eigenvalue on the negative real axis (a mode that changes sign every
 * step) contributes zero at half steps on either side of the branch cut.
 * nx <= 4096, m <= 256.  Synchronises `stream` (the rank goes to the host). */
vp_status vp_dmd_fit(vp_ctx* ctx, int32_t nx, int32_t m, const double* Y_dev, const double* Yp_dev,
                     double tol, int32_t r_max, int32_t* r_out, double* B_dev, double* Bpinv_dev,
                     double* A_dev, double* S_dev, double* sigma_dev, void* stream);
/* DMD coordinates beta_i = Bpinv Phi_i of q potentials (q x nx) -> beta (q x r);
 * Pi_i = W^-1 beta_i. */
vp_status vp_dmd_coords(vp_ctx* ctx, int32_t nx, int32_t r, const double* Bpinv_dev, int32_t q,
                        const double* Phi_dev, double* beta_dev, void* stream);
/* Gaussian radial basis interpolation (Sec. 4.2, coordinates of parameters
 * outside the sample): through q points eta_s (q x dim) with values (q x K),
 * kernel exp(-(eps |eta - eta_j|)^2), evaluated at p points eta (p x dim)
 * into out (p x K).  q (q + K) doubles must fit in 200 KB. */
vp_status vp_rbf_interpolate(vp_ctx* ctx, int32_t dim, int32_t q, const double* eta_s_dev,
                             int32_t K, const double* values_dev, int32_t p, const double* eta_dev,
                             double eps, double* out_dev, void* stream);
/* DMD potential (eq. DMD_approx_potential_subset) at s = (ksteps + half / 2) dt
 * after the last window state: Phi_i = B A^ksteps S^half beta_i for p
 * coordinate rows beta (p x r) -> Phi (p x nx). */
vp_status vp_dmd_potential(vp_ctx* ctx, int32_t nx, int32_t r, const double* B_dev,
                           const double* A_dev, const double* S_dev, int32_t p,
                           const double* beta_dev, int32_t ksteps, int32_t half, double* Phi_dev,
                           void* stream);

/* ------------------------------------------ DMD-DEIM reduced dynamics */
/* The DMD-DEIM reduced model of eq. UZredhyp integrated by the partitioned
 * Runge-Kutta scheme of Sec. 5 (eq. discrete_dynROM) following Algorithm 2.
 * A vp_hyper object owns the sliding windows and the DMD and DEIM operators
 * of one reduced problem (grid, N, n, p) with a parameter subsample.  Each
 * interval tau (one call step):
 *  1. the field of the sampled parameters at the entering state (U, Z_sub)
 *     gives the potentials Phi^i_{tau-1} and the DEIM data columns
 *     Lambda^0(X_r^i) Phi^i (eq. Ydeim); both enter windows of T + 1 entries;
 *  2. while the windows hold T entries or fewer the interval is the
 *     subsampled reduced step (vp_basis_update with the subsample);
 *  3. afterwards: DMD of the potential windows (vp_dmd_fit, tolerance
 *     dmd_tol), coordinates of the sampled parameters from Phi_{tau-1},
 *     Gaussian RBF interpolation to all p parameters (width 0.3 / mean
 *     nearest-neighbour distance of the sampled parameters), the DMD potential
 *     at the coefficient stage time t_{tau-1} + dt/2; the DEIM basis of the
 *     data window (d vectors), its indices (all of them on the first DMD-DEIM
 *     interval and every k_deim intervals after it, else n_up of them by
 *     vp_deim_indices_update) and weights; then the PRK2 step whose
 *     coefficient stage uses the DMD-DEIM gradient g^DD of eq. grHDD (its X
 *     part needs the d DEIM rows of U only, independent of N), while the basis
 *     stages keep the field of the sampled parameters (eq. UZhypred_basis).
 * The FP32-based forms only (arith 1 or 2).  The DMD rank is read on the
 * host once per interval (one stream synchronisation). */
typedef struct vp_hyper vp_hyper;
typedef struct vp_hyper_opts {
  int32_t nsub;            /* sampled parameters p* (n <= p* <= p) */
  const int32_t* sub_idx;  /* device, p* column indices (e.g. vp_param_subsample) */
  int32_t dim;             /* parameter dimension */
  const double* eta;       /* device, p x dim parameters (RBF coordinates) */
  int32_t T;               /* window length (T >= 1, p* T <= 256) */
  int32_t d;               /* DEIM points (d <= min(p* (T + 1), 128)) */
  int32_t n_up;            /* renewed indices per interval (0 .. d) */
  int32_t k_deim;          /* all indices renewed every k_deim intervals (>= 1) */
  double dmd_tol;          /* Algorithm 1 tolerance relative to sigma_1 */
  int32_t r_max;           /* DMD rank cap (<= 64) */
} vp_hyper_opts;
vp_status vp_hyper_create(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                          const vp_hyper_opts* opts, vp_hyper** out);
/* nsteps intervals from (Q, Z) in place; opts, trace, iters and kstate as in
 * vp_basis_update (opts->nsub / sub_idx are ignored: the object's subsample
 * is used).  Intervals continue the object's windows across calls. */
vp_status vp_hyper_step(vp_hyper* h, double* Q_dev, double* Z_dev, double dt, int32_t nsteps,
                        const vp_step_opts* opts, double* trace_dev, int32_t* iters_dev,
                        double* kstate_dev, void* stream);
/* State of the last interval: intervals done, DMD-DEIM intervals done, DMD
 * rank (0 before the first DMD-DEIM interval); idx_dev (nullable, d int32)
 * receives the current DEIM indices, Phi_dev (nullable, p x Nx) the DMD
 * potentials at the last coefficient stage time. */
vp_status vp_hyper_info(vp_hyper* h, int32_t* intervals, int32_t* hyper_intervals, int32_t* r_dmd,
                        int32_t* idx_dev, double* Phi_dev, void* stream);
vp_status vp_hyper_destroy(vp_hyper* h);

/* -------------------------------------------------- deposit, no allocation */
/* The paper has no counterpart to this call; it exists for callers that may
 * not allocate device memory (their pool or fixed memory plan owns it all,
 * or the device-wide synchronisation of cudaFree is unacceptable).
 * Same result as vp_deposit_cic (bit-identical counts), without a context:
 * the fixed-point charge counts live in one device array that the library
 * declares at file scope, 131072 int64 (1 MiB), held by every GPU that loads
 * the library until the process exits.  Nothing is allocated: no cudaMalloc,
 * cudaFree or allocating library routine.
 * - Limit: p * Nx <= 131072; larger requests return VP_EUNSUPPORTED and
 *   launch nothing.
 * - Works on the caller's current device, in its primary context (the one
 *   the CUDA runtime uses).  The first call on each device looks up the
 *   array's device address (cudaGetSymbolAddress); make that first call
 *   before any stream capture.
 * - Invalid arguments (a non-finite L, mp, Mq or background included) return
 *   VP_EINVAL; a failed launch returns VP_ECUDA for this call's own launches
 *   only.
 * - All calls on a device share the array.  Each call clears the part it uses
 *   before depositing, but calls whose work overlaps on the GPU (two streams,
 *   two host threads) race on it and give wrong results: serialise them. */
vp_status vp_deposit_cic_noalloc(const vp_grid* grid, int64_t N, int32_t p, const double* X_dev,
                                 int64_t ldx, double* rho_dev, void* stream);

/* ---------------------------------------------------------------- loading */
/* Macro-particles of p samples on the device (Sec. 6.1, eq.
 * initial_distribution): particle l of sample i sits at x = F_x^-1(u_x),
 * v = F_v^-1(u_v), F_x the CDF of (1 + alpha cos kx)/L on [0, L), F_v the CDF
 * of the family's Gaussian mixture truncated to [-10, 10].
 * mode 0, quiet start: u_x = phi_2(l) (base-2 radical inverse), u_v =
 * (l + 1/2)/N (2-D Hammersley set); seed unused.
 * mode 1, seeded: one Philox4x32-10 block per particle (Salmon et al. 2011)
 * with counter (l mod 2^32, l div 2^32, i, 0) and key (seed mod 2^32,
 * seed div 2^32); u_x = (w0 >> 5, w1 >> 6) and u_v = (w2 >> 5, w3 >> 6) as
 * 53-bit fractions.
 * family: 0 Landau damping (k = 0.5; eta_i = {alpha, sigma, unused}),
 * 1 two-stream (k = 0.2; eta_i = {v0, sigma, alpha}: streams at +-v0, weights
 * 1/2), 2 bump-on-tail (k = 0.5; eta_i = {vb, alpha, sigma_b}: 0.9 N(0,1) +
 * 0.1 N(vb, sigma_b^2)).  eta_dev: p x 3 doubles; X_dev, V_dev: p x N.
 * Inverses are solved to ~1e-14 relative; values agree with an FP64 host
 * evaluation of the same inverse CDFs to that level, not bit for bit. */
vp_status vp_load_particles(vp_ctx* ctx, int32_t family, int32_t mode, uint64_t seed, int64_t N,
                            int32_t p, const double* eta_dev, double* X_dev, double* V_dev,
                            void* stream);

/* ------------------------------------------------------------ checkpoint */
/* A reduced state as one host byte image: a header of 8 int64 {magic
 * "VPSTATE1", version 1, N, n, p, step, has_k, 0}, then Q (N x 2n), Z (2n x p)
 * and, with has_k, the fixed-point state k (2n x p) that warm-starts
 * vp_basis_update.  Restarting from an image continues bit for bit: the step
 * reads nothing else (the grid and options are the caller's). */
size_t vp_state_bytes(int64_t N, int32_t n, int32_t p, int32_t with_k);
/* Copies device Q, Z, K (K nullable) into `host` (host_bytes >= vp_state_bytes)
 * and synchronises `stream`. */
vp_status vp_state_export(vp_ctx* ctx, int64_t N, int32_t n, int32_t p, const double* Q_dev,
                          const double* Z_dev, const double* K_dev, int64_t step, void* host,
                          size_t host_bytes, void* stream);
/* Checks magic, version and sizes against (N, n, p), copies the image into
 * device Q, Z and (if K_dev is given; the image must then hold k) K, returns
 * the step count in *step (nullable) and synchronises `stream`.  Mismatch or
 * truncation: VP_EINVAL, nothing copied. */
vp_status vp_state_import(vp_ctx* ctx, const void* host, size_t host_bytes, int64_t N, int32_t n,
                          int32_t p, double* Q_dev, double* Z_dev, double* K_dev, int64_t* step,
                          void* stream);

/* --------------------------------------------------------------- serving */
/* Many-query serving of the parametric reduced model (Sec. 6: one query = one
 * parameter set of p samples, evolved from its own start).  A server owns one
 * device, an HBM budget and a number of slots.  Queries wait in FIFO order
 * and are admitted while a slot is free and their device bytes fit in what
 * the budget has left; each admitted query runs on its own context, stream and
 * host thread: particle load (vp_load_particles), truncated complex SVD start
 * (vp_init_csvd) with the rank chosen at t = 0 from the singular values:
 * n = the smallest k in [n_min, n_max] whose relative tail energy
 * sum_{j>k} sigma_j^2 / sum_j sigma_j^2 < rank_tol (n_max if none), lowered
 * while sigma_n < 1e-6 sigma_1 so that S(Z) stays invertible; then nsteps
 * partitioned RK2 steps (vp_basis_update, warm-started, in chunks of 16
 * steps; arith 2 re-orthonormalises each step).  The grid is
 * q = -1, m = 1, omega = L/N with a neutralising background.  Every kernel is
 * deterministic, so a query's result is the same alone or beside others. */
typedef struct vp_server vp_server;

typedef struct vp_query {
  int32_t family;   /* as vp_load_particles */
  int32_t loading;  /* vp_load_particles mode: 0 quiet start, 1 Philox-seeded */
  uint64_t seed;    /* key of the seeded loading */
  int32_t p;        /* samples, 1..256 */
  int64_t N;        /* particles per sample, 2..2^31-1 */
  int32_t Nx;       /* grid nodes, 3..1024 */
  int32_t n_max;    /* largest reduced rank n (2n columns), 1..min(p, 40) */
  int32_t n_min;    /* smallest reduced rank, 1..n_max */
  double rank_tol;  /* relative tail energy left out by the rank (e.g. 1e-8) */
  double dt;
  int32_t nsteps;
  int32_t arith;        /* as vp_step_opts.arith */
  const double* eta;    /* host, p x 3; copied at submit */
  double* trace_host;   /* host (nullable), nsteps x p x 2: E and H entering each step */
  double* zeta_host;    /* host (nullable), 2 n_max x p: final Z (first 2n x p written) */
} vp_query;

typedef struct vp_result {
  int32_t status;     /* VP_OK, VP_EAGAIN (cancelled) or the first error */
  int32_t n;          /* reduced rank chosen */
  int32_t steps_done;
  int32_t max_iters;  /* largest fixed-point iteration count of a step */
  double t_submit, t_admit, t_start, t_done; /* seconds since server creation;
                                                t_start: end of the start phase */
} vp_result;

/* hbm_budget: device bytes all running queries may hold together;
 * max_slots >= 1 queries run at once. */
vp_status vp_server_create(vp_server** out, int device, size_t hbm_budget, int max_slots);
/* Queue a query.  The caller's output buffers must stay valid until the poll
 * that returns it.  VP_EINVAL: bad sizes; VP_EUNSUPPORTED: 4 n_max^2 +
 * 2 n_max p > 25600; VP_ENOMEM: the query alone exceeds the budget; VP_EBUSY:
 * 4096 queries waiting or the server is stopping. */
vp_status vp_serve_submit(vp_server* srv, const vp_query* q, uint64_t* ticket);
/* Wait up to timeout_ms (0: do not wait) for a query.  VP_OK: done, *res
 * filled (res->status is the query's own status) and the ticket released;
 * VP_EAGAIN (timeout_ms = 0) / VP_ETIMEDOUT: not done yet, ticket kept;
 * VP_EINVAL: unknown or released ticket. */
vp_status vp_serve_poll(vp_server* srv, uint64_t ticket, vp_result* res, int32_t timeout_ms);
/* Cancel a query: a waiting query finishes at once with status VP_EAGAIN; a
 * running one stops at its next 16-step boundary with VP_EAGAIN. */
vp_status vp_serve_cancel(vp_server* srv, uint64_t ticket);
/* Counters (each nullable). */
vp_status vp_server_stats(vp_server* srv, int64_t* submitted, int64_t* completed, int32_t* active,
                          int32_t* pending, size_t* used_bytes);
/* Let waiting and running queries finish for up to drain_timeout_ms (0: not
 * at all), then drop the waiting ones, cancel the running ones at their next
 * 16-step boundary, join every thread and free.  Returns VP_ETIMEDOUT when
 * queries were still waiting or running at the timeout (the server is freed
 * all the same), VP_EINVAL for a negative timeout. */
vp_status vp_server_destroy(vp_server* srv, int32_t drain_timeout_ms);

/* ---------------------------------------------------------------- tuning */
/* Launch shape of the FP32-based particle kernels (arith 1 and 2): each
 * knob sizes its kernel's grid for this many resident blocks per SM (1..32).
 * Defaults {4, 4, 4, 8, 8} (measured on the two-stream workload).  The paper
 * has no counterpart. */
typedef enum vp_tune_knob {
  VP_TUNE_DEPOSIT_LP = 0, VP_TUNE_PROJECT_LP, VP_TUNE_BASIS_M_LP, VP_TUNE_GRAM_LP,
  VP_TUNE_AFFINE_LP, VP_TUNE_COUNT
} vp_tune_knob;
vp_status vp_tune_set(vp_ctx* ctx, int32_t knob, int32_t blocks_per_sm);
/* Tensor-core kernels of the FP32 form (arith = 2; tcgen05, kind::tf32, FP32
 * values split into TF32 pieces, FP32 accumulation in tensor memory), one
 * bit each: the reconstruction X_r = U_X Z of the deposit (Sec. 3.2; 2n <= 64
 * a multiple of 4, sample chunks of 16 or 32), the projection g_X = U_X^T G
 * (eq. grads; 2n <= 64), the Gram matrices X^H Y and U_V^T U_V (2n <= 64),
 * the basis velocity Gamma zeta^H (Sec. 3.2, 5; 2n <= 64) and the row
 * combinations sum_t X_t C_t of the basis velocity, the Cayley retraction and
 * the tangent velocity (2n <= 64).  A kernel whose bit is clear, or whose
 * shape does not apply, runs on the FP32 CUDA cores. */
typedef enum vp_tc_kernel {
  VP_TC_DEPOSIT = 1, VP_TC_PROJECT = 2, VP_TC_GRAM = 4, VP_TC_BASIS_M = 8, VP_TC_AFFINE = 16,
  VP_TC_ALL = 31,
  /* the default leaves the deposit on the CUDA cores: its cell and weight
   * come from the position, whose two-piece TF32 split (2^-22 of each
   * operand) measurably adds to the energy error of a step */
  VP_TC_DEFAULT = VP_TC_PROJECT | VP_TC_GRAM | VP_TC_BASIS_M | VP_TC_AFFINE
} vp_tc_kernel;
/* mask: an OR of vp_tc_kernel bits (default VP_TC_DEFAULT; 0: all SIMT).
 * Values outside [0, VP_TC_ALL]: VP_EINVAL. */
vp_status vp_tensor_cores(vp_ctx* ctx, int32_t mask);
vp_status vp_tune_get(vp_ctx* ctx, int32_t knob, int32_t* blocks_per_sm);
/* Autotuner: on the caller's state (Q N x 2n, Z 2n x p; read only) times
 * every knob's kernel at 1, 2, 3, 4, 6 and 8 blocks per SM (`reps` launches
 * each, CUDA events on `stream`), keeps the fastest in the context and
 * writes the choices to chosen[VP_TUNE_COUNT] (nullable).  Results of later
 * calls change only by the order of partial sums.  Synchronises `stream`. */
vp_status vp_autotune(vp_ctx* ctx, const vp_grid* grid, int64_t N, int32_t n, int32_t p,
                      const double* Q_dev, const double* Z_dev, int32_t arith, int32_t reps,
                      int32_t* chosen, void* stream);

/* --------------------------------------------------------------- batched */
/* Many independent reduced models advanced together (each its own grid, N,
 * n, p, dt and state; Sec. 5 steps).  The three phases of a step (field,
 * energies and basis stage with the first fixed-point rounds; further
 * rounds; Z update, tangent velocity and Cayley retraction) are captured
 * once for all instances into three CUDA graphs whose instances are parallel
 * branches.  A step launches the first graph, checks every instance's
 * convergence with one small kernel and one synchronisation of `stream`,
 * launches the rounds graph until all have converged (converged instances
 * return at once), then the last graph.  Per instance the kernels and their
 * order are those of vp_basis_update with arith 1 or 2 and a warm-started
 * fixed point, so each instance's state equals (bit for bit) that of its own
 * vp_basis_update call with kstate.  The paper has no batched form. */
typedef struct vp_batch vp_batch;

typedef struct vp_batch_item {
  vp_grid grid;
  int64_t N;
  int32_t n, p;
  double dt;
  double* Q_dev;       /* N x 2n, advanced in place */
  double* Z_dev;       /* 2n x p, advanced in place */
  double* kstate_dev;  /* 2n x p warm start (nullable: internal, zero at creation) */
  double* trace_dev;   /* nullable: trace_capacity x p x 2, E and H entering each step */
  int32_t trace_capacity;
  int32_t* iters_dev;  /* nullable: trace_capacity fixed-point iteration counts */
} vp_batch_item;

/* opts: arith 1 or 2 (others as vp_basis_update; reortho honoured).
 * rounds_first / rounds_more: fixed-point rounds in the first and in the
 * repeated graph.  scratch_per_instance: workspace budget of each instance's
 * context (0: 16 GiB).  The items' buffers must stay valid until destroy.
 * Synchronises the device. */
vp_status vp_batch_create(vp_batch** out, int device, const vp_batch_item* items, int32_t count,
                          const vp_step_opts* opts, int32_t rounds_first, int32_t rounds_more,
                          size_t scratch_per_instance);
/* nsteps steps of every instance on `stream` (one synchronisation per
 * convergence check; returns after the last step has finished).  The first
 * instance error found is returned (vp_batch_last_error names the instance). */
vp_status vp_batch_step(vp_batch* b, int32_t nsteps, void* stream);
/* Steps done, kernel launches made so far, kernel nodes of the three graphs. */
vp_status vp_batch_info(const vp_batch* b, int64_t* steps_done, int64_t* launches,
                        int64_t* graph_nodes);
/* Message of the last error of b; b = NULL: of the last failed vp_batch_create
 * on the calling thread. */
const char* vp_batch_last_error(const vp_batch* b);
vp_status vp_batch_destroy(vp_batch* b);

/* ------------------------------------------------------------ self-test */
/* Failure-detection check of the bounded waits: launches one block that waits
 * on an mbarrier nothing completes, `spins` polls (1 .. 2^22), after which it
 * records VP_ETIMEDOUT in the status word (read by vp_ctx_sync_status) and
 * ends.  The library's own waits (bulk copies completing on mbarriers) use
 * 2^22 polls and report the same way.  The paper has no counterpart. */
vp_status vp_selftest_wait(vp_ctx* ctx, int32_t spins, void* stream);

/* ------------------------------------------------------------ profiling */
/* Kernels of the library, for launch counts and event timing.  One id may
 * cover a family of kernels: VP_K_DEIM the DEIM basis, indices, weights and
 * snapshot columns; VP_K_DMD the DMD fit, coordinates, RBF interpolation and
 * predicted potentials; VP_K_JACOBI_SYM the real symmetric Jacobi of both;
 * VP_K_HYPER the per-interval window and operator work of vp_hyper_step;
 * VP_K_INIT the complex-SVD start and the re-orthonormalisation factor;
 * VP_K_DEPOSIT_DIAG the double-float deposit of the FP64-accurate energy
 * diagnostic in the FP32 form (arith = 2), apart from its FP32 deposits;
 * VP_K_PROJECT_TC the projection, VP_K_DEPOSIT_TC the deposit and
 * VP_K_GRAM_TC the Gram matrices (complex pairs and the real G_V),
 * VP_K_BASIS_M_TC the basis velocity product Gamma zeta^H and VP_K_AFFINE_TC
 * the row combinations sum_t X_t C_t of the FP32 form with their
 * contractions on the tensor cores. */
typedef enum vp_kernel {
  VP_K_DEPOSIT = 0, VP_K_RHO, VP_K_POISSON, VP_K_GATHER, VP_K_FULL_STEP, VP_K_RECONSTRUCT,
  VP_K_DEPOSIT_REDUCED, VP_K_PROJECT, VP_K_BASIS_M, VP_K_GRAM, VP_K_GRAM_REAL, VP_K_REDUCE,
  VP_K_AFFINE, VP_K_CELL_GRADIENT, VP_K_SMALL_BASIS, VP_K_SMALL_CAYLEY, VP_K_SMALL_TANGENT,
  VP_K_COEFF_UPDATE, VP_K_AXPY, VP_K_ADD_LINEAR, VP_K_ENERGIES, VP_K_SPLIT, VP_K_DEPOSIT_LP,
  VP_K_PROJECT_LP, VP_K_BASIS_M_LP, VP_K_PREP_LP, VP_K_GRAM_LP, VP_K_GRAM_REAL_LP, VP_K_AFFINE_LP,
  VP_K_INIT, VP_K_LOAD, VP_K_SUBSET, VP_K_HYPER, VP_K_DEIM_ROUND, VP_K_DEIM, VP_K_DMD,
  VP_K_JACOBI_SYM, VP_K_DEPOSIT_DIAG, VP_K_PROJECT_TC, VP_K_DEPOSIT_TC,
  VP_K_GRAM_TC, VP_K_BASIS_M_TC, VP_K_AFFINE_TC, VP_K_COUNT
} vp_kernel;

/* Every launch is counted per kernel.  Kernels whose bit (1 << vp_kernel) is
 * set in `mask` are also timed: a CUDA event pair is recorded around each
 * launch on the launch stream and resolved at the next synchronisation
 * point (vp_profile_read synchronises the context's device).  mask = 0
 * stops timing. */
vp_status vp_profile_enable(vp_ctx* ctx, uint64_t mask);
/* Launch count, timed launches and summed event time (ms) of one kernel. */
vp_status vp_profile_read(vp_ctx* ctx, int32_t kernel, int64_t* launches, int64_t* timed,
                          double* ms_total);
vp_status vp_profile_reset(vp_ctx* ctx);
const char* vp_kernel_name(int32_t kernel);

#ifdef __cplusplus
}
#endif
#endif /* VP_H */
