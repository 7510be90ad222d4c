/*
 * dyson.h — C ABI of the GB300 lattice Dyson solver.
 *
 * Solves the lattice Dyson equation of Dirks, Mikelsons, Krishnamurthy and
 * Freericks (arXiv:1309.5994), Sec. IV.D, Eqs. (Glatt2) and (Ginvblockstruct),
 * on the discretised Kadanoff-Baym-Keldysh contour of Sec. IV.A / Fig. 1:
 *
 *     G = Lambda + Lambda W J G,
 *
 * for a trapped 2D Fermi-Hubbard lattice (Sec. II, Eq. (model)), where
 * Lambda_i(z,z') is the atomic-limit contour Green's function of site i
 * (Sec. III; the block-diagonal preconditioner B^-1 of Sec. IV.D with no
 * self-energy), J_ij(t) the nearest-neighbour hopping (diagonal in contour
 * time) and W(z) the contour quadrature weights.  The solve runs block column
 * by block column (one source site, all Nc source times) with the series in
 * powers of J of App. C, G <- Lambda delta_s + K G.
 *
 * Conventions (shared with the CPU oracle, each side implements them itself):
 *   sites   i = y*Lx + x, open boundaries;
 *   bonds   horizontal (x,y)-(x+1,y) first, index y*(Lx-1)+x; then vertical
 *           (x,y)-(x,y+1), index Ly*(Lx-1) + y*Lx + x;  Nb = Ly(Lx-1)+Lx(Ly-1);
 *   contour Nc = 2*Nt + Nm points in contour order: forward t_k = k*dt
 *           (index k), backward (index Nt+q carries t_{Nt-1-q}), imaginary
 *           tau_m = m*beta/Nm (index 2Nt+m); weights +dt, -dt, -i*beta/Nm;
 *   trap    V_i = curvature * |r_i|^2 about the geometric lattice centre,
 *           eps_i = V_i - U_i(0)/2 - mu (Eq. (onsitelevels)).
 *   complex numbers are interleaved (re, im) pairs of doubles.
 *
 * Ownership: the context owns every device buffer it allocates (Lambda, its
 * split-precision copies, hopping tables, observables, work buffers).  The
 * caller owns every pointer it passes in; none is retained after a call
 * returns.  All device work is ordered on the stream given to dyson_init.
 *
 * Threads and streams: a context is not thread-safe; calls on one context must
 * not overlap.  Distinct contexts may be used from distinct threads.  Every call
 * on a context (or batch) that computes returns only after its work on the
 * context's stream has finished (results written), so the caller needs no extra
 * synchronisation before reading them; device buffers the caller passes must not
 * be written by other streams while a call runs.  dyson_extrapolate_dt, which
 * takes no context, is asynchronous on the stream it is given.
 *
 * Errors: every int-returning call returns DYSON_OK (0) or a negative
 * DYSON_ERR_* code and never throws; dyson_last_error() describes the last
 * failure of a context.  No call falls back to a CPU implementation.
 */
#ifndef DYSON_H
#define DYSON_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  DYSON_OK = 0,
  DYSON_ERR_INVALID_ARG = -1,   /* a size, pointer or option is out of range            */
  DYSON_ERR_OOM = -2,           /* device allocation failed                              */
  DYSON_ERR_NOT_CONVERGED = -3, /* max_sweeps reached above tolerance (results written)  */
  DYSON_ERR_DIVERGED = -4,      /* the series does not converge: the FP64 update passes  */
                                /* 2^52 (rounding exceeds the result), an update or      */
                                /* residual is not finite, or refinement residuals grow  */
                                /* twice (spectral radius of Lambda W J above 1)         */
  DYSON_ERR_TIMEOUT = -5,       /* a bounded device wait expired                          */
  DYSON_ERR_CUDA = -6,          /* a CUDA runtime call failed                             */
  DYSON_ERR_STATE = -7          /* call order violated (e.g. solve before build_sigma)    */
};

/* Arithmetic of the sweeps (App. C series). */
enum {
  DYSON_PREC_F64 = 0,           /* complex128 sweeps on the FP64 pipes                   */
  DYSON_PREC_TF32X3_F64REF = 1  /* complex FP32 sweeps as 3xTF32 tcgen05 products with
                                   FP32 accumulation, refined by FP64 Dyson residuals     */
};

typedef struct dyson_ctx dyson_ctx;

typedef struct {
  int32_t Lx, Ly;               /* lattice sides, >= 1 each, Lx*Ly <= 65535               */
} dyson_lattice;

typedef struct {
  int32_t Nt;                   /* real-time points per branch, >= 1                      */
  int32_t Nm;                   /* imaginary-time points, >= 1; 2*Nt+Nm <= 2048            */
  double dt;                    /* real-time step, > 0                                    */
  double beta;                  /* inverse temperature of the initial state, > 0          */
} dyson_contour;

typedef struct {
  double curvature;             /* V_trap(r) = curvature * |r|^2                          */
  double mu;                    /* chemical potential of the initial state                */
} dyson_trap;

typedef struct {
  const double* U;              /* host, [Nr][Nt]: U_i(t_k) (U_i(0) also sets eps_i)      */
  const double* J;              /* host, [Nb][Nt]: J_b(t_k); the imaginary branch uses J_b(0) */
} dyson_drive;

typedef struct {
  int32_t sweeps;               /* total series sweeps over all chunks and refinements     */
  int32_t refinements;          /* FP64 residual evaluations (mixed precision)             */
  int32_t chunks;               /* column chunks processed                                 */
  int32_t status;               /* same code the call returned                             */
  double update;                /* last relative max-norm update of the series             */
  double residual;              /* last relative max-norm FP64 residual (mixed precision)  */
  double gemm_flops;            /* algorithmic contour-GEMM flops: 8 Nc^3 per site,
                                   block column and sweep, over every sweep performed      */
  double seconds;               /* wall time of the call                                   */
  int64_t kernel_launches;      /* CUDA kernels this call launched                         */
  int32_t inner_gmres;          /* 1 if a refinement used the GMRES inner solver (its      */
                                /* matvecs are counted in sweeps), else 0                  */
  int32_t host_syncs;           /* times the call waited for the device: norm and error     */
                                /* reads, one per GMRES step, one per graph replay of the   */
                                /* inner series (one per sweep without graphs)              */
} dyson_report;

/* Create a context on `device`, ordering work on `cuda_stream` (a cudaStream_t,
 * NULL for the legacy default stream).  Copies the host drive tables; allocates
 * Lambda storage (16*Nr*Nc^2 bytes) and small tables.  Sec. II (model),
 * Sec. IV.A (contour).  Returns INVALID_ARG for out-of-range sizes, OOM if the
 * device cannot hold Lambda. */
int dyson_init(dyson_ctx** out, const dyson_lattice* lattice, const dyson_contour* contour,
               const dyson_trap* trap, const dyson_drive* drive, int device, void* cuda_stream);

/* Build Lambda_i(z,z') of every site in FP64 on the device: Boltzmann weights
 * of H_0^(i)(0) (Eq. (Z)), the tabulated phases of Eq. (cumulanttabulation)
 * (left rule dt*sum_{m<k} E(t_m) on the real branches, -i*tau*E(0) on the
 * imaginary one) and the closed form of the two transition channels (Sec. III).
 * Equal contour points are 'lesser' on the forward and imaginary branches and
 * 'greater' on the backward branch. */
int dyson_build_sigma(dyson_ctx* ctx);

/* Copy Lambda, [Nr][Nc][Nc] complex128 (row z, column z'), into dst (caller
 * owned, 16*Nr*Nc*Nc bytes; device memory if on_device != 0, else host).
 * Returns STATE before dyson_build_sigma. */
int dyson_copy_sigma(dyson_ctx* ctx, double* dst, int on_device);

/* Solve block columns G(:, s) for the n_src source sites src_sites (host array,
 * each in [0, Nr), repeats allowed) with the App. C series, to a relative
 * max-norm update (F64) or FP64 residual (mixed precision) <= tol, relative to
 * max|Lambda_s|, within max_sweeps series sweeps per solve.  Columns are
 * processed in chunks sized to the free device memory.
 *   g_out: NULL, or a caller-owned DEVICE buffer of n_src*Nr*Nc*Nc complex128
 *          receiving G_js(z, z') at [q][j][z][z'] for source src_sites[q].
 * Observables of every source site are computed as a side effect (see
 * dyson_observables).  rep may be NULL. */
int dyson_solve_columns(dyson_ctx* ctx, const int32_t* src_sites, int64_t n_src, int precision,
                        double tol, int32_t max_sweeps, double* g_out, dyson_report* rep);

/* Solve n single vector columns G(:, (s_q, z'_q)): the response to one source site
 * s_q = sites[q] at one source time z'_q = times[q] (host arrays; 0 <= s < Nr,
 * 0 <= z' < Nc), the unit-vector right-hand sides of Sec. IV.D.  Same series,
 * precisions and tolerances as dyson_solve_columns; columns are solved in
 * groups of 32 (the last group padded with zero columns).  No observables.
 *   g_out: NULL or a caller-owned DEVICE buffer of n*Nr*Nc complex128 receiving
 *          G_{j s_q}(z, z'_q) at [q][j][z]. */
int dyson_solve_vector_columns(dyson_ctx* ctx, const int32_t* sites, const int32_t* times, int64_t n,
                               int precision, double tol, int32_t max_sweeps, double* g_out,
                               dyson_report* rep);

/* Transpose every site block Lambda_i in place (call again to undo).  While
 * transposed, solves return columns of G^T, i.e. rows of G: G^T solves the same
 * Dyson equation with Lambda_i^T because W and J commute and J is symmetric.
 * dyson_solve_columns returns DYSON_ERR_STATE in this state (its observables
 * need columns of G). */
int dyson_transpose_sigma(dyson_ctx* ctx);

/* Gradients of L = sum_i w_i n_i(t_k), the weighted density per spin at forward
 * time index t_index (Sec. III.A), with respect to every U_i(t_k) and J_b(t_k)
 * of the drive tables.  The paper has no gradient; the derivation is
 *   dG = (I + G W J) dLambda (I + W J G) + G W dJ G,
 * with the columns G e_i and rows e_i^T G (solved on transposed site blocks, see
 * dyson_transpose_sigma) at (i, t_index) for every site, and the derivative of
 * the closed form of Lambda (Sec. III) in U, which includes the dependence of
 * eps_i and of the Boltzmann weights on U_i(0).
 *   w       host, [Nr] site weights;
 *   loss    host, optional: L;
 *   grad_U  host, optional: [Nr][Nt];  grad_J host, optional: [Nb][Nt].
 * Solves 2 Nr vector columns with the given precision/tolerance; device memory
 * 16 (4 Nr^2 Nc + Nr Nc^2) bytes beyond the solves.  Gradients with respect to
 * scalar drive parameters follow by the chain rule through the tables. */
int dyson_adjoint(dyson_ctx* ctx, const double* w, int32_t t_index, int precision, double tol,
                  int32_t max_sweeps, double* loss, double* grad_U, double* grad_J, dyson_report* rep);

/* The same adjoint for L = sum_i w_density[i] n_i(t_f) + w_docc[i] D_i(t_f), the
 * double occupancy D of Eq. (docc) read as dyson_observables reads it (App. B's
 * one-sided difference; t_index >= 1).  Either weight array may be NULL, not both.
 * D is real-linear in the same column G e_(i, t_f), through its entries at
 * (i, t_f), (i, t_f - 1) and the neighbours (j, t_f), so the gradient needs the
 * rows of G at (i, t_f) and (i, t_f - 1): 2 Nr transposed vector-column solves
 * besides the Nr columns.  It also takes D's explicit dependence on U_i(t_f)
 * (1/U), U_i(0) (through eps_i) and J_ij(t_f) (through e_kin).  Layouts and
 * codes as dyson_adjoint. */
int dyson_adjoint_obs(dyson_ctx* ctx, const double* w_density, const double* w_docc, int32_t t_index,
                      int precision, double tol, int32_t max_sweeps, double* loss, double* grad_U, double* grad_J,
                      dyson_report* rep);

/* Observables of the sites solved so far (Sec. III.A, Eq. (docc), App. B):
 * density per spin n_i(t_k), kinetic energy ekin_i(t_k) and double occupancy
 * D_i(t_k), each [Nr][Nt] doubles.  Sites never solved hold NaN; D_i(t_0) is
 * NaN (the difference quotient needs t_{k-1}).  The kinetic energy is
 * Re[-i sum_j J_ij G_ji(t,t)]: the solved G is that of hopping +J, the gauge
 * image of Eq. (model) on the bipartite lattice.  Each pointer may be NULL;
 * on_device != 0 means the pointers are device memory, else host memory. */
int dyson_observables(dyson_ctx* ctx, double* n, double* ekin, double* docc, int on_device);

/* Local Green's functions: solves the block columns of the sites src[0..n_src)
 * as dyson_solve_columns does (same precision, tolerance, report and codes;
 * observables are recorded too) and writes only their diagonal blocks,
 * gloc[s][z][z'] = G_ss(z, z'), DEVICE memory [Nr][Nc][Nc] complex128 (rows of
 * sites not in src are left untouched).  With DYSON_SYMMETRY_C4V one site per
 * orbit is solved and every other requested site receives its representative's
 * block (G_{g(r), g(r)} = G_{r, r}, App. A; the representative's own row is
 * written too, requested or not); this holds while the installed local
 * blocks are C4v-invariant too, as they stay when every self-energy step is fed
 * local Green's functions of this kind.  The input of the self-energy step below. */
int dyson_local_greens(dyson_ctx* ctx, const int32_t* src_sites, int64_t n_src, int precision, double tol,
                       int32_t max_sweeps, double* gloc, dyson_report* rep);

/* Self-energy step of the strong-coupling expansion (Sec. III, Eqs. (selfcons),
 * (defnSigma), (defnSigmatilde); Sec. IV.C, Eq. (Sigmamix)).  From the local
 * Green's functions gloc of every site (DEVICE [Nr][Nc][Nc] complex128, e.g. from
 * dyson_local_greens over all sites):
 *   Sigma~_i(a, d) = - sum_{j in NN(i)} sum_{b, c} K_i(a, b; c, d) W_c J_ij(c) Gloc_j(c, b) J_ji(b) W_b,
 * K_i the second-order cumulant of the isolated site i summed over the
 * neighbour's spin, evaluated on the fly from the site's phases (O(Nc^4) per
 * site, FP64); Sigma = G0^-1 * Sigma~ * G0^-1 (Eq. (defnSigma); G0 = the atomic
 * Lambda of the last dyson_build_sigma) is mixed as Sigma = mix Sigma_new +
 * (1 - mix) Sigma_old (Sigma_old = 0 after dyson_build_sigma; being linear in
 * Sigma~, the mixing is applied to Sigma~), and the local block
 *   B_i = G0_i (G0_i - Sigma~_i)^-1 G0_i,
 * the solution of the local Dyson equation B = G0 + G0 * Sigma * B, replaces
 * Lambda_i for the following solves (all precisions).  The two turning points of
 * the discretised contour make G0 - Sigma~ singular by one rank; the system is
 * completed along those directions, which leaves B unchanged.
 *   sigma_tilde  DEVICE [Nr][Nc][Nc] complex128 or NULL: receives Sigma~_new;
 *   criterion    host or NULL: N_bd^-1 |Sigma~_new - Sigma~_old|_F + |Sigma~_new - Sigma~_old|_max
 *                (N_bd = Nr Nc^2 block-diagonal entries), Sec. IV.C's measure taken on Sigma~
 *                (Sigma itself divides by a singular value of G0 that falls exponentially
 *                with the real-time branch length).
 * With DYSON_SYMMETRY_C4V set, the cumulant contraction runs for one site per
 * orbit and the other sites take their representative's (App. A); gloc must
 * then be C4v-invariant, as dyson_local_greens under C4v returns it.
 * dyson_build_sigma returns to Sigma = 0.  Device memory: 7 Nr Nc^2 complex128.
 * Returns INVALID_ARG for mix outside (0, 1] or a NULL gloc, STATE before
 * dyson_build_sigma or with Lambda transposed, DIVERGED if a local system is
 * singular.  dyson_adjoint and dyson_adjoint_obs return STATE while a local block
 * is installed (they differentiate the atomic Lambda). */
int dyson_selfenergy_step(dyson_ctx* ctx, const double* gloc, double mix, double* sigma_tilde, double* criterion);

/* Mixing of the self-energy steps: depth 0 (the default) is the linear mixing of
 * Eq. (Sigmamix); depth 1..6 replaces it by Anderson acceleration of the fixed-point
 * iteration Sigma~ -> Sigma~_new (an addition to the paper, same fixed point): with
 * the residual f = Sigma~_new - Sigma~ and the differences dF_i, dX_i of the last
 * depth residuals and iterates, gamma minimises |f - sum_i gamma_i dF_i|_2 and
 *   Sigma~ <- Sigma~ + mix f - sum_i gamma_i (dX_i + mix dF_i).
 * The history restarts here and at dyson_build_sigma.  Device memory: 2 depth + 3
 * more Nr Nc^2 complex128 arrays on the first Anderson step.  INVALID_ARG for a depth
 * outside 0..6. */
#define DYSON_SELFENERGY_MAX_ANDERSON 6
int dyson_selfenergy_set_anderson(dyson_ctx* ctx, int32_t depth);

/* Delta t -> 0 extrapolation (Sec. IV.D).  The same tables computed on n_grids
 * contours whose steps are h_b = h_0 / m_b (integer divisors, m_0 = 1 < m_1 <
 * ...; the real-time grid of contour b has at least m_b (nt[0] - 1) + 1
 * points, e.g. m_b nt[0] with m_b times the points on every branch) are
 * combined at the coarsest grid's times
 * t_k = k h_0, which are index k m_b of grid b, with the weights of the
 * polynomial of degree n_grids - 1 through the points (h_b, f_b) evaluated at
 * h = 0 (Lagrange form):
 *     out[r][k] = sum_b values[b][r][k m_b] prod_{c != b} h_c / (h_c - h_b).
 * n_grids = 3 is the paper's quadratic extrapolation, 2 the linear one it
 * cross-checks with.
 *   values  host array of n_grids DEVICE pointers; values[b] is [rows][nt[b]]
 *           doubles (e.g. a table of dyson_observables on the context of grid b);
 *   nt      host, [n_grids] time points per row;  m  host, [n_grids] divisors;
 *   out     device, [rows][nt[0]] doubles (may not alias an input).
 * NaN inputs (D at t = 0) give NaN.  Runs on `stream` (NULL: the legacy default
 * stream) of `device`.  Returns DYSON_ERR_INVALID_ARG for n_grids outside 1..4,
 * divisors that do not start at 1 or do not increase, a grid shorter than
 * m_b (nt[0] - 1) + 1, rows < 1 or a NULL pointer (message in
 * dyson_last_error(NULL)), DYSON_ERR_CUDA if the launch fails. */
#define DYSON_EXTRAPOLATE_MAX_GRIDS 4
int dyson_extrapolate_dt(int32_t n_grids, const double* const* values, const int32_t* nt, const int32_t* m,
                         int32_t rows, double* out, int device, void* stream);

void dyson_destroy(dyson_ctx* ctx);
const char* dyson_last_error(const dyson_ctx* ctx);

/* Kernel kinds timed by the optional per-launch CUDA-event profiler. */
enum {
  DYSON_KERNEL_SWEEP_F64 = 0,     /* FP64 series sweep (gather + complex GEMM)               */
  DYSON_KERNEL_SWEEP_F32 = 1,     /* FP32 CUDA-core sweep                                    */
  DYSON_KERNEL_SWEEP_TC = 2,      /* 3xTF32 tcgen05 sweep GEMM (split + MMA + epilogue)      */
  DYSON_KERNEL_RESIDUAL_F64 = 3,  /* FP64 Dyson residual r = Lambda delta + K G - G          */
  DYSON_KERNEL_RESIDUAL_SPLIT = 4,/* the same residual from BF16 slice products on tcgen05   */
  DYSON_KERNEL_SWEEP_TC_PAIR = 5, /* the same GEMM on CTA pairs (tcgen05 cta_group::2, M=256) */
  DYSON_KERNEL_GATHER_TC = 6,     /* neighbour gather X = J d of the tensor-core sweep        */
  DYSON_KERNEL_SELFENERGY = 7,    /* connected cumulant contraction of the self-energy step  */
  DYSON_KERNEL_SWEEP_TC_FUSED = 8,/* fused gather + 3xTF32 GEMM on CTA pairs (one launch/sweep)*/
  DYSON_KERNEL_KINDS = 9
};

/* Enable (1) or disable (0) event timing of every sweep/residual launch on the
 * context's stream and reset the counters.  Timing adds two events per launch. */
int dyson_profile(dyson_ctx* ctx, int enable);

/* Launch count and summed device time (ms) of one DYSON_KERNEL_* kind since
 * the last dyson_profile call. */
int dyson_profile_query(dyson_ctx* ctx, int kind, int64_t* launches, double* total_ms);

/* CUDA kernels launched by this context since dyson_init (-1 for NULL). */
int64_t dyson_launch_count(const dyson_ctx* ctx);

/* Cap the number of block columns solved together (0 = size from free memory). */
int dyson_set_chunk(dyson_ctx* ctx, int32_t block_columns);

/* Form of the 3xTF32 tensor-core sweep (App. C's series step; Sec. IV.D's
 * blocked application of the local blocks to many right-hand sides).
 *   SINGLE_CTA  a gather launch writes X = J d to global memory, then one CTA
 *               per 128 x 256 output tile multiplies (the default);
 *   CTA_PAIR    the same gather, then clusters of two CTAs on 256 x 256 tiles
 *               with tcgen05 cta_group::2 MMAs;
 *   FUSED_PAIR  one launch per sweep: CTA pairs whose producer warps gather the
 *               four neighbour rows of d straight into the MMA's shared-memory
 *               operand (X never reaches global memory); tiles of 256 rows x 256
 *               columns, two TMEM accumulators;
 *   FUSED_PAIR_WIDE  the fused form with tiles of 512 rows x 256 columns (X
 *               gathered once per site and column tile, one accumulator set).
 * The pair forms need Nc % 128 == 0 (FUSED_PAIR_WIDE: Nc % 256 == 0) and a
 * device that co-schedules CTA pairs; otherwise the single-CTA form runs.  All
 * give the same results to FP32 rounding; which is fastest depends on the
 * shape, which is what dyson_autotune measures.  Returns INVALID_ARG for an
 * unknown variant. */
enum {
  DYSON_SWEEP_SINGLE_CTA = 0,
  DYSON_SWEEP_CTA_PAIR = 1,
  DYSON_SWEEP_FUSED_PAIR = 2,
  DYSON_SWEEP_FUSED_PAIR_WIDE = 3
};
int dyson_set_sweep_variant(dyson_ctx* ctx, int variant);

/* Time limit of the bounded waits in the tensor-core pipelines (the sweep and the
 * split-product residual kernels), in seconds; 0 restores the default of 2 s.  The
 * limit is held per device, so it applies to every context on ctx's device.  A wait
 * that runs out raises the CTA's error flag; the CTA lets its in-flight copies and
 * MMAs land (those drain waits keep the default limit), frees its tensor memory and
 * exits, and the solve returns DYSON_ERR_TIMEOUT with the context still usable.  The
 * paper has no counterpart: the call exists so that tests can make a healthy pipeline
 * run out of time and check that path.  INVALID_ARG for a limit outside [0, 60]. */
int dyson_set_wait_limit(dyson_ctx* ctx, double seconds);

/* Sweeps per captured CUDA graph of the inner series (App. C) on the fused tensor-core
 * sweep: the series runs from replays of a graph of `sweeps` sweeps, each followed by a
 * one-warp kernel that applies the series' stopping rule on the device and lets the
 * remaining sweeps of a replay return at once (the replayed sweeps take their sweep
 * number for support truncation from the device).  One host synchronisation per replay
 * instead of one per sweep; results and sweep counts are the same as with 0, which keeps
 * one synchronisation per sweep.  The graph is captured on a private stream and launched
 * on the context's stream; not used while that stream is being captured by the caller.
 * Default 16; INVALID_ARG unless even and in 0..64. */
int dyson_set_graph_sweeps(dyson_ctx* ctx, int sweeps);

/* Point-group symmetry of the problem (App. A).  DYSON_SYMMETRY_C4V: on a
 * square lattice with the centred trap and drive tables invariant under the
 * eight operations of C4v (checked exactly here; INVALID_ARG otherwise),
 * dyson_solve_columns solves one source per symmetry orbit, the smallest site
 * index of the orbit, about Nr/8 block columns for all sources.  It fills the
 * other sources' observables by copies, and their G, when g_out is given, by
 * the site permutation G_{j,s} = G_{g^-1(j),r} for s = g(r).  The report
 * counts the solved representatives only.  dyson_local_greens and
 * dyson_selfenergy_step use the same reduction (see there).  The invariance is
 * checked on the drive tables; local blocks installed by the self-energy step
 * are taken to be invariant.  DYSON_SYMMETRY_NONE (the default) solves every
 * source. */
enum { DYSON_SYMMETRY_NONE = 0, DYSON_SYMMETRY_C4V = 1 };
int dyson_set_symmetry(dyson_ctx* ctx, int mode);

/* Autotuner of the tensor-core sweep.  On this context's Lambda it times two
 * warm-up and three timed sweeps for each candidate: every sweep variant the
 * contour allows (DYSON_SWEEP_SINGLE_CTA; DYSON_SWEEP_CTA_PAIR and
 * DYSON_SWEEP_FUSED_PAIR where Nc is a multiple of 128; DYSON_SWEEP_FUSED_PAIR_WIDE
 * where it is a multiple of 256) times every chunk of 1, 2, 4, ... block columns up to
 * max_block_columns and to what fits in 85 % of free device memory; unless the inner
 * solver is DYSON_INNER_SERIES, also only chunks that leave room for the GMRES basis
 * of the full restart length, so that a switch to GMRES does not restart early.  Then it
 * sets the context to the fastest (dyson_set_sweep_variant and dyson_set_chunk;
 * candidates are tried largest chunk first, in the variant order above, and a later
 * one wins only when it is more than 2 % faster, so that timing noise does not
 * flip the choice) and, when out is not NULL, reports the choice and every candidate's measured
 * sweep throughput in vector columns per second.  Needs a built, upright Lambda
 * and Nc % 64 == 0; the work buffers keep the largest candidate's size. */
enum { DYSON_TUNE_MAX_CANDIDATES = 32 };
typedef struct {
  int32_t sweep_variant;          /* chosen DYSON_SWEEP_*                                   */
  int32_t chunk_block_columns;    /* chosen block columns per chunk                         */
  double vector_columns_per_s;    /* measured sweep throughput of the choice                */
  int32_t n_candidates;
  int32_t cand_variant[DYSON_TUNE_MAX_CANDIDATES];
  int32_t cand_chunk[DYSON_TUNE_MAX_CANDIDATES];
  double cand_vector_columns_per_s[DYSON_TUNE_MAX_CANDIDATES];
} dyson_tuning;
int dyson_autotune(dyson_ctx* ctx, int32_t max_block_columns, dyson_tuning* out);

/* Inner solver of the mixed-precision path (DYSON_PREC_TF32X3_F64REF), between
 * FP64 residual refinements:
 *   SERIES  the series of App. C in FP32;
 *   GMRES   the preconditioned GMRES of App. C (preconditioner Lambda, the
 *           block-diagonal B^-1; initial guess the preconditioned right-hand
 *           side), restarted every `restart` iterations (0 = 40; at most 60,
 *           and fewer when the Krylov basis does not fit in free memory);
 *   AUTO    (the default) the series, switching to GMRES for the rest of a chunk
 *           when the series diverges, its transient peak leaves FP32 no correct
 *           digit (long contours), it runs through max_sweeps in one refinement
 *           (spectral radius near 1), or the refined residual grows.
 * GMRES keeps restart + 4 FP32 chunk states (8 Nr Nc bytes per vector column
 * each).  The FP64 path (DYSON_PREC_F64) always runs the series.
 * Returns INVALID_ARG for an unknown solver or a restart outside 0..60. */
enum { DYSON_INNER_SERIES = 0, DYSON_INNER_GMRES = 1, DYSON_INNER_AUTO = 2 };
int dyson_set_inner_solver(dyson_ctx* ctx, int solver, int32_t restart);

/* Support truncation (Sec. IV.D: the iterates spread from the localised start
 * one hop per application of the hopping).  The first right-hand side of a
 * solve, Lambda delta_s, is non-zero only on each column's source site, so after
 * n series sweeps a column vanishes beyond lattice distance n of its source.
 * When enabled (the default), the first inner series of the mixed-precision path
 * on the tensor cores skips every (site, 256-column) tile that is still zero:
 * the results are bit-identical, the work of the early sweeps shrinks.  Later
 * refinements (whose residuals are dense), GMRES, the FP64 and the CUDA-core FP32
 * sweeps are not truncated.  Truncated sweeps use the single-CTA kernel. */
int dyson_set_support_truncation(dyson_ctx* ctx, int enable);

/* ---------------------------------------------------------------------------
 * Batched solves of several problem instances.  The paper solves one trap at a
 * time; this entry point serves scans over many traps, lattices and drives.
 * Each context keeps its own lattice, contour, trap, drive and Lambda, and its
 * block columns are solved exactly as dyson_solve_columns(precision =
 * DYSON_PREC_TF32X3_F64REF) solves them (the series of App. C refined with
 * FP64-accurate residuals).  What the instances share is the inner FP32
 * series.  Every sweep is ONE gather launch and ONE persistent tensor-core
 * launch over the tiles of all instances still iterating, followed by a check
 * kernel that applies each instance's stopping rule on the device.  Blocks of
 * graph_sweeps sweeps are captured once as a CUDA graph and replayed with no
 * host round trip inside a block.  An instance whose series diverges (spectral
 * radius of Lambda W J above 1) is afterwards solved alone with the GMRES inner
 * solver of App. C, unless its context was set to DYSON_INNER_SERIES.
 *
 * Requirements: every context is on the same device and stream, its Lambda is
 * built and upright, and its contour suits the tensor-core path with the
 * split-product residual (Nc a multiple of 64, Nc <= 256).  The block columns
 * of one instance are solved as one chunk: DYSON_ERR_OOM if they do not fit.
 *
 * Ownership: the batch holds pointers to the contexts, not the contexts.
 * Destroy the batch before its contexts.
 * ------------------------------------------------------------------------- */
typedef struct dyson_batch dyson_batch;
enum { DYSON_BATCH_MAX_INSTANCES = 64 };

/* Group n contexts (1 <= n <= DYSON_BATCH_MAX_INSTANCES, no duplicates) into a batch. */
int dyson_batch_create(dyson_batch** out, dyson_ctx* const* ctxs, int32_t n);

/* Solve the block columns src[k][0..n_src[k]) of instance k, for every k, to a
 * relative FP64 Dyson residual <= tol; max_sweeps bounds each inner series.
 * graph_sweeps = sweeps per graph replay (0 = 8; odd values are rounded up).
 * g_out: NULL, or per instance NULL or a device buffer [n_src[k]][Nr][Nc][Nc]
 * complex128 (the layout of dyson_solve_columns).  reports: NULL or n entries.
 * Observables are read afterwards per context with dyson_observables.
 * Returns the first non-OK instance status (NOT_CONVERGED, DIVERGED), or an
 * error code; dyson_batch_last_error describes it. */
int dyson_batch_solve(dyson_batch* b, const int32_t* const* src, const int32_t* n_src, double tol,
                      int32_t max_sweeps, int32_t graph_sweeps, double* const* g_out, dyson_report* reports);

/* Kernels launched by the batch's sweep graphs (3 per sweep; -1 for NULL). */
int64_t dyson_batch_launch_count(const dyson_batch* b);
const char* dyson_batch_last_error(const dyson_batch* b);
void dyson_batch_destroy(dyson_batch* b);

/* ---------------------------------------------------------------------------
 * Allocation-free solve of one block column.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * while they run (a device heap owned and pre-reserved by another framework's
 * pool, latency-bound loops where cudaMalloc's implicit synchronisation is not
 * acceptable, tools that may not change a library's memory footprint).
 *
 * It runs the same FP64 series as dyson_solve_columns(precision = F64) for one
 * source site, but its only scratch memory (one block-column state and two
 * norm words) is a file-scope device array of DYSON_NOALLOC_MAX_STATE_BYTES +
 * 256 bytes that every GPU loading the library holds until the process exits.
 * It calls no cudaMalloc, cudaFree or other allocating routine.
 *
 *   lambda  device, [Nr][Nc][Nc] complex128 Lambda (e.g. from dyson_copy_sigma
 *           with on_device = 1);
 *   J       device, [Nb][Nt] hopping table (bond order as above; may be NULL
 *           when Nr = 1);
 *   g_out   device, [Nr][Nc][Nc] complex128, receives G_js(z, z') at [j][z][z'];
 *   sweeps_out  host, optional: sweeps performed;
 *   work is ordered on cuda_stream (NULL: legacy default stream) of the
 *   current device, and the call returns after it has completed.
 * Sizes with Nr*Nc*Nc*16 > DYSON_NOALLOC_MAX_STATE_BYTES are rejected with
 * INVALID_ARG (see dyson_noalloc_last_error).  Returns OK, NOT_CONVERGED
 * (g_out holds the last iterate), DIVERGED, INVALID_ARG or CUDA.
 *
 * With CUDA's lazy module loading the array is committed on a device when the
 * module that holds it is first loaded there: by dyson_init on that device, or
 * else by the first call of this function on it, which also looks up the
 * array's device address (cudaGetSymbolAddress with that device current).  A
 * caller whose heap another framework will take must therefore create a
 * context, or make one call, on each device before that happens.  The call
 * synchronises: it copies each sweep's norm to the host and waits for it, so
 * it blocks the host until the solve is done and cannot be called while its
 * stream is being captured into a CUDA graph.  All calls share the one array
 * and it keeps the previous call's contents (the call clears what must start
 * at zero): calls that overlap on the GPU, from several threads or streams,
 * race on it. */
#define DYSON_NOALLOC_MAX_STATE_BYTES (16u << 20)

int dyson_solve_block_column_noalloc(const double* lambda, const double* J, int32_t Lx, int32_t Ly, int32_t Nt,
                                     int32_t Nm, double dt, double beta, int32_t source, double tol,
                                     int32_t max_sweeps, double* g_out, int32_t* sweeps_out, void* cuda_stream);

/* Message of the last failing dyson_solve_block_column_noalloc call on this thread. */
const char* dyson_noalloc_last_error(void);

/* Library version string. */
const char* dyson_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DYSON_H */
