// Internal declarations shared by the translation units of the Dyson library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dyson.h"

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------

// Contour conventions (Sec. IV.A; the index order of the discretised contour):
// points 0..Nt-1 forward at t_k = k dt, Nt..2Nt-1 backward at t_{2Nt-1-z},
// 2Nt..Nc-1 imaginary (physical time 0); quadrature weights +dt, -dt, -i beta/Nm.
__device__ __forceinline__ int contour_time_index(int z, int Nt) {
  return z < Nt ? z : (z < 2 * Nt ? 2 * Nt - 1 - z : 0);
}
__device__ __forceinline__ double2 contour_weight(int z, int Nt, int Nm, double dt, double beta) {
  return z < Nt ? make_double2(dt, 0.0) : (z < 2 * Nt ? make_double2(-dt, 0.0) : make_double2(0.0, -beta / Nm));
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// max of non-negative doubles through their ordered bit patterns
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* p, double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ULL);  // NaN -> +inf: never converges
  atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// ---------------------------------------------------------------------------
// kernel launchers (all asynchronous on `s`)
// ---------------------------------------------------------------------------

// K1: atomic-limit functions.  eps [Nr], Lam [Nr][Nc][Nc] complex128.
void launch_build_sigma(const double* U, int Lx, int Ly, int Nt, int Nm, double dt, double beta,
                        double curvature, double mu, double* eps, double2* phase,
                        double2* lam, cudaStream_t s);
// contour hopping weights JW[b][z] = W(z) J_b(t(z)) (complex128) and Jz[b][z] = J_b(t(z)) (fp32)
void launch_hopping_tables(const double* J, int Nb, int Nt, int Nm, double dt, double beta,
                           double2* JW, float* Jz, cudaStream_t s);
// Lambda' = Lambda * W as complex64 (SIMT FP32 path)
void launch_lam_c64(const double2* lam, int Nr, int Nt, int Nm, double dt, double beta,
                    float2* lam32, cudaStream_t s);
// Lambda' = Lambda * W as the real 2Nc x 2Nc embedding [[Re,-Im],[Im,Re]], split in
// TF32 hi + lo parts (tcgen05 path).  hi/lo: [Nr][2Nc][2Nc] fp32.
void launch_lam_emb_split(const double2* lam, int Nr, int Nt, int Nm, double dt, double beta,
                          float* hi, float* lo, cudaStream_t s);

// transpose every Nc x Nc block of lam in place
void launch_transpose_blocks(double2* lam, int Nr, int Nc, cudaStream_t s);

// Chunk state: FP64 [Nr][ncol][Nc] complex128, FP32 [Nr][ncol][2Nc] planar.  Vector
// column n has the source (src_site[n], src_time[n]) (site -1: a zero padding column);
// norms and scales are kept per group of gs consecutive columns (q = n / gs).
void launch_init_rhs(const double2* lam, const int* src_site, const int* src_time, int Nr, int Nc, int ncol,
                     int gs, double2* G, unsigned long long* scale, cudaStream_t s);
// K3: out = B + K Gin (mode 0), or B + K Gin - Gin (mode 1); norm[q] = max |out - Gin| (mode 0)
// or max |out| (mode 1).  If out32 != nullptr (mode 1 only) the result is written as FP32
// planar state instead of into out.
void launch_sweep_f64(const double2* lam, const double2* JW, const int* nbr, const int* nbond,
                      const double2* Gin, double2* out, float* out32, const int* src_site, const int* src_time,
                      int Nr, int Nc, int ncol, int gs, int mode, unsigned long long* norm, cudaStream_t s);
// SIMT FP32 sweep: dout = r + K din over planar FP32 state; norm[q] = max |dout - din|
void launch_sweep_f32_simt(const float2* lam32, const float* Jz, const int* nbr, const int* nbond,
                           const float* r, const float* din, float* dout, int Nr, int Nc, int ncol, int gs,
                           unsigned long long* norm, cudaStream_t s);
// out[n][j][z] = G[j][n][z] for the first nv vector columns
void launch_export_vectors(const double2* G, int Nr, int Nc, int ncol, int nv, double2* out, cudaStream_t s);
// FP64 interleaved state -> FP32 planar state
void launch_to_planar32(const double2* G, float* out, size_t n_el, int Nc, cudaStream_t s);
// G64 += d32
void launch_accumulate(double2* G, const float* d, int Nr, int Nc, int ncol, cudaStream_t s);
// observables of the block columns of a chunk
void launch_observables(const double2* G, const int* src_site, int nq, const int* nbr,
                        const int* nbond, const double* Jtab, const double* eps, const double* U,
                        int Nr, int Nt, int Nc, int ncol, double dt, double* obs, cudaStream_t s);
// diagonal blocks of a chunk of block columns: out[s][z][z'] = G_ss(z, z') for each source s
void launch_export_diagonal(const double2* G, const int* src_site, int Nc, int ncol, int nq, double2* out,
                            cudaStream_t s);
// self-energy state: forget G0 (after a new Lambda build), free
void se_invalidate(dyson_ctx* c);
void se_release(dyson_ctx* c);
// [j][q*Nc+z'][z] -> user layout [q][j][z][z']
void launch_export(const double2* G, int Nr, int Nc, int nq, double2* out, cudaStream_t s);

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

struct dyson_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int Lx = 0, Ly = 0, Nr = 0, Nb = 0, Nt = 0, Nm = 0, Nc = 0;
  double dt = 0, beta = 0, curvature = 0, mu = 0;
  std::vector<double> U, J;          // host copies of the drive tables
  bool j_uniform = false;            // every bond carries the same J(t) row
  // inner series under captured graphs: sweeps per graph (0: one host synchronisation per
  // sweep); while a graph is captured, the flag its fused sweeps read (0: the series stopped)
  int graph_sweeps = 16;
  const int* sweep_run = nullptr;
  const int* sweep_count = nullptr;  // while capturing: the device count of sweeps done
  cudaStream_t cap_stream = nullptr; // private stream the series graph is captured on (lazy)
  void* d_series = nullptr;          // device stopping state of the captured series
  void* h_series = nullptr;          // pinned mirror
  double* d_rref = nullptr;          // reference norms of the current inner solve
  int rref_cap = 0;

  // device tables
  double* dU = nullptr;              // [Nr][Nt]
  double* dJ = nullptr;              // [Nb][Nt]
  int* d_nbr = nullptr;              // [Nr][4] neighbour site or -1
  int* d_nbond = nullptr;            // [Nr][4] bond index
  double* d_eps = nullptr;           // [Nr]
  double2* d_phase = nullptr;        // [Nr][2][Nc]
  double2* d_lam = nullptr;          // [Nr][Nc][Nc]
  double2* d_JW = nullptr;           // [Nb][Nc]
  float* d_Jz = nullptr;             // [Nb][Nc]
  float2* d_lam32 = nullptr;         // [Nr][Nc][Nc] (lazy)
  float* d_lam_hi = nullptr;         // [Nr][2Nc][2Nc] (lazy)
  float* d_lam_lo = nullptr;
  double* d_obs = nullptr;           // [3][Nr][Nt]
  bool sigma_built = false;
  bool sigma_transposed = false;     // every Lambda_i block transposed: solves give rows of G

  // work buffers, grown on demand
  void* work = nullptr;
  size_t work_bytes = 0;
  int* d_src_site = nullptr;         // per vector column of the current chunk
  int* d_src_time = nullptr;
  int src_cap = 0;
  std::vector<int> h_src_site, h_src_time;
  unsigned long long* d_norm = nullptr;   // [2 * max block columns]
  unsigned long long* h_norm = nullptr;   // pinned mirror
  int norm_cap = 0;

  bool lam32_built = false;
  bool lam_split_built = false;
  bool tc_enabled = true;            // 3xTF32 tcgen05 sweep allowed where the contour fits it
  bool use_tc = false;               // chosen for the current solve
  int tc_variant = 0;                // DYSON_SWEEP_SINGLE_CTA or DYSON_SWEEP_CTA_PAIR
  int max_refinements = 12;
  int chunk_override = 0;
  int64_t launches = 0;              // kernels launched by this context since dyson_init
  int64_t host_syncs = 0;            // host waits for the device in solves (reported per call)

  // optional per-launch event timing
  struct Pending {
    int kind;
    cudaEvent_t a, b;
  };
  bool profiling = false;
  std::vector<Pending> pending;
  double prof_ms[DYSON_KERNEL_KINDS] = {};
  int64_t prof_launches[DYSON_KERNEL_KINDS] = {};

  void* tc = nullptr;                // tensor-core module state (tensor maps, workspace)
  void* adj = nullptr;               // adjoint buffers (columns, rows, gathers, M, results)
  size_t adj_bytes = 0;
  void* oz = nullptr;                // split-product residual state (slices, scales, maps)
  void* gm = nullptr;                // GMRES inner-solver state (Krylov basis, rotations)
  std::vector<int> h_nbr, h_nbond;   // host copies of the neighbour tables
  int symmetry = 0;                  // DYSON_SYMMETRY_NONE or DYSON_SYMMETRY_C4V
  std::vector<int> sym_rep, sym_op;  // per site: orbit representative, an operation taking it there
  int* d_sym_perm = nullptr;         // [8][Nr]: site j <- g^{-1}(j) for each operation g
  int inner_solver = 2;              // DYSON_INNER_SERIES, DYSON_INNER_GMRES or DYSON_INNER_AUTO
  int gmres_restart = 40;            // restart length (capped by free memory)
  bool support_trunc = true;         // skip tiles outside the first series' support (dyson_set_support_truncation)
  int* d_act = nullptr;              // [Nr][column tiles] first live sweep per tile
  size_t act_bytes = 0;
  void* se = nullptr;                // self-energy step state (atomic G0, its pseudo-inverse, mixed T)
  bool se_installed = false;         // Lambda holds the local block of a self-energy step
  bool oz_enabled = true;            // split-product residual allowed where 2 Nc <= 512
  bool use_oz = false;               // chosen for the current solve

  std::string err;
};

int ctx_fail(dyson_ctx* c, int code, const std::string& msg);
// load the allocation-free entry point's module on `device` (current) and look up its
// scratch array, so the array is committed at context creation (noalloc.cu)
int noalloc_reserve_scratch(int device);

// Adjoint of L = sum_i Re(beta_i . c_i) with beta'_i = i beta_i: per site i the
// coefficient of the row at (i, kf) (b0), at (i, kf - 1) (b1) and at (j, kf) for
// the neighbour in slot s (bj[s]).
struct AdjCoef {
  double2 b0, b1, bj[4];
};
int adjoint_contract_obs(dyson_ctx* c, const double2* C, const double2* R1, const double2* R2,
                         const AdjCoef* coef_dev, const double* wn_dev, const double* wd_dev, const double* ones_dev,
                         int kf, double2* psi, double2* gam, double2* rho, double2* M, double* loss_dev,
                         double* gU_dev, double* gJ_dev);
#define DY_CUDA(ctx, call)                                                              \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ctx_fail((ctx), e_ == cudaErrorMemoryAllocation ? DYSON_ERR_OOM : DYSON_ERR_CUDA, \
                      std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)
