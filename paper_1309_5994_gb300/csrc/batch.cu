// Batched mixed-precision solves of several problem instances (dyson_batch_*).
//
// Each instance is a context of its own (lattice, contour, trap, drive, Lambda)
// solving its block columns with the series of App. C refined by FP64 residuals,
// exactly as dyson_solve_columns(precision = TF32X3_F64REF) does.  What is
// shared is the inner FP32 series: every sweep is ONE gather launch and ONE
// persistent tensor-core launch over the tiles of all instances still
// iterating (an instance table on the device, k_tc.cu), followed by a one-block
// check kernel that applies the inner stopping rule per instance on the device
// and clears the instance's activity flag when it stops.  A block of
// graph_sweeps sweeps is captured once as a CUDA graph and replayed until no
// instance is active, so the host reads one word per replay instead of
// synchronising after every sweep.  The FP64 residual refinement (split-product
// residual, k_oz.cu) runs per instance between inner solves.  An instance whose
// series diverges (spectral radius of K above 1) is then solved alone with the
// GMRES of App. C (k_gmres.cu).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <limits>
#include <vector>

#include "common.cuh"
#include "detail.cuh"
#include "oz.cuh"
#include "tc.cuh"

using namespace dyson_detail;

static_assert(DYSON_BATCH_MAX_INSTANCES == TC_MAX_INSTANCES, "one tensor-core launch serves the whole batch");

namespace {

struct BatchCheck {                 // what the check kernel reads per instance
  unsigned long long* norm;         // ng update max-norm words (bits of a non-negative double)
  const double* rref;               // ng reference norms of the current inner solve
  int ng;
  int max_sweeps;
};

struct BatchStop {                  // inner-series stopping state per instance
  double best, peak, last;
  double target;                     // update at which this refinement's series stops
  double hist[kStallSweeps];         // the last kStallSweeps updates (ring)
  int since_best, sweeps, diverged, since_peak;
};

// Stopping rule of the inner series (the refinement's target, kStallDrop, kStallSweeps, kFlatRatio) per
// active instance; clears the norm words for the next sweep and counts the
// instances still active.  One block.
__global__ void k_batch_check(const BatchCheck* __restrict__ chk, int n, int* __restrict__ active,
                              BatchStop* __restrict__ st, int* __restrict__ n_active) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    if (!active[k]) continue;
    const BatchCheck C = chk[k];
    double upd = 0.0;
    bool bad = false;
    for (int q = 0; q < C.ng; ++q) {
      const double v = __longlong_as_double((long long)C.norm[q]) / fmax(C.rref[q], 1e-300);
      if (!(v == v)) bad = true;
      else upd = fmax(upd, v);
      C.norm[q] = 0ull;
    }
    BatchStop S = st[k];
    S.sweeps += 1;
    S.last = upd;
    bool stop = false;
    if (bad || !(upd < kDivergedGrowth) || upd > kSeriesPeakMax) {
      // not finite, or a transient the FP32 series cannot carry: hand the
      // instance to the GMRES of App. C after the batch
      S.diverged = 1;
      stop = true;
    } else {
      if (upd > S.peak) {                              // the stall is judged on the decay after the peak
        S.peak = upd;
        S.best = upd;
        S.since_best = 0;
        S.since_peak = 0;
      } else {
        S.since_peak += 1;
        if (upd < S.best) {
          S.best = upd;
          S.since_best = 0;
        } else {
          S.since_best += 1;
        }
      }
      const double ago = S.hist[S.sweeps % kStallSweeps];
      S.hist[S.sweeps % kStallSweeps] = upd;
      stop = (upd <= S.target && (upd < S.peak || upd == 0.0)) ||
             (S.since_best >= kStallSweeps && S.best < kStallDrop * S.peak) ||
             (S.since_peak >= kStallSweeps && upd < kStallDrop * S.peak && upd > kFlatRatio * ago) ||
             S.sweeps >= C.max_sweeps;
    }
    st[k] = S;
    if (stop) active[k] = 0;
    else atomicAdd(&cnt, 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) *n_active = cnt;
}

// per-instance host state of one batched solve
struct Inst {
  dyson_ctx* c = nullptr;
  int nq = 0, ncol = 0, ng = 0;
  double2* G = nullptr;
  float *r32 = nullptr, *da = nullptr, *db = nullptr;
  std::vector<double> scale, rref;
  double prev_res = std::numeric_limits<double>::infinity();
  int strikes = 0;
  int status = DYSON_ERR_NOT_CONVERGED;
  bool done = false;
  int64_t launches0 = 0;
  dyson_report rep{};
};

}  // namespace

struct dyson_batch {
  std::vector<dyson_ctx*> ctx;
  int device = 0;
  cudaStream_t stream = nullptr;     // the contexts' stream
  cudaStream_t gstream = nullptr;    // capture/replay stream of the sweep graph
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::string err;
  int64_t launches = 0;
  // device tables (sized for ctx.size() instances)
  TcInst* d_tab = nullptr;
  TcInst* h_tab = nullptr;           // pinned
  BatchCheck* d_chk = nullptr;
  BatchStop* d_stop = nullptr;
  BatchStop* h_stop = nullptr;       // pinned
  int* d_active = nullptr;
  int* h_active = nullptr;           // pinned
  int* d_nactive = nullptr;
  int* h_nactive = nullptr;          // pinned
  double* d_rref = nullptr;
  double* h_rref = nullptr;          // pinned
  size_t rref_cap = 0;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int bfail(dyson_batch* b, int code, const std::string& m) {
  if (b) b->err = m;
  else fail_noctx(code, m);
  return code;
}

#define DYB_CUDA(b, call)                                                          \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      cudaGetLastError();                                                          \
      return bfail(b, DYSON_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    }                                                                              \
  } while (0)

void free_graph(dyson_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
}

}  // namespace

extern "C" {

int dyson_batch_create(dyson_batch** out, dyson_ctx* const* ctxs, int32_t n) {
  if (!out) return fail_noctx(DYSON_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!ctxs || n < 1 || n > DYSON_BATCH_MAX_INSTANCES)
    return fail_noctx(DYSON_ERR_INVALID_ARG, "a batch holds 1.." + std::to_string(DYSON_BATCH_MAX_INSTANCES) +
                                                 " contexts");
  for (int k = 0; k < n; ++k) {
    if (!ctxs[k]) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context in the batch");
    if (ctxs[k]->device != ctxs[0]->device || ctxs[k]->stream != ctxs[0]->stream)
      return fail_noctx(DYSON_ERR_INVALID_ARG, "batched contexts must share one device and one stream");
    for (int j = 0; j < k; ++j)
      if (ctxs[j] == ctxs[k]) return fail_noctx(DYSON_ERR_INVALID_ARG, "a context appears twice in the batch");
  }
  DeviceGuard g(ctxs[0]->device);
  auto* b = new dyson_batch;
  b->ctx.assign(ctxs, ctxs + n);
  b->device = ctxs[0]->device;
  b->stream = ctxs[0]->stream;
  cudaError_t e = cudaSuccess;
  if ((e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_tab, n * sizeof(TcInst))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&b->h_tab, n * sizeof(TcInst))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_chk, n * sizeof(BatchCheck))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_stop, n * sizeof(BatchStop))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&b->h_stop, n * sizeof(BatchStop))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_active, n * sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&b->h_active, n * sizeof(int))) != cudaSuccess ||
      (e = cudaMalloc((void**)&b->d_nactive, sizeof(int))) != cudaSuccess ||
      (e = cudaMallocHost((void**)&b->h_nactive, sizeof(int))) != cudaSuccess) {
    cudaGetLastError();
    dyson_batch_destroy(b);
    return fail_noctx(e == cudaErrorMemoryAllocation ? DYSON_ERR_OOM : DYSON_ERR_CUDA,
                      std::string("batch set-up: ") + cudaGetErrorString(e));
  }
  *out = b;
  return DYSON_OK;
}

int dyson_batch_solve(dyson_batch* b, const int32_t* const* src, const int32_t* n_src, double tol,
                      int32_t max_sweeps, int32_t graph_sweeps, double* const* g_out, dyson_report* reports) {
  if (!b) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL batch");
  const int n = (int)b->ctx.size();
  if (!src || !n_src) return bfail(b, DYSON_ERR_INVALID_ARG, "NULL source arrays");
  if (!(tol > 0) || max_sweeps < 1 || graph_sweeps < 0)
    return bfail(b, DYSON_ERR_INVALID_ARG, "need tol > 0, max_sweeps >= 1 and graph_sweeps >= 0");
  // sweeps per graph replay; even, so every replay starts from the state slot buf[0]
  int S = graph_sweeps > 0 ? graph_sweeps : 8;
  S += S & 1;
  const auto t0 = std::chrono::steady_clock::now();
  DeviceGuard g(b->device);
  std::vector<Inst> I(n);
  int rc;
  // ---- per-instance set-up: tables, work buffers, right-hand sides ----
  size_t rref_total = 0;
  for (int k = 0; k < n; ++k) {
    Inst& X = I[k];
    dyson_ctx* c = X.c = b->ctx[k];
    X.launches0 = c->launches;
    if (!c->sigma_built || c->sigma_transposed)
      return bfail(b, DYSON_ERR_STATE, "instance " + std::to_string(k) + ": Lambda not built or transposed");
    if (n_src[k] < 1 || !src[k]) return bfail(b, DYSON_ERR_INVALID_ARG, "every instance needs a source site");
    for (int q = 0; q < n_src[k]; ++q)
      if (src[k][q] < 0 || src[k][q] >= c->Nr) return bfail(b, DYSON_ERR_INVALID_ARG, "source site out of range");
    if ((rc = prepare_tables(c, DYSON_PREC_TF32X3_F64REF))) return bfail(b, rc, c->err);
    if (!c->use_tc || !c->use_oz)
      return bfail(b, DYSON_ERR_INVALID_ARG,
                   "instance " + std::to_string(k) + ": batched solves need Nc % 64 == 0 and 2 Nc <= 512");
    X.nq = n_src[k];
    X.ncol = X.nq * c->Nc;
    X.ng = X.nq;
    size_t col_bytes = 0;
    if (chunk_columns(c, DYSON_PREC_TF32X3_F64REF, c->Nc, X.ncol, &col_bytes) < X.ncol)
      return bfail(b, DYSON_ERR_OOM, "instance " + std::to_string(k) + ": its block columns do not fit at once");
    if ((rc = ensure_work(c, (size_t)X.ncol * col_bytes)) || (rc = ensure_cols(c, X.ncol, X.ng)))
      return bfail(b, rc, c->err);
    c->h_src_site.resize(X.ncol);
    c->h_src_time.resize(X.ncol);
    for (int q = 0; q < X.nq; ++q)
      for (int z = 0; z < c->Nc; ++z) {
        c->h_src_site[q * c->Nc + z] = src[k][q];
        c->h_src_time[q * c->Nc + z] = z;
      }
    if ((rc = upload_sources(c, X.ncol))) return bfail(b, rc, c->err);
    const size_t n_el = (size_t)c->Nr * X.ncol * c->Nc;
    X.G = (double2*)c->work;
    X.r32 = (float*)(X.G + n_el);
    X.da = X.r32 + 2 * n_el;
    X.db = X.da + 2 * n_el;
    DYB_CUDA(b, cudaMemsetAsync(X.G, 0, n_el * sizeof(double2), c->stream));
    DYB_CUDA(b, cudaMemsetAsync(c->d_norm, 0, 2 * (size_t)X.ng * sizeof(unsigned long long), c->stream));
    launch_init_rhs(c->d_lam, c->d_src_site, c->d_src_time, c->Nr, c->Nc, X.ncol, c->Nc, X.G, c->d_norm + X.ng,
                    c->stream);
    launch_to_planar32(X.G, X.r32, n_el, c->Nc, c->stream);
    c->launches += 2;
    DYB_CUDA(b, cudaMemsetAsync(X.G, 0, n_el * sizeof(double2), c->stream));
    if ((rc = read_norms(c, X.ng, true))) return bfail(b, rc, c->err);
    X.scale.resize(X.ng);
    for (int q = 0; q < X.ng; ++q) X.scale[q] = bits_to_double(c->h_norm[X.ng + q]);
    X.rref = X.scale;
    rref_total += X.ng;
  }
  // ---- device tables: instances, check entries, reference norms ----
  if (b->rref_cap < rref_total) {
    if (b->d_rref) cudaFree(b->d_rref);
    if (b->h_rref) cudaFreeHost(b->h_rref);
    b->d_rref = nullptr;
    b->h_rref = nullptr;
    b->rref_cap = 0;
    DYB_CUDA(b, cudaMalloc((void**)&b->d_rref, rref_total * sizeof(double)));
    DYB_CUDA(b, cudaMallocHost((void**)&b->h_rref, rref_total * sizeof(double)));
    b->rref_cap = rref_total;
  }
  std::vector<BatchCheck> chk(n);
  std::vector<size_t> rref_off(n);
  std::vector<CUtensorMap> m_hi(n), m_lo(n), m_x(n);
  int tiles = 0, gblocks = 0;
  size_t off = 0;
  for (int k = 0; k < n; ++k) {
    Inst& X = I[k];
    TcInst* e = &b->h_tab[k];
    if ((rc = tc_fill_instance(X.c, X.ncol, X.c->Nc, X.r32, X.da, X.db, X.c->d_norm, b->d_active + k, e, &m_hi[k],
                               &m_lo[k], &m_x[k])))
      return bfail(b, rc, X.c->err);
    e->tile0 = tiles;
    e->gblk0 = gblocks;
    tiles += tc_instance_tiles(*e);
    gblocks += tc_instance_gather_blocks(*e);
    rref_off[k] = off;
    chk[k] = BatchCheck{X.c->d_norm, b->d_rref + off, X.ng, max_sweeps};
    off += X.ng;
  }
  // every context's set-up work precedes the tables and the graph
  DYB_CUDA(b, cudaStreamSynchronize(b->stream));
  DYB_CUDA(b, cudaMemcpyAsync(b->d_tab, b->h_tab, n * sizeof(TcInst), cudaMemcpyHostToDevice, b->stream));
  DYB_CUDA(b, cudaMemcpyAsync(b->d_chk, chk.data(), n * sizeof(BatchCheck), cudaMemcpyHostToDevice, b->stream));
  DYB_CUDA(b, cudaStreamSynchronize(b->stream));

  // ---- the sweep graph: S x (gather, GEMM, check) over the whole table ----
  free_graph(b);
  {
    dyson_ctx* c0 = b->ctx[0];
    const int64_t l0 = c0->launches;
    cudaGraph_t graph = nullptr;
    DYB_CUDA(b, cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
    int cap_rc = DYSON_OK;
    for (int s = 0; s < S && cap_rc == DYSON_OK; ++s) {
      cap_rc = tc_launch_table(c0, b->d_tab, n, tiles, gblocks, s & 1, TC_GATHER | TC_GEMM, b->gstream,
                               m_hi.data(), m_lo.data(), m_x.data());
      if (cap_rc == DYSON_OK) k_batch_check<<<1, 256, 0, b->gstream>>>(b->d_chk, n, b->d_active, b->d_stop, b->d_nactive);
    }
    cudaError_t ce = cudaStreamEndCapture(b->gstream, &graph);
    c0->launches = l0;
    if (cap_rc != DYSON_OK) {
      if (graph) cudaGraphDestroy(graph);
      return bfail(b, cap_rc, c0->err);
    }
    if (ce != cudaSuccess) {
      cudaGetLastError();
      return bfail(b, DYSON_ERR_CUDA, std::string("sweep graph capture: ") + cudaGetErrorString(ce));
    }
    ce = cudaGraphInstantiate(&b->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
      return bfail(b, DYSON_ERR_CUDA, std::string("sweep graph instantiation: ") + cudaGetErrorString(ce));
    }
  }

  // ---- refinements: batched inner series, per-instance FP64 residuals ----
  dyson_ctx* c0 = b->ctx[0];
  const int max_ref = c0->max_refinements;
  for (int ref = 0; ref < max_ref; ++ref) {
    int n_live = 0;
    for (int k = 0; k < n; ++k) {
      Inst& X = I[k];
      b->h_active[k] = X.done ? 0 : 1;
      std::memset(&b->h_stop[k], 0, sizeof(BatchStop));
      b->h_stop[k].best = std::numeric_limits<double>::infinity();
      b->h_stop[k].target = inner_target(kInnerTarget, tol, X.prev_res);
      if (X.done) continue;
      ++n_live;
      const size_t n32 = (size_t)X.c->Nr * X.ncol * 2 * X.c->Nc;
      DYB_CUDA(b, cudaMemcpyAsync(X.da, X.r32, n32 * sizeof(float), cudaMemcpyDeviceToDevice, b->stream));
      DYB_CUDA(b, cudaMemsetAsync(X.c->d_norm, 0, (size_t)X.ng * sizeof(unsigned long long), b->stream));
      std::copy(X.rref.begin(), X.rref.end(), b->h_rref + rref_off[k]);
    }
    if (n_live == 0) break;
    DYB_CUDA(b, cudaMemcpyAsync(b->d_active, b->h_active, n * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    DYB_CUDA(b, cudaMemcpyAsync(b->d_stop, b->h_stop, n * sizeof(BatchStop), cudaMemcpyHostToDevice, b->stream));
    DYB_CUDA(b, cudaMemcpyAsync(b->d_rref, b->h_rref, rref_total * sizeof(double), cudaMemcpyHostToDevice,
                                b->stream));
    DYB_CUDA(b, cudaEventRecord(b->ev_in, b->stream));
    DYB_CUDA(b, cudaStreamWaitEvent(b->gstream, b->ev_in, 0));
    // replay until every instance has stopped (the check kernel also stops an
    // instance at max_sweeps, so the bound below is never the one that ends it)
    for (int rep = 0; rep <= max_sweeps / S + 1; ++rep) {
      DYB_CUDA(b, cudaGraphLaunch(b->exec, b->gstream));
      b->launches += 3 * (int64_t)S;
      DYB_CUDA(b, cudaMemcpyAsync(b->h_nactive, b->d_nactive, sizeof(int), cudaMemcpyDeviceToHost, b->gstream));
      DYB_CUDA(b, cudaStreamSynchronize(b->gstream));
      if ((rc = tc_check_error(c0))) return bfail(b, rc, c0->err);
      if (*b->h_nactive == 0) break;
    }
    DYB_CUDA(b, cudaEventRecord(b->ev_out, b->gstream));
    DYB_CUDA(b, cudaStreamWaitEvent(b->stream, b->ev_out, 0));
    DYB_CUDA(b, cudaMemcpyAsync(b->h_stop, b->d_stop, n * sizeof(BatchStop), cudaMemcpyDeviceToHost, b->stream));
    DYB_CUDA(b, cudaStreamSynchronize(b->stream));
    // G += d, then the FP64-accurate residual, per live instance
    for (int k = 0; k < n; ++k) {
      Inst& X = I[k];
      if (X.done) continue;
      dyson_ctx* c = X.c;
      const BatchStop& St = b->h_stop[k];
      X.rep.sweeps += St.sweeps;
      X.rep.update = St.last;
      X.rep.gemm_flops += St.sweeps * sweep_flops(c, X.ncol);
      if (St.diverged) {
        X.status = DYSON_ERR_DIVERGED;
        X.done = true;
        continue;
      }
      const float* d = (St.sweeps & 1) ? X.db : X.da;     // sweep s writes buf[s & 1]
      launch_accumulate(X.G, d, c->Nr, c->Nc, X.ncol, c->stream);
      c->launches += 1;
      DYB_CUDA(b, cudaMemsetAsync(c->d_norm, 0, (size_t)X.ng * sizeof(unsigned long long), c->stream));
      if ((rc = oz_residual(c, X.ncol, c->Nc, X.G, X.r32, tol))) return bfail(b, rc, c->err);
    }
    for (int k = 0; k < n; ++k) {
      Inst& X = I[k];
      if (X.done) continue;
      dyson_ctx* c = X.c;
      if ((rc = read_norms(c, X.ng, false))) return bfail(b, rc, c->err);
      if ((rc = oz_check_error(c))) return bfail(b, rc, c->err);
      X.rep.refinements += 1;
      X.rep.gemm_flops += sweep_flops(c, X.ncol);
      const double res = rel_max(c->h_norm, X.scale.data(), X.ng);
      X.rep.residual = res;
      for (int q = 0; q < X.ng; ++q) X.rref[q] = std::max(bits_to_double(c->h_norm[q]), 1e-300);
      if (!(res < kDivergedGrowth)) {
        X.status = DYSON_ERR_DIVERGED;
        X.done = true;
      } else if (res <= tol) {
        X.status = DYSON_OK;
        X.done = true;
      } else if (res > kRefineContract * X.prev_res && ++X.strikes >= kRefineStrikes) {
        X.status = DYSON_ERR_DIVERGED;
        X.done = true;
      }
      X.prev_res = res;
    }
  }
  // ---- instances whose series diverged: the GMRES of App. C, one context at a
  //      time (unless the context asked for the series alone) ----
  for (int k = 0; k < n; ++k) {
    Inst& X = I[k];
    dyson_ctx* c = X.c;
    if (X.status != DYSON_ERR_DIVERGED || c->inner_solver == DYSON_INNER_SERIES) continue;
    const int saved = c->inner_solver;
    c->inner_solver = DYSON_INNER_GMRES;
    double2* G = nullptr;
    rc = solve_mixed(c, X.ncol, c->Nc, DYSON_PREC_TF32X3_F64REF, tol, max_sweeps, &G, &X.rep);
    c->inner_solver = saved;
    if (rc != DYSON_OK && rc != DYSON_ERR_NOT_CONVERGED && rc != DYSON_ERR_DIVERGED) return bfail(b, rc, c->err);
    X.status = rc;
    X.G = G;
  }
  // ---- observables and optional export per instance ----
  int status = DYSON_OK;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int k = 0; k < n; ++k) {
    Inst& X = I[k];
    dyson_ctx* c = X.c;
    launch_observables(X.G, c->d_src_site, X.nq, c->d_nbr, c->d_nbond, c->dJ, c->d_eps, c->dU, c->Nr, c->Nt, c->Nc,
                       X.ncol, c->dt, c->d_obs, c->stream);
    c->launches += 1;
    if (g_out && g_out[k]) {
      launch_export(X.G, c->Nr, c->Nc, X.nq, (double2*)g_out[k], c->stream);
      c->launches += 1;
    }
    if (X.status != DYSON_OK && status == DYSON_OK) status = X.status;
    X.rep.status = X.status;
    X.rep.chunks = 1;
    X.rep.seconds = secs;
    X.rep.kernel_launches = c->launches - X.launches0;
    if (reports) reports[k] = X.rep;
  }
  DYB_CUDA(b, cudaGetLastError());
  DYB_CUDA(b, cudaStreamSynchronize(b->stream));
  if (status == DYSON_ERR_NOT_CONVERGED) b->err = "an instance reached its refinement limit above tolerance";
  if (status == DYSON_ERR_DIVERGED) b->err = "an instance's series diverged";
  return status;
}

int64_t dyson_batch_launch_count(const dyson_batch* b) { return b ? b->launches : -1; }

const char* dyson_batch_last_error(const dyson_batch* b) { return b ? b->err.c_str() : ""; }

void dyson_batch_destroy(dyson_batch* b) {
  if (!b) return;
  DeviceGuard g(b->device);
  if (b->gstream) cudaStreamSynchronize(b->gstream);
  free_graph(b);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  void* dptrs[] = {b->d_tab, b->d_chk, b->d_stop, b->d_active, b->d_nactive, b->d_rref};
  for (void* p : dptrs)
    if (p) cudaFree(p);
  void* hptrs[] = {b->h_tab, b->h_stop, b->h_active, b->h_nactive, b->h_rref};
  for (void* p : hptrs)
    if (p) cudaFreeHost(p);
  delete b;
}

}  // extern "C"
