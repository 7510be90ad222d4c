// Entry points of the C ABI declared in include/dyson.h.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>

#include "common.cuh"
#include "detail.cuh"
#include "gmres.cuh"
#include "oz.cuh"
#include "symmetry.cuh"
#include "tc.cuh"

namespace dyson_detail {

thread_local std::string g_noctx_err;

int fail_noctx(int code, const std::string& m) {
  g_noctx_err = m;
  return code;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

double bits_to_double(unsigned long long b) {
  double d;
  std::memcpy(&d, &b, sizeof d);
  return d;
}

// -------------------------------------------------------------------------
void flush_timers(dyson_ctx* c) {
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.kind] += ms;
      c->prof_launches[p.kind] += 1;
    }
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  c->pending.clear();
}

int ensure_work(dyson_ctx* c, size_t bytes) {
  if (c->work_bytes >= bytes) return DYSON_OK;
  if (c->work) cudaFree(c->work);
  c->work = nullptr;
  c->work_bytes = 0;
  cudaError_t e = cudaMalloc(&c->work, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, DYSON_ERR_OOM, "work buffer of " + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  c->work_bytes = bytes;
  return DYSON_OK;
}

// per-vector-column source arrays (ncol entries) and per-group norm/scale words (ng groups)
int ensure_cols(dyson_ctx* c, int ncol, int ng) {
  if (c->src_cap < ncol) {
    if (c->d_src_site) cudaFree(c->d_src_site);
    if (c->d_src_time) cudaFree(c->d_src_time);
    c->d_src_site = c->d_src_time = nullptr;
    c->src_cap = 0;
    DY_CUDA(c, dalloc(&c->d_src_site, ncol));
    DY_CUDA(c, dalloc(&c->d_src_time, ncol));
    c->src_cap = ncol;
  }
  if (c->norm_cap < ng) {
    if (c->d_norm) cudaFree(c->d_norm);
    if (c->h_norm) cudaFreeHost(c->h_norm);
    c->d_norm = nullptr;
    c->h_norm = nullptr;
    c->norm_cap = 0;
    DY_CUDA(c, dalloc(&c->d_norm, 2 * (size_t)ng));
    DY_CUDA(c, cudaMallocHost((void**)&c->h_norm, 2 * (size_t)ng * sizeof(unsigned long long)));
    c->norm_cap = ng;
  }
  return DYSON_OK;
}

// copy the host source arrays of the current chunk to the device
int upload_sources(dyson_ctx* c, int ncol) {
  DY_CUDA(c, cudaMemcpyAsync(c->d_src_site, c->h_src_site.data(), ncol * sizeof(int), cudaMemcpyHostToDevice,
                             c->stream));
  DY_CUDA(c, cudaMemcpyAsync(c->d_src_time, c->h_src_time.data(), ncol * sizeof(int), cudaMemcpyHostToDevice,
                             c->stream));
  return DYSON_OK;
}

// read norm[0..ng) (and scale[ng..2ng) when with_scale) to the host
int read_norms(dyson_ctx* c, int ng, bool with_scale) {
  DY_CUDA(c, cudaMemcpyAsync(c->h_norm, c->d_norm, (with_scale ? 2 : 1) * (size_t)ng * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  c->host_syncs += 1;
  flush_timers(c);
  return DYSON_OK;
}

// max over groups of norm[q] / ref[q] (groups with ref = 0 hold only padding columns)
double rel_max(const unsigned long long* norm, const double* ref, int ng) {
  double m = 0.0;
  for (int q = 0; q < ng; ++q) {
    double v = bits_to_double(norm[q]) / std::max(ref[q], 1e-300);
    if (!(v == v)) return std::numeric_limits<double>::infinity();
    m = std::max(m, v);
  }
  return m;
}


// algorithmic contour-GEMM flops of one sweep over ncol vector columns
double sweep_flops(const dyson_ctx* c, int ncol) { return 8.0 * c->Nc * (double)c->Nc * c->Nr * ncol; }

// Plain FP64 series over the chunk (ncol vector columns, norm groups of gs columns):
// G <- B + K G until the relative update <= tol
int solve_f64(dyson_ctx* c, int ncol, int gs, double tol, int max_sweeps, double2** result, dyson_report* r) {
  const int ng = ncol / gs;
  const size_t n_el = (size_t)c->Nr * ncol * c->Nc;
  double2* Ga = (double2*)c->work;
  double2* Gb = Ga + n_el;
  DY_CUDA(c, cudaMemsetAsync(Ga, 0, n_el * sizeof(double2), c->stream));
  DY_CUDA(c, cudaMemsetAsync(c->d_norm, 0, 2 * (size_t)ng * sizeof(unsigned long long), c->stream));
  launch_init_rhs(c->d_lam, c->d_src_site, c->d_src_time, c->Nr, c->Nc, ncol, gs, Ga, c->d_norm + ng, c->stream);
  c->launches += 1;
  int rc = read_norms(c, ng, true);
  if (rc) return rc;
  std::vector<double> scale(ng);
  for (int q = 0; q < ng; ++q) scale[q] = bits_to_double(c->h_norm[ng + q]);
  *result = Ga;
  int status = DYSON_ERR_NOT_CONVERGED;
  for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
    DY_CUDA(c, cudaMemsetAsync(c->d_norm, 0, (size_t)ng * sizeof(unsigned long long), c->stream));
    {
      KernelTimer t(c, DYSON_KERNEL_SWEEP_F64);
      launch_sweep_f64(c->d_lam, c->d_JW, c->d_nbr, c->d_nbond, Ga, Gb, nullptr, c->d_src_site, c->d_src_time,
                       c->Nr, c->Nc, ncol, gs, 0, c->d_norm, c->stream);
      c->launches += 1;
    }
    DY_CUDA(c, cudaGetLastError());
    if ((rc = read_norms(c, ng, false))) return rc;
    std::swap(Ga, Gb);
    double upd = rel_max(c->h_norm, scale.data(), ng);
    r->sweeps += 1;
    r->gemm_flops += sweep_flops(c, ncol);
    r->update = upd;
    if (!(upd < kDivergedF64)) {
      status = DYSON_ERR_DIVERGED;
      break;
    }
    if (upd <= tol) {
      status = DYSON_OK;
      break;
    }
  }
  *result = Ga;
  return status;
}

// Stopping state of the inner series, the same fields the host loop of inner_solve keeps;
// on the device for sweeps replayed from a captured graph.
struct SeriesState {
  double best, peak, last;
  double hist[kStallSweeps];           // the last kStallSweeps updates (ring)
  int since_best, since_peak, sweeps;
  int run;                             // 1 while the series goes on (read by the fused sweep)
  int outcome;
};
enum { SERIES_RUNNING = 0, SERIES_STOPPED, SERIES_EXHAUSTED, SERIES_ABORTED, SERIES_NOT_FINITE };

// After one sweep of a captured series: the update max_q norm_q / rref_q (norm words
// cleared for the next sweep) and the stopping rule of inner_solve's host loop, in the
// same order.  One warp; returns at once once the series has stopped.
__global__ void k_series_check(unsigned long long* __restrict__ norm, const double* __restrict__ rref, int ng,
                               int max_sweeps, double target, double abort_peak, SeriesState* __restrict__ S) {
  if (!S->run) return;
  double m = 0.0;
  int bad = 0;
  for (int q = threadIdx.x; q < ng; q += 32) {
    const double v = __longlong_as_double((long long)norm[q]) / fmax(rref[q], 1e-300);
    if (!(v == v)) bad = 1;
    else m = fmax(m, v);
    norm[q] = 0ull;
  }
  for (int o = 16; o > 0; o >>= 1) {
    m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if (threadIdx.x != 0) return;
  const double upd = bad ? __longlong_as_double(0x7ff0000000000000ll) : m;
  const int sweep = ++S->sweeps;
  S->last = upd;
  if (!(upd < kDivergedGrowth)) {
    S->outcome = SERIES_NOT_FINITE;
    S->run = 0;
    return;
  }
  if (upd > S->peak) {
    S->peak = upd;
    S->best = upd;
    S->since_best = 0;
    S->since_peak = 0;
  } else {
    ++S->since_peak;
    if (upd < S->best) {
      S->best = upd;
      S->since_best = 0;
    } else {
      ++S->since_best;
    }
  }
  const double ago = S->hist[sweep % kStallSweeps];
  S->hist[sweep % kStallSweeps] = upd;
  int out = SERIES_RUNNING;
  if (S->peak > abort_peak) out = SERIES_ABORTED;
  else if ((upd <= target && (upd < S->peak || upd == 0.0)) ||
           (S->since_best >= kStallSweeps && S->best < kStallDrop * S->peak) ||
           (S->since_peak >= kStallSweeps && upd < kStallDrop * S->peak && upd > kFlatRatio * ago))
    out = SERIES_STOPPED;
  else if (sweep >= max_sweeps)
    out = SERIES_EXHAUSTED;
  if (out != SERIES_RUNNING) {
    S->outcome = out;
    S->run = 0;
  }
}

// one 3xTF32 tensor-core sweep dout = r + K din with per-kind event timing: the
// fused gather + GEMM launch, or the gather launch and the GEMM launch
int tc_timed_sweep(dyson_ctx* c, int ncol, int gs, const float* r, const float* din, float* dout, const int* act,
                   int sweep, int rform = TC_R_DENSE) {
  if (tc_uses_fused(c)) {
    KernelTimer t(c, DYSON_KERNEL_SWEEP_TC_FUSED);
    return tc_sweep(c, ncol, gs, r, din, dout, TC_GATHER | TC_GEMM, act, sweep, rform);
  }
  int rc;
  {
    KernelTimer t(c, DYSON_KERNEL_GATHER_TC);
    if ((rc = tc_sweep(c, ncol, gs, r, din, dout, TC_GATHER, act, sweep))) return rc;
  }
  KernelTimer t(c, tc_uses_pair(c) && !act ? DYSON_KERNEL_SWEEP_TC_PAIR : DYSON_KERNEL_SWEEP_TC);
  return tc_sweep(c, ncol, gs, r, din, dout, TC_GEMM, act, sweep);
}

// inner solve d <- r + K d in FP32 (SIMT or 3xTF32 tensor cores)
// act (optional): support truncation of the tensor-core sweeps (tc_sweep), valid
// while every column of r32 is zero off its source site
// r_on_sources: r32 is non-zero only on each column's source site (the first right-hand side)
// With the fused sweep the series runs from replays of a captured graph of
// c->graph_sweeps sweeps, each followed by k_series_check: one host synchronisation per
// replay instead of one per sweep.  The replayed sweeps take their sweep number (for the
// support table) from the device count of sweeps done.
int inner_solve(dyson_ctx* c, int ncol, int gs, int precision, float* r32, float* da, float* db, int max_sweeps,
                const std::vector<double>& rref, float** dres, dyson_report* rep, double* peak_out,
                double abort_peak = std::numeric_limits<double>::infinity(), const int* act = nullptr,
                bool* exhausted = nullptr, double target = kInnerTarget, bool r_on_sources = false) {
  if (exhausted) *exhausted = false;
  const int ng = ncol / gs;
  const size_t n32 = (size_t)c->Nr * ncol * 2 * c->Nc;
  DY_CUDA(c, cudaMemcpyAsync(da, r32, n32 * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  if (act) DY_CUDA(c, cudaMemsetAsync(db, 0, n32 * sizeof(float), c->stream));   // skipped tiles stay 0
  const int rform = r_on_sources ? TC_R_ON_SOURCES : TC_R_DENSE;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  // (not inside a caller's own capture of the stream)
  const bool graph = c->graph_sweeps > 0 && precision == DYSON_PREC_TF32X3_F64REF && c->use_tc &&
                     tc_uses_fused(c) && cudaStreamIsCapturing(c->stream, &cap) == cudaSuccess &&
                     cap == cudaStreamCaptureStatusNone;
  const int eager_until = graph ? 0 : max_sweeps;
  SeriesState S = {};
  S.best = std::numeric_limits<double>::infinity();
  S.run = 1;
  int rc;
  while (S.run && S.sweeps < std::min(max_sweeps, eager_until)) {
    const int sweep = S.sweeps + 1;
    DY_CUDA(c, cudaMemsetAsync(c->d_norm, 0, (size_t)ng * sizeof(unsigned long long), c->stream));
    if (precision == DYSON_PREC_TF32X3_F64REF && c->use_tc) {
      if ((rc = tc_timed_sweep(c, ncol, gs, r32, da, db, act, sweep, rform))) return rc;
    } else {
      KernelTimer t(c, DYSON_KERNEL_SWEEP_F32);
      launch_sweep_f32_simt(c->d_lam32, c->d_Jz, c->d_nbr, c->d_nbond, r32, da, db, c->Nr, c->Nc, ncol, gs,
                            c->d_norm, c->stream);
      c->launches += 1;
    }
    DY_CUDA(c, cudaGetLastError());
    // one synchronisation per sweep: the norms and the pipeline's error flag come back together
    if (c->use_tc && (rc = tc_error_enqueue(c))) return rc;
    if ((rc = read_norms(c, ng, false))) return rc;
    if (c->use_tc && (rc = tc_error_status(c))) return rc;
    std::swap(da, db);
    const double upd = rel_max(c->h_norm, rref.data(), ng);
    S.sweeps = sweep;
    S.last = upd;
    rep->sweeps += 1;
    rep->gemm_flops += sweep_flops(c, ncol);
    rep->update = upd;
    if (!(upd < kDivergedGrowth)) return ctx_fail(c, DYSON_ERR_DIVERGED, "FP32 series update not finite");
    // stopping rule of the inner series (detail.cuh); the stall is judged only on
    // the decay after the latest peak (k_series_check applies the same, in this order)
    if (upd > S.peak) {
      S.peak = upd;
      S.best = upd;
      S.since_best = 0;
      S.since_peak = 0;
    } else {
      ++S.since_peak;
      if (upd < S.best) {
        S.best = upd;
        S.since_best = 0;
      } else {
        ++S.since_best;
      }
    }
    const double ago = S.hist[sweep % kStallSweeps];     // the update kStallSweeps sweeps ago
    S.hist[sweep % kStallSweeps] = upd;
    if (S.peak > abort_peak) {
      if (peak_out) *peak_out = S.peak;
      return DYSON_ERR_DIVERGED;                           // the caller switches to GMRES
    }
    if ((upd <= target && (upd < S.peak || upd == 0.0)) ||  // on the decay, not before the peak
        (S.since_best >= kStallSweeps && S.best < kStallDrop * S.peak) ||
        (S.since_peak >= kStallSweeps && upd < kStallDrop * S.peak && upd > kFlatRatio * ago)) {
      S.run = 0;
      S.outcome = SERIES_STOPPED;
    } else if (sweep == max_sweeps) {
      S.run = 0;
      S.outcome = SERIES_EXHAUSTED;
    }
  }
  if (S.run && graph) {
    // the rest of the series from a captured graph of S_g sweeps (even, so that every
    // replay starts from da), each followed by its check
    const int Sg = c->graph_sweeps;
    if (!c->d_series) {
      DY_CUDA(c, cudaMalloc(&c->d_series, sizeof(SeriesState)));
      DY_CUDA(c, cudaMallocHost(&c->h_series, sizeof(SeriesState)));
    }
    if (c->rref_cap < ng) {
      if (c->d_rref) cudaFree(c->d_rref);
      c->d_rref = nullptr;
      c->rref_cap = 0;
      DY_CUDA(c, cudaMalloc(&c->d_rref, (size_t)ng * sizeof(double)));
      c->rref_cap = ng;
    }
    SeriesState* hS = static_cast<SeriesState*>(c->h_series);
    SeriesState* dS = static_cast<SeriesState*>(c->d_series);
    *hS = S;
    if ((rc = tc_prepare_sweep(c, ncol))) return rc;     // nothing to allocate or encode while capturing
    DY_CUDA(c, cudaMemcpyAsync(c->d_rref, rref.data(), (size_t)ng * sizeof(double), cudaMemcpyHostToDevice,
                               c->stream));                // pageable: complete when the call returns
    DY_CUDA(c, cudaMemcpyAsync(dS, hS, sizeof(SeriesState), cudaMemcpyHostToDevice, c->stream));
    DY_CUDA(c, cudaMemsetAsync(c->d_norm, 0, (size_t)ng * sizeof(unsigned long long), c->stream));
    const int64_t launches0 = c->launches;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    // captured on a private stream (any stream of the caller's, the default one included,
    // can then launch it); the context's launches go there while capturing
    if (!c->cap_stream) DY_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = c->stream;
    DY_CUDA(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    c->stream = c->cap_stream;
    c->sweep_run = &dS->run;
    c->sweep_count = &dS->sweeps;
    int cap_rc = DYSON_OK;
    for (int k = 0; k < Sg && cap_rc == DYSON_OK; ++k) {
      cap_rc = tc_sweep(c, ncol, gs, r32, k % 2 ? db : da, k % 2 ? da : db, TC_GATHER | TC_GEMM, act, 0, rform);
      if (cap_rc == DYSON_OK)
        k_series_check<<<1, 32, 0, c->stream>>>(c->d_norm, c->d_rref, ng, max_sweeps, target, abort_peak, dS);
    }
    c->sweep_run = nullptr;
    c->sweep_count = nullptr;
    c->stream = user;
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &g);
    if (cap_rc) {
      if (g) cudaGraphDestroy(g);
      return cap_rc;
    }
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    if (ce != cudaSuccess) return ctx_fail(c, DYSON_ERR_CUDA, std::string("inner series graph: ") + cudaGetErrorString(ce));
    c->launches = launches0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) {
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
    }
    rc = DYSON_OK;
    while (rc == DYSON_OK) {
      const int before = hS->sweeps;
      if (e0) cudaEventRecord(e0, c->stream);
      cudaError_t le = cudaGraphLaunch(ge, c->stream);
      if (e1) cudaEventRecord(e1, c->stream);
      if (le == cudaSuccess && c->use_tc) rc = tc_error_enqueue(c);
      if (le == cudaSuccess && rc == DYSON_OK)
        le = cudaMemcpyAsync(hS, dS, sizeof(SeriesState), cudaMemcpyDeviceToHost, c->stream);
      if (le == cudaSuccess && rc == DYSON_OK) le = cudaStreamSynchronize(c->stream);
      if (le != cudaSuccess) {
        rc = ctx_fail(c, DYSON_ERR_CUDA, std::string("inner series graph: ") + cudaGetErrorString(le));
        break;
      }
      c->host_syncs += 1;
      if (rc || (c->use_tc && (rc = tc_error_status(c)))) break;
      const int n_run = hS->sweeps - before;
      c->launches += 2 * Sg;
      rep->sweeps += n_run;
      rep->gemm_flops += n_run * sweep_flops(c, ncol);
      rep->update = hS->last;
      float ms = 0.f;
      if (e0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
        c->prof_ms[DYSON_KERNEL_SWEEP_TC_FUSED] += ms;     // the replay, its checks included
        c->prof_launches[DYSON_KERNEL_SWEEP_TC_FUSED] += n_run;
      }
      if (!hS->run) {
        if (n_run % 2) std::swap(da, db);                  // the last sweep wrote db
        break;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGraphExecDestroy(ge);
    if (rc) return rc;
    S = *hS;
    if (S.outcome == SERIES_NOT_FINITE) return ctx_fail(c, DYSON_ERR_DIVERGED, "FP32 series update not finite");
    if (S.outcome == SERIES_ABORTED) {
      if (peak_out) *peak_out = S.peak;
      return DYSON_ERR_DIVERGED;
    }
  }
  if (S.outcome == SERIES_EXHAUSTED && exhausted) *exhausted = true;
  *dres = da;
  if (peak_out) *peak_out = S.peak;
  return DYSON_OK;
}

// out = zero + K in: one FP32 sweep with a zero right-hand side (the GMRES matvec)
int matvec_f32(dyson_ctx* c, int ncol, int gs, int precision, const float* zero, const float* in, float* out) {
  int rc;
  if (precision == DYSON_PREC_TF32X3_F64REF && c->use_tc) {
    if ((rc = tc_timed_sweep(c, ncol, gs, zero, in, out, nullptr, 0, TC_R_ZERO))) return rc;
  } else {
    KernelTimer t(c, DYSON_KERNEL_SWEEP_F32);
    launch_sweep_f32_simt(c->d_lam32, c->d_Jz, c->d_nbr, c->d_nbond, zero, in, out, c->Nr, c->Nc, ncol, gs,
                          c->d_norm, c->stream);
    c->launches += 1;
  }
  DY_CUDA(c, cudaGetLastError());
  return DYSON_OK;
}

// Support truncation (NEXT-2 of the build plan; Sec. IV.D): the first right-hand
// side Lambda delta_s is non-zero only on the source site of each column, and a
// sweep spreads an iterate by one hop, so after n sweeps a column is zero beyond
// lattice distance n of its source.  act[i][t] = min over the columns of 256-column
// tile t of the distance from site i to the column's source: the first sweep at
// which the tile can be non-zero.  Uploaded to c->d_act; nullptr when it cannot help.
const int* support_table(dyson_ctx* c, int ncol) {
  const int NT = (ncol + TC_TILE_COLS - 1) / TC_TILE_COLS;
  std::vector<int> act((size_t)c->Nr * NT, std::numeric_limits<int>::max());
  int far = 0;
  for (int t = 0; t < NT; ++t) {
    const int v1 = std::min(ncol, (t + 1) * TC_TILE_COLS);
    int last = -1;
    for (int v = t * TC_TILE_COLS; v < v1; ++v) {
      const int s = c->h_src_site[v];
      if (s == last || s < 0) continue;                  // padding columns (site -1) stay zero
      last = s;
      const int sx = s % c->Lx, sy = s / c->Lx;
      for (int i = 0; i < c->Nr; ++i) {
        const int d = std::abs(i % c->Lx - sx) + std::abs(i / c->Lx - sy);
        int& a = act[(size_t)i * NT + t];
        a = std::min(a, d);
      }
    }
  }
  for (int a : act) far = std::max(far, a);
  if (far < 2) return nullptr;                           // every tile is live from the first sweeps
  const size_t bytes = act.size() * sizeof(int);
  if (c->act_bytes < bytes) {
    if (c->d_act) cudaFree(c->d_act);
    c->d_act = nullptr;
    c->act_bytes = 0;
    if (cudaMalloc(&c->d_act, bytes) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;                                    // optional: run untruncated
    }
    c->act_bytes = bytes;
  }
  // pageable source: the copy completes before the call returns
  if (cudaMemcpyAsync(c->d_act, act.data(), bytes, cudaMemcpyHostToDevice, c->stream) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return c->d_act;
}

// complex FP32 series refined by FP64 residuals: G += solve(r), r = B + K G - G
int solve_mixed(dyson_ctx* c, int ncol, int gs, int precision, double tol, int max_sweeps, double2** result,
                dyson_report* rep) {
  const int ng = ncol / gs;
  const size_t n_el = (size_t)c->Nr * ncol * c->Nc;
  double2* G = (double2*)c->work;
  float* r32 = (float*)(G + n_el);
  float* da = r32 + 2 * n_el;
  float* db = da + 2 * n_el;
  int rc;
  // r = B (FP32), scale = max |B| per group; G = 0
  DY_CUDA(c, cudaMemsetAsync(G, 0, n_el * sizeof(double2), c->stream));
  DY_CUDA(c, cudaMemsetAsync(c->d_norm, 0, 2 * (size_t)ng * sizeof(unsigned long long), c->stream));
  launch_init_rhs(c->d_lam, c->d_src_site, c->d_src_time, c->Nr, c->Nc, ncol, gs, G, c->d_norm + ng, c->stream);
  launch_to_planar32(G, r32, n_el, c->Nc, c->stream);
  c->launches += 2;
  DY_CUDA(c, cudaMemsetAsync(G, 0, n_el * sizeof(double2), c->stream));
  if ((rc = read_norms(c, ng, true))) return rc;
  std::vector<double> scale(ng), rref(ng);
  for (int q = 0; q < ng; ++q) rref[q] = scale[q] = bits_to_double(c->h_norm[ng + q]);
  // the caller reads the chunk state (observables, export) whatever the status
  *result = G;
  int status = DYSON_ERR_NOT_CONVERGED;
  double prev_res = std::numeric_limits<double>::infinity();
  int strikes = 0;
  // inner solver: the series of App. C, or its GMRES.  AUTO starts with the series
  // and switches to GMRES for the rest of the chunk when the series cannot serve:
  // it diverges, its transient peak times the FP32 rounding leaves no correct
  // digit, it uses its whole sweep budget, or the refined residual grows.
  bool gmres = c->inner_solver == DYSON_INNER_GMRES;
  const bool may_switch = c->inner_solver == DYSON_INNER_AUTO;
  const MatvecFn mv = [&](const float* zero, const float* in, float* out) {
    return matvec_f32(c, ncol, gs, precision, zero, in, out);
  };
  for (int ref = 0; ref < c->max_refinements; ++ref) {
    float* d = nullptr;
    if (gmres) {
      rc = gmres_inner_solve(c, ncol, r32, da, max_sweeps, inner_target(kGmresTarget, tol, prev_res), rep, mv);
      d = da;
      rep->inner_gmres = 1;
    } else {
      double peak = 0.0;
      // the first right-hand side lives on the source sites: truncate its sweeps
      const int* act = ref == 0 && c->support_trunc && c->use_tc && precision == DYSON_PREC_TF32X3_F64REF
                           ? support_table(c, ncol)
                           : nullptr;
      bool exhausted = false;
      rc = inner_solve(c, ncol, gs, precision, r32, da, db, max_sweeps, rref, &d, rep, &peak,
                       may_switch ? kSeriesPeakMax : std::numeric_limits<double>::infinity(), act, &exhausted,
                       inner_target(kInnerTarget, tol, prev_res), ref == 0);
      if (rc == DYSON_ERR_DIVERGED && may_switch) {
        gmres = true;                                    // redo this refinement with GMRES
        --ref;
        continue;
      }
      // a series that used its whole sweep budget converges too slowly (spectral radius
      // near 1): its correction is kept, the following refinements use GMRES
      if (rc == DYSON_OK && exhausted && may_switch) gmres = true;
    }
    if (rc == DYSON_ERR_DIVERGED) {
      status = rc;
      break;
    }
    if (rc) return rc;
    launch_accumulate(G, d, c->Nr, c->Nc, ncol, c->stream);
    c->launches += 1;
    DY_CUDA(c, cudaMemsetAsync(c->d_norm, 0, (size_t)ng * sizeof(unsigned long long), c->stream));
    if (c->use_oz) {
      KernelTimer t(c, DYSON_KERNEL_RESIDUAL_SPLIT);
      if ((rc = oz_residual(c, ncol, gs, G, r32, tol))) return rc;
    } else {
      KernelTimer t(c, DYSON_KERNEL_RESIDUAL_F64);
      launch_sweep_f64(c->d_lam, c->d_JW, c->d_nbr, c->d_nbond, G, nullptr, r32, c->d_src_site, c->d_src_time,
                       c->Nr, c->Nc, ncol, gs, 1, c->d_norm, c->stream);
      c->launches += 1;
    }
    DY_CUDA(c, cudaGetLastError());
    if (c->use_oz && (rc = oz_error_enqueue(c))) return rc;   // read with the norms: one synchronisation
    if ((rc = read_norms(c, ng, false))) return rc;
    if (c->use_oz && (rc = oz_error_status(c))) return rc;
    rep->refinements += 1;
    rep->gemm_flops += sweep_flops(c, ncol);
    double res = rel_max(c->h_norm, scale.data(), ng);
    rep->residual = res;
    for (int q = 0; q < ng; ++q) rref[q] = std::max(bits_to_double(c->h_norm[q]), 1e-300);
    if (!(res < kDivergedGrowth)) {
      status = DYSON_ERR_DIVERGED;
      break;
    }
    if (res <= tol) {
      status = DYSON_OK;
      break;
    }
    if (res > kRefineContract * prev_res) {
      if (may_switch && !gmres) {
        gmres = true;                                    // the series does not contract: use GMRES
      } else if (++strikes >= kRefineStrikes) {
        status = DYSON_ERR_DIVERGED;
        break;
      }
    }
    prev_res = res;
  }
  return status;
}

}  // namespace dyson_detail

using namespace dyson_detail;

int ctx_fail(dyson_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  else g_noctx_err = msg;
  return code;
}

extern "C" {

const char* dyson_version(void) { return "gb300-dyson 0.1 (sm_103a)"; }

const char* dyson_last_error(const dyson_ctx* ctx) { return ctx ? ctx->err.c_str() : g_noctx_err.c_str(); }

int dyson_init(dyson_ctx** out, const dyson_lattice* L, const dyson_contour* C, const dyson_trap* T,
               const dyson_drive* D, int device, void* stream) {
  if (!out) return fail_noctx(DYSON_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!L || !C || !T || !D || !D->U || !D->J) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL argument");
  if (L->Lx < 1 || L->Ly < 1 || (int64_t)L->Lx * L->Ly > 65535)
    return fail_noctx(DYSON_ERR_INVALID_ARG, "lattice must have 1..65535 sites");
  if (C->Nt < 1 || C->Nm < 1 || 2 * (int64_t)C->Nt + C->Nm > 2048)
    return fail_noctx(DYSON_ERR_INVALID_ARG, "need Nt >= 1, Nm >= 1 and 2*Nt+Nm <= 2048");
  if (!(C->dt > 0) || !(C->beta > 0) || !std::isfinite(C->dt) || !std::isfinite(C->beta))
    return fail_noctx(DYSON_ERR_INVALID_ARG, "dt and beta must be positive and finite");
  if (!std::isfinite(T->curvature) || !std::isfinite(T->mu))
    return fail_noctx(DYSON_ERR_INVALID_ARG, "trap parameters must be finite");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return fail_noctx(DYSON_ERR_INVALID_ARG, "no such CUDA device");
  DeviceGuard g(device);
  // commit the allocation-free entry point's static scratch on this device now, not at
  // its first call (lazy module loading); optional, so a failure only clears the error
  if (noalloc_reserve_scratch(device) != DYSON_OK) cudaGetLastError();
  auto* c = new dyson_ctx;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  c->Lx = L->Lx;
  c->Ly = L->Ly;
  c->Nr = L->Lx * L->Ly;
  c->Nb = L->Ly * (L->Lx - 1) + L->Lx * (L->Ly - 1);
  c->Nt = C->Nt;
  c->Nm = C->Nm;
  c->Nc = 2 * C->Nt + C->Nm;
  c->dt = C->dt;
  c->beta = C->beta;
  c->curvature = T->curvature;
  c->mu = T->mu;
  c->U.assign(D->U, D->U + (size_t)c->Nr * c->Nt);
  c->J.assign(D->J, D->J + (size_t)c->Nb * c->Nt);
  for (double v : c->U)
    if (!std::isfinite(v)) {
      delete c;
      return fail_noctx(DYSON_ERR_INVALID_ARG, "U table holds a non-finite value");
    }
  for (double v : c->J)
    if (!std::isfinite(v)) {
      delete c;
      return fail_noctx(DYSON_ERR_INVALID_ARG, "J table holds a non-finite value");
    }
  c->j_uniform = true;
  for (int b = 1; b < c->Nb && c->j_uniform; ++b)
    c->j_uniform = std::equal(c->J.begin() + (size_t)b * c->Nt, c->J.begin() + (size_t)(b + 1) * c->Nt, c->J.begin());

  // neighbour slots (+x, -x, +y, -y) with their bond indices
  std::vector<int> nbr((size_t)c->Nr * 4, -1), nbond((size_t)c->Nr * 4, -1);
  for (int y = 0; y < c->Ly; ++y)
    for (int x = 0; x < c->Lx; ++x) {
      int i = y * c->Lx + x;
      if (x + 1 < c->Lx) { nbr[i * 4 + 0] = i + 1; nbond[i * 4 + 0] = y * (c->Lx - 1) + x; }
      if (x > 0) { nbr[i * 4 + 1] = i - 1; nbond[i * 4 + 1] = y * (c->Lx - 1) + x - 1; }
      int vb = c->Ly * (c->Lx - 1);
      if (y + 1 < c->Ly) { nbr[i * 4 + 2] = i + c->Lx; nbond[i * 4 + 2] = vb + y * c->Lx + x; }
      if (y > 0) { nbr[i * 4 + 3] = i - c->Lx; nbond[i * 4 + 3] = vb + (y - 1) * c->Lx + x; }
    }
  c->h_nbr = nbr;
  c->h_nbond = nbond;
  const size_t NcNc = (size_t)c->Nc * c->Nc;
  auto bail = [&](cudaError_t e, const char* what) {
    int code = e == cudaErrorMemoryAllocation ? DYSON_ERR_OOM : DYSON_ERR_CUDA;
    cudaGetLastError();
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    dyson_destroy(c);
    return fail_noctx(code, m);
  };
  cudaError_t e;
  if ((e = dalloc(&c->dU, c->U.size())) || (e = dalloc(&c->dJ, c->J.size())) ||
      (e = dalloc(&c->d_nbr, nbr.size())) || (e = dalloc(&c->d_nbond, nbond.size())) ||
      (e = dalloc(&c->d_eps, (size_t)c->Nr)) || (e = dalloc(&c->d_phase, (size_t)c->Nr * (2 * c->Nc + 2))) ||
      (e = dalloc(&c->d_lam, (size_t)c->Nr * NcNc)) || (e = dalloc(&c->d_JW, (size_t)c->Nb * c->Nc)) ||
      (e = dalloc(&c->d_Jz, (size_t)c->Nb * c->Nc)) || (e = dalloc(&c->d_obs, 3 * (size_t)c->Nr * c->Nt)))
    return bail(e, "device allocation");
  std::vector<double> nan_obs(3 * (size_t)c->Nr * c->Nt, std::numeric_limits<double>::quiet_NaN());
  if ((e = cudaMemcpyAsync(c->dU, c->U.data(), c->U.size() * 8, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->dJ, c->J.data(), c->J.size() * 8, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->d_nbr, nbr.data(), nbr.size() * 4, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->d_nbond, nbond.data(), nbond.size() * 4, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaMemcpyAsync(c->d_obs, nan_obs.data(), nan_obs.size() * 8, cudaMemcpyHostToDevice, c->stream)) ||
      (e = cudaStreamSynchronize(c->stream)))
    return bail(e, "table upload");
  *out = c;
  return DYSON_OK;
}

int dyson_build_sigma(dyson_ctx* c) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  DeviceGuard g(c->device);
  launch_build_sigma(c->dU, c->Lx, c->Ly, c->Nt, c->Nm, c->dt, c->beta, c->curvature, c->mu, c->d_eps,
                     c->d_phase, c->d_lam, c->stream);
  launch_hopping_tables(c->dJ, c->Nb, c->Nt, c->Nm, c->dt, c->beta, c->d_JW, c->d_Jz, c->stream);
  c->launches += c->Nb > 0 ? 3 : 2;
  DY_CUDA(c, cudaGetLastError());
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  c->sigma_built = true;
  c->lam32_built = c->lam_split_built = false;
  oz_invalidate(c);
  se_invalidate(c);                                      // Sigma = 0: Lambda is the atomic G0 again
  return DYSON_OK;
}

int dyson_copy_sigma(dyson_ctx* c, double* dst, int on_device) {
  if (!c || !dst) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL argument");
  if (!c->sigma_built) return ctx_fail(c, DYSON_ERR_STATE, "dyson_build_sigma has not run");
  DeviceGuard g(c->device);
  DY_CUDA(c, cudaMemcpyAsync(dst, c->d_lam, (size_t)c->Nr * c->Nc * c->Nc * sizeof(double2),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  return DYSON_OK;
}

}  // extern "C"

namespace dyson_detail {

// Build the reduced-precision copies of Lambda a solve needs and pick the sweep
// and residual kernels (sets c->use_tc, c->use_oz).
int prepare_tables(dyson_ctx* c, int precision) {
  c->use_tc = c->use_oz = false;
  if (precision == DYSON_PREC_F64) return DYSON_OK;
  const bool tc = c->tc_enabled && tc_supported(c, c->Nc);
  if (!tc && !c->lam32_built) {
    if (!c->d_lam32) DY_CUDA(c, dalloc(&c->d_lam32, (size_t)c->Nr * c->Nc * c->Nc));
    launch_lam_c64(c->d_lam, c->Nr, c->Nt, c->Nm, c->dt, c->beta, c->d_lam32, c->stream);
    c->launches += 1;
    c->lam32_built = true;
  }
  if (tc && !c->lam_split_built) {
    size_t n = (size_t)c->Nr * 4 * c->Nc * c->Nc;
    if (!c->d_lam_hi) DY_CUDA(c, dalloc(&c->d_lam_hi, n));
    if (!c->d_lam_lo) DY_CUDA(c, dalloc(&c->d_lam_lo, n));
    launch_lam_emb_split(c->d_lam, c->Nr, c->Nt, c->Nm, c->dt, c->beta, c->d_lam_hi, c->d_lam_lo, c->stream);
    c->launches += 1;
    c->lam_split_built = true;
  }
  c->use_tc = tc;
  c->use_oz = tc && c->oz_enabled && oz_supported(c);
  return DYSON_OK;
}

// Largest number of vector columns, a multiple of `unit` and at most `want`, whose
// work state fits in 85 % of the free device memory.  F64: two complex128 states;
// mixed: complex128 G + three FP32 states (+ the FP32 gather buffer of the
// tensor-core sweep, + the BF16 slices of the split-product residual).
int64_t chunk_columns(dyson_ctx* c, int precision, int64_t unit, int64_t want, size_t* bytes_per_col) {
  const double per_el = precision == DYSON_PREC_F64
                            ? 32.0
                            : (c->use_tc ? 48.0 : 40.0) + (c->use_oz ? (double)oz_bytes_per_element() : 0.0);
  const double col_bytes = per_el * c->Nr * (double)c->Nc;
  *bytes_per_col = (size_t)col_bytes;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
  const double budget = 0.85 * (double)(free_b + c->work_bytes);
  int64_t cols = (int64_t)(budget / col_bytes);
  if (c->chunk_override > 0) cols = std::min<int64_t>(cols, (int64_t)c->chunk_override * unit);
  cols = std::min<int64_t>(cols, want);
  cols = std::min<int64_t>(cols, (int64_t)1 << 24);
  return (cols / unit) * unit;
}

int solve_chunk(dyson_ctx* c, int ncol, int gs, int precision, double tol, int max_sweeps, double2** G,
                dyson_report* rep) {
  int rc = upload_sources(c, ncol);
  if (rc) return rc;
  return precision == DYSON_PREC_F64 ? solve_f64(c, ncol, gs, tol, max_sweeps, G, rep)
                                     : solve_mixed(c, ncol, gs, precision, tol, max_sweeps, G, rep);
}

int check_solve_args(dyson_ctx* c, int precision, double tol, int max_sweeps) {
  if (!c->sigma_built) return ctx_fail(c, DYSON_ERR_STATE, "dyson_build_sigma has not run");
  if (precision != DYSON_PREC_F64 && precision != DYSON_PREC_TF32X3_F64REF)
    return ctx_fail(c, DYSON_ERR_INVALID_ARG, "unknown precision");
  if (!(tol > 0) || max_sweeps < 1) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "need tol > 0 and max_sweeps >= 1");
  return DYSON_OK;
}

struct ReportScope {
  dyson_ctx* c;
  dyson_report rep;
  dyson_report* out;
  int64_t launches0, syncs0;
  std::chrono::steady_clock::time_point t0;
  ReportScope(dyson_ctx* cc, dyson_report* o) : c(cc), out(o), launches0(cc->launches), syncs0(cc->host_syncs) {
    std::memset(&rep, 0, sizeof rep);
    t0 = std::chrono::steady_clock::now();
  }
  int finish(int code) {
    rep.status = code;
    rep.kernel_launches = c->launches - launches0;
    rep.host_syncs = (int32_t)(c->host_syncs - syncs0);
    rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (out) *out = rep;
    return code;
  }
};

int fold_status(int status, int st) {
  if (st != DYSON_OK && status == DYSON_OK) return st;
  return status;
}

}  // namespace dyson_detail

extern "C" {

namespace {

// block-column solves; g_out: full block columns, gloc: diagonal blocks G_ss at row s (either may be NULL)
int solve_columns_impl(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                       int32_t max_sweeps, double* g_out, double* gloc, dyson_report* rep_out) {
  ReportScope R(c, rep_out);
  int rc = check_solve_args(c, precision, tol, max_sweeps);
  if (rc) return R.finish(rc);
  if (c->sigma_transposed)
    return R.finish(ctx_fail(c, DYSON_ERR_STATE, "Lambda is transposed: block columns and observables need it upright"));
  if (n_src < 1 || !src) return R.finish(ctx_fail(c, DYSON_ERR_INVALID_ARG, "need at least one source site"));
  for (int64_t q = 0; q < n_src; ++q)
    if (src[q] < 0 || src[q] >= c->Nr) return R.finish(ctx_fail(c, DYSON_ERR_INVALID_ARG, "source site out of range"));
  DeviceGuard g(c->device);
  if ((rc = prepare_tables(c, precision))) return R.finish(rc);
  size_t col_bytes = 0;
  const int64_t cols = chunk_columns(c, precision, c->Nc, n_src * (int64_t)c->Nc, &col_bytes);
  if (cols < c->Nc) return R.finish(ctx_fail(c, DYSON_ERR_OOM, "one block column does not fit in device memory"));
  const int64_t chunk = cols / c->Nc;
  if ((rc = ensure_work(c, (size_t)cols * col_bytes))) return R.finish(rc);
  if ((rc = ensure_cols(c, (int)cols, (int)chunk))) return R.finish(rc);

  int status = DYSON_OK;
  for (int64_t start = 0; start < n_src; start += chunk) {
    const int nq = (int)std::min<int64_t>(chunk, n_src - start);
    const int ncol = nq * c->Nc;
    c->h_src_site.resize(ncol);
    c->h_src_time.resize(ncol);
    for (int q = 0; q < nq; ++q)
      for (int z = 0; z < c->Nc; ++z) {
        c->h_src_site[q * c->Nc + z] = src[start + q];
        c->h_src_time[q * c->Nc + z] = z;
      }
    double2* G = nullptr;
    int st = solve_chunk(c, ncol, c->Nc, precision, tol, max_sweeps, &G, &R.rep);
    if (st != DYSON_OK && st != DYSON_ERR_NOT_CONVERGED && st != DYSON_ERR_DIVERGED) return R.finish(st);
    if (!G) return R.finish(ctx_fail(c, DYSON_ERR_STATE, "solve produced no state"));
    status = fold_status(status, st);
    R.rep.chunks += 1;
    launch_observables(G, c->d_src_site, nq, c->d_nbr, c->d_nbond, c->dJ, c->d_eps, c->dU, c->Nr, c->Nt, c->Nc,
                       ncol, c->dt, c->d_obs, c->stream);
    c->launches += 1;
    if (g_out) {
      launch_export(G, c->Nr, c->Nc, nq, (double2*)g_out + (size_t)start * c->Nr * c->Nc * c->Nc, c->stream);
      c->launches += 1;
    }
    if (gloc) {
      launch_export_diagonal(G, c->d_src_site, c->Nc, ncol, nq, (double2*)gloc, c->stream);
      c->launches += 1;
    }
    DY_CUDA(c, cudaGetLastError());
  }
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  flush_timers(c);
  if (status == DYSON_ERR_NOT_CONVERGED) ctx_fail(c, status, "max_sweeps or refinement limit reached above tolerance");
  if (status == DYSON_ERR_DIVERGED) ctx_fail(c, status, "series diverged (update not finite or past the rounding limit, or refinement residual growing)");
  return R.finish(status);
}

}  // namespace

int dyson_solve_columns(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                        int32_t max_sweeps, double* g_out, dyson_report* rep_out) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (c->symmetry == DYSON_SYMMETRY_C4V)
    return solve_columns_c4v(c, src, n_src, precision, tol, max_sweeps, g_out, rep_out);
  return solve_columns_impl(c, src, n_src, precision, tol, max_sweeps, g_out, nullptr, rep_out);
}

int dyson_local_greens(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                       int32_t max_sweeps, double* gloc, dyson_report* rep_out) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (!gloc) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "gloc is NULL");
  if (c->symmetry == DYSON_SYMMETRY_C4V)
    return local_greens_c4v(c, src, n_src, precision, tol, max_sweeps, gloc, rep_out);
  return solve_columns_impl(c, src, n_src, precision, tol, max_sweeps, nullptr, gloc, rep_out);
}

int dyson_solve_vector_columns(dyson_ctx* c, const int32_t* sites, const int32_t* times, int64_t n, int precision,
                               double tol, int32_t max_sweeps, double* g_out, dyson_report* rep_out) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  ReportScope R(c, rep_out);
  int rc = check_solve_args(c, precision, tol, max_sweeps);
  if (rc) return R.finish(rc);
  if (n < 1 || !sites || !times) return R.finish(ctx_fail(c, DYSON_ERR_INVALID_ARG, "need at least one column"));
  for (int64_t q = 0; q < n; ++q)
    if (sites[q] < 0 || sites[q] >= c->Nr || times[q] < 0 || times[q] >= c->Nc)
      return R.finish(ctx_fail(c, DYSON_ERR_INVALID_ARG, "column source out of range"));
  DeviceGuard g(c->device);
  if ((rc = prepare_tables(c, precision))) return R.finish(rc);
  constexpr int GS = 32;                                   // norm group; columns padded to a multiple
  const int64_t padded = (n + GS - 1) / GS * GS;
  size_t col_bytes = 0;
  const int64_t chunk = chunk_columns(c, precision, GS, padded, &col_bytes);
  if (chunk < GS) return R.finish(ctx_fail(c, DYSON_ERR_OOM, "32 vector columns do not fit in device memory"));
  if ((rc = ensure_work(c, (size_t)chunk * col_bytes))) return R.finish(rc);
  if ((rc = ensure_cols(c, (int)chunk, (int)(chunk / GS)))) return R.finish(rc);
  int status = DYSON_OK;
  for (int64_t start = 0; start < padded; start += chunk) {
    const int ncol = (int)std::min<int64_t>(chunk, padded - start);
    c->h_src_site.assign(ncol, -1);
    c->h_src_time.assign(ncol, 0);
    const int nv = (int)std::min<int64_t>(ncol, n - start);
    for (int k = 0; k < nv; ++k) {
      c->h_src_site[k] = sites[start + k];
      c->h_src_time[k] = times[start + k];
    }
    double2* G = nullptr;
    int st = solve_chunk(c, ncol, GS, precision, tol, max_sweeps, &G, &R.rep);
    if (st != DYSON_OK && st != DYSON_ERR_NOT_CONVERGED && st != DYSON_ERR_DIVERGED) return R.finish(st);
    if (!G) return R.finish(ctx_fail(c, DYSON_ERR_STATE, "solve produced no state"));
    status = fold_status(status, st);
    R.rep.chunks += 1;
    if (g_out) {
      launch_export_vectors(G, c->Nr, c->Nc, ncol, nv, (double2*)g_out + (size_t)start * c->Nr * c->Nc, c->stream);
      c->launches += 1;
    }
    DY_CUDA(c, cudaGetLastError());
  }
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  flush_timers(c);
  if (status == DYSON_ERR_NOT_CONVERGED) ctx_fail(c, status, "max_sweeps or refinement limit reached above tolerance");
  if (status == DYSON_ERR_DIVERGED) ctx_fail(c, status, "series diverged (update not finite or past the rounding limit, or refinement residual growing)");
  return R.finish(status);
}

int dyson_adjoint_obs(dyson_ctx* c, const double* w_density, const double* w_docc, int32_t t_index, int precision,
                      double tol, int32_t max_sweeps, double* loss, double* grad_U, double* grad_J,
                      dyson_report* rep_out) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  ReportScope R(c, rep_out);
  int rc = check_solve_args(c, precision, tol, max_sweeps);
  if (rc) return R.finish(rc);
  if (c->sigma_transposed) return R.finish(ctx_fail(c, DYSON_ERR_STATE, "Lambda is transposed"));
  if (c->se_installed)
    return R.finish(ctx_fail(c, DYSON_ERR_STATE, "the adjoint differentiates the atomic Lambda: rebuild it first"));
  if ((!w_density && !w_docc) || t_index < 0 || t_index >= c->Nt || (w_docc && t_index < 1))
    return R.finish(ctx_fail(c, DYSON_ERR_INVALID_ARG, "need weights, 0 <= t_index < Nt (>= 1 with D weights)"));
  DeviceGuard g(c->device);
  const int Nr = c->Nr, Nc = c->Nc, Nt = c->Nt;
  const bool docc = w_docc != nullptr;
  const size_t colbuf = (size_t)Nr * Nr * Nc;                 // double2 elements of C (and the rows, psi, gamma, rho)
  const size_t nbuf = docc ? 6 : 5;
  const size_t need = (nbuf * colbuf + (size_t)Nr * Nc * Nc) * sizeof(double2) + (size_t)Nr * sizeof(AdjCoef) +
                      ((size_t)3 * Nr + 1 + (size_t)Nr * Nt + (size_t)std::max(c->Nb, 1) * Nt) * sizeof(double);
  if (c->adj_bytes < need) {
    if (c->adj) cudaFree(c->adj);
    c->adj = nullptr;
    c->adj_bytes = 0;
    cudaError_t e = cudaMalloc(&c->adj, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return R.finish(ctx_fail(c, DYSON_ERR_OOM, "adjoint buffers"));
    }
    c->adj_bytes = need;
  }
  double2* C = (double2*)c->adj;
  double2* R1 = C + colbuf;
  double2* R2 = docc ? R1 + colbuf : nullptr;
  double2* psi = (docc ? R2 : R1) + colbuf;
  double2* gam = psi + colbuf;
  double2* rho = gam + colbuf;
  double2* M = rho + colbuf;
  AdjCoef* coef_dev = (AdjCoef*)(M + (size_t)Nr * Nc * Nc);
  double* wn_dev = (double*)(coef_dev + Nr);
  double* wd_dev = wn_dev + Nr;
  double* ones_dev = wd_dev + Nr;
  double* loss_dev = ones_dev + Nr;
  double* gU_dev = loss_dev + 1;
  double* gJ_dev = gU_dev + (size_t)Nr * Nt;
  // coefficients beta'_i = i beta_i of the rows (see k_adjoint.cu): the density
  // n_i = Im c_i(i, kf) gives b0 += w; the double occupancy D_i of Eq. (docc) gives
  // b0 += i v / (dt U) - v eps / U, b1 = -i v / (dt U), bj = -v J_ij / U
  std::vector<double> eps(Nr);
  DY_CUDA(c, cudaMemcpyAsync(eps.data(), c->d_eps, Nr * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  std::vector<AdjCoef> coef(Nr);
  std::vector<double> ones(Nr, 1.0);
  for (int i = 0; i < Nr; ++i) {
    AdjCoef& k = coef[i];
    std::memset(&k, 0, sizeof k);
    if (w_density) k.b0.x += w_density[i];
    if (docc && w_docc[i] != 0.0) {
      const double v = w_docc[i], U = c->U[(size_t)i * Nt + t_index];
      k.b0.x += -v * eps[i] / U;
      k.b0.y += v / (c->dt * U);
      k.b1.y = -v / (c->dt * U);
      for (int s = 0; s < 4; ++s)
        if (c->h_nbr[i * 4 + s] >= 0) k.bj[s].x = -v * c->J[(size_t)c->h_nbond[i * 4 + s] * Nt + t_index] / U;
    }
  }
  DY_CUDA(c, cudaMemcpyAsync(coef_dev, coef.data(), Nr * sizeof(AdjCoef), cudaMemcpyHostToDevice, c->stream));
  DY_CUDA(c, cudaMemcpyAsync(ones_dev, ones.data(), Nr * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (w_density)
    DY_CUDA(c, cudaMemcpyAsync(wn_dev, w_density, Nr * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  if (docc) DY_CUDA(c, cudaMemcpyAsync(wd_dev, w_docc, Nr * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  // columns G e_i at (i, kf); rows of G (columns of G^T) at (i, kf) and, for D, (i, kf - 1)
  std::vector<int32_t> sites(2 * (size_t)Nr), times(2 * (size_t)Nr);
  for (int i = 0; i < Nr; ++i) {
    sites[i] = sites[Nr + i] = i;
    times[i] = t_index;
    times[Nr + i] = t_index - 1;
  }
  dyson_report r1, r2;
  int st1 = dyson_solve_vector_columns(c, sites.data(), times.data(), Nr, precision, tol, max_sweeps,
                                       (double*)C, &r1);
  if (st1 != DYSON_OK && st1 != DYSON_ERR_NOT_CONVERGED) return R.finish(st1);
  if ((rc = dyson_transpose_sigma(c))) return R.finish(rc);
  int st2 = dyson_solve_vector_columns(c, sites.data(), times.data(), docc ? 2 * Nr : Nr, precision, tol,
                                       max_sweeps, (double*)R1, &r2);
  if ((rc = dyson_transpose_sigma(c))) return R.finish(rc);
  if (st2 != DYSON_OK && st2 != DYSON_ERR_NOT_CONVERGED) return R.finish(st2);
  R.rep.sweeps = r1.sweeps + r2.sweeps;
  R.rep.refinements = r1.refinements + r2.refinements;
  R.rep.chunks = r1.chunks + r2.chunks;
  R.rep.gemm_flops = r1.gemm_flops + r2.gemm_flops;
  R.rep.update = std::max(r1.update, r2.update);
  R.rep.residual = std::max(r1.residual, r2.residual);
  R.rep.inner_gmres = r1.inner_gmres | r2.inner_gmres;
  if ((rc = adjoint_contract_obs(c, C, R1, R2, coef_dev, w_density ? wn_dev : nullptr, docc ? wd_dev : nullptr,
                                 ones_dev, t_index, psi, gam, rho, M, loss_dev, gU_dev, gJ_dev)))
    return R.finish(rc);
  if (loss) DY_CUDA(c, cudaMemcpyAsync(loss, loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (grad_U)
    DY_CUDA(c, cudaMemcpyAsync(grad_U, gU_dev, (size_t)Nr * Nt * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (grad_J && c->Nb > 0)
    DY_CUDA(c, cudaMemcpyAsync(grad_J, gJ_dev, (size_t)c->Nb * Nt * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  const int status = fold_status(st1, st2);
  if (status == DYSON_ERR_NOT_CONVERGED) ctx_fail(c, status, "max_sweeps or refinement limit reached above tolerance");
  return R.finish(status);
}

int dyson_adjoint(dyson_ctx* c, const double* w, int32_t t_index, int precision, double tol, int32_t max_sweeps,
                  double* loss, double* grad_U, double* grad_J, dyson_report* rep_out) {
  if (c && !w) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "bad weights or time");
  return dyson_adjoint_obs(c, w, nullptr, t_index, precision, tol, max_sweeps, loss, grad_U, grad_J, rep_out);
}

int dyson_transpose_sigma(dyson_ctx* c) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (!c->sigma_built) return ctx_fail(c, DYSON_ERR_STATE, "dyson_build_sigma has not run");
  DeviceGuard g(c->device);
  launch_transpose_blocks(c->d_lam, c->Nr, c->Nc, c->stream);
  c->launches += 1;
  DY_CUDA(c, cudaGetLastError());
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  c->sigma_transposed = !c->sigma_transposed;
  c->lam32_built = c->lam_split_built = false;
  oz_invalidate(c);
  return DYSON_OK;
}

int dyson_observables(dyson_ctx* c, double* n, double* ekin, double* docc, int on_device) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  DeviceGuard g(c->device);
  size_t cnt = (size_t)c->Nr * c->Nt;
  double* dst[3] = {n, ekin, docc};
  for (int k = 0; k < 3; ++k)
    if (dst[k])
      DY_CUDA(c, cudaMemcpyAsync(dst[k], c->d_obs + k * cnt, cnt * sizeof(double),
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  return DYSON_OK;
}

int dyson_profile(dyson_ctx* c, int enable) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  flush_timers(c);
  c->profiling = enable != 0;
  for (int k = 0; k < DYSON_KERNEL_KINDS; ++k) {
    c->prof_ms[k] = 0.0;
    c->prof_launches[k] = 0;
  }
  return DYSON_OK;
}

int dyson_profile_query(dyson_ctx* c, int kind, int64_t* launches, double* total_ms) {
  if (!c || kind < 0 || kind >= DYSON_KERNEL_KINDS) return fail_noctx(DYSON_ERR_INVALID_ARG, "bad kernel kind");
  flush_timers(c);
  if (launches) *launches = c->prof_launches[kind];
  if (total_ms) *total_ms = c->prof_ms[kind];
  return DYSON_OK;
}

int64_t dyson_launch_count(const dyson_ctx* c) { return c ? c->launches : -1; }

int dyson_set_chunk(dyson_ctx* c, int32_t block_columns) {
  if (!c || block_columns < 0) return fail_noctx(DYSON_ERR_INVALID_ARG, "bad chunk size");
  c->chunk_override = block_columns;
  return DYSON_OK;
}

int dyson_set_inner_solver(dyson_ctx* c, int solver, int32_t restart) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (solver != DYSON_INNER_SERIES && solver != DYSON_INNER_GMRES && solver != DYSON_INNER_AUTO)
    return ctx_fail(c, DYSON_ERR_INVALID_ARG, "unknown inner solver");
  if (restart < 0 || restart > 60) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "restart length must be 0..60");
  c->inner_solver = solver;
  c->gmres_restart = restart > 0 ? restart : 40;
  return DYSON_OK;
}

int dyson_set_support_truncation(dyson_ctx* c, int enable) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  c->support_trunc = enable != 0;
  return DYSON_OK;
}

int dyson_set_wait_limit(dyson_ctx* c, double seconds) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (!(seconds >= 0.0) || seconds > 60.0) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "limit must be in [0, 60] s");
  DeviceGuard g(c->device);
  const unsigned long long ns = seconds == 0.0 ? 2000000000ull : (unsigned long long)(seconds * 1e9);
  int rc = tc_set_wait_limit(c, ns);
  if (rc) return rc;
  return oz_set_wait_limit(c, ns);
}

int dyson_set_graph_sweeps(dyson_ctx* c, int sweeps) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (sweeps < 0 || sweeps > 64 || sweeps % 2) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "sweeps must be even, 0..64");
  c->graph_sweeps = sweeps;
  return DYSON_OK;
}

int dyson_set_sweep_variant(dyson_ctx* c, int variant) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (variant < DYSON_SWEEP_SINGLE_CTA || variant > DYSON_SWEEP_FUSED_PAIR_WIDE)
    return ctx_fail(c, DYSON_ERR_INVALID_ARG, "unknown sweep variant");
  c->tc_variant = variant;
  return DYSON_OK;
}

void dyson_destroy(dyson_ctx* c) {
  if (!c) return;
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  flush_timers(c);
  tc_release(c);
  oz_release(c);
  gmres_release(c);
  se_release(c);
  if (c->d_sym_perm) cudaFree(c->d_sym_perm);
  void* ptrs[] = {c->dU, c->dJ, c->d_nbr, c->d_nbond, c->d_eps, c->d_phase, c->d_lam, c->d_JW, c->d_Jz,
                  c->d_lam32, c->d_lam_hi, c->d_lam_lo, c->d_obs, c->work, c->d_src_site, c->d_src_time,
                  c->d_norm, c->adj, c->d_act, c->d_series, c->d_rref};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_norm) cudaFreeHost(c->h_norm);
  if (c->h_series) cudaFreeHost(c->h_series);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"
