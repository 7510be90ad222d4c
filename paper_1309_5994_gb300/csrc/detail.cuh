// Host helpers of the solve drivers (capi.cu), shared with the batched driver (batch.cu).
#pragma once
#include <string>

#include "common.cuh"

namespace dyson_detail {

// make device d current for the scope, restoring the previous device after
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(d);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// a relative update above this (or not finite) counts as divergence
constexpr double kDivergedGrowth = 1e200;
// An FP64 series whose relative update passes 2^52 has partial sums whose
// rounding alone exceeds the result: it cannot converge to anything, and a
// transient of the real-time series never comes near (about 2e7 on the longest
// contours).  The FP64 series stops there with DYSON_ERR_DIVERGED.
constexpr double kDivergedF64 = 4503599627370496.0;

// Stopping rule of the FP32 inner series.  Its update first grows (the transient
// of the real-time series), falls factorially after its peak, then settles at
// the FP32 rounding level of the partial sums: stop at kInnerTarget, or once it
// sits kStallDrop below its peak and has not improved for kStallSweeps sweeps
// (improvement counted from the latest peak, never during the growth).
constexpr double kInnerTarget = 4e-7;
// A refinement only has to take the residual from its previous value r_prev to the
// tolerance: its inner solve stops at an update of kInnerSlack * tol / r_prev (at
// most kInnerCap; never below kInnerTarget or kGmresTarget).  The update overstates
// nothing by more than a few times, so the slack of 10 keeps the next residual
// below the tolerance.
constexpr double kInnerSlack = 0.1;
constexpr double kInnerCap = 1e-2;
inline double inner_target(double floor_target, double tol, double prev_res) {
  if (!(prev_res < 1e300)) return floor_target;
  const double t = kInnerSlack * tol / prev_res;
  return t > kInnerCap ? kInnerCap : (t > floor_target ? t : floor_target);
}
constexpr double kStallDrop = 1e-4;
constexpr int kStallSweeps = 4;
// The same floor seen earlier: on its FP32 floor the update fluctuates, so new minima
// keep resetting the count above, while the decay itself has stopped.  The series also
// stops once the update, kStallDrop below its peak, fell by less than a factor
// kFlatRatio over the last kStallSweeps sweeps (the decay after the peak is factorial:
// a factor 3 to 10 over four sweeps until the floor).
constexpr double kFlatRatio = 0.8;

// Refinement that grows the residual: a residual above kRefineContract times the
// previous one, kRefineStrikes times, means the series of App. C does not
// converge for this problem (spectral radius of K above 1); the solve ends with
// DYSON_ERR_DIVERGED instead of spending its refinement budget.  A residual that
// falls, however slowly, keeps the solve going (NOT_CONVERGED at the limit).
constexpr double kRefineContract = 1.0;
constexpr int kRefineStrikes = 2;

// An inner series whose update peaked above this (relative to the right-hand
// side) carries FP32 rounding of about kSeriesPeakMax * 6e-8 > 1e-2 in its result,
// too little for refinement to gain; with DYSON_INNER_AUTO the chunk continues
// with GMRES.  Contours of the length of the 16x16 benchmark peak near 1e4.
constexpr double kSeriesPeakMax = 1e5;
// relative residual at which the FP32 GMRES inner solve stops (its rounding floor
// is near 1e-6; the FP64 refinement supplies the rest)
constexpr double kGmresTarget = 4e-6;

// per-kernel-kind timing with events on the library stream
// -------------------------------------------------------------------------
struct KernelTimer {
  dyson_ctx* c;
  int kind;
  cudaEvent_t a = nullptr, b = nullptr;
  KernelTimer(dyson_ctx* cc, int k) : c(cc), kind(k) {
    if (!c->profiling) return;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, c->stream);
  }
  ~KernelTimer() {
    if (!a) return;
    cudaEventRecord(b, c->stream);
    c->pending.push_back({kind, a, b});
  }
};

int fail_noctx(int code, const std::string& m);           // error without a context
double bits_to_double(unsigned long long b);
void flush_timers(dyson_ctx* c);                          // fold finished event timings into the profile
int ensure_work(dyson_ctx* c, size_t bytes);              // grow the work buffer
int ensure_cols(dyson_ctx* c, int ncol, int ng);          // source arrays and norm words for a chunk
int upload_sources(dyson_ctx* c, int ncol);               // host source arrays -> device
int read_norms(dyson_ctx* c, int ng, bool with_scale);    // norm (and scale) words -> host, synchronises
double rel_max(const unsigned long long* norm, const double* ref, int ng);
double sweep_flops(const dyson_ctx* c, int ncol);         // algorithmic contour-GEMM flops of one sweep
// reduced-precision copies of Lambda; sets c->use_tc, c->use_oz
int prepare_tables(dyson_ctx* c, int precision);
// mixed-precision solve of the chunk whose sources are on the device (G in c->work)
int solve_mixed(dyson_ctx* c, int ncol, int gs, int precision, double tol, int max_sweeps, double2** result,
                dyson_report* rep);
// vector columns per chunk that fit in device memory (multiple of unit, at most want)
int64_t chunk_columns(dyson_ctx* c, int precision, int64_t unit, int64_t want, size_t* bytes_per_col);

}  // namespace dyson_detail
