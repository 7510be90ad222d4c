// Autotuner of the tensor-core sweep (dyson_autotune): measures, on the
// context's own Lambda and right-hand sides, the sweep throughput of every
// candidate (sweep variant x block columns per chunk) and keeps the fastest.
//
// A candidate's chunk is set up exactly as the mixed-precision solve sets it up
// (right-hand sides Lambda delta_s of the first sources, FP32 planar state),
// then two warm-up and three timed sweeps run back to back on the context's
// stream; CUDA events give the device time.  A candidate replaces the best so far
// only when it is more than 2 % faster.  Candidates are tried from the
// largest chunk down, so the work buffers are allocated once.  The chunk sizes
// are powers of two up to the caller's cap and to what fits in 85 % of free
// device memory; the CTA-pair and fused variants are tried where Nc allows them.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "detail.cuh"
#include "tc.cuh"

using namespace dyson_detail;

namespace {

// device time (ms) of `timed` sweeps over a chunk of nq block columns
int time_sweeps(dyson_ctx* c, int nq, int warm, int timed, double* ms_per_sweep) {
  const int ncol = nq * c->Nc;
  c->h_src_site.resize(ncol);
  c->h_src_time.resize(ncol);
  for (int q = 0; q < nq; ++q)
    for (int z = 0; z < c->Nc; ++z) {
      c->h_src_site[q * c->Nc + z] = q % c->Nr;
      c->h_src_time[q * c->Nc + z] = z;
    }
  int rc;
  if ((rc = ensure_cols(c, ncol, nq)) || (rc = upload_sources(c, ncol))) return rc;
  const size_t n_el = (size_t)c->Nr * ncol * c->Nc;
  double2* G = (double2*)c->work;
  float* r32 = (float*)(G + n_el);
  float* da = r32 + 2 * n_el;
  float* db = da + 2 * n_el;
  DY_CUDA(c, cudaMemsetAsync(G, 0, n_el * sizeof(double2), c->stream));
  launch_init_rhs(c->d_lam, c->d_src_site, c->d_src_time, c->Nr, c->Nc, ncol, c->Nc, G, c->d_norm + nq, c->stream);
  launch_to_planar32(G, r32, n_el, c->Nc, c->stream);
  DY_CUDA(c, cudaMemcpyAsync(da, r32, 2 * n_el * sizeof(float), cudaMemcpyDeviceToDevice, c->stream));
  c->launches += 2;
  cudaEvent_t e0, e1;
  DY_CUDA(c, cudaEventCreate(&e0));
  DY_CUDA(c, cudaEventCreate(&e1));
  for (int s = 0; s < warm + timed; ++s) {
    if (s == warm) DY_CUDA(c, cudaEventRecord(e0, c->stream));
    if ((rc = tc_sweep(c, ncol, c->Nc, r32, da, db, TC_GATHER | TC_GEMM))) break;
    std::swap(da, db);
  }
  if (rc == DYSON_OK) {
    DY_CUDA(c, cudaEventRecord(e1, c->stream));
    DY_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    DY_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    *ms_per_sweep = ms / timed;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == DYSON_OK) rc = tc_check_error(c);
  return rc;
}

}  // namespace

extern "C" {

int dyson_autotune(dyson_ctx* c, int32_t max_block_columns, dyson_tuning* out) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (max_block_columns < 1) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "max_block_columns must be >= 1");
  if (!c->sigma_built || c->sigma_transposed) return ctx_fail(c, DYSON_ERR_STATE, "Lambda not built or transposed");
  DeviceGuard g(c->device);
  int rc;
  if ((rc = prepare_tables(c, DYSON_PREC_TF32X3_F64REF))) return rc;
  if (!c->use_tc) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "the tensor-core sweep needs Nc % 64 == 0");
  size_t col_bytes = 0;
  const int64_t cap = chunk_columns(c, DYSON_PREC_TF32X3_F64REF, c->Nc, (int64_t)max_block_columns * c->Nc,
                                    &col_bytes) / c->Nc;
  if (cap < 1) return ctx_fail(c, DYSON_ERR_OOM, "one block column does not fit in device memory");
  // a chunk whose inner solve may switch to GMRES (DYSON_INNER_AUTO or _GMRES) must leave
  // room for the Krylov basis of the full restart length (restart + 4 FP32 states), or
  // GMRES would restart early and converge far more slowly than the sweeps timed here
  int64_t cap_gm = cap;
  if (c->inner_solver != DYSON_INNER_SERIES) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
      const int m = c->gmres_restart > 0 ? c->gmres_restart : 40;
      const double per_block = (double)c->Nc * ((double)col_bytes + (m + 4.0) * c->Nr * 2.0 * c->Nc * sizeof(float));
      const double avail = 0.8 * (double)(free_b + c->work_bytes);
      cap_gm = std::max<int64_t>(1, std::min<int64_t>(cap, (int64_t)(avail / per_block)));
    }
  }

  std::vector<int> chunks;
  for (int64_t k = 1; k <= cap_gm; k *= 2) chunks.push_back((int)k);
  if (chunks.back() != cap_gm) chunks.push_back((int)cap_gm);
  std::reverse(chunks.begin(), chunks.end());
  if ((rc = ensure_work(c, (size_t)chunks.front() * c->Nc * col_bytes))) return rc;
  std::vector<int> variants = {DYSON_SWEEP_SINGLE_CTA};
  const int saved_variant = c->tc_variant;
  c->tc_variant = DYSON_SWEEP_CTA_PAIR;
  if (tc_uses_pair(c)) variants.push_back(DYSON_SWEEP_CTA_PAIR);
  for (int v : {DYSON_SWEEP_FUSED_PAIR, DYSON_SWEEP_FUSED_PAIR_WIDE}) {
    c->tc_variant = v;
    if (tc_uses_fused(c)) variants.push_back(v);
  }
  c->tc_variant = saved_variant;

  dyson_tuning T;
  std::memset(&T, 0, sizeof T);
  double best = -1.0;
  for (int nq : chunks)
    for (int v : variants) {
      c->tc_variant = v;
      double ms = 0.0;
      if ((rc = time_sweeps(c, nq, 2, 3, &ms))) {
        c->tc_variant = saved_variant;
        return rc;
      }
      const double rate = (double)nq * c->Nc / (ms * 1e-3);
      if (T.n_candidates < DYSON_TUNE_MAX_CANDIDATES) {
        T.cand_variant[T.n_candidates] = v;
        T.cand_chunk[T.n_candidates] = nq;
        T.cand_vector_columns_per_s[T.n_candidates] = rate;
        ++T.n_candidates;
      }
      // a later candidate must beat the best by 2 %: within timing noise the earlier one
      // (larger chunk, single-CTA form) is kept, so repeated tuning gives one answer
      if (rate > best * 1.02) {
        best = rate;
        T.sweep_variant = v;
        T.chunk_block_columns = nq;
        T.vector_columns_per_s = rate;
      }
    }
  c->tc_variant = T.sweep_variant;
  c->chunk_override = T.chunk_block_columns;
  flush_timers(c);
  if (out) *out = T;
  return DYSON_OK;
}

}  // extern "C"
