// Delta t -> 0 extrapolation of tables computed on refined contours (Sec. IV.D):
// out[r][k] = sum_b w_b values_b[r][k m_b], w_b the Lagrange weights at step 0 of
// the steps h_b = h_0 / m_b, computed on the host in FP64.
#include <string>

#include "detail.cuh"
#include "dyson.h"

using namespace dyson_detail;

namespace {

struct ExtrapArgs {
  const double* v[DYSON_EXTRAPOLATE_MAX_GRIDS];
  double w[DYSON_EXTRAPOLATE_MAX_GRIDS];
  int nt[DYSON_EXTRAPOLATE_MAX_GRIDS];
  int m[DYSON_EXTRAPOLATE_MAX_GRIDS];
  int n;
};

// one thread per output entry (rows x nt[0]); the grid strides over the table
__global__ void k_extrapolate_dt(const __grid_constant__ ExtrapArgs a, double* __restrict__ out, long long total) {
  const int nt0 = a.nt[0];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / nt0;
    const int k = (int)(e - r * nt0);
    double acc = 0.0;
    for (int b = 0; b < a.n; ++b) acc = fma(a.w[b], a.v[b][r * a.nt[b] + (long long)k * a.m[b]], acc);
    out[e] = acc;
  }
}

}  // namespace

extern "C" int dyson_extrapolate_dt(int32_t n_grids, const double* const* values, const int32_t* nt,
                                    const int32_t* m, int32_t rows, double* out, int device, void* stream) {
  if (n_grids < 1 || n_grids > DYSON_EXTRAPOLATE_MAX_GRIDS)
    return fail_noctx(DYSON_ERR_INVALID_ARG, "n_grids must be 1.." + std::to_string(DYSON_EXTRAPOLATE_MAX_GRIDS));
  if (!values || !nt || !m || !out) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL argument");
  if (rows < 1 || nt[0] < 1) return fail_noctx(DYSON_ERR_INVALID_ARG, "need rows >= 1 and nt[0] >= 1");
  if (m[0] != 1) return fail_noctx(DYSON_ERR_INVALID_ARG, "the coarsest grid's divisor m[0] must be 1");
  ExtrapArgs a;
  a.n = n_grids;
  for (int b = 0; b < n_grids; ++b) {
    if (!values[b]) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL table");
    if (b > 0 && m[b] <= m[b - 1]) return fail_noctx(DYSON_ERR_INVALID_ARG, "divisors must increase");
    if ((int64_t)nt[b] < (int64_t)m[b] * (nt[0] - 1) + 1)
      return fail_noctx(DYSON_ERR_INVALID_ARG, "grid " + std::to_string(b) + " is shorter than the coarse grid");
    a.v[b] = values[b];
    a.nt[b] = nt[b];
    a.m[b] = m[b];
    // L_b(0) = prod_{c != b} h_c / (h_c - h_b) with h = 1 / m (the scale h_0 cancels)
    double w = 1.0;
    for (int c = 0; c < n_grids; ++c)
      if (c != b) {
        const double hc = 1.0 / m[c], hb = 1.0 / m[b];
        w *= hc / (hc - hb);
      }
    a.w[b] = w;
  }
  DeviceGuard g(device);
  const long long total = (long long)rows * nt[0];
  const int threads = 256;
  const long long want = (total + threads - 1) / threads;
  const int blocks = (int)(want < 4096 ? want : 4096);
  k_extrapolate_dt<<<blocks, threads, 0, (cudaStream_t)stream>>>(a, out, total);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail_noctx(DYSON_ERR_CUDA, std::string("extrapolation launch: ") + cudaGetErrorString(e));
  return DYSON_OK;
}
