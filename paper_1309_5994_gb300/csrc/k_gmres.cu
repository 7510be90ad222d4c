// Preconditioned GMRES of App. C as the inner solver of the mixed-precision path.
//
// The refinement needs d with (I - K) d = r (r: the FP64-accurate residual,
// rounded to the FP32 planar state).  With the block-diagonal preconditioner
// P = B^{-1} of App. C the preconditioned operator is I - K, the initial guess
// is u0 = P b (here r itself) and the first residue is z0 = r - (I - K) r = K r.
// Per column (vector column n of the chunk, its own Krylov space):
//   q_0 = z0 / |z0|;  for j = 0, 1, ...:
//     w = (I - K) q_j                      (K: the 3xTF32 tensor-core sweep with a zero r)
//     two passes of classical Gram-Schmidt: h_ij += <q_i, w>, w -= h_ij q_i (i <= j)
//     h_{j+1,j} = |w|,  q_{j+1} = w / h_{j+1,j}
//     complex Givens rotations reduce the Hessenberg column; |g_{j+1}| is the
//     preconditioned residual of the current iterate
//   until max_n |g_{j+1}| / |r_n| <= tol or j + 1 = m (restart from the iterate);
//   then y = R^{-1} g and d = u0 + sum_i y_i q_i.
// Vectors are FP32 planar states [Nr][ncol][2Nc]; reductions, rotations and the
// small triangular solves are FP64.  The series stalls where the FP32 rounding of
// its transient partial sums is amplified beyond 1 (long contours) or diverges
// (spectral radius of K above 1); GMRES converges in both cases because each
// Krylov vector is normalised and the residual is minimised.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "detail.cuh"
#include "gmres.cuh"
#include "tc.cuh"

using namespace dyson_detail;

namespace {

constexpr int GM_THREADS = 256;

struct GmState {
  float* Q = nullptr;                 // m + 1 Krylov vectors
  float* zero = nullptr;              // zero right-hand side of the matvec
  float* u = nullptr;                 // K q_j
  float* w = nullptr;                 // the vector being orthogonalised
  double2* h = nullptr;               // [ncol][m + 1] first-pass projections of the current column
  double2* h2 = nullptr;              // [ncol][m + 1] second-pass projections
  double* nrm = nullptr;              // [ncol] |w|^2 after orthogonalisation
  double* nrm0 = nullptr;             // [ncol] |(I - K) q_j|^2 before it
  double* nrm1 = nullptr;             // [ncol] |w|^2 after the first pass
  double* bnorm = nullptr;            // [ncol] |r|
  double* beta = nullptr;             // [ncol] |z0| of the current cycle
  double* cs = nullptr;               // [ncol][m] Givens cosines
  double2* sn = nullptr;              // [ncol][m] Givens sines
  double2* g = nullptr;               // [ncol][m + 1] rotated right-hand side
  double2* R = nullptr;               // [ncol][m][m] rotated Hessenberg (column j at R[n][.][j])
  double2* y = nullptr;               // [ncol][m]
  unsigned long long* res = nullptr;  // max over columns of |g_{j+1}| / |r| (bits of a double)
  unsigned long long* h_res = nullptr;
  size_t vsz = 0;
  int m = 0, ncol = 0;
};

GmState* gstate(dyson_ctx* c) {
  if (!c->gm) c->gm = new GmState();
  return static_cast<GmState*>(c->gm);
}

__device__ __forceinline__ double2 gm_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 gm_conj(double2 a) { return make_double2(a.x, -a.y); }

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  __syncthreads();
  return t;   // valid in thread 0
}

// Second Gram-Schmidt pass only where the first lost most of the vector: the
// test of Daniel, Gragg, Kaufman and Stewart, |w| < 0.7 |(I - K) q_j|.
__device__ __forceinline__ bool reorth_needed(const double* after, const double* before, int n) {
  return after[n] < 0.49 * before[n];
}

// h[n][i] += <Q_i[n], a[n] - b[n]>  (b may be null) over a chunk of sites;
// blocks with i = 0 also add |a - b|^2 to nrm0[n] when nrm0 is given.  With a
// gate (after, before), columns that need no second pass are skipped.
// grid: (basis vectors, ncol, site chunks) - the basis index runs fastest, so the
// blocks of one (column, chunk) follow each other and re-read a, b from L2.
__global__ void __launch_bounds__(GM_THREADS) k_gm_dots(const float* __restrict__ Q, size_t vsz,
                                                        const float* __restrict__ a, const float* __restrict__ b,
                                                        int Nr, int Nc, int ncol, int sites_per_blk,
                                                        double2* __restrict__ h, int hstride,
                                                        double* __restrict__ nrm0, const double* __restrict__ after,
                                                        const double* __restrict__ before) {
  __shared__ double sh[GM_THREADS / 32];
  const int i = blockIdx.x, n = blockIdx.y;
  if (after && !reorth_needed(after, before, n)) return;
  const int s0 = blockIdx.z * sites_per_blk, s1 = min(Nr, s0 + sites_per_blk);
  const float* __restrict__ q = Q + (size_t)i * vsz;
  const bool self = nrm0 && i == 0;
  // Each warp walks the block's sites (stride: warps per block), its lanes the
  // contour index, four elements per lane at a time (independent loads in
  // flight).  FP32 products are summed in FP32 within a site and in FP64 across
  // sites - GB300's FP64 pipe is too slow for a product per element.
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  double re = 0.0, im = 0.0, sq = 0.0;
  for (int s = s0 + warp; s < s1; s += nwarps) {
    const size_t base = ((size_t)s * ncol + n) * 2 * Nc;
    const float* __restrict__ ar = a + base;
    const float* __restrict__ br = b ? b + base : nullptr;
    const float* __restrict__ qr_ = q + base;
    float sre = 0.f, sim = 0.f, ssq = 0.f;
    for (int z0 = lane; z0 < Nc; z0 += 128) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int z = z0 + 32 * k;
        if (z < Nc) {
          float wr = ar[z], wi = ar[Nc + z];
          if (br) {
            wr -= br[z];
            wi -= br[Nc + z];
          }
          const float qre = qr_[z], qim = qr_[Nc + z];
          sre = fmaf(qre, wr, fmaf(qim, wi, sre));    // conj(q) w
          sim = fmaf(qre, wi, fmaf(-qim, wr, sim));
          if (self) ssq = fmaf(wr, wr, fmaf(wi, wi, ssq));
        }
      }
    }
    re += sre;
    im += sim;
    sq += ssq;
  }
  re = block_sum(re, sh);
  im = block_sum(im, sh);
  if (self) sq = block_sum(sq, sh);
  if (threadIdx.x == 0) {
    atomicAdd(&h[(size_t)n * hstride + i].x, re);
    atomicAdd(&h[(size_t)n * hstride + i].y, im);
    if (self) atomicAdd(&nrm0[n], sq);
  }
}

// nrm[n] += |a[n]|^2; grid (Nr, ncol)
__global__ void __launch_bounds__(GM_THREADS) k_gm_norm2(const float* __restrict__ a, int Nc, int ncol,
                                                         double* __restrict__ nrm) {
  __shared__ double sh[GM_THREADS / 32];
  const int s = blockIdx.x, n = blockIdx.y;
  const size_t base = ((size_t)s * ncol + n) * 2 * Nc;
  float part = 0.f;
  for (int z = threadIdx.x; z < 2 * Nc; z += blockDim.x) part = fmaf(a[base + z], a[base + z], part);
  const double acc = block_sum((double)part, sh);
  if (threadIdx.x == 0) atomicAdd(&nrm[n], acc);
}

// out = a - b + c elementwise over the whole chunk state
__global__ void k_gm_lin3(const float* __restrict__ a, const float* __restrict__ b, const float* __restrict__ c,
                          float* __restrict__ out, size_t n4) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n4; e += (size_t)gridDim.x * blockDim.x) {
    const float4 x = reinterpret_cast<const float4*>(a)[e];
    const float4 y = reinterpret_cast<const float4*>(b)[e];
    const float4 z = reinterpret_cast<const float4*>(c)[e];
    reinterpret_cast<float4*>(out)[e] = make_float4(x.x - y.x + z.x, x.y - y.y + z.y, x.z - y.z + z.z, x.w - y.w + z.w);
  }
}

// v <- sqrt(v)
__global__ void k_gm_sqrt(double* __restrict__ v, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = sqrt(fmax(v[i], 0.0));
}

// w[n] = (a[n] - b[n]) - sum_{i < nvec} h[n][i] Q_i[n]  (b may be null), nrm[n] += |w[n]|^2.
// With a gate (after, before): columns that need no second pass keep w and
// take nrm[n] = after[n].  grid: (Nr, ncol)
// (a and w may be the same array: each element is read, then written, by one thread)
__global__ void __launch_bounds__(GM_THREADS) k_gm_update(const float* __restrict__ Q, size_t vsz, int nvec,
                                                          const double2* __restrict__ h, int hstride,
                                                          const float* a, const float* __restrict__ b, float* w,
                                                          int Nc, int ncol, double* __restrict__ nrm,
                                                          const double* __restrict__ after,
                                                          const double* __restrict__ before) {
  __shared__ double sh[GM_THREADS / 32];
  __shared__ float2 hs[64];
  const int s = blockIdx.x, n = blockIdx.y;
  if (after && !reorth_needed(after, before, n)) {
    if (s == 0 && threadIdx.x == 0) atomicAdd(&nrm[n], after[n]);
    return;
  }
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    const double2 v = h[(size_t)n * hstride + i];
    hs[i] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const size_t base = ((size_t)s * ncol + n) * 2 * Nc;
  double acc = 0.0;
  for (int z = threadIdx.x; z < Nc; z += blockDim.x) {
    float wr = a[base + z], wi = a[base + Nc + z];
    if (b) {
      wr -= b[base + z];
      wi -= b[base + Nc + z];
    }
    const float* qz = Q + base + z;
    int i = 0;
    for (; i + 4 <= nvec; i += 4) {                      // four independent loads in flight
      float qr[4], qi[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        qr[k] = qz[(size_t)(i + k) * vsz];
        qi[k] = qz[(size_t)(i + k) * vsz + Nc];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 c = hs[i + k];
        wr -= c.x * qr[k] - c.y * qi[k];
        wi -= c.x * qi[k] + c.y * qr[k];
      }
    }
    for (; i < nvec; ++i) {
      const float qr = qz[(size_t)i * vsz], qi = qz[(size_t)i * vsz + Nc];
      const float2 c = hs[i];
      wr -= c.x * qr - c.y * qi;
      wi -= c.x * qi + c.y * qr;
    }
    w[base + z] = wr;
    w[base + Nc + z] = wi;
    acc += fmaf(wr, wr, wi * wi);
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0 && nrm) atomicAdd(&nrm[n], acc);
}

// out[n] = scale[n] * x[n] with scale = 1 / sqrt(nrm[n]) (0 where nrm = 0); grid (Nr, ncol)
__global__ void __launch_bounds__(GM_THREADS) k_gm_scale(const float* __restrict__ x, const double* __restrict__ nrm,
                                                         float* __restrict__ out, int Nc, int ncol) {
  const int s = blockIdx.x, n = blockIdx.y;
  const double v = nrm[n];
  const float f = v > 0.0 ? (float)(1.0 / sqrt(v)) : 0.f;
  const size_t base = ((size_t)s * ncol + n) * 2 * Nc;
  for (int z = threadIdx.x; z < 2 * Nc; z += blockDim.x) out[base + z] = f * x[base + z];
}

// out[n] = x0[n] + sum_{i < nvec} y[n][i] Q_i[n]; grid (Nr, ncol)
// (x0 and out may be the same array)
__global__ void __launch_bounds__(GM_THREADS) k_gm_combine(const float* __restrict__ Q, size_t vsz, int nvec,
                                                           const double2* __restrict__ y, int ystride,
                                                           const float* x0, float* out, int Nc, int ncol) {
  __shared__ float2 ys[64];
  const int s = blockIdx.x, n = blockIdx.y;
  for (int i = threadIdx.x; i < nvec; i += blockDim.x) {
    const double2 v = y[(size_t)n * ystride + i];
    ys[i] = make_float2((float)v.x, (float)v.y);
  }
  __syncthreads();
  const size_t base = ((size_t)s * ncol + n) * 2 * Nc;
  for (int z = threadIdx.x; z < Nc; z += blockDim.x) {
    float xr = x0[base + z], xi = x0[base + Nc + z];
    const float* qz = Q + base + z;
    int i = 0;
    for (; i + 4 <= nvec; i += 4) {
      float qr[4], qi[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        qr[k] = qz[(size_t)(i + k) * vsz];
        qi[k] = qz[(size_t)(i + k) * vsz + Nc];
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float2 c = ys[i + k];
        xr += c.x * qr[k] - c.y * qi[k];
        xi += c.x * qi[k] + c.y * qr[k];
      }
    }
    for (; i < nvec; ++i) {
      const float qr = qz[(size_t)i * vsz], qi = qz[(size_t)i * vsz + Nc];
      const float2 c = ys[i];
      xr += c.x * qr - c.y * qi;
      xi += c.x * qi + c.y * qr;
    }
    out[base + z] = xr;
    out[base + Nc + z] = xi;
  }
}

// Start of a cycle, per column: beta = sqrt(nrm), g = (beta, 0, ...).
__global__ void k_gm_start(int ncol, int m, const double* __restrict__ nrm, double* __restrict__ beta,
                           double2* __restrict__ g) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncol) return;
  const double b = sqrt(fmax(nrm[n], 0.0));
  beta[n] = b;
  for (int i = 0; i <= m; ++i) g[(size_t)n * (m + 1) + i] = make_double2(i == 0 ? b : 0.0, 0.0);
}

// Column j of the Hessenberg matrix, per column n: apply the earlier rotations,
// make rotation j, rotate g, keep the reduced column in R, and fold the new
// residual |g_{j+1}| / |r| into res (max over columns).
__global__ void k_gm_givens(int j, int ncol, int m, const double2* __restrict__ h, const double2* __restrict__ h2,
                            const double* __restrict__ nrm,
                            const double* __restrict__ bnorm, double* __restrict__ cs, double2* __restrict__ sn,
                            double2* __restrict__ g, double2* __restrict__ R, unsigned long long* __restrict__ res) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncol) return;
  const double2* h1c = h + (size_t)n * (m + 1);
  const double2* h2c = h2 + (size_t)n * (m + 1);
  auto hc = [&](int i) { return make_double2(h1c[i].x + h2c[i].x, h1c[i].y + h2c[i].y); };
  double* c_ = cs + (size_t)n * m;
  double2* s_ = sn + (size_t)n * m;
  double2* gn = g + (size_t)n * (m + 1);
  double2* Rn = R + (size_t)n * m * m;
  double2 col_i = hc(0);
  for (int i = 0; i < j; ++i) {
    const double2 next = hc(i + 1);
    // [a; b] <- [c a + s b; -conj(s) a + c b]
    const double2 a = col_i;
    const double2 top = make_double2(c_[i] * a.x + gm_mul(s_[i], next).x, c_[i] * a.y + gm_mul(s_[i], next).y);
    const double2 sa = gm_mul(gm_conj(s_[i]), a);
    col_i = make_double2(-sa.x + c_[i] * next.x, -sa.y + c_[i] * next.y);
    Rn[(size_t)i * m + j] = top;
  }
  const double2 a = col_i;                           // entry j after the earlier rotations
  const double bsub = sqrt(fmax(nrm[n], 0.0));       // h_{j+1,j}, real and non-negative
  const double aa = sqrt(a.x * a.x + a.y * a.y);
  double c, rr;
  double2 s, r;
  if (aa == 0.0) {
    c = 0.0;
    s = make_double2(1.0, 0.0);
    r = make_double2(bsub, 0.0);
  } else {
    rr = sqrt(aa * aa + bsub * bsub);
    c = aa / rr;
    s = make_double2(bsub * a.x / (rr * aa), bsub * a.y / (rr * aa));
    r = make_double2(a.x / aa * rr, a.y / aa * rr);
  }
  c_[j] = c;
  s_[j] = s;
  Rn[(size_t)j * m + j] = r;
  const double2 gj = gn[j];
  gn[j] = make_double2(c * gj.x, c * gj.y);
  const double2 t = gm_mul(gm_conj(s), gj);
  gn[j + 1] = make_double2(-t.x, -t.y);
  const double bn = bnorm[n];
  const double rel = bn > 0.0 ? sqrt(t.x * t.x + t.y * t.y) / bn : 0.0;
  atomicMax(res, (unsigned long long)__double_as_longlong(rel == rel ? rel : 1e300));
}

// y = R^{-1} g over the first d rows, per column
__global__ void k_gm_backsolve(int d, int ncol, int m, const double2* __restrict__ R, const double2* __restrict__ g,
                               double2* __restrict__ y) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ncol) return;
  const double2* Rn = R + (size_t)n * m * m;
  const double2* gn = g + (size_t)n * (m + 1);
  double2* yn = y + (size_t)n * m;
  for (int i = d - 1; i >= 0; --i) {
    double2 acc = gn[i];
    for (int k = i + 1; k < d; ++k) {
      const double2 p = gm_mul(Rn[(size_t)i * m + k], yn[k]);
      acc.x -= p.x;
      acc.y -= p.y;
    }
    const double2 di = Rn[(size_t)i * m + i];
    const double den = di.x * di.x + di.y * di.y;
    yn[i] = den > 0.0 ? make_double2((acc.x * di.x + acc.y * di.y) / den, (acc.y * di.x - acc.x * di.y) / den)
                      : make_double2(0.0, 0.0);
  }
}

template <class T>
int gm_alloc(dyson_ctx* c, T** p, size_t count) {
  if (*p) cudaFree(*p);
  *p = nullptr;
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, DYSON_ERR_OOM, std::string("GMRES buffers: ") + cudaGetErrorString(e));
  }
  return DYSON_OK;
}

// buffers for ncol columns of vsz floats and restart length m
int gm_prepare(dyson_ctx* c, size_t vsz, int ncol, int m) {
  GmState* st = gstate(c);
  if (st->vsz == vsz && st->ncol == ncol && st->m == m) return DYSON_OK;
  int rc;
  if ((rc = gm_alloc(c, &st->Q, (size_t)(m + 1) * vsz)) || (rc = gm_alloc(c, &st->zero, vsz)) ||
      (rc = gm_alloc(c, &st->u, vsz)) || (rc = gm_alloc(c, &st->w, vsz)) ||
      (rc = gm_alloc(c, &st->h, (size_t)ncol * (m + 1))) || (rc = gm_alloc(c, &st->h2, (size_t)ncol * (m + 1))) ||
      (rc = gm_alloc(c, &st->nrm, ncol)) || (rc = gm_alloc(c, &st->nrm0, ncol)) ||
      (rc = gm_alloc(c, &st->nrm1, ncol)) ||
      (rc = gm_alloc(c, &st->bnorm, ncol)) || (rc = gm_alloc(c, &st->beta, ncol)) ||
      (rc = gm_alloc(c, &st->cs, (size_t)ncol * m)) || (rc = gm_alloc(c, &st->sn, (size_t)ncol * m)) ||
      (rc = gm_alloc(c, &st->g, (size_t)ncol * (m + 1))) || (rc = gm_alloc(c, &st->R, (size_t)ncol * m * m)) ||
      (rc = gm_alloc(c, &st->y, (size_t)ncol * m)) || (rc = gm_alloc(c, &st->res, 1))) {
    st->vsz = 0;
    return rc;
  }
  if (!st->h_res) DY_CUDA(c, cudaMallocHost((void**)&st->h_res, sizeof(unsigned long long)));
  DY_CUDA(c, cudaMemsetAsync(st->zero, 0, vsz * sizeof(float), c->stream));
  st->vsz = vsz;
  st->ncol = ncol;
  st->m = m;
  return DYSON_OK;
}

}  // namespace

int gmres_restart_length(dyson_ctx* c, int ncol) {
  const size_t vbytes = (size_t)c->Nr * ncol * 2 * c->Nc * sizeof(float);
  GmState* st = static_cast<GmState*>(c->gm);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 0;
  const size_t held = st ? (size_t)(st->m + 4) * st->vsz * sizeof(float) : 0;
  const double budget = 0.8 * (double)(free_b + held);
  const int fit = (int)(budget / (double)vbytes) - 4;
  return std::max(0, std::min(c->gmres_restart > 0 ? c->gmres_restart : 40, std::min(fit, 60)));
}

int gmres_inner_solve(dyson_ctx* c, int ncol, const float* r, float* x, int max_iters, double tol,
                      dyson_report* rep, const MatvecFn& matvec) {
  if (ncol > 65535 || c->Nr > 65535) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "GMRES chunks hold <= 65535 columns");
  const int m = gmres_restart_length(c, ncol);
  if (m < 2) return ctx_fail(c, DYSON_ERR_OOM, "GMRES needs room for at least 3 Krylov vectors");
  const size_t vsz = (size_t)c->Nr * ncol * 2 * c->Nc;
  int rc = gm_prepare(c, vsz, ncol, m);
  if (rc) return rc;
  GmState* st = gstate(c);
  cudaStream_t s = c->stream;
  const int Nc = c->Nc;
  const dim3 grid_el(c->Nr, ncol);
  // dot blocks: enough (basis x column x chunk) blocks without tiny chunks
  const int chunks = (int)std::max<int64_t>(1, std::min<int64_t>(c->Nr, 4096 / std::max(1, ncol)));
  const int sites_per_blk = (c->Nr + chunks - 1) / chunks;
  const int nchunk = (c->Nr + sites_per_blk - 1) / sites_per_blk;
  const int cb = (ncol + 127) / 128;
  const size_t n4 = vsz / 4;
  const int lin_grid = (int)std::min<size_t>((n4 + 255) / 256, 152 * 16);
  const size_t hbytes = (size_t)ncol * (m + 1) * sizeof(double2);

  // |r| per column, and the iterate starts at u0 = r
  DY_CUDA(c, cudaMemsetAsync(st->bnorm, 0, ncol * sizeof(double), s));
  k_gm_norm2<<<grid_el, GM_THREADS, 0, s>>>(r, Nc, ncol, st->bnorm);
  k_gm_sqrt<<<cb, 128, 0, s>>>(st->bnorm, ncol);
  DY_CUDA(c, cudaMemcpyAsync(x, r, vsz * sizeof(float), cudaMemcpyDeviceToDevice, s));
  c->launches += 2;
  int its = 0;
  double rel = INFINITY;
  while (its < max_iters) {
    // residue of the iterate: z0 = r - (I - K) x = r - x + K x
    if ((rc = matvec(st->zero, x, st->u))) return rc;
    rep->sweeps += 1;
    rep->gemm_flops += sweep_flops(c, ncol);
    k_gm_lin3<<<lin_grid, 256, 0, s>>>(r, x, st->u, st->w, n4);
    DY_CUDA(c, cudaMemsetAsync(st->nrm, 0, ncol * sizeof(double), s));
    k_gm_norm2<<<grid_el, GM_THREADS, 0, s>>>(st->w, Nc, ncol, st->nrm);
    k_gm_start<<<cb, 128, 0, s>>>(ncol, m, st->nrm, st->beta, st->g);
    k_gm_scale<<<grid_el, GM_THREADS, 0, s>>>(st->w, st->nrm, st->Q, Nc, ncol);
    c->launches += 4;
    int d = 0;
    for (int j = 0; j < m && its < max_iters; ++j) {
      ++its;
      float* qj = st->Q + (size_t)j * vsz;
      // u = K q_j, so w = (I - K) q_j = q_j - u
      if ((rc = matvec(st->zero, qj, st->u))) return rc;
      rep->sweeps += 1;
      rep->gemm_flops += sweep_flops(c, ncol);
      // classical Gram-Schmidt: h = <Q, q_j - u>, w = q_j - u - Q h; then, for the
      // columns that lost most of their length, a second pass h2 = <Q, w>, w -= Q h2
      DY_CUDA(c, cudaMemsetAsync(st->h, 0, hbytes, s));
      DY_CUDA(c, cudaMemsetAsync(st->h2, 0, hbytes, s));
      DY_CUDA(c, cudaMemsetAsync(st->nrm0, 0, ncol * sizeof(double), s));
      DY_CUDA(c, cudaMemsetAsync(st->nrm1, 0, ncol * sizeof(double), s));
      DY_CUDA(c, cudaMemsetAsync(st->nrm, 0, ncol * sizeof(double), s));
      k_gm_dots<<<dim3(j + 1, ncol, nchunk), GM_THREADS, 0, s>>>(st->Q, vsz, qj, st->u, c->Nr, Nc, ncol,
                                                                 sites_per_blk, st->h, m + 1, st->nrm0, nullptr,
                                                                 nullptr);
      k_gm_update<<<grid_el, GM_THREADS, 0, s>>>(st->Q, vsz, j + 1, st->h, m + 1, qj, st->u, st->w, Nc, ncol,
                                                  st->nrm1, nullptr, nullptr);
      k_gm_dots<<<dim3(j + 1, ncol, nchunk), GM_THREADS, 0, s>>>(st->Q, vsz, st->w, nullptr, c->Nr, Nc, ncol,
                                                                 sites_per_blk, st->h2, m + 1, nullptr, st->nrm1,
                                                                 st->nrm0);
      k_gm_update<<<grid_el, GM_THREADS, 0, s>>>(st->Q, vsz, j + 1, st->h2, m + 1, st->w, nullptr, st->w, Nc, ncol,
                                                  st->nrm, st->nrm1, st->nrm0);
      k_gm_scale<<<grid_el, GM_THREADS, 0, s>>>(st->w, st->nrm, st->Q + (size_t)(j + 1) * vsz, Nc, ncol);
      DY_CUDA(c, cudaMemsetAsync(st->res, 0, sizeof(unsigned long long), s));
      k_gm_givens<<<cb, 128, 0, s>>>(j, ncol, m, st->h, st->h2, st->nrm, st->bnorm, st->cs, st->sn, st->g, st->R,
                                     st->res);
      DY_CUDA(c, cudaMemcpyAsync(st->h_res, st->res, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
      DY_CUDA(c, cudaGetLastError());
      DY_CUDA(c, cudaStreamSynchronize(s));
      c->host_syncs += 1;
      flush_timers(c);
      c->launches += 6;
      d = j + 1;
      rel = bits_to_double(*st->h_res);
      rep->update = rel;
      if (!(rel < kDivergedGrowth)) return ctx_fail(c, DYSON_ERR_DIVERGED, "GMRES residual not finite");
      if (rel <= tol) break;
    }
    // x += Q_d y,  y = R^{-1} g
    k_gm_backsolve<<<cb, 128, 0, s>>>(d, ncol, m, st->R, st->g, st->y);
    k_gm_combine<<<grid_el, GM_THREADS, 0, s>>>(st->Q, vsz, d, st->y, m, x, x, Nc, ncol);
    c->launches += 2;
    DY_CUDA(c, cudaGetLastError());
    if (rel <= tol) break;
  }
  return DYSON_OK;
}

void gmres_release(dyson_ctx* c) {
  GmState* st = static_cast<GmState*>(c->gm);
  if (!st) return;
  void* ptrs[] = {st->Q, st->zero, st->u, st->w, st->h, st->h2, st->nrm, st->nrm0, st->nrm1, st->bnorm, st->beta,
                  st->cs, st->sn, st->g, st->R, st->y, st->res};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (st->h_res) cudaFreeHost(st->h_res);
  delete st;
  c->gm = nullptr;
}
