// Series sweeps of App. C on CUDA cores, chunk set-up, observables and export.
//
// Chunk state layout ("vector-column major"): for site i and vector column
// n = q*Nc + z' (block column q, source time z'), the Nc rows z are contiguous.
//   FP64: G[i][n][z] complex128 (interleaved)
//   FP32: S[i][n][0:Nc] real parts, S[i][n][Nc:2Nc] imaginary parts
// One sweep computes, for every site i,
//   out_i = B_i + Lambda_i * X_i,   X_i(n, zb) = W(zb) sum_{j in NN(i)} J_ij(zb) G_j(n, zb),
// with B_i(n, z) = Lambda_i(z, z') when i is the source of block column q.
#include "common.cuh"

namespace {

constexpr int TZ = 64, TN = 64;

// max over the 64 columns of a tile, one global atomic per column group (gs columns) touched
__device__ void tile_norm_flush(unsigned long long* smax, int n0, int ncol, int gs,
                                unsigned long long* __restrict__ norm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = 0;
    int qcur = -1;
    for (int c = 0; c < TN; ++c) {
      int n = n0 + c;
      if (n >= ncol) break;
      int q = n / gs;
      if (q != qcur) {
        if (qcur >= 0 && m) atomicMax(norm + qcur, m);
        qcur = q;
        m = 0;
      }
      if (smax[c] > m) m = smax[c];
    }
    if (qcur >= 0 && m) atomicMax(norm + qcur, m);
  }
}

__device__ __forceinline__ unsigned long long nonneg_bits(double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ULL);
  return (unsigned long long)__double_as_longlong(v);
}

// K3: FP64 sweep (MODE 0) or FP64 Dyson residual (MODE 1).  Tile 64 rows z x 64
// vector columns n per CTA, 256 threads, 4x4 complex outputs per thread.
template <int MODE>
__global__ __launch_bounds__(256) void k_sweep_f64(
    const double2* __restrict__ lam, const double2* __restrict__ JW, const int* __restrict__ nbr,
    const int* __restrict__ nbond, const double2* __restrict__ Gin, double2* __restrict__ out,
    float* __restrict__ out32, const int* __restrict__ src_site, const int* __restrict__ src_time, int Nc,
    int ncol, int gs, unsigned long long* __restrict__ norm) {
  constexpr int KT = 16;
  __shared__ double2 As[TZ][KT + 1];
  __shared__ double2 Xs[TN][KT + 1];
  __shared__ unsigned long long smax[TN];
  const int i = blockIdx.z;
  const int n0 = blockIdx.x * TN, z0 = blockIdx.y * TZ;
  const int tid = threadIdx.x, tz = tid & 15, tn = tid >> 4;
  int nb[4], bd[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    nb[s] = nbr[i * 4 + s];
    bd[s] = nbond[i * 4 + s];
  }
  const double2 zero = make_double2(0.0, 0.0);
  double2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = zero;

  const double2* lam_i = lam + (size_t)i * Nc * Nc;
  for (int k0 = 0; k0 < Nc; k0 += KT) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + 256 * r, row = e >> 4, col = e & 15;
      int z = z0 + row, k = k0 + col;
      As[row][col] = (z < Nc && k < Nc) ? lam_i[(size_t)z * Nc + k] : zero;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int e = tid + 256 * r, row = e >> 4, col = e & 15;
      int n = n0 + row, k = k0 + col;
      double2 x = zero;
      if (n < ncol && k < Nc) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (nb[s] >= 0) {
            double2 w = JW[(size_t)bd[s] * Nc + k];
            double2 g = Gin[((size_t)nb[s] * ncol + n) * Nc + k];
            x.x += w.x * g.x - w.y * g.y;
            x.y += w.x * g.y + w.y * g.x;
          }
        }
      }
      Xs[row][col] = x;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KT; ++kk) {
      double2 a[4], x[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[tz + 16 * r][kk];
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = Xs[tn + 16 * c][kk];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[r][c].x = fma(a[r].x, x[c].x, acc[r][c].x);
          acc[r][c].x = fma(-a[r].y, x[c].y, acc[r][c].x);
          acc[r][c].y = fma(a[r].x, x[c].y, acc[r][c].y);
          acc[r][c].y = fma(a[r].y, x[c].x, acc[r][c].y);
        }
    }
    __syncthreads();
  }

#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int n = n0 + tn + 16 * c;
    double m = 0.0;
    if (n < ncol) {
      const int zp = src_time[n];
      const bool src = (src_site[n] == i);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int z = z0 + tz + 16 * r;
        if (z < Nc) {
          double2 y = acc[r][c];
          if (src) {
            double2 b = lam_i[(size_t)z * Nc + zp];
            y.x += b.x;
            y.y += b.y;
          }
          size_t off = ((size_t)i * ncol + n) * Nc + z;
          double2 g = Gin[off];
          double dx = y.x - g.x, dy = y.y - g.y;
          if (MODE == 0) {
            out[off] = y;
          } else if (out32) {
            size_t o2 = ((size_t)i * ncol + n) * (2 * Nc) + z;
            out32[o2] = (float)dx;
            out32[o2 + Nc] = (float)dy;
          } else {
            out[off] = make_double2(dx, dy);
          }
          m = fmax(m, sqrt(dx * dx + dy * dy));
        }
      }
    }
    unsigned long long mb = nonneg_bits(m);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o, 16);
      mb = v > mb ? v : mb;
    }
    if (tz == 0) smax[tn + 16 * c] = mb;
  }
  tile_norm_flush(smax, n0, ncol, gs, norm);
}

// SIMT FP32 sweep over planar state: dout = r + Lambda' X, Lambda' = Lambda * W (complex64),
// X(n, zb) = sum_j J_ij(zb) din_j(n, zb).  norm[q] = max |dout - din|.
__global__ __launch_bounds__(256) void k_sweep_f32_simt(
    const float2* __restrict__ lam32, const float* __restrict__ Jz, const int* __restrict__ nbr,
    const int* __restrict__ nbond, const float* __restrict__ r, const float* __restrict__ din,
    float* __restrict__ dout, int Nc, int ncol, int gs, unsigned long long* __restrict__ norm) {
  constexpr int KT = 32;
  __shared__ float2 As[TZ][KT + 1];
  __shared__ float2 Xs[TN][KT + 1];
  __shared__ unsigned long long smax[TN];
  const int i = blockIdx.z;
  const int n0 = blockIdx.x * TN, z0 = blockIdx.y * TZ;
  const int tid = threadIdx.x, tz = tid & 15, tn = tid >> 4;
  const int N2 = 2 * Nc;
  int nb[4], bd[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    nb[s] = nbr[i * 4 + s];
    bd[s] = nbond[i * 4 + s];
  }
  float2 acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = make_float2(0.f, 0.f);
  const float2* lam_i = lam32 + (size_t)i * Nc * Nc;
  for (int k0 = 0; k0 < Nc; k0 += KT) {
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      int e = tid + 256 * rr, row = e >> 5, col = e & 31;
      int z = z0 + row, k = k0 + col;
      As[row][col] = (z < Nc && k < Nc) ? lam_i[(size_t)z * Nc + k] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int rr = 0; rr < 8; ++rr) {
      int e = tid + 256 * rr, row = e >> 5, col = e & 31;
      int n = n0 + row, k = k0 + col;
      float xr = 0.f, xi = 0.f;
      if (n < ncol && k < Nc) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          if (nb[s] >= 0) {
            float j = Jz[(size_t)bd[s] * Nc + k];
            const float* g = din + ((size_t)nb[s] * ncol + n) * N2;
            xr = fmaf(j, g[k], xr);
            xi = fmaf(j, g[Nc + k], xi);
          }
        }
      }
      Xs[row][col] = make_float2(xr, xi);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KT; ++kk) {
      float2 a[4], x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = As[tz + 16 * q][kk];
#pragma unroll
      for (int c = 0; c < 4; ++c) x[c] = Xs[tn + 16 * c][kk];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[q][c].x = fmaf(a[q].x, x[c].x, acc[q][c].x);
          acc[q][c].x = fmaf(-a[q].y, x[c].y, acc[q][c].x);
          acc[q][c].y = fmaf(a[q].x, x[c].y, acc[q][c].y);
          acc[q][c].y = fmaf(a[q].y, x[c].x, acc[q][c].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    int n = n0 + tn + 16 * c;
    double m = 0.0;
    if (n < ncol) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        int z = z0 + tz + 16 * q;
        if (z < Nc) {
          size_t off = ((size_t)i * ncol + n) * N2 + z;
          float yr = r[off] + acc[q][c].x, yi = r[off + Nc] + acc[q][c].y;
          float dr = yr - din[off], di = yi - din[off + Nc];
          dout[off] = yr;
          dout[off + Nc] = yi;
          m = fmax(m, (double)sqrtf(dr * dr + di * di));
        }
      }
    }
    unsigned long long mb = nonneg_bits(m);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) {
      unsigned long long v = __shfl_xor_sync(0xffffffffu, mb, o, 16);
      mb = v > mb ? v : mb;
    }
    if (tz == 0) smax[tn + 16 * c] = mb;
  }
  tile_norm_flush(smax, n0, ncol, gs, norm);
}

// B = Lambda delta_s e_{z'}: for vector column n with source (s, z'), G[s][n][z] =
// Lambda_s[z][z'] (one warp per column; s < 0 marks a padding column that stays
// zero); scale[n / gs] = max |B| over the group.  G must be zeroed before.
__global__ void k_init_rhs(const double2* __restrict__ lam, const int* __restrict__ src_site,
                           const int* __restrict__ src_time, int Nc, int ncol, int gs, double2* __restrict__ G,
                           unsigned long long* __restrict__ scale) {
  const int n = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (n >= ncol) return;
  const int s = src_site[n], zp = src_time[n];
  if (s < 0) return;
  const double2* L = lam + (size_t)s * Nc * Nc;
  double m = 0.0;
  for (int z = lane; z < Nc; z += 32) {
    const double2 v = L[(size_t)z * Nc + zp];
    G[((size_t)s * ncol + n) * Nc + z] = v;
    m = fmax(m, sqrt(v.x * v.x + v.y * v.y));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) atomicMax(scale + n / gs, nonneg_bits(m));
}

__global__ void k_accumulate(double2* __restrict__ G, const float* __restrict__ d, int Nc, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    size_t col = e / Nc;
    int z = (int)(e - col * Nc);
    const float* dc = d + col * 2 * Nc;
    double2 g = G[e];
    g.x += (double)dc[z];
    g.y += (double)dc[Nc + z];
    G[e] = g;
  }
}

__global__ void k_to_planar32(const double2* __restrict__ G, float* __restrict__ out, int Nc, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    size_t col = e / Nc;
    int z = (int)(e - col * Nc);
    double2 g = G[e];
    out[col * 2 * Nc + z] = (float)g.x;
    out[col * 2 * Nc + Nc + z] = (float)g.y;
  }
}

// K5: n, ekin, D of the source site of each block column (Sec. III.A, Eq. docc, App. B);
// block column q holds vector columns q*Nc .. q*Nc + Nc - 1 of one source site
__global__ void k_observables(const double2* __restrict__ G, const int* __restrict__ src_site,
                              const int* __restrict__ nbr, const int* __restrict__ nbond,
                              const double* __restrict__ Jtab, const double* __restrict__ eps,
                              const double* __restrict__ U, int Nr, int Nt, int Nc, int ncol, double dt,
                              double* __restrict__ obs) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  int q = blockIdx.y;
  if (k >= Nt) return;
  int s = src_site[(size_t)q * Nc];
  size_t n = (size_t)q * Nc + k;  // source time t_k on the forward branch
  double2 geq = G[((size_t)s * ncol + n) * Nc + k];
  double dens = geq.y;            // Re(-i g) = Im g
  double ax = 0.0, ay = 0.0;
  for (int slot = 0; slot < 4; ++slot) {
    int j = nbr[s * 4 + slot];
    if (j < 0) continue;
    double Jv = Jtab[(size_t)nbond[s * 4 + slot] * Nt + k];
    double2 g = G[((size_t)j * ncol + n) * Nc + k];
    ax += Jv * g.x;
    ay += Jv * g.y;
  }
  double ekin = ay;               // Re(-i acc)
  double D = __longlong_as_double(0x7ff8000000000000ULL);
  if (k >= 1) {
    double2 gm = G[((size_t)s * ncol + n) * Nc + (k - 1)];
    double dre = (geq.x - gm.x) / dt;
    D = (dre - eps[s] * dens - ekin) / U[(size_t)s * Nt + k];
  }
  size_t o = (size_t)s * Nt + k;
  obs[o] = dens;
  obs[(size_t)Nr * Nt + o] = ekin;
  obs[2 * (size_t)Nr * Nt + o] = D;
}

// out[q][j][z][z'] = G[j][q*Nc + z'][z]
__global__ void k_export(const double2* __restrict__ G, int Nr, int Nc, int nq, double2* __restrict__ out) {
  __shared__ double2 t[32][33];
  int j = blockIdx.y, q = blockIdx.z;
  int ncol = nq * Nc, tiles = (Nc + 31) / 32;
  int z0 = (blockIdx.x % tiles) * 32, zp0 = (blockIdx.x / tiles) * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    int zp = zp0 + r, z = z0 + threadIdx.x;
    if (z < Nc && zp < Nc) t[r][threadIdx.x] = G[((size_t)j * ncol + (size_t)q * Nc + zp) * Nc + z];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    int z = z0 + r, zp = zp0 + threadIdx.x;
    if (z < Nc && zp < Nc) out[(((size_t)q * Nr + j) * Nc + z) * Nc + zp] = t[threadIdx.x][r];
  }
}

// out[n][j][z] = G[j][n][z] for the first nv vector columns
__global__ void k_export_vectors(const double2* __restrict__ G, int Nr, int Nc, int ncol, int nv,
                                 double2* __restrict__ out) {
  const size_t total = (size_t)nv * Nr * Nc;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int z = (int)(e % Nc);
    const size_t rest = e / Nc;
    const int j = (int)(rest % Nr);
    const size_t n = rest / Nr;
    out[e] = G[((size_t)j * ncol + n) * Nc + z];
  }
}

int grid_for(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  return (int)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

}  // namespace

void launch_init_rhs(const double2* lam, const int* src_site, const int* src_time, int Nr, int Nc, int ncol, int gs,
                     double2* G, unsigned long long* scale, cudaStream_t s) {
  (void)Nr;
  k_init_rhs<<<(ncol + 7) / 8, 256, 0, s>>>(lam, src_site, src_time, Nc, ncol, gs, G, scale);
}

void launch_sweep_f64(const double2* lam, const double2* JW, const int* nbr, const int* nbond,
                      const double2* Gin, double2* out, float* out32, const int* src_site, const int* src_time,
                      int Nr, int Nc, int ncol, int gs, int mode, unsigned long long* norm, cudaStream_t s) {
  dim3 grd((ncol + TN - 1) / TN, (Nc + TZ - 1) / TZ, Nr);
  if (mode == 0)
    k_sweep_f64<0><<<grd, 256, 0, s>>>(lam, JW, nbr, nbond, Gin, out, nullptr, src_site, src_time, Nc, ncol, gs,
                                       norm);
  else
    k_sweep_f64<1><<<grd, 256, 0, s>>>(lam, JW, nbr, nbond, Gin, out, out32, src_site, src_time, Nc, ncol, gs,
                                       norm);
}

void launch_sweep_f32_simt(const float2* lam32, const float* Jz, const int* nbr, const int* nbond,
                           const float* r, const float* din, float* dout, int Nr, int Nc, int ncol, int gs,
                           unsigned long long* norm, cudaStream_t s) {
  dim3 grd((ncol + TN - 1) / TN, (Nc + TZ - 1) / TZ, Nr);
  k_sweep_f32_simt<<<grd, 256, 0, s>>>(lam32, Jz, nbr, nbond, r, din, dout, Nc, ncol, gs, norm);
}

void launch_export_vectors(const double2* G, int Nr, int Nc, int ncol, int nv, double2* out, cudaStream_t s) {
  const size_t total = (size_t)nv * Nr * Nc;
  k_export_vectors<<<grid_for(total, 256), 256, 0, s>>>(G, Nr, Nc, ncol, nv, out);
}

void launch_accumulate(double2* G, const float* d, int Nr, int Nc, int ncol, cudaStream_t s) {
  size_t total = (size_t)Nr * ncol * Nc;
  k_accumulate<<<grid_for(total, 256), 256, 0, s>>>(G, d, Nc, total);
}

void launch_to_planar32(const double2* G, float* out, size_t n_el, int Nc, cudaStream_t s) {
  k_to_planar32<<<grid_for(n_el, 256), 256, 0, s>>>(G, out, Nc, n_el);
}

void launch_observables(const double2* G, const int* src_site, int nq, const int* nbr, const int* nbond,
                        const double* Jtab, const double* eps, const double* U, int Nr, int Nt, int Nc,
                        int ncol, double dt, double* obs, cudaStream_t s) {
  k_observables<<<dim3((Nt + 127) / 128, nq), 128, 0, s>>>(G, src_site, nbr, nbond, Jtab, eps, U, Nr, Nt, Nc,
                                                          ncol, dt, obs);
}

void launch_export(const double2* G, int Nr, int Nc, int nq, double2* out, cudaStream_t s) {
  int tiles = (Nc + 31) / 32;
  dim3 grd(tiles * tiles, Nr, nq), blk(32, 8);
  k_export<<<grd, blk, 0, s>>>(G, Nr, Nc, nq, out);
}
