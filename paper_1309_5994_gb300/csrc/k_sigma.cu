// K1: atomic-limit contour Green's functions Lambda_i (Sec. III) in FP64, the
// contour hopping tables and the reduced-precision copies of Lambda * W.
#include "common.cuh"

namespace {

// contour point z -> branch (0 forward, 1 backward, 2 imaginary) and grid index
__device__ __forceinline__ int branch_of(int z, int Nt) { return z < Nt ? 0 : (z < 2 * Nt ? 1 : 2); }
__device__ __forceinline__ int time_of(int z, int Nt) { return contour_time_index(z, Nt); }
// quadrature weight of the contour measure: +dt, -dt, -i*beta/Nm
__device__ __forceinline__ double2 weight_of(int z, int Nt, int Nm, double dt, double beta) {
  return contour_weight(z, Nt, Nm, dt, beta);
}

// One thread per site: eps_i (Eq. onsitelevels), log Boltzmann weights of
// H_0^(i)(0) (Eq. Z) and the channel phases Phi_p(z) (Eq. cumulanttabulation).
// phase layout per site: [2][Nc] Phi_p(z) followed by (log a_1, log b_1),
// (log a_2, log b_2).
__global__ void k_site_tables(const double* __restrict__ U, int Lx, int Ly, int Nt, int Nm, double dt,
                              double beta, double curvature, double mu, double* __restrict__ eps_out,
                              double2* __restrict__ phase) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int Nr = Lx * Ly;
  if (i >= Nr) return;
  int Nc = 2 * Nt + Nm;
  int x = i % Lx, y = i / Lx;
  double rx = x - 0.5 * (Lx - 1), ry = y - 0.5 * (Ly - 1);
  const double* Ui = U + (size_t)i * Nt;
  double eps = curvature * (rx * rx + ry * ry) - 0.5 * Ui[0] - mu;
  eps_out[i] = eps;

  // Boltzmann weights of the four states {0, dn, up, d} with energies
  // {0, eps, eps, 2 eps + U(0)}, normalised in log space
  double e0 = 0.0, e1 = -beta * eps, e3 = -beta * (2.0 * eps + Ui[0]);
  double m = fmax(e0, fmax(e1, e3));
  double logZ = m + log(exp(e0 - m) + 2.0 * exp(e1 - m) + exp(e3 - m));
  double l0 = e0 - logZ, ls = e1 - logZ, ld = e3 - logZ;

  double2* ph = phase + (size_t)i * (2 * Nc + 2);
  // real branches: Phi_p(t_k) = dt * sum_{m<k} E_p(t_m), E_1 = eps, E_2 = eps + U(t)
  double s1 = 0.0, s2 = 0.0;
  for (int k = 0; k < Nt; ++k) {
    double p1 = s1 * dt, p2 = s2 * dt;
    ph[k] = make_double2(p1, 0.0);                      // forward point k
    ph[2 * Nt - 1 - k] = make_double2(p1, 0.0);         // backward point carrying t_k
    ph[Nc + k] = make_double2(p2, 0.0);
    ph[Nc + 2 * Nt - 1 - k] = make_double2(p2, 0.0);
    s1 += eps;
    s2 += eps + Ui[k];
  }
  // imaginary branch: Phi_p(-i tau) = -i tau E_p(0)
  double dtau = beta / Nm;
  for (int mm = 0; mm < Nm; ++mm) {
    double tau = mm * dtau;
    ph[2 * Nt + mm] = make_double2(0.0, -tau * eps);
    ph[Nc + 2 * Nt + mm] = make_double2(0.0, -tau * (eps + Ui[0]));
  }
  ph[2 * Nc] = make_double2(l0, ls);      // channel 1: a = rho_0, b = rho_sigma
  ph[2 * Nc + 1] = make_double2(ls, ld);  // channel 2: a = rho_sigma, b = rho_d
}

// Lambda_i(z, z') = -i sum_p exp(-i (Phi_p(z) - Phi_p(z'))) * (a_p if z later than z', else -b_p)
__global__ void k_lambda(const double2* __restrict__ phase, int Nt, int Nm, double2* __restrict__ lam) {
  int Nc = 2 * Nt + Nm;
  int zp = blockIdx.x * blockDim.x + threadIdx.x;
  int z = blockIdx.y * blockDim.y + threadIdx.y;
  int i = blockIdx.z;
  if (z >= Nc || zp >= Nc) return;
  const double2* ph = phase + (size_t)i * (2 * Nc + 2);
  bool later = (z > zp) || (z == zp && branch_of(z, Nt) == 1);
  double re = 0.0, im = 0.0;
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    double2 a = ph[p * Nc + z], b = ph[p * Nc + zp];
    double dr = a.x - b.x, di = a.y - b.y;           // dPhi = dr + i di;  -i dPhi = di - i dr
    double2 lw = ph[2 * Nc + p];
    double mag = exp((later ? lw.x : lw.y) + di);
    double sn, cs;
    sincos(dr, &sn, &cs);
    double sg = later ? 1.0 : -1.0;
    re += sg * mag * cs;
    im -= sg * mag * sn;
  }
  // multiply by -i: (re + i im)(-i) = im - i re
  lam[((size_t)i * Nc + z) * Nc + zp] = make_double2(im, -re);
}

__global__ void k_hopping(const double* __restrict__ J, int Nb, int Nt, int Nm, double dt, double beta,
                          double2* __restrict__ JW, float* __restrict__ Jz) {
  int Nc = 2 * Nt + Nm;
  int z = blockIdx.x * blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (z >= Nc) return;
  double j = J[(size_t)b * Nt + time_of(z, Nt)];
  double2 w = weight_of(z, Nt, Nm, dt, beta);
  JW[(size_t)b * Nc + z] = make_double2(w.x * j, w.y * j);
  Jz[(size_t)b * Nc + z] = (float)j;
}

__global__ void k_lam_c64(const double2* __restrict__ lam, int Nt, int Nm, double dt, double beta,
                          float2* __restrict__ out, size_t total) {
  int Nc = 2 * Nt + Nm;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int zb = (int)(e % Nc);
    double2 v = cmul(lam[e], weight_of(zb, Nt, Nm, dt, beta));
    out[e] = make_float2((float)v.x, (float)v.y);
  }
}

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// real embedding [[Re, -Im], [Im, Re]] of Lambda * W, split as hi + lo in TF32
__global__ void k_lam_emb_split(const double2* __restrict__ lam, int Nt, int Nm, double dt, double beta,
                                float* __restrict__ hi, float* __restrict__ lo, int Nr) {
  int Nc = 2 * Nt + Nm, N2 = 2 * Nc;
  size_t total = (size_t)Nr * N2 * N2;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    int k = (int)(e % N2);
    int m = (int)((e / N2) % N2);
    size_t i = e / ((size_t)N2 * N2);
    int z = m % Nc, zb = k % Nc;
    double2 v = cmul(lam[(i * Nc + z) * Nc + zb], weight_of(zb, Nt, Nm, dt, beta));
    double x = (m < Nc) == (k < Nc) ? v.x : (m < Nc ? -v.y : v.y);
    float f = (float)x;
    float h = to_tf32(f);
    hi[e] = h;
    lo[e] = to_tf32((float)(x - (double)h));
  }
}

// In-place transpose of each Nc x Nc block: the CTA of tile pair (bi, bj), bi <= bj,
// swaps tile (bi, bj) with the transpose of tile (bj, bi) through shared memory.
__global__ void k_transpose_blocks(double2* __restrict__ lam, int Nc) {
  __shared__ double2 ta[32][33], tb[32][33];
  const int tiles = (Nc + 31) / 32;
  const int bi = blockIdx.x / tiles, bj = blockIdx.x % tiles;
  if (bi > bj) return;
  double2* L = lam + (size_t)blockIdx.y * Nc * Nc;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int zi = bi * 32 + r, zj = bj * 32 + threadIdx.x;
    if (zi < Nc && zj < Nc) ta[r][threadIdx.x] = L[(size_t)zi * Nc + zj];
    const int yi = bj * 32 + r, yj = bi * 32 + threadIdx.x;
    if (yi < Nc && yj < Nc) tb[r][threadIdx.x] = L[(size_t)yi * Nc + yj];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int zi = bi * 32 + r, zj = bj * 32 + threadIdx.x;     // (bi, bj) <- transpose of (bj, bi)
    if (zi < Nc && zj < Nc) L[(size_t)zi * Nc + zj] = tb[threadIdx.x][r];
    const int yi = bj * 32 + r, yj = bi * 32 + threadIdx.x;     // (bj, bi) <- transpose of (bi, bj)
    if (yi < Nc && yj < Nc) L[(size_t)yi * Nc + yj] = ta[threadIdx.x][r];
  }
}

int grid_for(size_t total, int threads) {
  size_t b = (total + threads - 1) / threads;
  return (int)(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

}  // namespace

void launch_build_sigma(const double* U, int Lx, int Ly, int Nt, int Nm, double dt, double beta,
                        double curvature, double mu, double* eps, double2* phase, double2* lam,
                        cudaStream_t s) {
  int Nr = Lx * Ly, Nc = 2 * Nt + Nm;
  k_site_tables<<<(Nr + 127) / 128, 128, 0, s>>>(U, Lx, Ly, Nt, Nm, dt, beta, curvature, mu, eps, phase);
  dim3 blk(32, 8), grd((Nc + 31) / 32, (Nc + 7) / 8, Nr);
  k_lambda<<<grd, blk, 0, s>>>(phase, Nt, Nm, lam);
}

void launch_hopping_tables(const double* J, int Nb, int Nt, int Nm, double dt, double beta, double2* JW,
                           float* Jz, cudaStream_t s) {
  if (Nb == 0) return;
  int Nc = 2 * Nt + Nm;
  k_hopping<<<dim3((Nc + 127) / 128, Nb), 128, 0, s>>>(J, Nb, Nt, Nm, dt, beta, JW, Jz);
}

void launch_lam_c64(const double2* lam, int Nr, int Nt, int Nm, double dt, double beta, float2* lam32,
                    cudaStream_t s) {
  int Nc = 2 * Nt + Nm;
  size_t total = (size_t)Nr * Nc * Nc;
  k_lam_c64<<<grid_for(total, 256), 256, 0, s>>>(lam, Nt, Nm, dt, beta, lam32, total);
}

void launch_lam_emb_split(const double2* lam, int Nr, int Nt, int Nm, double dt, double beta, float* hi,
                          float* lo, cudaStream_t s) {
  int Nc = 2 * Nt + Nm;
  size_t total = (size_t)Nr * 4 * Nc * Nc;
  k_lam_emb_split<<<grid_for(total, 256), 256, 0, s>>>(lam, Nt, Nm, dt, beta, hi, lo, Nr);
}

void launch_transpose_blocks(double2* lam, int Nr, int Nc, cudaStream_t s) {
  const int tiles = (Nc + 31) / 32;
  k_transpose_blocks<<<dim3(tiles * tiles, Nr), dim3(32, 8), 0, s>>>(lam, Nc);
}
