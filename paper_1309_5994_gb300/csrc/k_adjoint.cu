// Gradients of L = sum_i Re(beta_i . c_i), c_i = G e_i the column at (i, z_f) and
// beta_i a sparse complex weight vector (no paper counterpart).  The site
// density n_i(t_f) = Im c_i(i, z_f) and the double occupancy D_i(t_f) of
// Eq. (docc) are both of this form.  From G = (I - K)^{-1} Lambda, K = Lambda W J:
//     dG = (I + G W J) dLambda (I + W J G) + G W dJ G,
// so with the effective rows psi_i = sum_a beta_ia r_a (r_a^T = e_a^T G: rows come
// from the same solver on transposed site blocks), gamma_i = e_i + W J c_i and
// rho_i = beta_i + W J psi_i:
//   dL/dJ_b(t_k) = Re sum_i sum_{z in Z_k} W(z) (psi_i(l,z) c_i(m,z) + psi_i(m,z) c_i(l,z)),
//   dL/dU_l(t_k) = Re sum_{z,z'} dLambda_l/dU_l(t_k)(z,z') M_l(z',z),  M_l = sum_i gamma_i[l] rho_i[l]^T,
// plus D's explicit dependence on U(t_f), U(0) and J(t_f).  The kernels carry
// beta' = i beta (real for the density) and take imaginary parts: Re(x) = Im(i x).
// The derivative of the closed form (Sec. III): U(t_k), k >= 1, only moves the
// channel-2 phase on real points later than t_k, so
//   dL/dU_l(t_k) = -dt Re sum_{real z, m(z) > k} (rowsum_2 - colsum_2)(z),
//   T_p(z,z') = Lambda^(p)(z,z') M(z',z),  rowsum_p(z) = sum_z' T_p,  colsum_p(z') = sum_z T_p;
// U(0) also moves the level eps = V - U(0)/2 - mu, every phase and the Boltzmann
// weights, and takes the full chain rule.
//
// Layouts: C, rows and psi [i][j][z] complex128 (column i of G or of G^T is [Nr][Nc]).
#include "common.cuh"

namespace {

__device__ __forceinline__ int time_of(int z, int Nt) { return contour_time_index(z, Nt); }
__device__ __forceinline__ bool is_imag(int z, int Nt) { return z >= 2 * Nt; }
__device__ __forceinline__ double2 weight_of(int z, int Nt, int Nm, double dt, double beta) {
  return contour_weight(z, Nt, Nm, dt, beta);
}
__device__ __forceinline__ void bond_sites(int b, int Lx, int Ly, int* l, int* m) {
  const int hb = Ly * (Lx - 1);
  if (b < hb) {
    const int y = b / (Lx - 1), x = b % (Lx - 1);
    *l = y * Lx + x;
    *m = *l + 1;
  } else {
    const int bb = b - hb, y = bb / Lx, x = bb % Lx;
    *l = y * Lx + x;
    *m = *l + Lx;
  }
}

// L = sum_i w_i Im C_i(i, z_f)
// one CTA per bond: gJ[b][k] = sum_i w_i Im[sum_{z in Z_k} W(z)(r_i(l,z) c_i(m,z) + r_i(m,z) c_i(l,z))]
__global__ void k_adj_bonds(const double2* __restrict__ C, const double2* __restrict__ R, const double* __restrict__ w,
                            int Lx, int Ly, int Nt, int Nm, double dt, double beta, double* __restrict__ gJ) {
  extern __shared__ double bins[];                   // [Nt]
  const int Nr = Lx * Ly, Nc = 2 * Nt + Nm, b = blockIdx.x;
  int l, m;
  bond_sites(b, Lx, Ly, &l, &m);
  for (int k = threadIdx.x; k < Nt; k += blockDim.x) bins[k] = 0.0;
  __syncthreads();
  for (int z = threadIdx.x; z < Nc; z += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int i = 0; i < Nr; ++i) {
      const double wi = w[i];
      if (wi == 0.0) continue;
      const size_t base = (size_t)i * Nr;
      const double2 rl = R[(base + l) * Nc + z], cm = C[(base + m) * Nc + z];
      const double2 rm = R[(base + m) * Nc + z], cl = C[(base + l) * Nc + z];
      sr += wi * (rl.x * cm.x - rl.y * cm.y + rm.x * cl.x - rm.y * cl.y);
      si += wi * (rl.x * cm.y + rl.y * cm.x + rm.x * cl.y + rm.y * cl.x);
    }
    const double2 W = weight_of(z, Nt, Nm, dt, beta);
    atomicAdd(&bins[time_of(z, Nt)], W.x * si + W.y * sr);   // Im(W S)
  }
  __syncthreads();
  for (int k = threadIdx.x; k < Nt; k += blockDim.x) gJ[(size_t)b * Nt + k] = bins[k];
}

// Gam[l][i][z] = delta_il delta_{z zf} + W(z) sum_{m in NN(l)} J_lm(z) X_i(m, z) for X = C (gamma) or R (rho)
__global__ void k_adj_gather(const double2* __restrict__ X, const int* __restrict__ nbr, const int* __restrict__ nbond,
                             const double* __restrict__ Jtab, int Nr, int Nt, int Nm, double dt, double beta, int zf,
                             double2* __restrict__ out) {
  const int Nc = 2 * Nt + Nm;
  const size_t li = (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (li >= (size_t)Nr * Nr) return;
  const int l = (int)(li / Nr), i = (int)(li % Nr);
  for (int z = threadIdx.x & 31; z < Nc; z += 32) {
    double ar = 0.0, ai = 0.0;
    const int tk = time_of(z, Nt);
    for (int s = 0; s < 4; ++s) {
      const int m = nbr[l * 4 + s];
      if (m < 0) continue;
      const double Jv = Jtab[(size_t)nbond[l * 4 + s] * Nt + tk];
      const double2 x = X[((size_t)i * Nr + m) * Nc + z];
      ar += Jv * x.x;
      ai += Jv * x.y;
    }
    double2 v = cmul(weight_of(z, Nt, Nm, dt, beta), make_double2(ar, ai));
    if (l == i && z == zf) v.x += 1.0;
    out[li * Nc + z] = v;
  }
}

// M_l[z'][z] = sum_i w_i Gam[l][i][z'] P[l][i][z]; CTA: one site, a 32 x 32 tile
__global__ __launch_bounds__(256) void k_adj_M(const double2* __restrict__ Gam, const double2* __restrict__ P,
                                               const double* __restrict__ w, int Nr, int Nc,
                                               double2* __restrict__ M) {
  __shared__ double2 ga[16][33], pb[16][33];
  const int l = blockIdx.z, t0 = blockIdx.y * 32, u0 = blockIdx.x * 32;   // rows z' (t), columns z (u)
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[2][2] = {};
  for (int i0 = 0; i0 < Nr; i0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int ii = e / 32, c = e % 32, i = i0 + ii;
      double2 g = make_double2(0.0, 0.0), p = make_double2(0.0, 0.0);
      if (i < Nr) {
        const size_t base = ((size_t)l * Nr + i) * Nc;
        if (t0 + c < Nc) {
          g = Gam[base + t0 + c];
          g.x *= w[i];
          g.y *= w[i];
        }
        if (u0 + c < Nc) p = P[base + u0 + c];
      }
      ga[ii][c] = g;
      pb[ii][c] = p;
    }
    __syncthreads();
    for (int ii = 0; ii < 16; ++ii)
      for (int a = 0; a < 2; ++a) {
        const double2 g = ga[ii][ty + 16 * a];
        for (int bb = 0; bb < 2; ++bb) {
          const double2 p = pb[ii][tx + 16 * bb];
          acc[a][bb].x = fma(g.x, p.x, fma(-g.y, p.y, acc[a][bb].x));
          acc[a][bb].y = fma(g.x, p.y, fma(g.y, p.x, acc[a][bb].y));
        }
      }
    __syncthreads();
  }
  for (int a = 0; a < 2; ++a)
    for (int bb = 0; bb < 2; ++bb) {
      const int t = t0 + ty + 16 * a, u = u0 + tx + 16 * bb;
      if (t < Nc && u < Nc) M[((size_t)l * Nc + t) * Nc + u] = acc[a][bb];
    }
}

// channel part Lambda^(p)(z, z') of the closed form, from the phase table of k_site_tables
__device__ __forceinline__ double2 channel(const double2* ph, int Nc, int Nt, int p, int z, int zp) {
  const bool later = (z > zp) || (z == zp && z >= Nt && z < 2 * Nt);
  const double2 a = ph[p * Nc + z], b = ph[p * Nc + zp];
  const double dr = a.x - b.x, di = a.y - b.y;
  const double2 lw = ph[2 * Nc + p];
  const double mag = exp((later ? lw.x : lw.y) + di);
  double sn, cs;
  sincos(dr, &sn, &cs);
  const double sg = later ? 1.0 : -1.0;
  // -i * sg * mag * (cs - i sn) = -sg mag sn - i sg mag cs
  return make_double2(-sg * mag * sn, -sg * mag * cs);
}

// one CTA per site l: gU[l][k]
__global__ void k_adj_U(const double2* __restrict__ M, const double2* __restrict__ phase, int Nt, int Nm, double dt,
                        double beta, double* __restrict__ gU) {
  extern __shared__ double sh[];                      // D[Nc] (re), bins[Nt], red[64]
  const int Nc = 2 * Nt + Nm, l = blockIdx.x;
  double* D = sh;
  double* bins = sh + Nc;
  double* red = bins + Nt;
  const double2* ph = phase + (size_t)l * (2 * Nc + 2);
  const double2* Ml = M + (size_t)l * Nc * Nc;
  const double dtau = beta / Nm;
  // log weights and their U(0)-derivatives: dl_0 = -beta rho_s, dl_s = beta/2 - beta rho_s, dl_d = -beta rho_s
  const double rho_s = exp(ph[2 * Nc].y);
  const double dl0 = -beta * rho_s, dls = 0.5 * beta - beta * rho_s, dld = -beta * rho_s;
  const double dla[2] = {dl0, dls}, dlb[2] = {dls, dld};
  // d Phi_p(z) / d U(0) (see the derivation in the header)
  auto dphi = [&](int p, int z) -> double2 {
    if (is_imag(z, Nt)) {
      const double tau = (z - 2 * Nt) * dtau;
      return p == 0 ? make_double2(0.0, 0.5 * tau) : make_double2(0.0, -0.5 * tau);
    }
    const int m = time_of(z, Nt);
    return make_double2(p == 0 ? -0.5 * dt * m : dt * (-0.5 * m + (m > 0 ? 1.0 : 0.0)), 0.0);
  };
  double acc0r = 0.0, acc0i = 0.0;                   // U(0) chain rule, sum_{z,z'} T_p dlog_p
  // pass 1: rows (rowsum) and the weight-derivative terms
  for (int z = threadIdx.x; z < Nc; z += blockDim.x) {
    double2 row[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    for (int zp = 0; zp < Nc; ++zp) {
      const double2 m = Ml[(size_t)zp * Nc + z];
      const bool later = (z > zp) || (z == zp && z >= Nt && z < 2 * Nt);
      for (int p = 0; p < 2; ++p) {
        const double2 t = cmul(channel(ph, Nc, Nt, p, z, zp), m);
        row[p].x += t.x;
        row[p].y += t.y;
        const double wgt = later ? dla[p] : dlb[p];
        acc0r += wgt * t.x;
        acc0i += wgt * t.y;
      }
    }
    // phase part of the U(0) derivative: -i sum_z dPhi_p(z) rowsum_p(z)
    for (int p = 0; p < 2; ++p) {
      const double2 d = dphi(p, z);
      const double2 t = cmul(make_double2(d.y, -d.x), row[p]);   // -i d * row
      acc0r += t.x;
      acc0i += t.y;
    }
    D[z] = is_imag(z, Nt) ? 0.0 : row[1].x;          // Re rowsum_2 on real points
  }
  __syncthreads();
  // pass 2: columns (colsum)
  for (int zp = threadIdx.x; zp < Nc; zp += blockDim.x) {
    double2 col[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};
    for (int z = 0; z < Nc; ++z) {
      const double2 m = Ml[(size_t)zp * Nc + z];
      for (int p = 0; p < 2; ++p) {
        const double2 t = cmul(channel(ph, Nc, Nt, p, z, zp), m);
        col[p].x += t.x;
        col[p].y += t.y;
      }
    }
    for (int p = 0; p < 2; ++p) {                     // +i sum_z' dPhi_p(z') colsum_p(z')
      const double2 d = dphi(p, zp);
      const double2 t = cmul(make_double2(-d.y, d.x), col[p]);
      acc0r += t.x;
      acc0i += t.y;
    }
    if (!is_imag(zp, Nt)) D[zp] -= col[1].x;           // D = Re(rowsum_2 - colsum_2)
  }
  __syncthreads();
  // reduce the U(0) sum: gU[l][0] = Re(-i acc0) = Im(acc0)
  double v = acc0i;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) s0 += red[k];
    // bins by real time index, then suffix sums: gU[k] = -dt sum_{m > k} bin[m] (k >= 1)
    for (int k = 0; k < Nt; ++k) bins[k] = 0.0;
    for (int z = 0; z < 2 * Nt; ++z) bins[time_of(z, Nt)] += D[z];
    double suffix = 0.0;
    for (int k = Nt - 1; k >= 1; --k) {
      gU[(size_t)l * Nt + k] = -dt * suffix;
      suffix += bins[k];
    }
    gU[(size_t)l * Nt + 0] = s0;
  }
}

// Effective rows psi_i = sum_a beta'_ia r_a: rows at (i, kf), (i, kf - 1) and
// (j, kf) for the neighbour slots j of i, with the coefficients of AdjCoef.
// Layout [i][l][z]; one warp per (i, l).
__global__ void k_adj_psi(const double2* __restrict__ R1, const double2* __restrict__ R2,
                          const AdjCoef* __restrict__ coef, const int* __restrict__ nbr, int Nr, int Nc,
                          double2* __restrict__ psi) {
  const size_t il = (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (il >= (size_t)Nr * Nr) return;
  const int i = (int)(il / Nr), l = (int)(il % Nr);
  const AdjCoef cf = coef[i];
  int js[4];
  for (int s = 0; s < 4; ++s) js[s] = nbr[i * 4 + s];
  for (int z = threadIdx.x & 31; z < Nc; z += 32) {
    double2 acc = cmul(cf.b0, R1[((size_t)i * Nr + l) * Nc + z]);
    if (R2) {
      const double2 t = cmul(cf.b1, R2[((size_t)i * Nr + l) * Nc + z]);
      acc.x += t.x;
      acc.y += t.y;
    }
    for (int s = 0; s < 4; ++s) {
      if (js[s] < 0 || (cf.bj[s].x == 0.0 && cf.bj[s].y == 0.0)) continue;
      const double2 t = cmul(cf.bj[s], R1[((size_t)js[s] * Nr + l) * Nc + z]);
      acc.x += t.x;
      acc.y += t.y;
    }
    psi[il * Nc + z] = acc;
  }
}

// rho_i += beta'_i (its few non-zero entries); rho layout [l][i][z]
__global__ void k_adj_rho_add(const AdjCoef* __restrict__ coef, const int* __restrict__ nbr, int Nr, int Nc, int kf,
                              double2* __restrict__ rho) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nr) return;
  const AdjCoef cf = coef[i];
  auto add = [&](int l, int z, double2 v) {
    double2& r = rho[((size_t)l * Nr + i) * Nc + z];
    r.x += v.x;
    r.y += v.y;
  };
  add(i, kf, cf.b0);
  if (kf >= 1) add(i, kf - 1, cf.b1);
  for (int s = 0; s < 4; ++s)
    if (nbr[i * 4 + s] >= 0) add(nbr[i * 4 + s], kf, cf.bj[s]);
}

// Loss L = sum_i wn_i n_i + wd_i D_i from the columns, and the explicit dependence
// of D_i on U_i(t_f), U_i(0) (through eps_i) and J_ij(t_f), added to gU and gJ.
__global__ void k_adj_obs_terms(const double2* __restrict__ C, const double* __restrict__ wn,
                                const double* __restrict__ wd, const double* __restrict__ eps,
                                const double* __restrict__ Utab, const double* __restrict__ Jtab,
                                const int* __restrict__ nbr, const int* __restrict__ nbond, int Nr, int Nt, int Nc,
                                int kf, double dt, double* __restrict__ loss, double* __restrict__ gU,
                                double* __restrict__ gJ) {
  double s = 0.0;
  for (int i = threadIdx.x; i < Nr; i += blockDim.x) {
    const double2* ci = C + (size_t)i * Nr * Nc;
    const double n = ci[(size_t)i * Nc + kf].y;
    if (wn) s += wn[i] * n;
    if (wd && wd[i] != 0.0) {
      const double U = Utab[(size_t)i * Nt + kf];
      double ekin = 0.0;
      for (int q = 0; q < 4; ++q) {
        const int j = nbr[i * 4 + q];
        if (j >= 0) ekin += Jtab[(size_t)nbond[i * 4 + q] * Nt + kf] * ci[(size_t)j * Nc + kf].y;
      }
      const double D = ((ci[(size_t)i * Nc + kf].x - ci[(size_t)i * Nc + kf - 1].x) / dt - eps[i] * n - ekin) / U;
      s += wd[i] * D;
      atomicAdd(&gU[(size_t)i * Nt + kf], wd[i] * (-D / U));
      atomicAdd(&gU[(size_t)i * Nt + 0], wd[i] * n / (2.0 * U));
      for (int q = 0; q < 4; ++q) {
        const int j = nbr[i * 4 + q];
        if (j >= 0) atomicAdd(&gJ[(size_t)nbond[i * 4 + q] * Nt + kf], wd[i] * (-ci[(size_t)j * Nc + kf].y / U));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += part[k];
    *loss = t;
  }
}

}  // namespace

int adjoint_contract_obs(dyson_ctx* c, const double2* C, const double2* R1, const double2* R2,
                         const AdjCoef* coef_dev, const double* wn_dev, const double* wd_dev, const double* ones_dev,
                         int kf, double2* psi, double2* gam, double2* rho, double2* M, double* loss_dev,
                         double* gU_dev, double* gJ_dev) {
  const int Nr = c->Nr, Nc = c->Nc, Nt = c->Nt;
  const size_t warps = (size_t)Nr * Nr;
  const unsigned wblocks = (unsigned)((warps + 7) / 8);
  k_adj_psi<<<wblocks, 256, 0, c->stream>>>(R1, R2, coef_dev, c->d_nbr, Nr, Nc, psi);
  if (c->Nb > 0)
    k_adj_bonds<<<c->Nb, 256, Nt * sizeof(double), c->stream>>>(C, psi, ones_dev, c->Lx, c->Ly, Nt, c->Nm, c->dt,
                                                                  c->beta, gJ_dev);
  k_adj_gather<<<wblocks, 256, 0, c->stream>>>(C, c->d_nbr, c->d_nbond, c->dJ, Nr, Nt, c->Nm, c->dt, c->beta, kf,
                                               gam);
  k_adj_gather<<<wblocks, 256, 0, c->stream>>>(psi, c->d_nbr, c->d_nbond, c->dJ, Nr, Nt, c->Nm, c->dt, c->beta, -1,
                                               rho);
  k_adj_rho_add<<<(Nr + 127) / 128, 128, 0, c->stream>>>(coef_dev, c->d_nbr, Nr, Nc, kf, rho);
  const int tiles = (Nc + 31) / 32;
  k_adj_M<<<dim3(tiles, tiles, Nr), 256, 0, c->stream>>>(gam, rho, ones_dev, Nr, Nc, M);
  const size_t shmem = (size_t)(Nc + Nt + 64) * sizeof(double);
  k_adj_U<<<Nr, 256, shmem, c->stream>>>(M, c->d_phase, Nt, c->Nm, c->dt, c->beta, gU_dev);
  k_adj_obs_terms<<<1, 256, 0, c->stream>>>(C, wn_dev, wd_dev, c->d_eps, c->dU, c->dJ, c->d_nbr, c->d_nbond, Nr, Nt,
                                            Nc, kf, c->dt, loss_dev, gU_dev, gJ_dev);
  c->launches += (c->Nb > 0 ? 9 : 8);
  DY_CUDA(c, cudaGetLastError());
  return DYSON_OK;
}
