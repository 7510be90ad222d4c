// Self-energy step of the strong-coupling expansion (Sec. III, Eqs. (selfcons),
// (defnSigma), (defnSigmatilde); Sec. IV.C, Eq. (Sigmamix) and its convergence rule).
//
// Given the local Green's functions Gloc_j = G_jj of the last lattice solve:
//   F_i(c, b)      = sum_{j in NN(i)} W_c J_ij(c) Gloc_j(c, b) J_ji(b) W_b
//   Sigma~_i(a, d) = - sum_{b,c} K_i(a, b; c, d) F_i(c, b),
//   K = sum_{s1} [G2_{up s1}(a,b;c,d) + G0(a,c) G0(b,d) delta_{up s1} - G0(a,d) G0(b,c)],
// the second-order cumulant of the isolated site summed over the neighbour's spin.
// The disconnected terms contract to G0 F G0 and G0 tr(G0 F) (batched complex
// GEMMs); the connected part, the two-particle function G2 of the site, is
// evaluated on the fly (Sec. III: no [Nc]^4 tensor is stored).  Its Hamiltonian is
// diagonal in the number basis, so each operator of the T_C-ordered product moves
// a basis state to one other state with the phase exp(-/+ i Phi_p(z)) of its
// channel p (p = 1: the other spin is empty, energy eps; p = 2: it is occupied,
// energy eps + U), and the trace is a sum over the four initial states.  For
// fixed (a, b, d) the contour order of the four operators changes only where the
// creator's point c passes a, b or d, so c runs through at most four intervals,
// each with one operator order.  A host-built table gives, for each order, spin
// case and initial state, the fermionic sign and the four channels; the kernel
// adds per interval the coefficient of exp(i Phi_p(c)) F(c, b) for p = 1, 2.  The
// interval sums over the real branches come from prefix sums over c (unit-modulus
// factors there, so no cancellation), the imaginary branch is summed directly:
// O(Nc^3 (1 + Nm)) per site instead of the paper's O(Nc^4), all in FP64 (the
// imaginary-branch factors span exp(+-beta E); there each summand is a product,
// which keeps its relative precision, and a physical, bounded term).
//
// Then Sigma = G0^-1 * Sigma~ * G0^-1 enters the lattice solve through the local
// Dyson equation B = G0 + G0 * Sigma * B, whose matrix solution
//   B_i = G0_i (G0_i - Sigma~_i)^-1 G0_i
// replaces Lambda_i and needs no inverse of G0.  On the discretised contour the
// turning points (last forward / first backward point, last backward / first
// imaginary point) carry one time each, so G0 and Sigma~ share equal columns
// (right null vector v = e_{Nt-1} - e_{Nt}) and equal rows (left null vector
// u = e_{2Nt-1} - e_{2Nt}); the singular system is completed to
// G0 - Sigma~ + u v^T / 2, which leaves B unchanged.  Mixing (Eq. (Sigmamix)) acts
// on Sigma~ (Sigma is linear in it), and so does the convergence measure
// N_bd^-1 |dSigma~|_F + |dSigma~|_max: forming Sigma itself would divide by the
// exponentially small singular value the atomic G0 develops on long real-time
// branches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "detail.cuh"
#include "dyson.h"

using namespace dyson_detail;

void oz_invalidate(dyson_ctx* c);

namespace {

// ---------------------------------------------------------------------------
// operator-path table
// ---------------------------------------------------------------------------
// operators of G2_{up s1}(a, b; c, d) in product order: kind 0 = c_up(a), 1 = c_s1(b),
// 2 = c+_s1(c), 3 = c+_up(d).  An order is four kinds, latest first, coded
// o0*64 + o1*16 + o2*4 + o3.  Entry [code][spin case * 4 + initial state]:
//   bit 0 valid, bit 1 sign negative, bits 2..5 channel - 1 of kinds 0..3, bits 6..7 state class
//   (0: |0>, 1: one particle, 2: doubly occupied).  The sign includes (-i)^2 = -1.
constexpr int PATHS = 8;

uint32_t path_entry(const int o[4], int spin_case, int nu) {
  // permutation parity of the order against the product order 0 1 2 3
  int inv = 0;
  for (int x = 0; x < 4; ++x)
    for (int y = x + 1; y < 4; ++y)
      if (o[x] > o[y]) ++inv;
  int sign = (inv & 1) ? -1 : 1;
  sign = -sign;                                          // (-i)^2
  int state = nu, ch[4] = {0, 0, 0, 0};
  for (int u = 3; u >= 0; --u) {                        // earliest operator acts first
    const int kind = o[u];
    const bool up = kind == 0 || kind == 3 || spin_case == 0;
    const bool creator = kind >= 2;
    const int n_up = (state >> 1) & 1, n_dn = state & 1;
    const int occ = up ? n_up : n_dn, other = up ? n_dn : n_up;
    if (creator == (occ != 0)) return 0;                 // create on occupied / remove from empty
    if (!up && n_up) sign = -sign;                       // c_dn carries the Jordan-Wigner string of up
    ch[kind] = other;                                    // channel 2 when the other spin is present
    state ^= up ? 2 : 1;
  }
  if (state != nu) return 0;
  const int cls = nu == 0 ? 0 : (nu == 3 ? 2 : 1);
  uint32_t e = 1u | (sign < 0 ? 2u : 0u);
  for (int k = 0; k < 4; ++k) e |= (uint32_t)ch[k] << (2 + k);
  return e | ((uint32_t)cls << 6);
}

std::vector<uint32_t> path_table() {
  std::vector<uint32_t> t(256 * PATHS, 0);
  int o[4];
  for (o[0] = 0; o[0] < 4; ++o[0])
    for (o[1] = 0; o[1] < 4; ++o[1])
      for (o[2] = 0; o[2] < 4; ++o[2])
        for (o[3] = 0; o[3] < 4; ++o[3]) {
          if (o[0] == o[1] || o[0] == o[2] || o[0] == o[3] || o[1] == o[2] || o[1] == o[3] || o[2] == o[3]) continue;
          const int code = o[0] * 64 + o[1] * 16 + o[2] * 4 + o[3];
          for (int sc = 0; sc < 2; ++sc)
            for (int nu = 0; nu < 4; ++nu) t[code * PATHS + sc * 4 + nu] = path_entry(o, sc, nu);
        }
  return t;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int branch_bwd(int z, int Nt) { return z >= Nt && z < 2 * Nt; }
// T_C keys: contour index, then the equal-point rule (creators later on the forward
// and imaginary branches, annihilators later on the backward branch), then the
// product order (kind 0 latest among equals)
__device__ __forceinline__ int key_ann(int z, int Nt, int kind) { return ((2 * z + branch_bwd(z, Nt)) << 2) | (3 - kind); }
__device__ __forceinline__ int key_cre(int z, int Nt, int kind) { return ((2 * z + 1 - branch_bwd(z, Nt)) << 2) | (3 - kind); }
// first creator point c (kind 2) whose key exceeds K
__device__ __forceinline__ int first_c_above(int K, int Nt) {
  const int z = K >> 3;
  return key_cre(z, Nt, 2) > K ? z : z + 1;
}

__device__ __forceinline__ double2 cexp_phase(double2 phi, double sgn) {
  // exp(sgn * (-i) * phi) for phi = dr + i di:  -i phi = di - i dr
  double s, c;
  sincos(-sgn * phi.x, &s, &c);
  const double m = exp(sgn * phi.y);
  return make_double2(m * c, m * s);
}

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

// FT_i[b][c] = F_i(c, b) = sum_s JW_s(c) Gloc_{nb s}(c, b) JW_s(b); 32 x 32 tiles through shared memory
__global__ void k_se_hyb(const double2* __restrict__ gloc, const double2* __restrict__ JW, const int* __restrict__ nbr,
                         const int* __restrict__ nbond, int Nc, double2* __restrict__ FT) {
  __shared__ double2 tile[32][33];
  const int i = blockIdx.z;
  const int c0 = blockIdx.y * 32, b0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8
  double2 acc[4];
  for (int r = 0; r < 4; ++r) acc[r] = make_double2(0.0, 0.0);
  for (int s = 0; s < 4; ++s) {
    const int j = nbr[i * 4 + s];
    if (j < 0) continue;
    const double2* jw = JW + (size_t)nbond[i * 4 + s] * Nc;
    for (int r = 0; r < 4; ++r) {
      const int c = c0 + ty + 8 * r, b = b0 + tx;
      if (c < Nc && b < Nc) acc[r] = cadd(acc[r], cmul(cmul(jw[c], gloc[((size_t)j * Nc + c) * Nc + b]), jw[b]));
    }
  }
  for (int r = 0; r < 4; ++r) tile[ty + 8 * r][tx] = acc[r];
  __syncthreads();
  for (int r = 0; r < 4; ++r) {
    const int b = b0 + ty + 8 * r, c = c0 + tx;
    if (b < Nc && c < Nc) FT[((size_t)i * Nc + b) * Nc + c] = tile[tx][ty + 8 * r];
  }
}

// Prefix sums over the real branches of the creator terms:
// Q_i[p][b][c] = sum_{c' < c} exp(+i Phi_p(c')) F_i(c', b),  c = 0..2Nt (2Nt + 1 entries).
// On the real branches |exp(+i Phi)| = 1, so differences of these sums lose nothing to
// cancellation; the imaginary branch, whose factors span exp(+-beta E), is summed directly.
__global__ void k_se_prefix(const double2* __restrict__ phase, const double2* __restrict__ FT, int Nt, int Nm,
                            const int* __restrict__ sites, double2* __restrict__ Q) {
  const int Nc = 2 * Nt + Nm, R = 2 * Nt;
  const int i = sites ? sites[blockIdx.y] : blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * Nc) return;
  const int p = t / Nc, b = t % Nc;
  const double2* ph = phase + (size_t)i * (2 * Nc + 2) + (size_t)p * Nc;
  const double2* f = FT + ((size_t)i * Nc + b) * Nc;
  double2* q = Q + (((size_t)i * 2 + p) * Nc + b) * (R + 1);
  double2 acc = make_double2(0.0, 0.0);
  q[0] = acc;
  for (int c = 0; c < R; ++c) {
    acc = cfma(cexp_phase(ph[c], -1.0), f[c], acc);
    q[c + 1] = acc;
  }
}

// connected part: conn_i(a, d) = sum_{b,c} [G2_{up up} + G2_{up dn}](a, b; c, d) F_i(c, b)
// grid (ceil(Nc^2 / 256), sites), 256 threads, one (a, d) per thread; blockIdx.y indexes `sites`
// (all sites in order when NULL).  Per b the creator point c
// runs through four intervals of fixed operator order: their real-branch parts come from the
// prefix sums Q, their imaginary-branch parts are summed directly.
constexpr int CONN_THREADS = 256;
__global__ void __launch_bounds__(CONN_THREADS) k_se_conn(const uint32_t* __restrict__ paths,
                                                           const double2* __restrict__ phase,
                                                           const double2* __restrict__ FT,
                                                           const double2* __restrict__ Q, int Nt, int Nm,
                                                           const int* __restrict__ sites,
                                                           double2* __restrict__ conn) {
  extern __shared__ double2 sm[];
  const int Nc = 2 * Nt + Nm, R = 2 * Nt;
  const int i = sites ? sites[blockIdx.y] : blockIdx.y;
  double2* em = sm;                  // [2][Nc] exp(-i Phi_p(z)): annihilator factors
  double2* ep = em + 2 * Nc;         // [2][Nc] exp(+i Phi_p(z)): creator factors
  double2* Qs = ep + 2 * Nc;         // [2][R + 1] prefix sums of the current b
  double2* Pi = Qs + 2 * (R + 1);    // [2][Nm] exp(+i Phi_p(c)) F(c, b) on the imaginary branch
  uint32_t* tab = reinterpret_cast<uint32_t*>(Pi + 2 * Nm);   // [256][PATHS]
  __shared__ double rho[3];
  const double2* ph = phase + (size_t)i * (2 * Nc + 2);
  for (int e = threadIdx.x; e < 2 * Nc; e += blockDim.x) {
    em[e] = cexp_phase(ph[e], 1.0);
    ep[e] = cexp_phase(ph[e], -1.0);
  }
  for (int e = threadIdx.x; e < 256 * PATHS; e += blockDim.x) tab[e] = paths[e];
  if (threadIdx.x == 0) {
    const double2 l1 = ph[2 * Nc], l2 = ph[2 * Nc + 1];  // (log rho_0, log rho_s), (log rho_s, log rho_d)
    rho[0] = exp(l1.x);
    rho[1] = exp(l1.y);
    rho[2] = exp(l2.y);
  }
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = e < Nc * Nc;
  const int a = live ? e / Nc : 0, d = live ? e % Nc : 0;
  const int Ka = key_ann(a, Nt, 0), Kd = key_cre(d, Nt, 3);
  double2 acc = make_double2(0.0, 0.0);
  __syncthreads();
  // products of the factors at a and d for the four channel pairs (pa, pd)
  double2 fad[4];
#pragma unroll
  for (int pa = 0; pa < 2; ++pa)
#pragma unroll
    for (int pd = 0; pd < 2; ++pd) fad[pa * 2 + pd] = cmul(em[pa * Nc + a], ep[pd * Nc + d]);
  const double2* Fi = FT + (size_t)i * Nc * Nc;
  const double2* Qi = Q + (size_t)i * 2 * Nc * (R + 1);
  for (int b = 0; b < Nc; ++b) {
    __syncthreads();                                   // the previous b's tables are no longer read
    for (int x = threadIdx.x; x < 2 * (R + 1); x += blockDim.x) {
      const int p = x / (R + 1), c = x % (R + 1);
      Qs[x] = Qi[((size_t)p * Nc + b) * (R + 1) + c];
    }
    for (int x = threadIdx.x; x < Nm; x += blockDim.x) {
      const double2 f = Fi[(size_t)b * Nc + R + x];
      Pi[x] = cmul(ep[R + x], f);
      Pi[Nm + x] = cmul(ep[Nc + R + x], f);
    }
    __syncthreads();
    const int Kb = key_ann(b, Nt, 1);
    // the three fixed operators, latest first
    int k0 = 0, k1 = 1, k2 = 3;                          // kinds
    int K0 = Ka, K1 = Kb, K2 = Kd;
    if (K1 > K0) { int t = K0; K0 = K1; K1 = t; t = k0; k0 = k1; k1 = t; }
    if (K2 > K1) { int t = K1; K1 = K2; K2 = t; t = k1; k1 = k2; k2 = t; }
    if (K1 > K0) { int t = K0; K0 = K1; K1 = t; t = k0; k0 = k1; k1 = t; }
    const int n0 = first_c_above(K0, Nt), n1 = first_c_above(K1, Nt), n2 = first_c_above(K2, Nt);
    const double2 fb0 = em[b], fb1 = em[Nc + b];
    // coefficients of P_1(c), P_2(c) on the four c intervals
    double2 A[4][2];
#pragma unroll
    for (int iv = 0; iv < 4; ++iv) {
      // iv = number of fixed operators earlier than c
      const int code = iv == 0 ? (k0 * 64 + k1 * 16 + k2 * 4 + 2)
                     : iv == 1 ? (k0 * 64 + k1 * 16 + 2 * 4 + k2)
                     : iv == 2 ? (k0 * 64 + 2 * 16 + k1 * 4 + k2)
                               : (2 * 64 + k0 * 16 + k1 * 4 + k2);
      double2 s1 = make_double2(0.0, 0.0), s2 = make_double2(0.0, 0.0);
#pragma unroll
      for (int q = 0; q < PATHS; ++q) {
        const uint32_t t = tab[code * PATHS + q];
        if (!(t & 1u)) continue;
        const double w = ((t & 2u) ? -1.0 : 1.0) * rho[(t >> 6) & 3u];
        const int pad = ((t & 4u) ? 2 : 0) + ((t & 32u) ? 1 : 0);
        const double2 f1 = pad == 0 ? fad[0] : pad == 1 ? fad[1] : pad == 2 ? fad[2] : fad[3];
        double2 v = cmul(f1, (t & 8u) ? fb1 : fb0);
        v.x *= w;
        v.y *= w;
        if (t & 16u) s2 = cadd(s2, v);
        else s1 = cadd(s1, v);
      }
      A[iv][0] = s1;
      A[iv][1] = s2;
    }
    // real branches: interval iv covers [lo, hi) with lo/hi from (0, n2, n1, n0, Nc), clipped to R
    {
      const int bnd[5] = {0, min(n2, R), min(n1, R), min(n0, R), R};
#pragma unroll
      for (int iv = 0; iv < 4; ++iv) {
        const double2 q1 = make_double2(Qs[bnd[iv + 1]].x - Qs[bnd[iv]].x, Qs[bnd[iv + 1]].y - Qs[bnd[iv]].y);
        const double2 q2 = make_double2(Qs[R + 1 + bnd[iv + 1]].x - Qs[R + 1 + bnd[iv]].x,
                                        Qs[R + 1 + bnd[iv + 1]].y - Qs[R + 1 + bnd[iv]].y);
        acc = cfma(A[iv][0], q1, cfma(A[iv][1], q2, acc));
      }
    }
    // imaginary branch: direct
    for (int x = 0; x < Nm; ++x) {
      const int c = R + x;
      const bool g0 = c >= n0, g1 = c >= n1, g2 = c >= n2;
      const double2 x0 = g0 ? A[3][0] : g1 ? A[2][0] : g2 ? A[1][0] : A[0][0];
      const double2 x1 = g0 ? A[3][1] : g1 ? A[2][1] : g2 ? A[1][1] : A[0][1];
      acc = cfma(x0, Pi[x], cfma(x1, Pi[Nm + x], acc));
    }
  }
  if (live) conn[((size_t)i * Nc + a) * Nc + d] = acc;
}

// batched complex GEMM C_i = A_i B_i, 32 x 32 tiles
__global__ void k_zgemm(const double2* __restrict__ A, const double2* __restrict__ B, double2* __restrict__ C, int n) {
  __shared__ double2 As[32][33], Bs[32][33];
  const int i = blockIdx.z;
  const int row0 = blockIdx.y * 32, col0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;          // 32 x 8: each thread 4 rows
  const double2* Ai = A + (size_t)i * n * n;
  const double2* Bi = B + (size_t)i * n * n;
  double2 acc[4];
  for (int r = 0; r < 4; ++r) acc[r] = make_double2(0.0, 0.0);
  for (int k0 = 0; k0 < n; k0 += 32) {
    for (int r = 0; r < 4; ++r) {
      const int rr = ty + 8 * r;
      double2 av = make_double2(0.0, 0.0), bv = make_double2(0.0, 0.0);
      if (row0 + rr < n && k0 + tx < n) av = Ai[(size_t)(row0 + rr) * n + k0 + tx];
      As[rr][tx] = av;                                    // As[row][k]
      if (k0 + rr < n && col0 + tx < n) bv = Bi[(size_t)(k0 + rr) * n + col0 + tx];
      Bs[rr][tx] = bv;                                    // Bs[k][col]
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const double2 b = Bs[k][tx];
      for (int r = 0; r < 4; ++r) acc[r] = cfma(As[ty + 8 * r][k], b, acc[r]);
    }
    __syncthreads();
  }
  for (int r = 0; r < 4; ++r) {
    const int row = row0 + ty + 8 * r, col = col0 + tx;
    if (row < n && col < n) C[((size_t)i * n + row) * n + col] = acc[r];
  }
}

// tr_i = sum_{b,c} G0(b, c) F(c, b) = sum_{b,c} G0[b][c] FT[b][c]; one block per site
__global__ void k_se_trace(const double2* __restrict__ g0, const double2* __restrict__ FT, int Nc,
                           double2* __restrict__ tr) {
  const int i = blockIdx.x;
  const size_t n = (size_t)Nc * Nc, off = (size_t)i * n;
  double re = 0.0, im = 0.0;
  for (size_t e = threadIdx.x; e < n; e += blockDim.x) {
    const double2 v = cmul(g0[off + e], FT[off + e]);
    re += v.x;
    im += v.y;
  }
  __shared__ double sr[256], si[256];
  sr[threadIdx.x] = re;
  si[threadIdx.x] = im;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) tr[i] = make_double2(sr[0], si[0]);
}

// St = -conn - D1 + 2 tr G0
__global__ void k_se_combine(const double2* __restrict__ conn, const double2* __restrict__ D1,
                             const double2* __restrict__ tr, const double2* __restrict__ g0, size_t per_site,
                             size_t total, double2* __restrict__ St) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double2 t = tr[e / per_site];
    const double2 g = cmul(t, g0[e]);
    St[e] = make_double2(-conn[e].x - D1[e].x + 2.0 * g.x, -conn[e].y - D1[e].y + 2.0 * g.y);
  }
}

// M = G0 - Sigma~ + u v^T / 2 (u = e_{2Nt-1} - e_{2Nt}, v = e_{Nt-1} - e_{Nt}): the turning-point completion
__global__ void k_se_complete(const double2* __restrict__ g0, const double2* __restrict__ St, int Nc, int Nt,
                              size_t total, double2* __restrict__ M) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)((e / Nc) % Nc), c = (int)(e % Nc);
    double x = g0[e].x - St[e].x;
    const double su = r == 2 * Nt - 1 ? 1.0 : (r == 2 * Nt ? -1.0 : 0.0);
    const double sv = c == Nt - 1 ? 1.0 : (c == Nt ? -1.0 : 0.0);
    x += 0.5 * su * sv;
    M[e] = make_double2(x, g0[e].y - St[e].y);
  }
}

// out_i = A_i^T
__global__ void k_transpose(const double2* __restrict__ A, int n, double2* __restrict__ out) {
  __shared__ double2 tile[32][33];
  const int i = blockIdx.z;
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int row = r0 + r, col = c0 + threadIdx.x;
    if (row < n && col < n) tile[r][threadIdx.x] = A[((size_t)i * n + row) * n + col];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int row = c0 + r, col = r0 + threadIdx.x;
    if (row < n && col < n) {
      out[((size_t)i * n + row) * n + col] = tile[threadIdx.x][r];
    }
  }
}

// Gauss-Jordan elimination with partial pivoting, one block per site:
// A_i (n x n) is destroyed, R_i (n x n right-hand sides) becomes A_i^-1 R_i.
// A zero pivot sets err[i] = 1 and leaves the site's result undefined.
constexpr int GJ_THREADS = 256;
__global__ void __launch_bounds__(GJ_THREADS) k_gauss_jordan(double2* __restrict__ A, double2* __restrict__ R, int n,
                                                              int* __restrict__ err) {
  extern __shared__ double2 fcol[];                     // [n] multipliers of the current column
  __shared__ double best[GJ_THREADS];
  __shared__ int bidx[GJ_THREADS];
  __shared__ double2 pinv;
  __shared__ int piv, bad;
  const int i = blockIdx.x;
  double2* a = A + (size_t)i * n * n;
  double2* r = R + (size_t)i * n * n;
  if (threadIdx.x == 0) bad = 0;
  for (int k = 0; k < n; ++k) {
    // pivot: largest |a(row, k)| for row >= k
    double bv = -1.0;
    int bi = k;
    for (int row = k + threadIdx.x; row < n; row += blockDim.x) {
      const double2 v = a[(size_t)row * n + k];
      const double m = v.x * v.x + v.y * v.y;
      if (m > bv) {
        bv = m;
        bi = row;
      }
    }
    best[threadIdx.x] = bv;
    bidx[threadIdx.x] = bi;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s && (best[threadIdx.x + s] > best[threadIdx.x] ||
                              (best[threadIdx.x + s] == best[threadIdx.x] && bidx[threadIdx.x + s] < bidx[threadIdx.x]))) {
        best[threadIdx.x] = best[threadIdx.x + s];
        bidx[threadIdx.x] = bidx[threadIdx.x + s];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      piv = bidx[0];
      const double2 p = a[(size_t)piv * n + k];
      const double m = p.x * p.x + p.y * p.y;
      if (!(m > 0.0)) {
        bad = 1;
        pinv = make_double2(0.0, 0.0);
      } else {
        pinv = make_double2(p.x / m, -p.y / m);
      }
    }
    __syncthreads();
    // swap rows k and piv
    if (piv != k) {
      for (int col = threadIdx.x; col < n; col += blockDim.x) {
        double2 t = a[(size_t)k * n + col];
        a[(size_t)k * n + col] = a[(size_t)piv * n + col];
        a[(size_t)piv * n + col] = t;
        t = r[(size_t)k * n + col];
        r[(size_t)k * n + col] = r[(size_t)piv * n + col];
        r[(size_t)piv * n + col] = t;
      }
    }
    __syncthreads();
    // scale the pivot row
    for (int col = threadIdx.x; col < n; col += blockDim.x) {
      if (col > k) a[(size_t)k * n + col] = cmul(a[(size_t)k * n + col], pinv);
      r[(size_t)k * n + col] = cmul(r[(size_t)k * n + col], pinv);
    }
    for (int row = threadIdx.x; row < n; row += blockDim.x) fcol[row] = a[(size_t)row * n + k];
    __syncthreads();
    if (threadIdx.x == 0) a[(size_t)k * n + k] = make_double2(1.0, 0.0);
    // eliminate column k from every other row
    const size_t cols_a = (size_t)(n - k - 1), total = (size_t)n * (cols_a + n);
    for (size_t e = threadIdx.x; e < total; e += blockDim.x) {
      const int row = (int)(e / (cols_a + n));
      if (row == k) continue;
      const size_t cc = e % (cols_a + n);
      const double2 f = fcol[row];
      if (cc < cols_a) {
        const int col = k + 1 + (int)cc;
        const double2 v = cmul(f, a[(size_t)k * n + col]);
        a[(size_t)row * n + col].x -= v.x;
        a[(size_t)row * n + col].y -= v.y;
      } else {
        const int col = (int)(cc - cols_a);
        const double2 v = cmul(f, r[(size_t)k * n + col]);
        r[(size_t)row * n + col].x -= v.x;
        r[(size_t)row * n + col].y -= v.y;
      }
    }
    __syncthreads();
    for (int row = threadIdx.x; row < n; row += blockDim.x)
      if (row != k) a[(size_t)row * n + k] = make_double2(0.0, 0.0);
    __syncthreads();
  }
  if (threadIdx.x == 0 && bad) err[i] = 1;
}

// Sigma~ difference and mixing: (sum |dS|^2, max |dS|) per block, dS = Sn - Sm; then Sm = lambda Sn + (1 - lambda) Sm
constexpr int MIX_BLOCKS = 1024;
__global__ void k_se_mix(const double2* __restrict__ Sn, double2* __restrict__ Sm, size_t total, double lambda,
                         double* __restrict__ part, int update) {
  double ss = 0.0, mx = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double dx = Sn[e].x - Sm[e].x, dy = Sn[e].y - Sm[e].y;
    const double m2 = dx * dx + dy * dy;
    ss += m2;
    mx = fmax(mx, m2);
    if (update)
      Sm[e] = make_double2(lambda * Sn[e].x + (1.0 - lambda) * Sm[e].x, lambda * Sn[e].y + (1.0 - lambda) * Sm[e].y);
  }
  __shared__ double s1[256], s2[256];
  s1[threadIdx.x] = ss;
  s2[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      s1[threadIdx.x] += s1[threadIdx.x + s];
      s2[threadIdx.x] = fmax(s2[threadIdx.x], s2[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s1[0];
    part[2 * blockIdx.x + 1] = s2[0];
  }
}

// Anderson acceleration of the loop (an option; the paper mixes linearly): with the
// residual f = Sigma~_new - Sigma~ of the current iterate and the last m differences
// dF_i, dX_i of residuals and iterates, gamma minimises |f - sum gamma_i dF_i|_2 and
//   Sigma~ <- Sigma~ + lambda f - sum_i gamma_i (dX_i + lambda dF_i).
constexpr int AA_MAX = DYSON_SELFENERGY_MAX_ANDERSON;
struct AaVecs {
  const double2* dF[AA_MAX];
  const double2* dX[AA_MAX];
  int m;
};

// f = Sn - Sm; dF_slot = f - f_prev, dX_slot = Sm - x_prev (when have_prev); then f_prev = f, x_prev = Sm
__global__ void k_aa_push(const double2* __restrict__ Sn, const double2* __restrict__ Sm, double2* __restrict__ f,
                          double2* __restrict__ fprev, double2* __restrict__ xprev, double2* __restrict__ dF,
                          double2* __restrict__ dX, int have_prev, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double2 fe = make_double2(Sn[e].x - Sm[e].x, Sn[e].y - Sm[e].y);
    const double2 xe = Sm[e];
    if (have_prev) {
      dF[e] = make_double2(fe.x - fprev[e].x, fe.y - fprev[e].y);
      dX[e] = make_double2(xe.x - xprev[e].x, xe.y - xprev[e].y);
    }
    f[e] = fe;
    fprev[e] = fe;
    xprev[e] = xe;
  }
}

// per block: the Gram entries <dF_i, dF_j> (i <= j) and <dF_i, f>, complex, in a fixed order
__global__ void k_aa_dots(const __grid_constant__ AaVecs v, const double2* __restrict__ f, size_t total,
                          double* __restrict__ part) {
  constexpr int NDOT = AA_MAX * (AA_MAX + 1) / 2 + AA_MAX;
  double re[NDOT], im[NDOT];
#pragma unroll
  for (int q = 0; q < NDOT; ++q) re[q] = im[q] = 0.0;
  const int m = v.m;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    double2 a[AA_MAX];
#pragma unroll
    for (int i = 0; i < AA_MAX; ++i) a[i] = i < m ? v.dF[i][e] : make_double2(0.0, 0.0);
    const double2 fe = f[e];
    int q = 0;
#pragma unroll
    for (int i = 0; i < AA_MAX; ++i) {
#pragma unroll
      for (int j = i; j < AA_MAX; ++j, ++q) {      // conj(a_i) a_j
        re[q] += a[i].x * a[j].x + a[i].y * a[j].y;
        im[q] += a[i].x * a[j].y - a[i].y * a[j].x;
      }
    }
#pragma unroll
    for (int i = 0; i < AA_MAX; ++i, ++q) {        // conj(a_i) f
      re[q] += a[i].x * fe.x + a[i].y * fe.y;
      im[q] += a[i].x * fe.y - a[i].y * fe.x;
    }
  }
  __shared__ double red[256];
  for (int q = 0; q < NDOT; ++q) {
    for (int c = 0; c < 2; ++c) {
      red[threadIdx.x] = c ? im[q] : re[q];
      __syncthreads();
      for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
      }
      if (threadIdx.x == 0) part[((size_t)blockIdx.x * NDOT + q) * 2 + c] = red[0];
      __syncthreads();
    }
  }
}

struct AaCoef {
  double2 g[AA_MAX];
  double lambda;
};

// Sm <- Sm + lambda f - sum_i g_i (dX_i + lambda dF_i)
__global__ void k_aa_update(const __grid_constant__ AaVecs v, const __grid_constant__ AaCoef cf,
                            const double2* __restrict__ f, double2* __restrict__ Sm, size_t total) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    double2 x = Sm[e];
    x.x += cf.lambda * f[e].x;
    x.y += cf.lambda * f[e].y;
    for (int i = 0; i < v.m; ++i) {
      const double2 d = make_double2(v.dX[i][e].x + cf.lambda * v.dF[i][e].x, v.dX[i][e].y + cf.lambda * v.dF[i][e].y);
      const double2 t = cmul(cf.g[i], d);
      x.x -= t.x;
      x.y -= t.y;
    }
    Sm[e] = x;
  }
}

// out[s][z][z'] = G[s][q Nc + z'][z] for the block column q of source s (chunk state layout [site][col][z])
__global__ void k_export_diagonal(const double2* __restrict__ G, const int* __restrict__ src_site, int Nc, int ncol,
                                  double2* __restrict__ out) {
  __shared__ double2 tile[32][33];
  const int q = blockIdx.z;
  const int s = src_site[q * Nc];
  const int z0 = blockIdx.y * 32, zp0 = blockIdx.x * 32;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int zp = zp0 + r, z = z0 + threadIdx.x;
    if (zp < Nc && z < Nc) tile[r][threadIdx.x] = G[((size_t)s * ncol + (size_t)q * Nc + zp) * Nc + z];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int z = z0 + r, zp = zp0 + threadIdx.x;
    if (z < Nc && zp < Nc) out[((size_t)s * Nc + z) * Nc + zp] = tile[threadIdx.x][r];
  }
}

// ---------------------------------------------------------------------------
// state
// ---------------------------------------------------------------------------
struct SeState {
  int Nr = 0, Nc = 0;
  double2 *g0 = nullptr, *Sm = nullptr, *FT = nullptr, *conn = nullptr, *w1 = nullptr, *w2 = nullptr,
          *St = nullptr, *tr = nullptr, *Q = nullptr;
  uint32_t* paths = nullptr;
  double* part = nullptr;
  int* err = nullptr;
  int* reps = nullptr;               // [Nr] orbit representatives, when the context has C4v set
  bool ready = false;                // g0 holds the atomic Lambda of the current build, Sm the mixed Sigma~
  int aa_depth = 0;                  // 0: linear mixing; 1..AA_MAX: Anderson depth
  int aa_count = 0;                  // iterates seen since the last reset
  double2* aa_f = nullptr;           // current residual
  double2* aa_fprev = nullptr;
  double2* aa_xprev = nullptr;
  double2* aa_dF[AA_MAX] = {};
  double2* aa_dX[AA_MAX] = {};
  double* aa_part = nullptr;         // per-block partial inner products
};

void free_aa(SeState* st) {
  void* ptrs[] = {st->aa_f, st->aa_fprev, st->aa_xprev, st->aa_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  st->aa_f = st->aa_fprev = st->aa_xprev = nullptr;
  st->aa_part = nullptr;
  for (int i = 0; i < AA_MAX; ++i) {
    if (st->aa_dF[i]) cudaFree(st->aa_dF[i]);
    if (st->aa_dX[i]) cudaFree(st->aa_dX[i]);
    st->aa_dF[i] = st->aa_dX[i] = nullptr;
  }
}

void free_state(SeState* st) {
  void* ptrs[] = {st->g0, st->Sm, st->FT, st->conn, st->w1, st->w2, st->St, st->tr, st->Q, st->paths, st->part,
                  st->err, st->reps};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  free_aa(st);
}

// complex Gaussian elimination with partial pivoting of the m x m system (row-major), in place;
// false when a pivot vanishes
bool small_solve(std::vector<double2>& A, std::vector<double2>& b, int m) {
  for (int k = 0; k < m; ++k) {
    int p = k;
    double best = -1.0;
    for (int r = k; r < m; ++r) {
      const double v = A[r * m + k].x * A[r * m + k].x + A[r * m + k].y * A[r * m + k].y;
      if (v > best) {
        best = v;
        p = r;
      }
    }
    if (!(best > 0.0)) return false;
    if (p != k) {
      for (int c = 0; c < m; ++c) std::swap(A[k * m + c], A[p * m + c]);
      std::swap(b[k], b[p]);
    }
    const double2 pv = A[k * m + k];
    const double2 inv = make_double2(pv.x / best, -pv.y / best);
    for (int r = k + 1; r < m; ++r) {
      const double2 a = A[r * m + k];
      const double2 f = make_double2(a.x * inv.x - a.y * inv.y, a.x * inv.y + a.y * inv.x);
      for (int c = k; c < m; ++c) {
        const double2 t = A[k * m + c];
        A[r * m + c].x -= f.x * t.x - f.y * t.y;
        A[r * m + c].y -= f.x * t.y + f.y * t.x;
      }
      b[r].x -= f.x * b[k].x - f.y * b[k].y;
      b[r].y -= f.x * b[k].y + f.y * b[k].x;
    }
  }
  for (int k = m - 1; k >= 0; --k) {
    double2 acc = b[k];
    for (int c = k + 1; c < m; ++c) {
      acc.x -= A[k * m + c].x * b[c].x - A[k * m + c].y * b[c].y;
      acc.y -= A[k * m + c].x * b[c].y + A[k * m + c].y * b[c].x;
    }
    const double2 pv = A[k * m + k];
    const double d = pv.x * pv.x + pv.y * pv.y;
    b[k] = make_double2((acc.x * pv.x + acc.y * pv.y) / d, (acc.y * pv.x - acc.x * pv.y) / d);
  }
  return true;
}

dim3 tiles32(int n, int Nr) { return dim3((n + 31) / 32, (n + 31) / 32, Nr); }

int gemm(dyson_ctx* c, const double2* A, const double2* B, double2* C) {
  k_zgemm<<<tiles32(c->Nc, c->Nr), dim3(32, 8), 0, c->stream>>>(A, B, C, c->Nc);
  c->launches += 1;
  DY_CUDA(c, cudaGetLastError());
  return DYSON_OK;
}

// R <- A^-1 R for every site (A destroyed)
int solve(dyson_ctx* c, SeState* st, double2* A, double2* R, const char* what) {
  DY_CUDA(c, cudaMemsetAsync(st->err, 0, (size_t)c->Nr * sizeof(int), c->stream));
  k_gauss_jordan<<<c->Nr, GJ_THREADS, (size_t)c->Nc * sizeof(double2), c->stream>>>(A, R, c->Nc, st->err);
  c->launches += 1;
  DY_CUDA(c, cudaGetLastError());
  std::vector<int> h(c->Nr);
  DY_CUDA(c, cudaMemcpyAsync(h.data(), st->err, (size_t)c->Nr * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->Nr; ++i)
    if (h[i]) return ctx_fail(c, DYSON_ERR_DIVERGED, std::string(what) + ": singular matrix at site " + std::to_string(i));
  return DYSON_OK;
}

SeState* state(dyson_ctx* c) { return static_cast<SeState*>(c->se); }

int ensure_state(dyson_ctx* c) {
  SeState* st = state(c);
  if (st && st->Nr == c->Nr && st->Nc == c->Nc) return DYSON_OK;
  if (st) {
    free_state(st);
    delete st;
    c->se = nullptr;
  }
  st = new SeState();
  st->Nr = c->Nr;
  st->Nc = c->Nc;
  const size_t blk = (size_t)c->Nr * c->Nc * c->Nc * sizeof(double2);
  bool ok = true;
  double2** bufs[] = {&st->g0, &st->Sm, &st->FT, &st->conn, &st->w1, &st->w2, &st->St};
  for (double2** b : bufs) ok = ok && cudaMalloc(b, blk) == cudaSuccess;
  ok = ok && cudaMalloc(&st->Q, (size_t)c->Nr * 2 * c->Nc * (2 * c->Nt + 1) * sizeof(double2)) == cudaSuccess &&
       cudaMalloc(&st->tr, (size_t)c->Nr * sizeof(double2)) == cudaSuccess &&
       cudaMalloc(&st->paths, 256 * PATHS * sizeof(uint32_t)) == cudaSuccess &&
       cudaMalloc(&st->part, 2 * MIX_BLOCKS * sizeof(double)) == cudaSuccess &&
       cudaMalloc(&st->err, (size_t)c->Nr * sizeof(int)) == cudaSuccess &&
       cudaMalloc(&st->reps, (size_t)c->Nr * sizeof(int)) == cudaSuccess;
  const std::vector<uint32_t> tab = path_table();
  ok = ok && cudaMemcpy(st->paths, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {                                             // nothing half-built stays behind
    cudaGetLastError();
    free_state(st);
    delete st;
    return ctx_fail(c, DYSON_ERR_OOM, "self-energy buffers (7 Nr Nc^2 complex128 and the prefix tables)");
  }
  c->se = st;
  return DYSON_OK;
}

// G0 = the atomic Lambda of the current build; the mixed Sigma~ starts at 0
int prepare(dyson_ctx* c) {
  SeState* st = state(c);
  if (st->ready) return DYSON_OK;
  const size_t blk = (size_t)c->Nr * c->Nc * c->Nc * sizeof(double2);
  DY_CUDA(c, cudaMemcpyAsync(st->g0, c->d_lam, blk, cudaMemcpyDeviceToDevice, c->stream));
  DY_CUDA(c, cudaMemsetAsync(st->Sm, 0, blk, c->stream));
  st->ready = true;
  st->aa_count = 0;
  return DYSON_OK;
}

// Anderson update of st->Sm from the new Sigma~ in st->St (buffers allocated on first use)
int anderson_update(dyson_ctx* c, SeState* st, double mix) {
  const size_t n_el = (size_t)c->Nr * c->Nc * c->Nc, blk = n_el * sizeof(double2);
  const int m = st->aa_depth;
  constexpr int NDOT = AA_MAX * (AA_MAX + 1) / 2 + AA_MAX;
  if (!st->aa_f) {
    bool ok = cudaMalloc(&st->aa_f, blk) == cudaSuccess && cudaMalloc(&st->aa_fprev, blk) == cudaSuccess &&
              cudaMalloc(&st->aa_xprev, blk) == cudaSuccess &&
              cudaMalloc(&st->aa_part, (size_t)MIX_BLOCKS * NDOT * 2 * sizeof(double)) == cudaSuccess;
    for (int i = 0; i < AA_MAX && ok; ++i)
      ok = cudaMalloc(&st->aa_dF[i], blk) == cudaSuccess && cudaMalloc(&st->aa_dX[i], blk) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_aa(st);
      return ctx_fail(c, DYSON_ERR_OOM, "Anderson history buffers");
    }
  }
  const int slot = (st->aa_count - 1 + AA_MAX) % AA_MAX;   // where the newest difference pair goes
  const unsigned eblocks = (unsigned)std::min<size_t>((n_el + 255) / 256, 8192);
  k_aa_push<<<eblocks, 256, 0, c->stream>>>(st->St, st->Sm, st->aa_f, st->aa_fprev, st->aa_xprev,
                                            st->aa_dF[slot], st->aa_dX[slot], st->aa_count > 0 ? 1 : 0, n_el);
  c->launches += 1;
  const int mk = std::min(st->aa_count, m);
  st->aa_count += 1;
  AaVecs v{};
  v.m = mk;
  for (int i = 0; i < mk; ++i) {                           // the mk newest pairs
    const int sl = (slot - i + AA_MAX) % AA_MAX;
    v.dF[i] = st->aa_dF[sl];
    v.dX[i] = st->aa_dX[sl];
  }
  AaCoef cf{};
  cf.lambda = mix;
  if (mk > 0) {
    k_aa_dots<<<MIX_BLOCKS, 256, 0, c->stream>>>(v, st->aa_f, n_el, st->aa_part);
    c->launches += 1;
    std::vector<double> part((size_t)MIX_BLOCKS * NDOT * 2);
    DY_CUDA(c, cudaMemcpyAsync(part.data(), st->aa_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                               c->stream));
    DY_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<double2> dots(NDOT, make_double2(0.0, 0.0));
    for (int bk = 0; bk < MIX_BLOCKS; ++bk)
      for (int q = 0; q < NDOT; ++q) {
        dots[q].x += part[((size_t)bk * NDOT + q) * 2];
        dots[q].y += part[((size_t)bk * NDOT + q) * 2 + 1];
      }
    // normal equations (dF^H dF + reg) gamma = dF^H f
    std::vector<double2> A((size_t)mk * mk), rhs(mk);
    double trace = 0.0;
    int q = 0;
    for (int i = 0; i < AA_MAX; ++i)
      for (int j = i; j < AA_MAX; ++j, ++q) {
        if (i >= mk || j >= mk) continue;
        A[i * mk + j] = dots[q];
        A[j * mk + i] = make_double2(dots[q].x, -dots[q].y);
        if (i == j) trace += dots[q].x;
      }
    for (int i = 0; i < AA_MAX; ++i, ++q)
      if (i < mk) rhs[i] = dots[q];
    for (int i = 0; i < mk; ++i) A[i * mk + i].x += 1e-12 * trace;
    if (small_solve(A, rhs, mk))
      for (int i = 0; i < mk; ++i) cf.g[i] = rhs[i];
    else
      v.m = 0;                                             // degenerate history: plain mixing this step
  }
  k_aa_update<<<eblocks, 256, 0, c->stream>>>(v, cf, st->aa_f, st->Sm, n_el);
  c->launches += 1;
  DY_CUDA(c, cudaGetLastError());
  return DYSON_OK;
}

}  // namespace

void se_invalidate(dyson_ctx* c) {
  if (c->se) state(c)->ready = false;
  c->se_installed = false;
}

void se_release(dyson_ctx* c) {
  if (!c->se) return;
  free_state(state(c));
  delete state(c);
  c->se = nullptr;
}

void launch_export_diagonal(const double2* G, const int* src_site, int Nc, int ncol, int nq, double2* out,
                            cudaStream_t s) {
  k_export_diagonal<<<dim3((Nc + 31) / 32, (Nc + 31) / 32, nq), dim3(32, 8), 0, s>>>(G, src_site, Nc, ncol, out);
}

extern "C" int dyson_selfenergy_set_anderson(dyson_ctx* c, int32_t depth) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (depth < 0 || depth > AA_MAX)
    return ctx_fail(c, DYSON_ERR_INVALID_ARG, "Anderson depth must be 0.." + std::to_string(AA_MAX));
  DeviceGuard g(c->device);
  int rc;
  if ((rc = ensure_state(c))) return rc;
  state(c)->aa_depth = depth;
  state(c)->aa_count = 0;
  return DYSON_OK;
}

extern "C" int dyson_selfenergy_step(dyson_ctx* c, const double* gloc, double mix, double* sigma_tilde,
                                     double* criterion) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (!gloc) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "gloc is NULL");
  if (!(mix > 0.0 && mix <= 1.0)) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "mix must lie in (0, 1]");
  if (!c->sigma_built) return ctx_fail(c, DYSON_ERR_STATE, "dyson_build_sigma has not run");
  if (c->sigma_transposed) return ctx_fail(c, DYSON_ERR_STATE, "Lambda is transposed");
  DeviceGuard g(c->device);
  int rc;
  if ((rc = ensure_state(c)) || (rc = prepare(c))) return rc;
  SeState* st = state(c);
  const int Nr = c->Nr, Nc = c->Nc;
  const size_t n_el = (size_t)Nr * Nc * Nc;
  const double2* G = reinterpret_cast<const double2*>(gloc);
  // F (transposed), the connected contraction, the disconnected terms
  k_se_hyb<<<tiles32(Nc, Nr), dim3(32, 8), 0, c->stream>>>(G, c->d_JW, c->d_nbr, c->d_nbond, Nc, st->FT);
  const int R = 2 * c->Nt;
  const size_t smem = (4 * (size_t)Nc + 2 * (R + 1) + 2 * (size_t)c->Nm) * sizeof(double2) +
                      256 * PATHS * sizeof(uint32_t);
  if (smem > 48 * 1024)
    DY_CUDA(c, cudaFuncSetAttribute(k_se_conn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  // with C4v the contraction runs for one site per orbit; a site s = g(r) has F_s = F_r and
  // K_s = K_r (its neighbours' G_loc and its levels are images of r's), so conn_s = conn_r
  std::vector<int> reps;
  if (c->symmetry == DYSON_SYMMETRY_C4V && (int)c->sym_rep.size() == Nr)
    for (int i = 0; i < Nr; ++i)
      if (c->sym_rep[i] == i) reps.push_back(i);
  const int n_conn = reps.empty() ? Nr : (int)reps.size();
  const int* d_sites = nullptr;
  if (!reps.empty()) {
    DY_CUDA(c, cudaMemcpyAsync(st->reps, reps.data(), reps.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    d_sites = st->reps;
  }
  {
    KernelTimer t(c, DYSON_KERNEL_SELFENERGY);
    k_se_prefix<<<dim3((unsigned)((2 * Nc + 127) / 128), n_conn), 128, 0, c->stream>>>(c->d_phase, st->FT, c->Nt,
                                                                                      c->Nm, d_sites, st->Q);
    k_se_conn<<<dim3((unsigned)((Nc * Nc + CONN_THREADS - 1) / CONN_THREADS), n_conn), CONN_THREADS, smem,
                c->stream>>>(st->paths, c->d_phase, st->FT, st->Q, c->Nt, c->Nm, d_sites, st->conn);
  }
  if (!reps.empty()) {
    const size_t blk = (size_t)Nc * Nc;
    for (int i = 0; i < Nr; ++i)
      if (c->sym_rep[i] != i)
        DY_CUDA(c, cudaMemcpyAsync(st->conn + (size_t)i * blk, st->conn + (size_t)c->sym_rep[i] * blk,
                                   blk * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  }
  k_se_trace<<<Nr, 256, 0, c->stream>>>(st->g0, st->FT, Nc, st->tr);
  c->launches += 4;
  DY_CUDA(c, cudaGetLastError());
  // D1 = G0 F G0 (F = FT^T), Sigma~ = -conn - D1 + 2 tr(G0 F) G0
  k_transpose<<<tiles32(Nc, Nr), dim3(32, 8), 0, c->stream>>>(st->FT, Nc, st->w2);
  c->launches += 1;
  if ((rc = gemm(c, st->g0, st->w2, st->w1)) || (rc = gemm(c, st->w1, st->g0, st->w2))) return rc;
  const unsigned eblocks = (unsigned)std::min<size_t>((n_el + 255) / 256, 8192);
  k_se_combine<<<eblocks, 256, 0, c->stream>>>(st->conn, st->w2, st->tr, st->g0, (size_t)Nc * Nc, n_el, st->St);
  c->launches += 1;
  DY_CUDA(c, cudaGetLastError());
  if (sigma_tilde)
    DY_CUDA(c, cudaMemcpyAsync(sigma_tilde, st->St, n_el * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  // measure and mixing on Sigma~ (linear, Eq. (Sigmamix), or Anderson)
  k_se_mix<<<MIX_BLOCKS, 256, 0, c->stream>>>(st->St, st->Sm, n_el, mix, st->part, st->aa_depth == 0 ? 1 : 0);
  c->launches += 1;
  DY_CUDA(c, cudaGetLastError());
  std::vector<double> part(2 * MIX_BLOCKS);
  DY_CUDA(c, cudaMemcpyAsync(part.data(), st->part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (st->aa_depth > 0 && (rc = anderson_update(c, st, mix))) return rc;
  // B = G0 (G0 - Sigma~ + u v^T / 2)^-1 G0 replaces Lambda
  k_se_complete<<<eblocks, 256, 0, c->stream>>>(st->g0, st->Sm, Nc, c->Nt, n_el, st->w1);
  c->launches += 1;
  DY_CUDA(c, cudaMemcpyAsync(st->conn, st->g0, n_el * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  if ((rc = solve(c, st, st->w1, st->conn, "local Dyson equation"))) return rc;
  if ((rc = gemm(c, st->g0, st->conn, st->w2))) return rc;
  DY_CUDA(c, cudaMemcpyAsync(c->d_lam, st->w2, n_el * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  c->lam32_built = c->lam_split_built = false;
  oz_invalidate(c);
  c->se_installed = true;
  double ss = 0.0, mx = 0.0;
  for (int b = 0; b < MIX_BLOCKS; ++b) {
    ss += part[2 * b];
    mx = std::max(mx, part[2 * b + 1]);
  }
  if (criterion) *criterion = std::sqrt(ss) / (double)n_el + std::sqrt(mx);
  flush_timers(c);
  return DYSON_OK;
}
