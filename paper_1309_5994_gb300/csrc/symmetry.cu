// C4v irreducible-wedge solves (App. A).
//
// On an L x L lattice whose trap is centred and whose drive tables are
// invariant under the eight operations g of C4v (reflections in the two axes
// and the two diagonals, and their products), G_{g(a), g(b)} = G_{a, b}.  A
// block column of source s = g(r) is therefore the block column of r with its
// sites permuted, G_{j, s} = G_{g^-1(j), r}, and the observables of site s equal
// those of r.  Only one source per orbit (its representative, the orbit's
// smallest site index) is solved; the others are filled by copies.
#include <algorithm>
#include <map>
#include <vector>

#include "common.cuh"
#include "detail.cuh"
#include "symmetry.cuh"

using namespace dyson_detail;

namespace {

// (x, y) -> g(x, y) for the eight operations on an L x L lattice
void apply_op(int g, int L, int x, int y, int* ox, int* oy) {
  const int X = L - 1 - x, Y = L - 1 - y;
  switch (g) {
    case 0: *ox = x; *oy = y; break;
    case 1: *ox = X; *oy = y; break;
    case 2: *ox = x; *oy = Y; break;
    case 3: *ox = y; *oy = x; break;
    case 4: *ox = Y; *oy = X; break;
    case 5: *ox = X; *oy = Y; break;
    case 6: *ox = y; *oy = X; break;
    default: *ox = Y; *oy = x; break;
  }
}

// dst block of site j <- src block of site perm[j], blk elements per site
__global__ void k_permute_sites(const double2* __restrict__ src, double2* __restrict__ dst,
                                const int* __restrict__ perm, size_t blk) {
  const int j = blockIdx.y;
  const double2* s = src + (size_t)perm[j] * blk;
  double2* d = dst + (size_t)j * blk;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < blk; e += (size_t)gridDim.x * blockDim.x)
    d[e] = s[e];
}

}  // namespace

extern "C" int dyson_set_symmetry(dyson_ctx* c, int mode) {
  if (!c) return fail_noctx(DYSON_ERR_INVALID_ARG, "NULL context");
  if (mode == DYSON_SYMMETRY_NONE) {
    c->symmetry = mode;
    return DYSON_OK;
  }
  if (mode != DYSON_SYMMETRY_C4V) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "unknown symmetry");
  if (c->Lx != c->Ly) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "C4v needs a square lattice");
  const int L = c->Lx, Nr = c->Nr, Nt = c->Nt;
  std::vector<int> fwd(8 * (size_t)Nr);
  for (int g = 0; g < 8; ++g)
    for (int i = 0; i < Nr; ++i) {
      int ox, oy;
      apply_op(g, L, i % L, i / L, &ox, &oy);
      fwd[(size_t)g * Nr + i] = oy * L + ox;
    }
  // the drive must be invariant: U on sites, J on bonds
  std::map<std::pair<int, int>, int> bond_of;
  for (int i = 0; i < Nr; ++i)
    for (int q = 0; q < 4; ++q) {
      const int j = c->h_nbr[i * 4 + q];
      if (j >= 0) bond_of[{std::min(i, j), std::max(i, j)}] = c->h_nbond[i * 4 + q];
    }
  for (int g = 1; g < 8; ++g) {
    for (int i = 0; i < Nr; ++i) {
      const int gi = fwd[(size_t)g * Nr + i];
      for (int t = 0; t < Nt; ++t)
        if (c->U[(size_t)gi * Nt + t] != c->U[(size_t)i * Nt + t])
          return ctx_fail(c, DYSON_ERR_INVALID_ARG, "U is not C4v-invariant");
    }
    for (const auto& kv : bond_of) {
      const int a = fwd[(size_t)g * Nr + kv.first.first], b = fwd[(size_t)g * Nr + kv.first.second];
      const auto it = bond_of.find({std::min(a, b), std::max(a, b)});
      if (it == bond_of.end()) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "lattice bonds are not C4v-invariant");
      for (int t = 0; t < Nt; ++t)
        if (c->J[(size_t)it->second * Nt + t] != c->J[(size_t)kv.second * Nt + t])
          return ctx_fail(c, DYSON_ERR_INVALID_ARG, "J is not C4v-invariant");
    }
  }
  // representatives and, per site, an operation taking its representative to it
  c->sym_rep.assign(Nr, 0);
  c->sym_op.assign(Nr, 0);
  for (int i = 0; i < Nr; ++i) {
    int r = i;
    for (int g = 0; g < 8; ++g) r = std::min(r, fwd[(size_t)g * Nr + i]);
    c->sym_rep[i] = r;
    for (int g = 0; g < 8; ++g)
      if (fwd[(size_t)g * Nr + r] == i) {
        c->sym_op[i] = g;
        break;
      }
  }
  std::vector<int> inv(8 * (size_t)Nr);
  for (int g = 0; g < 8; ++g)
    for (int i = 0; i < Nr; ++i) inv[(size_t)g * Nr + fwd[(size_t)g * Nr + i]] = i;
  DeviceGuard dg(c->device);
  if (!c->d_sym_perm) DY_CUDA(c, cudaMalloc(&c->d_sym_perm, 8 * (size_t)Nr * sizeof(int)));
  DY_CUDA(c, cudaMemcpy(c->d_sym_perm, inv.data(), inv.size() * sizeof(int), cudaMemcpyHostToDevice));
  c->symmetry = mode;
  return DYSON_OK;
}

namespace {

// one representative per requested orbit, in order of first appearance; slot[r] = its position
int orbit_representatives(dyson_ctx* c, const int32_t* src, int64_t n_src, std::vector<int32_t>* reps,
                          std::vector<int>* slot) {
  if (n_src < 1 || !src) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "need at least one source site");
  for (int64_t q = 0; q < n_src; ++q)
    if (src[q] < 0 || src[q] >= c->Nr) return ctx_fail(c, DYSON_ERR_INVALID_ARG, "source site out of range");
  slot->assign(c->Nr, -1);
  reps->clear();
  for (int64_t q = 0; q < n_src; ++q) {
    const int r = c->sym_rep[src[q]];
    if ((*slot)[r] < 0) {
      (*slot)[r] = (int)reps->size();
      reps->push_back(r);
    }
  }
  return DYSON_OK;
}

// observables of each requested site s are those of its representative
void copy_observables(dyson_ctx* c, const int32_t* src, int64_t n_src) {
  const size_t NrNt = (size_t)c->Nr * c->Nt;
  for (int64_t q = 0; q < n_src; ++q) {
    const int s = src[q], r = c->sym_rep[s];
    if (s != r)
      for (int k = 0; k < 3; ++k)
        cudaMemcpyAsync(c->d_obs + k * NrNt + (size_t)s * c->Nt, c->d_obs + k * NrNt + (size_t)r * c->Nt,
                        c->Nt * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
  }
}

}  // namespace

int solve_columns_c4v(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                      int32_t max_sweeps, double* g_out, dyson_report* rep_out) {
  std::vector<int32_t> reps;
  std::vector<int> slot;
  int rc0 = orbit_representatives(c, src, n_src, &reps, &slot);
  if (rc0) return rc0;
  DeviceGuard dg(c->device);
  const size_t blk = (size_t)c->Nc * c->Nc;                  // one site's Nc x Nc block
  const size_t col = (size_t)c->Nr * blk;                    // one block column
  double2* tmp = nullptr;
  if (g_out) {
    cudaError_t e = cudaMalloc(&tmp, reps.size() * col * sizeof(double2));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return ctx_fail(c, DYSON_ERR_OOM, "C4v: block columns of the representatives");
    }
  }
  c->symmetry = DYSON_SYMMETRY_NONE;
  int rc = dyson_solve_columns(c, reps.data(), (int64_t)reps.size(), precision, tol, max_sweeps,
                               reinterpret_cast<double*>(tmp), rep_out);
  c->symmetry = DYSON_SYMMETRY_C4V;
  if (rc == DYSON_OK || rc == DYSON_ERR_NOT_CONVERGED || rc == DYSON_ERR_DIVERGED) {
    copy_observables(c, src, n_src);
    for (int64_t q = 0; q < n_src; ++q) {
      const int s = src[q], r = c->sym_rep[s];
      if (g_out) {                                           // G_{j,s} = G_{g^-1(j), r}
        const int g = c->sym_op[s];
        k_permute_sites<<<dim3((unsigned)std::min<size_t>((blk + 255) / 256, 64), c->Nr), 256, 0, c->stream>>>(
            tmp + (size_t)slot[r] * col, reinterpret_cast<double2*>(g_out) + (size_t)q * col,
            c->d_sym_perm + (size_t)g * c->Nr, blk);
        c->launches += 1;
      }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = ctx_fail(c, DYSON_ERR_CUDA, std::string("C4v fill: ") + cudaGetErrorString(e));
  }
  if (tmp) cudaFree(tmp);
  return rc;
}

int local_greens_c4v(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                     int32_t max_sweeps, double* gloc, dyson_report* rep_out) {
  std::vector<int32_t> reps;
  std::vector<int> slot;
  int rc = orbit_representatives(c, src, n_src, &reps, &slot);
  if (rc) return rc;
  DeviceGuard dg(c->device);
  c->symmetry = DYSON_SYMMETRY_NONE;
  rc = dyson_local_greens(c, reps.data(), (int64_t)reps.size(), precision, tol, max_sweeps, gloc, rep_out);
  c->symmetry = DYSON_SYMMETRY_C4V;
  if (rc == DYSON_OK || rc == DYSON_ERR_NOT_CONVERGED || rc == DYSON_ERR_DIVERGED) {
    copy_observables(c, src, n_src);
    const size_t blk = (size_t)c->Nc * c->Nc;
    double2* G = reinterpret_cast<double2*>(gloc);
    for (int64_t q = 0; q < n_src; ++q) {
      const int s = src[q], r = c->sym_rep[s];
      if (s != r)
        cudaMemcpyAsync(G + (size_t)s * blk, G + (size_t)r * blk, blk * sizeof(double2), cudaMemcpyDeviceToDevice,
                        c->stream);
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) rc = ctx_fail(c, DYSON_ERR_CUDA, std::string("C4v fill: ") + cudaGetErrorString(e));
  }
  return rc;
}
