// Allocation-free FP64 series solve of one block column.
//
// Some callers cannot allocate device memory while they run: code that executes
// inside a host process whose device heap is owned and pre-reserved by another
// framework (a memory pool that must not fragment, or one that is already full),
// real-time or embedded loops where cudaMalloc's latency and implicit
// synchronisation are not acceptable, and tools that may only call into a
// library without ever changing its memory footprint.  For them this file keeps
// all scratch memory of the solve in one file-scope device array of fixed size:
// it is reserved when the library is loaded on a GPU and stays reserved until the
// process exits.  The caller passes every input and output buffer.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace {

// scratch: the second state buffer of the ping-pong series plus two norm words.
// With CUDA's lazy module loading the array is committed on a device when this
// file's module is first loaded there: by dyson_init on that device, or by the
// first dyson_solve_block_column_noalloc call, whichever comes first.
constexpr size_t kStateBytes = (size_t)DYSON_NOALLOC_MAX_STATE_BYTES;
constexpr size_t kWordsBytes = 256;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStateBytes + kWordsBytes];

// device address of g_noalloc_scratch per device (the host symbol is only a stand-in)
std::mutex g_setup_mu;
void* g_scratch_dev[128] = {};

thread_local std::string g_noalloc_err;

int fail(int code, const std::string& m) {
  g_noalloc_err = m;
  return code;
}

__device__ __forceinline__ unsigned long long nonneg(double v) {
  if (!(v >= 0.0)) v = __longlong_as_double(0x7ff0000000000000ULL);
  return (unsigned long long)__double_as_longlong(v);
}

// G[j][z][z'] = Lambda_s[z][z'] if j == s else 0; words[1] = max |Lambda_s|
__global__ void k_na_init(const double2* __restrict__ lam, int Nr, int Nc, int s, double2* __restrict__ G,
                          unsigned long long* __restrict__ words) {
  size_t total = (size_t)Nr * Nc * Nc, blk = (size_t)Nc * Nc;
  double m = 0.0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    size_t j = e / blk;
    double2 v = make_double2(0.0, 0.0);
    if ((int)j == s) {
      v = lam[(size_t)s * blk + (e - j * blk)];
      m = fmax(m, sqrt(v.x * v.x + v.y * v.y));
    }
    G[e] = v;
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(words + 1, nonneg(m));
}

// one series sweep in the row-major block-column layout G[j][z][z']:
// out_i[z][z'] = B_i + sum_zb Lambda_i[z][zb] W(zb) sum_{j in NN(i)} J_ij(zb) in_j[zb][z'];
// words[0] = max |out - in|.  Tile 32 x 32 outputs, 256 threads, 2 x 2 per thread.
__global__ __launch_bounds__(256) void k_na_sweep(const double2* __restrict__ lam, const double* __restrict__ J,
                                                  int Lx, int Ly, int Nt, int Nm, double dt, double beta, int s,
                                                  const double2* __restrict__ gin, double2* __restrict__ gout,
                                                  unsigned long long* __restrict__ words) {
  constexpr int T = 32, KT = 16;
  __shared__ double2 As[T][KT + 1];
  __shared__ double2 Xs[KT][T + 1];
  const int Nc = 2 * Nt + Nm, i = blockIdx.z;
  const int z0 = blockIdx.y * T, c0 = blockIdx.x * T;
  const int tid = threadIdx.x, tc = tid & 15, tr = tid >> 4;
  const int x = i % Lx, y = i / Lx, hb = Ly * (Lx - 1);
  int nb[4], bd[4];
  nb[0] = x + 1 < Lx ? i + 1 : -1;   bd[0] = y * (Lx - 1) + x;
  nb[1] = x > 0 ? i - 1 : -1;        bd[1] = y * (Lx - 1) + x - 1;
  nb[2] = y + 1 < Ly ? i + Lx : -1;  bd[2] = hb + y * Lx + x;
  nb[3] = y > 0 ? i - Lx : -1;       bd[3] = hb + (y - 1) * Lx + x;
  const size_t blk = (size_t)Nc * Nc;
  const double2* L = lam + (size_t)i * blk;
  double2 acc[2][2] = {};
  for (int k0 = 0; k0 < Nc; k0 += KT) {
    for (int e = tid; e < T * KT; e += 256) {
      int r = e / KT, k = e % KT;
      int z = z0 + r, kk = k0 + k;
      As[r][k] = (z < Nc && kk < Nc) ? L[(size_t)z * Nc + kk] : make_double2(0.0, 0.0);
    }
    for (int e = tid; e < KT * T; e += 256) {
      int k = e / T, c = e % T;
      int kk = k0 + k, cc = c0 + c;
      double2 v = make_double2(0.0, 0.0);
      if (kk < Nc && cc < Nc) {
        double jr = 0.0, ji = 0.0;
        int tk = contour_time_index(kk, Nt);
        for (int q = 0; q < 4; ++q) {
          if (nb[q] < 0) continue;
          double Jv = J[(size_t)bd[q] * Nt + tk];
          double2 g = gin[(size_t)nb[q] * blk + (size_t)kk * Nc + cc];
          jr += Jv * g.x;
          ji += Jv * g.y;
        }
        v = cmul(contour_weight(kk, Nt, Nm, dt, beta), make_double2(jr, ji));
      }
      Xs[k][c] = v;
    }
    __syncthreads();
    for (int k = 0; k < KT; ++k) {
      for (int a = 0; a < 2; ++a) {
        double2 av = As[tr + 16 * a][k];
        for (int b = 0; b < 2; ++b) {
          double2 xv = Xs[k][tc + 16 * b];
          acc[a][b].x = fma(av.x, xv.x, fma(-av.y, xv.y, acc[a][b].x));
          acc[a][b].y = fma(av.x, xv.y, fma(av.y, xv.x, acc[a][b].y));
        }
      }
    }
    __syncthreads();
  }
  double m = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      int z = z0 + tr + 16 * a, c = c0 + tc + 16 * b;
      if (z >= Nc || c >= Nc) continue;
      double2 v = acc[a][b];
      if (i == s) {
        double2 bb = L[(size_t)z * Nc + c];
        v.x += bb.x;
        v.y += bb.y;
      }
      size_t off = (size_t)i * blk + (size_t)z * Nc + c;
      double2 g = gin[off];
      gout[off] = v;
      double dx = v.x - g.x, dy = v.y - g.y;
      m = fmax(m, sqrt(dx * dx + dy * dy));
    }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((tid & 31) == 0) atomicMax(words, nonneg(m));
}

// set-up once per device, with that device current: the device address of the scratch array
int scratch_address(int device, void** out) {
  if (device < 0 || device >= 128) return fail(DYSON_ERR_INVALID_ARG, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_dev[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(DYSON_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    }
    g_scratch_dev[device] = p;
  }
  *out = g_scratch_dev[device];
  return DYSON_OK;
}

double bits_to_d(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof d);
  return d;
}

}  // namespace

// dyson_init's set-up for `device` (current): loads this module and looks up the
// scratch address, so that the array is committed when a context is created
int noalloc_reserve_scratch(int device) {
  void* p = nullptr;
  return scratch_address(device, &p);
}

extern "C" const char* dyson_noalloc_last_error(void) { return g_noalloc_err.c_str(); }

extern "C" int dyson_solve_block_column_noalloc(const double* lambda, const double* J, int32_t Lx, int32_t Ly,
                                                int32_t Nt, int32_t Nm, double dt, double beta, int32_t source,
                                                double tol, int32_t max_sweeps, double* g_out, int32_t* sweeps_out,
                                                void* cuda_stream) {
  if (!lambda || !g_out) return fail(DYSON_ERR_INVALID_ARG, "lambda and g_out must be device pointers");
  if (Lx < 1 || Ly < 1 || (int64_t)Lx * Ly > 65535) return fail(DYSON_ERR_INVALID_ARG, "lattice must have 1..65535 sites");
  if (Nt < 1 || Nm < 1 || 2 * (int64_t)Nt + Nm > 2048) return fail(DYSON_ERR_INVALID_ARG, "need Nt, Nm >= 1, 2Nt+Nm <= 2048");
  const int Nr = Lx * Ly, Nc = 2 * Nt + Nm;
  const size_t bytes = (size_t)Nr * Nc * Nc * sizeof(double2);
  if (bytes > kStateBytes)
    return fail(DYSON_ERR_INVALID_ARG, "block column of " + std::to_string(bytes) + " bytes exceeds the " +
                                           std::to_string(kStateBytes) + "-byte static scratch (Nr*Nc*Nc*16 bytes)");
  if (Nr > 1 && !J) return fail(DYSON_ERR_INVALID_ARG, "J must be a device pointer");
  if (source < 0 || source >= Nr) return fail(DYSON_ERR_INVALID_ARG, "source site out of range");
  if (!(tol > 0) || max_sweeps < 1) return fail(DYSON_ERR_INVALID_ARG, "need tol > 0 and max_sweeps >= 1");
  if (!(dt > 0) || !(beta > 0)) return fail(DYSON_ERR_INVALID_ARG, "dt and beta must be positive");
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return fail(DYSON_ERR_CUDA, "no current CUDA device");
  void* scratch = nullptr;
  int rc = scratch_address(device, &scratch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double2* other = static_cast<double2*>(scratch);
  unsigned long long* words = reinterpret_cast<unsigned long long*>(static_cast<unsigned char*>(scratch) + kStateBytes);
  double2* cur = reinterpret_cast<double2*>(g_out);
  const double2* lam = reinterpret_cast<const double2*>(lambda);
#define NA_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(DYSON_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  NA_CUDA(cudaMemsetAsync(words, 0, 2 * sizeof(unsigned long long), st));
  k_na_init<<<152 * 4, 256, 0, st>>>(lam, Nr, Nc, source, cur, words);
  NA_CUDA(cudaGetLastError());
  unsigned long long h[2] = {0, 0};
  NA_CUDA(cudaMemcpyAsync(h, words, sizeof h, cudaMemcpyDeviceToHost, st));
  NA_CUDA(cudaStreamSynchronize(st));
  const double scale = std::max(bits_to_d(h[1]), 1e-300);
  dim3 grid((Nc + 31) / 32, (Nc + 31) / 32, Nr);
  int status = DYSON_ERR_NOT_CONVERGED, sweeps = 0;
  for (int sw = 1; sw <= max_sweeps; ++sw) {
    NA_CUDA(cudaMemsetAsync(words, 0, sizeof(unsigned long long), st));
    k_na_sweep<<<grid, 256, 0, st>>>(lam, J, Lx, Ly, Nt, Nm, dt, beta, source, cur, other, words);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemcpyAsync(h, words, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    NA_CUDA(cudaStreamSynchronize(st));
    std::swap(cur, other);
    sweeps = sw;
    double upd = bits_to_d(h[0]) / scale;
    if (!(upd < 4503599627370496.0)) {        // 2^52: partial-sum rounding exceeds the result
      status = DYSON_ERR_DIVERGED;
      break;
    }
    if (upd <= tol) {
      status = DYSON_OK;
      break;
    }
  }
  if (cur != reinterpret_cast<double2*>(g_out))
    NA_CUDA(cudaMemcpyAsync(g_out, cur, bytes, cudaMemcpyDeviceToDevice, st));
  NA_CUDA(cudaStreamSynchronize(st));
#undef NA_CUDA
  if (sweeps_out) *sweeps_out = sweeps;
  if (status == DYSON_ERR_NOT_CONVERGED) fail(status, "max_sweeps reached above tolerance");
  if (status == DYSON_ERR_DIVERGED) fail(status, "series diverged");
  return status;
}
