// FP64-accurate Dyson residual on the BF16 tensor cores:
//     r = B + (Lambda W) X - G,   X_i(n, k) = sum_{j in NN(i)} J_ij(k) G_j(n, k),
// the residual of the series of App. C that refines the FP32 sweeps.
//
// The real GEMM A X (A = [[Re,-Im],[Im,Re]] of Lambda W, per site 2Nc x 2Nc) is
// evaluated exactly enough in FP32 tensor-core arithmetic by splitting both
// operands into integer slices (the Ozaki scheme): every row of A and every
// column of X is scaled by a power of two into [-1, 1] and cut into S = 7 slices
// of 7 bits, v = sum_s q_s 2^{-7 s} with integers |q_s| <= 128.  A slice product
// sum_k A_s X_t is then an integer multiple of 2^{-7(s+t)} below 2^24 in
// magnitude for every diagonal s + t <= 5 when K = 2Nc <= 512, so BF16 inputs
// with FP32 accumulation are exact there.
// The 28 products with s + t <= 8 (truncation ~2^-50 of |A||X|) accumulate per
// diagonal in five TMEM accumulators, {2}, {3}, {4}, {5} exact and {6, 7, 8}
// rounded at 2^-24 of its own size (about 2^-48 of the result).  The epilogue
// adds them in FP64, rescales, and forms r = B + A X - G in FP64.  Solves whose
// tolerance is 1e-8 or looser use the first five slices of each operand and the
// 15 products with s + t <= 6 (X is split into five digits rounded at 2^-35 of its
// column scale, the Lambda slices are the first five of seven; truncation ~2^-35 of
// |A||X|, two orders below such a tolerance).
//
// Kernels: k_oz_aprep (once per Lambda), k_oz_xprep, or k_oz_xprep_sum where every
// bond carries the same J(t) (gather + scale + slice of X per residual), k_oz_gemm
// (persistent: TMA + tcgen05.mma kind::f16 into two
// accumulator sets + FP64 epilogue of the previous tile).  With five slices the
// accumulators of diagonals 2..6 are consecutive 48-column blocks and so are the X
// slices in a stage: A_s X_t for t = 1..6-s is one MMA (N = (6 - s) 48) into the
// blocks of diagonals s+1..6, five MMAs per k step for the fifteen products.
#include <algorithm>

#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"
#include "oz.cuh"
#include "ptx.cuh"

namespace {

constexpr int S = 7;                                      // slices stored
constexpr int S_SHORT = 5;                                 // slices used for tolerances >= 1e-8
constexpr double SHORT_TOL = 1e-8;
constexpr int BM = 128, BN = 48, BK = 32;                 // BK bf16 = 64-byte rows (64-byte swizzle)
constexpr int A_TILE = BM * BK * 2;                       // 8 KB per A slice tile
constexpr int X_TILE = BN * BK * 2;                       // 3 KB per X slice tile
// pipeline of one slice count: a stage holds SE A slices and SE X slices (55 KB for
// five, 77 KB for seven); as many stages as fit, at most four
template <int SE>
struct OzPipe {
  static constexpr int STAGE_BYTES = SE * (A_TILE + X_TILE);
  static constexpr int FIT = (227 * 1024 - 1024) / STAGE_BYTES;
  static constexpr int STAGES = FIT > 4 ? 4 : FIT;
  static constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
};
constexpr int THREADS = 384;                               // warps 4-11: epilogue, two per TMEM lane quarter
constexpr int EPI_CHUNK = 8;                               // accumulator columns per tcgen05.ld
constexpr int NACC = 5;                                    // diagonals {2}, {3}, {4}, {5}, {6, 7, 8}
constexpr uint32_t ACC_COLS = NACC * BN;                   // one tile's accumulators: 240 columns
constexpr uint32_t TMEM_COLS = 512;                        // two tiles' accumulators (double-buffered)

// kind::f16, D = F32, A = B = BF16, K-major, M = 128, N = 48
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

struct OzState {
  CUtensorMap amap, xmap;
  __nv_bfloat16* aslices = nullptr;   // [S][Nr][2Nc][2Nc]
  double* sigma = nullptr;            // [Nr][2Nc] row scales of A
  size_t a_bytes = 0;
  bool a_ready = false;
  __nv_bfloat16* xslices = nullptr;   // [S][Nr][ncol][2Nc]
  double* tau = nullptr;              // [Nr][ncol] column scales of X
  size_t x_bytes = 0, tau_bytes = 0;
  const void* xmap_ptr = nullptr;
  int xmap_ncol = -1;
  int* d_err = nullptr;
  int* h_err = nullptr;               // pinned mirror of d_err
  int num_sms = 1;
  bool smem_set = false;
};

__device__ __forceinline__ int time_of(int z, int Nt) { return contour_time_index(z, Nt); }
__device__ __forceinline__ double2 weight_of(int z, int Nt, int Nm, double dt, double beta) {
  return contour_weight(z, Nt, Nm, dt, beta);
}

// power of two >= max |v| (1 for an all-zero vector)
__device__ __forceinline__ double pow2_scale(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);           // mx = f 2^e, f in [0.5, 1)
  return ldexp(1.0, e);
}

constexpr int FIX = 7 * S;                                 // fixed-point bits of a scaled value

// the S slices of x (|x| <= sc, fix_over_sc = 2^FIX / sc): the fixed-point integer from one
// FP64 multiply and one conversion (the Lambda slices, built once)
__device__ __forceinline__ long long lambda_fixed(double x, double fix_over_sc) { return __double2ll_rn(x * fix_over_sc); }

// rint(x 2^k) where the scaling only shifts right (E - 1075 + k <= 0, i.e. |x 2^k| < 2^52):
// the mantissa shifted right by r with the half unit added first (ties away from zero).
// Every caller's column scale is at least the column's largest value, so this holds there.
__device__ __forceinline__ long long fixed_right(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int r = min(1075 - k - E, 63);                     // >= 0 by the condition above
  const long long v = E == 0 ? 0 : (long long)((M + ((1ull << r) >> 1)) >> r);
  return (b >> 63) ? -v : v;
}

// The first NS signed 7-bit digits of V (|V| <= 2^FIX) in one pass: for A = |V| plus 64 in
// every digit position below the top (and half a unit of the last kept digit when NS < S),
// digit s of A in base 128, less 64, is the balanced digit q_s in [-64, 63]; the top digit
// is A >> 7 (S - 1) <= 128.  Then sum_s q_s 2^{7 (S - s)} = |V| rounded to the last kept
// digit, and the digits of V are those of |V| with its sign.  Slice s holds q_s 2^{-7 s}.
template <int NS>
__device__ __forceinline__ void write_digits_fast(long long V, __nv_bfloat16* dst, size_t slice_stride) {
  static_assert(NS >= 1 && NS <= S, "digits kept");
  constexpr unsigned long long BIAS = [] {
    unsigned long long b = NS < S ? 1ull << (7 * (S - NS) - 1) : 0ull;
    for (int s = 2; s <= NS; ++s) b += 64ull << (7 * (S - s));
    return b;
  }();
  const bool neg = V < 0;
  const unsigned long long A = (unsigned long long)(neg ? -V : V) + BIAS;
#pragma unroll
  for (int s = 1; s <= NS; ++s) {
    const int sh = 7 * (S - s);
    const int q = s == 1 ? (int)(A >> sh) : (int)((A >> sh) & 127u) - 64;
    const float unit = __int_as_float((127 - 7 * s) << 23);                    // 2^{-7 s}
    dst[(size_t)(s - 1) * slice_stride] = __float2bfloat16_rn(__int2float_rn(neg ? -q : q) * unit);
  }
}

// Accumulator A of the slice products holds, for A < NACC - 1, sum q_s q_t 2^{-7 d} over
// the diagonal d = A + 2 exactly: an integer N below 2^24 in units of 2^{-7 d}, moved to
// the 2^-FIX fixed point by one exact scaling, an exact int32 conversion and a shift.
// The last accumulator (diagonals >= NACC + 1, rounded in FP32) is scaled by 2^FIX and
// rounded to the nearest integer; its magnitude stays below 2^-18 for K <= 512 (diagonal
// 6 sums at most 7 2^12 K 2^-42), so the integer fits in 32 bits, the conversion needs
// no 64-bit (FP64-pipe) instruction, and nothing but the part below 2^-FIX is lost.
template <int A>
__device__ __forceinline__ long long acc_to_fixed(float v) {
  if constexpr (A < NACC - 1) {
    constexpr int d = A + 2;
    const int N = __float2int_rn(v * __int_as_float((127 + 7 * d) << 23));   // v * 2^{7 d}, exact
    return (long long)N << (FIX - 7 * d);
  } else {
    return (long long)__float2int_rn(v * __int_as_float((127 + FIX) << 23));   // v * 2^FIX: |.| < 2^31
  }
}

__device__ __forceinline__ double emb_value(const double2* lrow, int k, int part, int Nc, int Nt, int Nm, double dt,
                                            double beta) {
  int kb = k < Nc ? k : k - Nc, kpart = k < Nc ? 0 : 1;
  double2 v = cmul(lrow[kb], weight_of(kb, Nt, Nm, dt, beta));
  return part == kpart ? v.x : (part == 0 ? -v.y : v.y);
}

// one warp per row (site i, row m) of the embedding of Lambda W; with Jrow set (hopping equal
// on every bond), column k also carries the factor J(t(k)) that the gather would apply to
// row k of X, so that X becomes the plain sum of the neighbours' columns
__global__ void k_oz_aprep(const double2* __restrict__ lam, const double* __restrict__ Jrow, int Nr, int Nt, int Nm,
                           double dt, double beta, __nv_bfloat16* __restrict__ as, double* __restrict__ sigma) {
  const int Nc = 2 * Nt + Nm, N2 = 2 * Nc;
  const size_t row = (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= (size_t)Nr * N2) return;
  const int i = (int)(row / N2), m = (int)(row % N2);
  const int z = m % Nc, part = m / Nc;
  const double2* lrow = lam + ((size_t)i * Nc + z) * Nc;
  auto value = [&](int k) {
    const double v = emb_value(lrow, k, part, Nc, Nt, Nm, dt, beta);
    return Jrow ? v * Jrow[time_of(k < Nc ? k : k - Nc, Nt)] : v;
  };
  double mx = 0.0;
  for (int k = lane; k < N2; k += 32) mx = fmax(mx, fabs(value(k)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const double sc = pow2_scale(mx);
  if (lane == 0) sigma[row] = sc;
  const double fix_over_sc = ldexp(1.0, FIX) / sc;
  const size_t stride = (size_t)Nr * N2 * N2;
  for (int k = lane; k < N2; k += 32) write_digits_fast<S>(lambda_fixed(value(k), fix_over_sc), as + row * N2 + k, stride);
}

// one warp per (site i, vector column n): X = sum_j J_ij G_j (FP64), column scale, slices.
// Warps walk the sites fastest for one column, so that the four reads of a neighbour's
// column meet in L1 or L2 instead of coming from HBM four times.
template <int NS>
__global__ void k_oz_xprep(const double2* __restrict__ G, const double* __restrict__ Jtab, const int* __restrict__ nbr,
                           const int* __restrict__ nbond, int Nr, int Nt, int Nc, int ncol,
                           __nv_bfloat16* __restrict__ xs, double* __restrict__ tau) {
  const size_t wi = (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (wi >= (size_t)Nr * ncol) return;
  const int i = (int)(wi % Nr), n = (int)(wi / Nr);
  const size_t w = (size_t)i * ncol + n;                   // slot of (i, n) in tau and in the slices
  const int N2 = 2 * Nc;
  int nb[4], bd[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    nb[q] = nbr[i * 4 + q];
    bd[q] = nbond[i * 4 + q];
  }
  // gather once into registers (Nc <= 256: at most 8 points per lane); the column max is
  // taken on the bit patterns of |x| (their unsigned order is the order of the values)
  constexpr int PER_LANE = 256 / 32;
  constexpr unsigned long long ABS = 0x7FFFFFFFFFFFFFFFull;
  double2 x[PER_LANE];
  unsigned long long mb = 0;
#pragma unroll
  for (int u = 0; u < PER_LANE; ++u) {
    const int z = lane + 32 * u;
    double xr = 0.0, xi = 0.0;
    if (z < Nc) {
      const int tk = time_of(z, Nt);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (nb[q] < 0) continue;
        const double Jv = Jtab[(size_t)bd[q] * Nt + tk];
        const double2 g = G[((size_t)nb[q] * ncol + n) * Nc + z];
        xr = fma(Jv, g.x, xr);
        xi = fma(Jv, g.y, xi);
      }
    }
    x[u] = make_double2(xr, xi);
    const unsigned long long br = (unsigned long long)__double_as_longlong(xr) & ABS;
    const unsigned long long bi = (unsigned long long)__double_as_longlong(xi) & ABS;
    mb = max(mb, max(br, bi));
  }
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, (unsigned long long)__shfl_xor_sync(0xffffffffu, mb, o));
  // scale sc = 2^e >= max |x| (the exponent of frexp), 1 for an all-zero column
  const int Emx = (int)((mb >> 52) & 0x7FF);
  const int e = Emx == 0 ? 0 : Emx - 1022;
  if (lane == 0) tau[w] = __longlong_as_double((long long)(e + 1023) << 52);
  const size_t stride = (size_t)Nr * ncol * N2;
  __nv_bfloat16* dst = xs + w * N2;
#pragma unroll
  for (int u = 0; u < PER_LANE; ++u) {
    const int z = lane + 32 * u;
    if (z < Nc) {
      write_digits_fast<NS>(fixed_right(x[u].x, FIX - e), dst + z, stride);
      write_digits_fast<NS>(fixed_right(x[u].y, FIX - e), dst + Nc + z, stride);
    }
  }
}

// The same where every bond carries the same J(t): the factor sits in the Lambda slices
// (k_oz_aprep with Jrow), and X = sum_j G_j needs only additions, done on the FP64 pipe
// (which this kernel leaves otherwise idle) while the integer pipe cuts the digits.
template <int NS>
__global__ void k_oz_xprep_sum(const double2* __restrict__ G, const int* __restrict__ nbr, int Nr, int Nc, int ncol,
                               __nv_bfloat16* __restrict__ xs, double* __restrict__ tau) {
  const size_t wi = (size_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (wi >= (size_t)Nr * ncol) return;
  const int i = (int)(wi % Nr), n = (int)(wi / Nr);
  const size_t w = (size_t)i * ncol + n;
  const int N2 = 2 * Nc;
  const double2* col[4];
  bool has[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = nbr[i * 4 + q];
    has[q] = j >= 0;
    col[q] = G + ((size_t)(has[q] ? j : i) * ncol + n) * Nc;
  }
  constexpr int PER_LANE = 256 / 32;
  double2 x[PER_LANE];
  unsigned int mb = 0;                                     // high words of |x|: their order is the values' order
#pragma unroll
  for (int u = 0; u < PER_LANE; ++u) {
    const int z = lane + 32 * u;
    double xr = 0.0, xi = 0.0;
    if (z < Nc) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (!has[q]) continue;
        const double2 g = col[q][z];
        xr += g.x;
        xi += g.y;
      }
    }
    x[u] = make_double2(xr, xi);
    mb = max(mb, max((unsigned int)__double2hiint(xr) & 0x7FFFFFFFu, (unsigned int)__double2hiint(xi) & 0x7FFFFFFFu));
  }
  for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
  const int Emx = (int)((mb >> 20) & 0x7FF);
  const int e = Emx == 0 ? 0 : Emx - 1022;
  if (lane == 0) tau[w] = __longlong_as_double((long long)(e + 1023) << 52);
  const size_t stride = (size_t)Nr * ncol * N2;
  __nv_bfloat16* dst = xs + w * N2;
#pragma unroll
  for (int u = 0; u < PER_LANE; ++u) {
    const int z = lane + 32 * u;
    if (z >= Nc) continue;
    write_digits_fast<NS>(fixed_right(x[u].x, FIX - e), dst + z, stride);
    write_digits_fast<NS>(fixed_right(x[u].y, FIX - e), dst + Nc + z, stride);
  }
}

struct Prod {
  int s, t, acc;
};
template <int SE>
__host__ __device__ constexpr Prod prod_of(int p) {
  // products of the first SE slices with s + t <= SE + 1, ordered by diagonal; accumulator min(d - 2, 4)
  int idx = 0;
  for (int d = 2; d <= SE + 1; ++d)
    for (int s = 1; s < d; ++s) {
      int t = d - s;
      if (s > SE || t > SE) continue;
      if (idx == p) return Prod{s, t, d - 2 < NACC - 1 ? d - 2 : NACC - 1};
      ++idx;
    }
  return Prod{0, 0, 0};
}

// Persistent: one CTA per SM walks the 128 x 48 output tiles (row tile fastest, then
// column tile, then site).  Warp roles: warp 0 TMA loads (SE A slices and SE X slices
// per k-block), warp 1 one thread issuing the slice products into one of two
// accumulator sets in TMEM, warps 4-7 the epilogue of the previous tile.  Every
// mbarrier wait is bounded; on expiry the CTA raises the error flag and drains.
template <int SE>
__global__ void __launch_bounds__(THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap xmap,
              const double* __restrict__ sigma, const double* __restrict__ tau, const double2* __restrict__ G,
              const double2* __restrict__ lam, const int* __restrict__ src_site, const int* __restrict__ src_time,
              int Nr, int Nc, int ncol, int gs, float* __restrict__ r32, unsigned long long* __restrict__ norm,
              int* __restrict__ err) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  constexpr int STAGES = OzPipe<SE>::STAGES, STAGE_BYTES = OzPipe<SE>::STAGE_BYTES;
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_holder;
  __shared__ WaitCtl wctl;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int N2 = 2 * Nc, KB = N2 / BK;
  const int MT = N2 / BM, NT = (ncol + BN - 1) / BN;
  const int tiles = MT * NT * Nr;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 256);                   // 8 epilogue warps
    }
    mbar_init(&drain, 1);
    wait_ctl_init(&wctl);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(&tmem_holder, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  volatile WaitCtl* abort_p = &wctl;
  auto stage_ptr = [&](int s) { return smem + (size_t)s * STAGE_BYTES; };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int g = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int mt = tile % MT, nt = (tile / MT) % NT, site = tile / (MT * NT);
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % STAGES;
          if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1, abort_p)) {
            ok = false;
            break;
          }
          uint8_t* st = stage_ptr(s);
          mbar_expect_tx(&full[s], SE * (A_TILE + X_TILE));
          for (int q = 0; q < SE; ++q) {
            tma_load_4d(st + q * A_TILE, &amap, &full[s], kb * BK, mt * BM, site, q);
            tma_load_4d(st + SE * A_TILE + q * X_TILE, &xmap, &full[s], kb * BK, nt * BN, site, q);
          }
        }
      }
      // let every copy this thread issued land before the CTA can exit
      for (int q = g > STAGES ? g - STAGES : 0; q < g; ++q)
        mbar_wait(&full[q % STAGES], (q / STAGES) & 1, abort_p, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int g = 0, t = 0;
      bool ok = true, any = false;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const int buf = t & 1;
        if (t >= 2 && !mbar_wait(&acc_empty[buf], ((t >> 1) - 1) & 1, abort_p)) break;
        ++t;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(buf * ACC_COLS);
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % STAGES;
          if (!mbar_wait(&full[s], (g / STAGES) & 1, abort_p)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t base = smem_u32(stage_ptr(s));
#pragma unroll
          for (int k16 = 0; k16 < BK / 16; ++k16) {
            if constexpr (SE + 1 == NACC + 1) {
              // the X slices lie back to back in the stage, so A_s times X_1 .. X_{SE+1-s} is one
              // MMA of N = (SE + 1 - s) BN whose column block t lands at accumulator s + t - 2:
              // D starts at accumulator s - 1.  SE MMAs per k step instead of SE (SE + 1) / 2,
              // each A slice read once from shared memory.
#pragma unroll
              for (int sl = 1; sl <= SE; ++sl) {
                const uint32_t n = (uint32_t)((SE + 1 - sl) * BN);
                const uint32_t idesc = (IDESC & ~(0x3Fu << 17)) | ((n >> 3) << 17);
                const uint64_t ad = sdesc_sw64(base + (sl - 1) * A_TILE + k16 * 32);
                const uint64_t xd = sdesc_sw64(base + SE * A_TILE + k16 * 32);
                // the first MMA of the tile (sl = 1 covers every accumulator) overwrites
                mma<0>(dacc + (uint32_t)((sl - 1) * BN), ad, xd, idesc, (kb == 0 && k16 == 0 && sl == 1) ? 0u : 1u);
              }
            } else {
#pragma unroll
              for (int p = 0; p < SE * (SE + 1) / 2; ++p) {
                const Prod pr = prod_of<SE>(p);
                const uint64_t ad = sdesc_sw64(base + (pr.s - 1) * A_TILE + k16 * 32);
                const uint64_t xd = sdesc_sw64(base + SE * A_TILE + (pr.t - 1) * X_TILE + k16 * 32);
                // the first product of each accumulator at the first k step overwrites it
                const bool first = (kb == 0 && k16 == 0 && (p == 0 || prod_of<SE>(p - 1).acc != pr.acc));
                mma<0>(dacc + (uint32_t)(pr.acc * BN), ad, xd, IDESC, first ? 0u : 1u);
              }
            }
          }
          mma_commit(&empty[s]);
          any = true;
        }
        if (ok) mma_commit(&acc_full[buf]);
      }
      if (any) {
        mma_commit(&drain);                               // all MMAs of this thread completed
        mbar_wait(&drain, 0, abort_p, false);
      }
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: warps 4-11, two per TMEM lane quarter ----------------
    const int q4 = warp & 3;                             // TMEM lane quarter (a warp reads lanes 32 (warp % 4) ..)
    const int half = (warp - 4) >> 2;                    // which half of the tile's column chunks
    int t = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const int mt = tile % MT, nt = (tile / MT) % NT, site = tile / (MT * NT);
      const int buf = t & 1;
      bool go = mbar_wait(&acc_full[buf], (t >> 1) & 1, abort_p);
      ++t;
      go = __all_sync(0xffffffffu, go);                 // tcgen05.ld below is warp-collective
      if (!go) break;
      tc_fence_after();
      const int m = mt * BM + q4 * 32 + lane;            // planar row: part m / Nc, contour row z = m % Nc
      const int z = m % Nc, part = m / Nc;
      const double sg = sigma[(size_t)site * N2 + m] * ldexp(1.0, -FIX);   // row scale / fixed-point unit
      const long long sgb = __double_as_longlong(sg);
      const uint32_t tacc = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * ACC_COLS);
      constexpr int CHUNKS = BN / EPI_CHUNK, PER_HALF = CHUNKS / 2;
      int qcur = (nt * BN + half * PER_HALF * EPI_CHUNK) / gs;
      float runmax = 0.f;
      for (int cc = 0; cc < PER_HALF; ++cc) {
        const int c = half * PER_HALF + cc;
        const int n0 = nt * BN + c * EPI_CHUNK;
        if (n0 >= ncol) break;                          // warp-uniform; ncol and gs are multiples of 32
        const int q = n0 / gs;
        if (q != qcur) {
          float mm = runmax;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
          if (lane == 0) atomicMax(norm + qcur, (unsigned long long)__double_as_longlong((double)mm));
          qcur = q;
          runmax = 0.f;
        }
        // the accumulators hold integer multiples of 2^{-7d}: sum them exactly in
        // 2^-FIX fixed point (int64), then convert once
        uint32_t r0[EPI_CHUNK], r1[EPI_CHUNK], r2[EPI_CHUNK], r3[EPI_CHUNK], r4[EPI_CHUNK];
        const uint32_t col = (uint32_t)(c * EPI_CHUNK);
        tmem_ld8(tacc + col, r0);
        tmem_ld8(tacc + (uint32_t)BN + col, r1);
        tmem_ld8(tacc + (uint32_t)(2 * BN) + col, r2);
        tmem_ld8(tacc + (uint32_t)(3 * BN) + col, r3);
        tmem_ld8(tacc + (uint32_t)(4 * BN) + col, r4);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < EPI_CHUNK; ++j) {
          const long long acc = acc_to_fixed<0>(__uint_as_float(r0[j])) + acc_to_fixed<1>(__uint_as_float(r1[j])) +
                                acc_to_fixed<2>(__uint_as_float(r2[j])) + acc_to_fixed<3>(__uint_as_float(r3[j])) +
                                acc_to_fixed<4>(__uint_as_float(r4[j]));
          const int n = n0 + j;
          const double2 gv = G[((size_t)site * ncol + n) * Nc + z];
          // sg tau = 2^es from the exponent fields (both are powers of two), by integer
          // arithmetic; a scale below the normal range drops terms below ~2^-960
          const long long pe = sgb + __double_as_longlong(tau[(size_t)site * ncol + n]) - (1023ll << 52);
          const double sc = pe > (1ll << 52) ? __longlong_as_double(pe) : 0.0;
          double rv = fma((double)acc, sc, -(part ? gv.y : gv.x));
          if (__builtin_expect(src_site[n] == site, 0)) {   // B = Lambda_s e_{z'} on the source site
            const double2 lv = lam[((size_t)site * Nc + z) * Nc + src_time[n]];
            rv += part ? lv.y : lv.x;
          }
          const float rf = (float)rv;
          r32[((size_t)site * ncol + n) * N2 + m] = rf;
          float d = fabsf(rf);
          d = (d == d) ? d : __int_as_float(0x7f800000);
          runmax = fmaxf(runmax, d);
        }
      }
      float mm = runmax;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
      if (lane == 0) atomicMax(norm + qcur, (unsigned long long)__double_as_longlong((double)mm));
      // this accumulator set may be overwritten by the MMAs of tile t + 2
      tc_fence_before();
      mbar_arrive(&acc_empty[buf]);
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && wctl.abort) atomicExch(err, 1);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 4D bf16 map [d3][d2][d1][d0] with a (32 x rows x 1 x 1) box and 64-byte swizzle
bool make_map4(CUtensorMap* m, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t d3, uint32_t rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[4] = {d0, d1, d2, d3};
  cuuint64_t strides[3] = {d0 * 2, d0 * d1 * 2, d0 * d1 * d2 * 2};
  cuuint32_t box[4] = {(cuuint32_t)BK, rows, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

OzState* state(dyson_ctx* c) {
  if (!c->oz) c->oz = new OzState();
  return static_cast<OzState*>(c->oz);
}

template <class T>
int grow(dyson_ctx* c, T** p, size_t* have, size_t bytes, const char* what) {
  if (*have >= bytes) return DYSON_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx_fail(c, DYSON_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
  }
  *have = bytes;
  return DYSON_OK;
}

}  // namespace

// Exactness of the diagonal-5 accumulator needs K = 2Nc <= 2^24 / (3 * 2^13) ~ 682.
bool oz_supported(dyson_ctx* c) { return c->Nc % 64 == 0 && 2 * c->Nc <= 512 && encode_fn() != nullptr; }

size_t oz_bytes_per_element() { return (size_t)S * 2 * 2; }   // X slices per complex state element

void oz_invalidate(dyson_ctx* c) {
  if (c->oz) static_cast<OzState*>(c->oz)->a_ready = false;
}

int oz_residual(dyson_ctx* c, int ncol, int gs, const double2* G, float* r32, double tol) {
  const bool short_split = tol >= SHORT_TOL;
  OzState* st = state(c);
  const int Nr = c->Nr, Nc = c->Nc, N2 = 2 * Nc;
  int rc;
  if (!st->d_err) {
    DY_CUDA(c, cudaMalloc(&st->d_err, sizeof(int)));
    DY_CUDA(c, cudaMemsetAsync(st->d_err, 0, sizeof(int), c->stream));
    DY_CUDA(c, cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  }
  if (!st->a_ready) {
    size_t abytes = (size_t)S * Nr * N2 * N2 * 2;
    if ((rc = grow(c, &st->aslices, &st->a_bytes, abytes, "Ozaki slices of Lambda"))) return rc;
    if (!st->sigma) DY_CUDA(c, cudaMalloc(&st->sigma, (size_t)Nr * N2 * sizeof(double)));
    size_t rows = (size_t)Nr * N2;
    const double* Jrow = c->j_uniform && c->Nb > 0 ? c->dJ : nullptr;   // bond 0's row stands for all
    k_oz_aprep<<<(unsigned)((rows + 7) / 8), 256, 0, c->stream>>>(c->d_lam, Jrow, Nr, c->Nt, c->Nm, c->dt, c->beta,
                                                                 st->aslices, st->sigma);
    c->launches += 1;
    if (!make_map4(&st->amap, st->aslices, N2, N2, Nr, S, BM))
      return ctx_fail(c, DYSON_ERR_CUDA, "cuTensorMapEncodeTiled failed for the Lambda slices");
    st->a_ready = true;
  }
  size_t xbytes = (size_t)S * Nr * ncol * N2 * 2;
  if ((rc = grow(c, &st->xslices, &st->x_bytes, xbytes, "Ozaki slices of X"))) return rc;
  if ((rc = grow(c, &st->tau, &st->tau_bytes, (size_t)Nr * ncol * sizeof(double), "Ozaki column scales"))) return rc;
  if (st->xmap_ptr != st->xslices || st->xmap_ncol != ncol) {
    if (!make_map4(&st->xmap, st->xslices, N2, ncol, Nr, S, BN))
      return ctx_fail(c, DYSON_ERR_CUDA, "cuTensorMapEncodeTiled failed for the X slices");
    st->xmap_ptr = st->xslices;
    st->xmap_ncol = ncol;
  }
  if (!st->smem_set) {
    DY_CUDA(c, cudaFuncSetAttribute(k_oz_gemm<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    OzPipe<S>::SMEM_BYTES));
    DY_CUDA(c, cudaFuncSetAttribute(k_oz_gemm<S_SHORT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    OzPipe<S_SHORT>::SMEM_BYTES));
    st->smem_set = true;
  }
  size_t warps = (size_t)Nr * ncol;
  const unsigned xblocks = (unsigned)((warps + 7) / 8);
  if (c->j_uniform && c->Nb > 0) {
    if (short_split)
      k_oz_xprep_sum<S_SHORT><<<xblocks, 256, 0, c->stream>>>(G, c->d_nbr, Nr, Nc, ncol, st->xslices, st->tau);
    else
      k_oz_xprep_sum<S><<<xblocks, 256, 0, c->stream>>>(G, c->d_nbr, Nr, Nc, ncol, st->xslices, st->tau);
  } else {
    if (short_split)
      k_oz_xprep<S_SHORT><<<xblocks, 256, 0, c->stream>>>(G, c->dJ, c->d_nbr, c->d_nbond, Nr, c->Nt, Nc, ncol,
                                                           st->xslices, st->tau);
    else
      k_oz_xprep<S><<<xblocks, 256, 0, c->stream>>>(G, c->dJ, c->d_nbr, c->d_nbond, Nr, c->Nt, Nc, ncol,
                                                     st->xslices, st->tau);
  }
  const long long tiles = (long long)(N2 / BM) * ((ncol + BN - 1) / BN) * Nr;
  const int grid = (int)std::min<long long>(tiles, st->num_sms);
  if (short_split)
    k_oz_gemm<S_SHORT><<<grid, THREADS, OzPipe<S_SHORT>::SMEM_BYTES, c->stream>>>(
        st->amap, st->xmap, st->sigma, st->tau, G, c->d_lam, c->d_src_site, c->d_src_time, Nr, Nc, ncol, gs, r32,
        c->d_norm, st->d_err);
  else
    k_oz_gemm<S><<<grid, THREADS, OzPipe<S>::SMEM_BYTES, c->stream>>>(
        st->amap, st->xmap, st->sigma, st->tau, G, c->d_lam, c->d_src_site, c->d_src_time, Nr, Nc, ncol, gs, r32,
        c->d_norm, st->d_err);
  c->launches += 2;
  DY_CUDA(c, cudaGetLastError());
  return DYSON_OK;
}

int oz_set_wait_limit(dyson_ctx* c, unsigned long long ns) {
  DY_CUDA(c, cudaMemcpyToSymbolAsync(ptx::g_wait_limit_ns, &ns, sizeof ns, 0, cudaMemcpyHostToDevice, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  return DYSON_OK;
}

int oz_error_enqueue(dyson_ctx* c) {
  OzState* st = static_cast<OzState*>(c->oz);
  if (!st || !st->d_err) return DYSON_OK;
  if (!st->h_err) DY_CUDA(c, cudaMallocHost(&st->h_err, sizeof(int)));
  *st->h_err = 0;
  DY_CUDA(c, cudaMemcpyAsync(st->h_err, st->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return DYSON_OK;
}

int oz_error_status(dyson_ctx* c) {
  OzState* st = static_cast<OzState*>(c->oz);
  if (!st || !st->h_err || !*st->h_err) return DYSON_OK;
  *st->h_err = 0;
  cudaMemsetAsync(st->d_err, 0, sizeof(int), c->stream);
  return ctx_fail(c, DYSON_ERR_TIMEOUT, "a residual pipeline wait exceeded its time limit");
}

int oz_check_error(dyson_ctx* c) {
  OzState* st = static_cast<OzState*>(c->oz);
  if (!st || !st->d_err) return DYSON_OK;
  int rc = oz_error_enqueue(c);
  if (rc) return rc;
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  c->host_syncs += 1;
  return oz_error_status(c);
}

void oz_release(dyson_ctx* c) {
  OzState* st = static_cast<OzState*>(c->oz);
  if (!st) return;
  void* ptrs[] = {st->aslices, st->sigma, st->xslices, st->tau, st->d_err};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (st->h_err) cudaFreeHost(st->h_err);
  delete st;
  c->oz = nullptr;
}
