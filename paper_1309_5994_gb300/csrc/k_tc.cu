// K2: one series sweep of App. C on the 5th-generation tensor cores,
//     d_out = r + (Lambda W) X,   X_i(n, k) = sum_{j in NN(i)} J_ij(k) d_in_j(n, k),
// over the FP32 planar chunk state (per vector column: Nc real parts, then Nc
// imaginary parts).  The complex product is the real GEMM of the embedding
// [[Re, -Im], [Im, Re]] (M = K = 2Nc) with the planar column vectors (N = vector
// columns), and FP32 accuracy comes from three TF32 products
//     A_hi X_hi + A_hi X_lo + A_lo X_hi
// accumulated in FP32 in tensor memory.
//
// Two launches per sweep:
//   k_tc_gather  X = sum_j J_ij d_j (FP32, coalesced float4, columns of all
//                sites visited block by block so neighbour rows hit in L2);
//   k_tc_gemm    persistent: one CTA per SM walks 128 x 256 output tiles (row
//                tile fastest, then column tile, then site, so X tiles and the
//                site's Lambda are shared through L2).  Warp roles:
//                  warp 0       TMA loads of A_hi, A_lo, X (128-byte swizzle, 2 stages)
//                  warps 4-7    split X into TF32 hi/lo in place in shared memory
//                  warp 1       one thread issues tcgen05.mma into one of two
//                               256-column TMEM accumulators
//                  warps 8-11   epilogue: tcgen05.ld, + r, store d_out, update norm
//                so the epilogue of one tile overlaps the MMAs of the next.
//   k_tc_gemm_pair  the same sweep on clusters of two CTAs (tcgen05 cta_group::2,
//                256 x 256 tiles, three 64 KB stages); selected per context with
//                dyson_set_sweep_variant.
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the CTA
// raises an error flag, lets in-flight copies and MMAs land, frees TMEM and
// exits, and the host returns DYSON_ERR_TIMEOUT.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "ptx.cuh"
#include "tc.cuh"

namespace {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 2;
static_assert(BN == TC_TILE_COLS, "support-truncation tables are laid out per GEMM column tile");
constexpr int PREFETCH = 4;                            // k-blocks of L2 prefetch ahead of the loads
constexpr int A_TILE = BM * BK * 4;                    // 16 KB
constexpr int X_TILE = BN * BK * 4;                    // 32 KB
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * X_TILE;   // A_hi, A_lo, X (-> X_hi), X_lo
constexpr int TMA_BYTES = 2 * A_TILE + X_TILE;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int THREADS = 384;
constexpr uint32_t ACC_COLS = BN;                      // one accumulator: 128 lanes x 256 fp32
constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;           // double-buffered

// kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

struct TcState {
  CUtensorMap a_hi, a_lo, x;
  const float* a_hi_ptr = nullptr;
  const float* a_lo_ptr = nullptr;
  int a_Nr = 0, a_Nc = 0;
  const float* x_ptr = nullptr;
  int x_ncol = -1;
  float* xbuf = nullptr;
  size_t xbuf_bytes = 0;
  int* d_err = nullptr;
  int* h_err = nullptr;              // pinned copy of d_err (tc_error_enqueue / tc_error_status)
  bool smem_set = false;
  int num_sms = 0;
  // CTA-pair kernel: X map with half-width boxes, co-resident clusters (0 = unused)
  CUtensorMap xh;
  int xh_ncol = -1;
  const float* xh_ptr = nullptr;
  int pair_clusters = -1;
  // fused gather + GEMM (k_tc_fused<GT>): co-resident clusters per GT (-1: not yet asked)
  int fused_clusters[2] = {-1, -1};
  // one-entry instance table of the single-context sweep (pinned host copy and device copy)
  TcInst* h_inst = nullptr;
  TcInst* d_inst = nullptr;
  bool inst_valid = false;
};

// Round to TF32 (10 explicit mantissa bits), to nearest with ties away from zero,
// by integer arithmetic on the bit pattern: adding half of the 13 dropped bits
// then clearing them rounds the magnitude (sign-magnitude encoding).  Two
// full-rate integer instructions instead of a conversion instruction.
__device__ __forceinline__ float to_tf32(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}

__device__ __forceinline__ unsigned long long nonneg_bits(float v) {
  double d = (v == v) ? (double)v : __longlong_as_double(0x7ff0000000000000ULL);
  return (unsigned long long)__double_as_longlong(d);
}

// ---------------------------------------------------------------------------
// gather: X[i][n][k] = sum_j J_ij(k mod Nc) d_j[n][k]
// grid: the instances' blocks back to back; within an instance one CTA per
// (block of 16 vector columns, site), column block outermost
// ---------------------------------------------------------------------------
constexpr int GATHER_COLS = 16;

// the instance whose range [key0, next key0) holds t (keys ascending, first key 0)
template <int FIELD>
__device__ __forceinline__ int find_inst(const TcInst* __restrict__ tab, int n, int t) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int key = FIELD == 0 ? tab[mid].tile0 : tab[mid].gblk0;
    if (key <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool inst_active(const TcInst& I) { return I.active == nullptr || *I.active != 0; }

// single instance: pointers and sizes as kernel parameters (32 registers, 8 blocks per SM)
// act (optional, [Nr][column tiles of BN]): the first sweep at which the tile can
// be non-zero; blocks of later tiles are skipped (support truncation)
__global__ __launch_bounds__(256) void k_tc_gather_one(const float* __restrict__ din, const float* __restrict__ Jz,
                                                       const int* __restrict__ nbr, const int* __restrict__ nbond,
                                                       float* __restrict__ X, int Nr, int Nc, int ncol,
                                                       const int* __restrict__ act, int sweep) {
  const int i = blockIdx.x % Nr;
  const int nblk = blockIdx.x / Nr;
  if (act && act[i * ((ncol + BN - 1) / BN) + (nblk * GATHER_COLS) / BN] > sweep) return;
  const int N2 = 2 * Nc;
  int nb[4], bd[4];
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    nb[s] = nbr[i * 4 + s];
    bd[s] = nbond[i * 4 + s];
  }
  const int per_col4 = N2 / 4;
  const int total4 = GATHER_COLS * per_col4;
  for (int e = threadIdx.x; e < total4; e += blockDim.x) {
    int c = e / per_col4, k = (e - c * per_col4) * 4;
    int n = nblk * GATHER_COLS + c;
    if (n >= ncol) break;
    int kz = k < Nc ? k : k - Nc;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if (nb[s] < 0) continue;
      float4 j = *reinterpret_cast<const float4*>(Jz + (size_t)bd[s] * Nc + kz);
      float4 g = *reinterpret_cast<const float4*>(din + ((size_t)nb[s] * ncol + n) * N2 + k);
      acc.x = fmaf(j.x, g.x, acc.x);
      acc.y = fmaf(j.y, g.y, acc.y);
      acc.z = fmaf(j.z, g.z, acc.z);
      acc.w = fmaf(j.w, g.w, acc.w);
    }
    *reinterpret_cast<float4*>(X + ((size_t)i * ncol + n) * N2 + k) = acc;
  }
}

// batched: the instance table; an instance's blocks follow the previous instance's
__global__ __launch_bounds__(256) void k_tc_gather(const TcInst* __restrict__ tab, int ninst, int parity) {
  // the instance's pointers and this site's neighbours, read once per block
  __shared__ const float* s_din;
  __shared__ const float* s_Jz;
  __shared__ float* s_X;
  __shared__ int s_nb[4], s_bd[4], s_dim[4];
  if (threadIdx.x == 0) {
    const TcInst& I = tab[find_inst<1>(tab, ninst, blockIdx.x)];
    const bool act = inst_active(I);
    const int b = blockIdx.x - I.gblk0;
    const int i = b % I.Nr;
    s_din = I.buf[parity];
    s_Jz = I.Jz;
    s_X = I.X;
    s_dim[0] = act ? I.Nc : 0;
    s_dim[1] = I.ncol;
    s_dim[2] = i;
    s_dim[3] = b / I.Nr;
    for (int q = 0; q < 4; ++q) {
      s_nb[q] = I.nbr[i * 4 + q];
      s_bd[q] = I.nbond[i * 4 + q];
    }
  }
  __syncthreads();
  const int Nc = s_dim[0];
  if (Nc == 0) return;                                  // converged instance
  const int ncol = s_dim[1], i = s_dim[2], nblk = s_dim[3];
  const int N2 = 2 * Nc;
  const int per_col4 = N2 / 4;
  const int total4 = GATHER_COLS * per_col4;
  for (int e = threadIdx.x; e < total4; e += blockDim.x) {
    int c = e / per_col4, k = (e - c * per_col4) * 4;
    int n = nblk * GATHER_COLS + c;
    if (n >= ncol) break;
    int kz = k < Nc ? k : k - Nc;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int nb = s_nb[s];
      if (nb < 0) continue;
      float4 j = *reinterpret_cast<const float4*>(s_Jz + (size_t)s_bd[s] * Nc + kz);
      float4 g = *reinterpret_cast<const float4*>(s_din + ((size_t)nb * ncol + n) * N2 + k);
      acc.x = fmaf(j.x, g.x, acc.x);
      acc.y = fmaf(j.y, g.y, acc.y);
      acc.z = fmaf(j.z, g.z, acc.z);
      acc.w = fmaf(j.w, g.w, acc.w);
    }
    *reinterpret_cast<float4*>(s_X + ((size_t)i * ncol + n) * N2 + k) = acc;
  }
}

// split an fp32 tile (float4 granules e = tt, tt + 128, ...) into TF32 hi in place and lo at x + bytes
template <int BYTES>
__device__ __forceinline__ void split_tile(uint8_t* x, int tt) {
  float4* xh = reinterpret_cast<float4*>(x);
  float4* xl = reinterpret_cast<float4*>(x + BYTES);
#pragma unroll 4
  for (int e = tt; e < BYTES / 16; e += 128) {
    float4 v = xh[e], h, l;
    h.x = to_tf32(v.x); l.x = to_tf32(v.x - h.x);
    h.y = to_tf32(v.y); l.y = to_tf32(v.y - h.y);
    h.z = to_tf32(v.z); l.z = to_tf32(v.z - h.z);
    h.w = to_tf32(v.w); l.w = to_tf32(v.w - h.w);
    xh[e] = h;
    xl[e] = l;
  }
}

// epilogue of one warp's 32 accumulator lanes x BN columns (TMEM address tacc):
// y = r + acc at planar row mg, columns n_first.., store y, and fold max|y - d_in|
// into norm[] per group of gs columns (gs a multiple of 32)
// (CH = 32 or 16 columns per tcgen05.ld; 16 keeps the register count of the 512-thread
// fused kernel below its limit)
// (RZERO: r is zero on this tile, its loads are skipped)
template <int CH = 32, bool RZERO = false>
__device__ __forceinline__ void epilogue_rows(uint32_t tacc, int mg, int n_first, int site, int ncol, int gs,
                                              size_t N2, const float* __restrict__ r, const float* __restrict__ din,
                                              float* __restrict__ dout, unsigned long long* __restrict__ norm,
                                              int lane) {
  using namespace ptx;
  int qcur = n_first / gs;
  float runmax = 0.f;
  for (int c = 0; c < BN / CH; ++c) {
    const int n0 = n_first + c * CH;
    if (n0 >= ncol) break;                          // uniform across the warp
    const int q = n0 / gs;
    if (q != qcur) {
      float m = runmax;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) atomicMax(norm + qcur, nonneg_bits(m));
      qcur = q;
      runmax = 0.f;
    }
    float rv[CH], dv[CH];
    uint32_t v[CH];
    const size_t base = ((size_t)site * ncol + n0) * N2 + mg;
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      rv[j] = RZERO ? 0.f : __ldcs(r + base + (size_t)j * N2);
      dv[j] = __ldcs(din + base + (size_t)j * N2);
    }
    if (CH == 32) tmem_ld32(tacc + (uint32_t)(c * CH), v);
    else tmem_ld16(tacc + (uint32_t)(c * CH), v);
    tmem_wait_ld();
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const float y = rv[j] + __uint_as_float(v[j]);
      float d = fabsf(y - dv[j]);
      d = (d == d) ? d : __int_as_float(0x7f800000);
      __stcs(dout + base + (size_t)j * N2, y);
      runmax = fmaxf(runmax, d);
    }
  }
  float m = runmax;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) atomicMax(norm + qcur, nonneg_bits(m));
}

// ---------------------------------------------------------------------------
// persistent GEMM + epilogue over the tiles of every instance of the table
// ---------------------------------------------------------------------------
// One 128 x 256 output tile of an instance, as every warp role decodes it.
struct TileRef {
  const TcInst* I;
  int k;                             // instance index (its tensor maps are maps.*[k])
  int KB, mt, nt, site;
  bool active;
};

// act/sweep: support truncation of a one-entry table (tiles whose act entry exceeds
// the sweep hold zeros and are skipped), act == nullptr: none
__device__ __forceinline__ TileRef decode_tile(const TcInst* __restrict__ tab, int ninst, int tile,
                                               const int* __restrict__ act, int sweep) {
  TileRef T;
  T.k = find_inst<0>(tab, ninst, tile);
  T.I = &tab[T.k];
  const int Nc = T.I->Nc;
  const int MT = (2 * Nc) / BM, NT = (T.I->ncol + BN - 1) / BN;
  const int lt = tile - T.I->tile0;
  T.KB = (2 * Nc) / BK;
  T.mt = lt % MT;
  T.nt = (lt / MT) % NT;
  T.site = lt / (MT * NT);
  T.active = inst_active(*T.I) && !(act && act[T.site * NT + T.nt] > sweep);
  return T;
}

template <int MAXI>
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ TcMaps<MAXI> maps, const TcInst* __restrict__ tab, int ninst, int tiles,
              int parity, int* __restrict__ err, const int* __restrict__ act, int sweep) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_tma[STAGES], full_split[STAGES], empty[STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_holder;
  __shared__ WaitCtl wctl;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_tma[s], 1);
      mbar_init(&full_split[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
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
      int g = 0;                                        // k-blocks issued by this CTA
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const TileRef T = decode_tile(tab, ninst, tile, act, sweep);
        if (!T.active) continue;
        const CUtensorMap* ma_hi = &maps.a_hi[T.k];
        const CUtensorMap* ma_lo = &maps.a_lo[T.k];
        const CUtensorMap* mx = &maps.x[T.k];
        // the next active tile of this CTA, for the L2 prefetch that runs ahead of the loads
        int t2 = tile + (int)gridDim.x;
        TileRef N;
        N.active = false;
        for (; t2 < tiles; t2 += gridDim.x) {
          N = decode_tile(tab, ninst, t2, act, sweep);
          if (N.active) break;
        }
        for (int kb = 0; kb < T.KB; ++kb, ++g) {
          const int s = g % STAGES;
          if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1, abort_p)) {
            ok = false;
            break;
          }
          uint8_t* st = stage_ptr(s);
          mbar_expect_tx(&full_tma[s], TMA_BYTES);
          tma_load_3d(st, ma_hi, &full_tma[s], kb * BK, T.mt * BM, T.site);
          tma_load_3d(st + A_TILE, ma_lo, &full_tma[s], kb * BK, T.mt * BM, T.site);
          tma_load_3d(st + 2 * A_TILE, mx, &full_tma[s], kb * BK, T.nt * BN, T.site);
          // warm L2 with the tiles of the k-block PREFETCH steps ahead: the stage
          // loads then see L2 latency instead of DRAM latency
          const int ahead = kb + PREFETCH;
          if (ahead < T.KB) {
            tma_prefetch_3d(ma_hi, ahead * BK, T.mt * BM, T.site);
            tma_prefetch_3d(ma_lo, ahead * BK, T.mt * BM, T.site);
            tma_prefetch_3d(mx, ahead * BK, T.nt * BN, T.site);
          } else if (N.active && ahead - T.KB < N.KB) {
            const int k2 = ahead - T.KB;
            tma_prefetch_3d(&maps.a_hi[N.k], k2 * BK, N.mt * BM, N.site);
            tma_prefetch_3d(&maps.a_lo[N.k], k2 * BK, N.mt * BM, N.site);
            tma_prefetch_3d(&maps.x[N.k], k2 * BK, N.nt * BN, N.site);
          }
        }
      }
      // let every copy this thread issued land before the CTA can exit
      for (int q = g > STAGES ? g - STAGES : 0; q < g; ++q)
        mbar_wait(&full_tma[q % STAGES], (q / STAGES) & 1, abort_p, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int g = 0, t = 0;
      bool ok = true, any = false;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        const TileRef T = decode_tile(tab, ninst, tile, act, sweep);
        if (!T.active) continue;
        const int buf = t & 1;
        if (t >= 2 && !mbar_wait(&acc_empty[buf], ((t >> 1) - 1) & 1, abort_p)) break;
        ++t;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(buf * ACC_COLS);
        for (int kb = 0; kb < T.KB; ++kb, ++g) {
          const int s = g % STAGES;
          if (!mbar_wait(&full_split[s], (g / STAGES) & 1, abort_p)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_hi = smem_u32(stage_ptr(s));
          const uint32_t a_lo = a_hi + A_TILE;
          const uint32_t x_hi = a_hi + 2 * A_TILE;
          const uint32_t x_lo = x_hi + X_TILE;
#pragma unroll
          for (int k8 = 0; k8 < BK / 8; ++k8) {
            const uint32_t off = k8 * 32;   // 8 TF32 values inside the 128-byte swizzle row
            const uint64_t dah = sdesc_sw128(a_hi + off), dal = sdesc_sw128(a_lo + off);
            const uint64_t dxh = sdesc_sw128(x_hi + off), dxl = sdesc_sw128(x_lo + off);
            mma<1>(dacc, dah, dxh, IDESC, (kb | k8) ? 1u : 0u);
            mma<1>(dacc, dah, dxl, IDESC, 1u);
            mma<1>(dacc, dal, dxh, IDESC, 1u);
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
  } else if (warp >= 4 && warp < 8) {
    // ---------------- split X into TF32 hi / lo ----------------
    const int tt = threadIdx.x - 128;
    int g = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
      const TileRef T = decode_tile(tab, ninst, tile, act, sweep);
      if (!T.active) continue;
      for (int kb = 0; kb < T.KB; ++kb, ++g) {
        const int s = g % STAGES;
        if (!mbar_wait(&full_tma[s], (g / STAGES) & 1, abort_p)) {
          ok = false;
          break;
        }
        split_tile<X_TILE>(stage_ptr(s) + 2 * A_TILE, tt);
        fence_async_smem();
        mbar_arrive(&full_split[s]);
      }
    }
  } else if (warp >= 8) {
    // ---------------- epilogue ----------------
    const int q4 = warp - 8;                            // TMEM lane quarter (warp % 4)
    int t = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      const TileRef T = decode_tile(tab, ninst, tile, act, sweep);
      if (!T.active) continue;
      const int buf = t & 1;
      bool go = mbar_wait(&acc_full[buf], (t >> 1) & 1, abort_p);
      ++t;
      go = __all_sync(0xffffffffu, go);                 // tcgen05.ld below is warp-collective
      if (!go) break;
      tc_fence_after();
      const TcInst& I = *T.I;
      epilogue_rows(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * ACC_COLS), T.mt * BM + q4 * 32 + lane,
                    T.nt * BN, T.site, I.ncol, I.gs, 2 * (size_t)I.Nc, I.r, I.buf[parity], I.buf[parity ^ 1],
                    I.norm, lane);
      // this accumulator may be overwritten by the MMAs of tile t + 2
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

// ---------------------------------------------------------------------------
// CTA-pair form (cluster of 2, tcgen05 cta_group::2): the pair computes a
// 256 x 256 tile with M = 256 MMAs.  CTA r of the pair loads Lambda rows
// 128 r .. 128 r + 127 of the tile and X columns 128 r .. 128 r + 127, splits only
// its half of X, and holds rows 128 r .. of the accumulator in its own TMEM.
// The even CTA's MMA thread reads both CTAs' shared memory, so per SM the TMA,
// split and MMA operand traffic through shared memory drop by a third, and
// three 64 KB stages fit.  Pipeline:
//   TMA (each CTA, own barrier) -> split (each CTA) -> arrive on the even CTA's
//   full_split -> MMAs -> commit multicast to both CTAs' empty / acc_full ->
//   epilogue (each CTA) -> arrive on the even CTA's acc_empty.
// ---------------------------------------------------------------------------
constexpr int PM = 256;                                 // tile rows per pair
constexpr int PX_TILE = (BN / 2) * BK * 4;              // 16 KB: one CTA's half of the X tile
constexpr int P_STAGES = 3;
constexpr int P_STAGE_BYTES = 2 * A_TILE + 2 * PX_TILE;  // A_hi, A_lo, X (-> X_hi), X_lo
constexpr int P_TMA_BYTES = 2 * A_TILE + PX_TILE;
constexpr int P_SMEM_BYTES = P_STAGES * P_STAGE_BYTES + 1024;
constexpr uint32_t P_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                             ((uint32_t)(PM >> 4) << 24);

__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm_pair(const __grid_constant__ CUtensorMap map_ahi, const __grid_constant__ CUtensorMap map_alo,
                   const __grid_constant__ CUtensorMap map_xh, const float* __restrict__ r,
                   const float* __restrict__ din, float* __restrict__ dout, int Nr, int Nc, int ncol, int gs,
                   unsigned long long* __restrict__ norm, int* __restrict__ err) {
  using namespace ptx;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_tma[P_STAGES], full_split[P_STAGES], empty[P_STAGES];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], drain;
  __shared__ uint32_t tmem_holder;
  __shared__ WaitCtl wctl;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int KB = (2 * Nc) / BK;
  const int MT = (2 * Nc) / PM, NT = (ncol + BN - 1) / BN;
  const int tiles = MT * NT * Nr;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P_STAGES; ++s) {
      mbar_init(&full_tma[s], 1);
      mbar_init(&full_split[s], 256);                   // 128 split threads of each CTA (even CTA's copy is used)
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 256);                    // 128 epilogue threads of each CTA
    }
    mbar_init(&drain, 1);
    wait_ctl_init(&wctl);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc_pair(&tmem_holder, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  cluster_sync();                                       // the peer's barriers exist before any remote arrive
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  volatile WaitCtl* abort_p = &wctl;
  auto stage_ptr = [&](int s) { return smem + (size_t)s * P_STAGE_BYTES; };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer (both CTAs) ----------------
      int g = 0;
      bool ok = true;
      for (int tile = pair; tile < tiles && ok; tile += npairs) {
        const int mt = tile % MT, nt = (tile / MT) % NT, site = tile / (MT * NT);
        const int row0 = mt * PM + (int)rank * BM;
        // a half tile wholly past the last column loads columns 0.. instead (its
        // products land in accumulator columns the epilogue never reads), so no
        // box lies entirely outside the tensor
        int col0 = nt * BN + (int)rank * (BN / 2);
        col0 = col0 < ncol ? col0 : 0;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % P_STAGES;
          if (g >= P_STAGES && !mbar_wait(&empty[s], ((g / P_STAGES) - 1) & 1, abort_p)) {
            ok = false;
            break;
          }
          uint8_t* st = stage_ptr(s);
          mbar_expect_tx(&full_tma[s], P_TMA_BYTES);
          tma_load_3d(st, &map_ahi, &full_tma[s], kb * BK, row0, site);
          tma_load_3d(st + A_TILE, &map_alo, &full_tma[s], kb * BK, row0, site);
          tma_load_3d(st + 2 * A_TILE, &map_xh, &full_tma[s], kb * BK, col0, site);
          {
            const int ahead = kb + PREFETCH;
            const int t2 = ahead < KB ? tile : tile + npairs;
            if (t2 < tiles && (ahead < KB || ahead - KB < KB)) {
              const int k2 = ahead < KB ? ahead : ahead - KB;
              const int m2 = t2 % MT, n2 = (t2 / MT) % NT, s2 = t2 / (MT * NT);
              tma_prefetch_3d(&map_ahi, k2 * BK, m2 * PM + (int)rank * BM, s2);
              tma_prefetch_3d(&map_alo, k2 * BK, m2 * PM + (int)rank * BM, s2);
              const int c2 = n2 * BN + (int)rank * (BN / 2);
              tma_prefetch_3d(&map_xh, k2 * BK, c2 < ncol ? c2 : 0, s2);
            }
          }
        }
      }
      for (int q = g > P_STAGES ? g - P_STAGES : 0; q < g; ++q)
        mbar_wait(&full_tma[q % P_STAGES], (q / P_STAGES) & 1, abort_p, false);
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---------------- MMA issuer (even CTA only) ----------------
      int g = 0, t = 0;
      bool ok = true, any = false;
      for (int tile = pair; tile < tiles && ok; tile += npairs, ++t) {
        const int buf = t & 1;
        if (t >= 2 && !mbar_wait_cluster(&acc_empty[buf], ((t >> 1) - 1) & 1, abort_p)) break;
        tc_fence_after();
        const uint32_t dacc = tmem + (uint32_t)(buf * ACC_COLS);
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % P_STAGES;
          if (!mbar_wait_cluster(&full_split[s], (g / P_STAGES) & 1, abort_p)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a_hi = smem_u32(stage_ptr(s));
          const uint32_t a_lo = a_hi + A_TILE;
          const uint32_t x_hi = a_hi + 2 * A_TILE;
          const uint32_t x_lo = x_hi + PX_TILE;
#pragma unroll
          for (int k8 = 0; k8 < BK / 8; ++k8) {
            const uint32_t off = k8 * 32;
            const uint64_t dah = sdesc_sw128(a_hi + off), dal = sdesc_sw128(a_lo + off);
            const uint64_t dxh = sdesc_sw128(x_hi + off), dxl = sdesc_sw128(x_lo + off);
            mma_pair_tf32(dacc, dah, dxh, P_IDESC, (kb | k8) ? 1u : 0u);
            mma_pair_tf32(dacc, dah, dxl, P_IDESC, 1u);
            mma_pair_tf32(dacc, dal, dxh, P_IDESC, 1u);
          }
          mma_commit_pair_mc(&empty[s], 0x3);
          any = true;
        }
        if (ok) mma_commit_pair_mc(&acc_full[buf], 0x3);
      }
      if (any) {
        mma_commit_pair_mc(&drain, 0x1);
        mbar_wait(&drain, 0, abort_p, false);
      }
    }
  } else if (warp >= 4 && warp < 8) {
    // ---------------- split own half of X (both CTAs) ----------------
    const int tt = threadIdx.x - 128;
    const uint32_t split_bar0 = mapa(smem_u32(&full_split[0]), 0);
    int g = 0;
    bool ok = true;
    for (int tile = pair; tile < tiles && ok; tile += npairs) {
      for (int kb = 0; kb < KB; ++kb, ++g) {
        const int s = g % P_STAGES;
        if (!mbar_wait(&full_tma[s], (g / P_STAGES) & 1, abort_p)) {
          ok = false;
          break;
        }
        split_tile<PX_TILE>(stage_ptr(s) + 2 * A_TILE, tt);
        fence_async_smem();
        mbar_arrive_remote(split_bar0 + (uint32_t)(s * sizeof(uint64_t)));
      }
    }
  } else if (warp >= 8) {
    // ---------------- epilogue (both CTAs, own 128 rows) ----------------
    const int q4 = warp - 8;
    const size_t N2 = 2 * (size_t)Nc;
    const uint32_t empty_bar0 = mapa(smem_u32(&acc_empty[0]), 0);
    int t = 0;
    for (int tile = pair; tile < tiles; tile += npairs, ++t) {
      const int mt = tile % MT, nt = (tile / MT) % NT, site = tile / (MT * NT);
      const int buf = t & 1;
      bool go = mbar_wait(&acc_full[buf], (t >> 1) & 1, abort_p);
      go = __all_sync(0xffffffffu, go);
      if (!go) break;
      tc_fence_after();
      epilogue_rows(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(buf * ACC_COLS),
                    mt * PM + (int)rank * BM + q4 * 32 + lane, nt * BN, site, ncol, gs, N2, r, din, dout, norm, lane);
      tc_fence_before();
      mbar_arrive_remote(empty_bar0 + (uint32_t)(buf * sizeof(uint64_t)));
    }
  }

  // both CTAs stay resident until the even CTA's MMAs (which read the odd CTA's
  // shared memory and write its TMEM) have drained and every remote arrive landed
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc_pair(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && wctl.abort) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// Fused sweep on CTA pairs: the neighbour gather is the producer of the MMA's
// B operand.  Eight warps per CTA read the four neighbour rows of d_in
// (coalesced float4 loads, all sixteen of a k-block issued back to back and one
// k-block ahead of their sums), scale them by J(k), sum, round the sum to TF32
// hi + lo and write both straight into the 128-byte-swizzled stage, so X never
// exists in global memory and only Lambda hi/lo travel by TMA.  The epilogue
// forms d_out = r + K d_in and the update norm max|d_out - d_in| as the unfused
// sweeps do (GMRES matvecs use it with r = 0).
// A tile is (site, 256-column tile, GT row groups of 256 rows):
//   GT = 1  tiles also run over the 2Nc / 256 row groups (each group-tile
//           gathers its own copy of X; the copies meet in L2); two TMEM
//           accumulators, so a tile's epilogue overlaps the next tile's MMAs;
//   GT = 2  one tile covers 512 rows (2Nc = 512 or a multiple): X is gathered
//           once per (site, column tile), the A stage holds both groups, and
//           the two accumulators fill TMEM, so the epilogue does not overlap.
// Sites are visited in bands of two lattice rows, column by column, so that
// a site's neighbours are read while they are still in L2.
// Warp roles (512 threads per CTA, both CTAs of the pair):
//   warp 0        TMA of this CTA's 128 rows of Lambda hi/lo per group (+ L2 prefetch)
//   warp 1        (even CTA) one thread issues the cta_group::2 MMAs
//   warp 2        one thread waits until this CTA's Lambda tiles of a stage have landed
//                 and its producer warps have written X, then arrives once on the even
//                 CTA's stage barrier (the only cluster-scope release per CTA and stage;
//                 producers arrive on a CTA-local barrier and never wait for TMA)
//   warps 4-11    gather producers: X columns 128 r .. 128 r + 127 of the tile
//   warps 12-15   epilogue: tcgen05.ld, + r, store, update norm
// Every wait is bounded like those of the other tcgen05 kernels.
// ---------------------------------------------------------------------------
constexpr int F_THREADS = 512;
constexpr int F_PROD_W0 = 4, F_PROD_WARPS = 8;
constexpr int F_EPI_W0 = 12;
constexpr int F_A_GROUP = 2 * A_TILE;                   // Lambda hi + lo, one row group, this CTA's 128 rows
constexpr int F_SITE_BAND = 2;                          // lattice rows per band of the site order
constexpr int F_RELAY_W = 2;                            // warp 2: relays "Lambda landed" to the even CTA
// registers per thread of each warpgroup once the roles split: the producers keep sixteen
// neighbour loads in flight one k-block ahead, more than the 128 a thread of a 512-thread
// block gets at launch; the TMA / MMA / relay warpgroup needs few
constexpr int F_REG_CTRL = 56, F_REG_PROD = 168, F_REG_EPI = 120;
constexpr int F_REGS_AT_LAUNCH = 65536 / F_THREADS;
static_assert(F_REG_CTRL + 2 * F_REG_PROD + F_REG_EPI <= 4 * F_REGS_AT_LAUNCH,
              "the warpgroups' register shares exceed the block's registers at launch");
static_assert(F_PROD_W0 == 4 && F_PROD_WARPS == 8 && F_EPI_W0 == 12 && F_THREADS == 512,
              "the register split assumes warpgroups {0-3: control, 4-11: producers, 12-15: epilogue}");
template <int GT>
struct FusedCfg {
  static constexpr int STAGE = GT * F_A_GROUP + 2 * PX_TILE;
  static constexpr int STAGES = GT == 1 ? 3 : 2;
  static constexpr int SMEM = STAGES * STAGE + 1024;
  static constexpr int NBUF = 2 / GT;                   // accumulator sets of GT x 256 columns
  static_assert(NBUF * GT * BN <= 512, "TMEM holds 512 columns");
};

// site of visit index v: bands of F_SITE_BAND lattice rows, walked column by column
__device__ __forceinline__ int band_site(int v, int Lx, int Ly) {
  const int band = v / (F_SITE_BAND * Lx);
  const int y0 = band * F_SITE_BAND;
  const int h = min(F_SITE_BAND, Ly - y0);
  const int w = v - band * F_SITE_BAND * Lx;
  return (y0 + w % h) * Lx + w / h;
}

struct FTile {
  int site, nt, gt;
  bool active;
};
__device__ __forceinline__ FTile fused_tile(int tile, int NGT, int NT, int Lx, int Ly, const int* __restrict__ act,
                                            int sweep) {
  FTile T;
  T.gt = tile % NGT;
  T.nt = (tile / NGT) % NT;
  T.site = band_site(tile / (NGT * NT), Lx, Ly);
  T.active = !(act && act[T.site * NT + T.nt] > sweep);
  return T;
}

template <int GT>
__global__ void __launch_bounds__(F_THREADS, 1)
    k_tc_fused(const __grid_constant__ CUtensorMap map_ahi, const __grid_constant__ CUtensorMap map_alo,
               const float* __restrict__ r, const float* __restrict__ din, float* __restrict__ dout,
               const int* __restrict__ rsrc, const float* __restrict__ Jz, const int* __restrict__ nbr,
               const int* __restrict__ nbond, int Lx,
               int Ly, int Nc, int ncol, int gs, unsigned long long* __restrict__ norm, int* __restrict__ err,
               const int* __restrict__ act, int sweep, const int* __restrict__ run,
               const int* __restrict__ sweeps_done) {
  using namespace ptx;
  using Cfg = FusedCfg<GT>;
  // a sweep of a captured graph after the series has stopped: nothing to do (every CTA
  // reads the same flag, before any barrier, cluster or TMEM step); in a captured graph
  // the sweep number (for the support table) is the device count of sweeps done, plus one
  if (run && *run == 0) return;
  if (sweeps_done) sweep = *sweeps_done + 1;
  constexpr int STAGES = Cfg::STAGES, NBUF = Cfg::NBUF, STAGE = Cfg::STAGE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_a[STAGES], xready[STAGES], full[STAGES], empty[STAGES];
  __shared__ __align__(8) uint64_t acc_full[NBUF], acc_empty[NBUF], drain;
  __shared__ uint32_t tmem_holder;
  __shared__ WaitCtl wctl;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank();
  const int pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
  const int N2 = 2 * Nc, KB = N2 / BK;
  const int NGT = N2 / (PM * GT);
  const int NT = (ncol + BN - 1) / BN;
  const int tiles = Lx * Ly * NT * NGT;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_a[s], 1);
      mbar_init(&xready[s], F_PROD_WARPS);              // this CTA's producer warps wrote X
      mbar_init(&full[s], 2);                           // each CTA's relay (even CTA's copy)
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 256);                    // 128 epilogue threads of each CTA
    }
    mbar_init(&drain, 1);
    wait_ctl_init(&wctl);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc_pair(&tmem_holder, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  volatile WaitCtl* abort_p = &wctl;
  auto stage_ptr = [&](int s) { return smem + (size_t)s * STAGE; };

  // each warpgroup sets its register budget first, in its own branch, so that the code of
  // each role is compiled against that budget
  if (warp < F_PROD_W0) {
    reg_budget<F_REG_CTRL, F_REGS_AT_LAUNCH>();
    if (warp == 0) {
      if (lane == 0) {
        // ---------------- TMA: Lambda hi / lo (each CTA its own rows) ----------------
        int g = 0;
        bool ok = true;
        for (int tile = pair; tile < tiles && ok; tile += npairs) {
          const FTile T = fused_tile(tile, NGT, NT, Lx, Ly, act, sweep);
          if (!T.active) continue;
          int t2 = tile + npairs;
          FTile N;
          N.active = false;
          for (; t2 < tiles; t2 += npairs) {
            N = fused_tile(t2, NGT, NT, Lx, Ly, act, sweep);
            if (N.active) break;
          }
          for (int kb = 0; kb < KB; ++kb, ++g) {
            const int s = g % STAGES;
            if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1, abort_p)) {
              ok = false;
              break;
            }
            uint8_t* st = stage_ptr(s);
            mbar_expect_tx(&full_a[s], GT * F_A_GROUP);
#pragma unroll
            for (int gi = 0; gi < GT; ++gi) {
              const int row0 = (T.gt * GT + gi) * PM + (int)rank * BM;
              tma_load_3d(st + gi * F_A_GROUP, &map_ahi, &full_a[s], kb * BK, row0, T.site);
              tma_load_3d(st + gi * F_A_GROUP + A_TILE, &map_alo, &full_a[s], kb * BK, row0, T.site);
            }
            const int ahead = kb + PREFETCH;
            const FTile* P = ahead < KB ? &T : (N.active && ahead - KB < KB ? &N : nullptr);
            if (P) {
              const int k2 = ahead < KB ? ahead : ahead - KB;
#pragma unroll
              for (int gi = 0; gi < GT; ++gi) {
                const int row0 = (P->gt * GT + gi) * PM + (int)rank * BM;
                tma_prefetch_3d(&map_ahi, k2 * BK, row0, P->site);
                tma_prefetch_3d(&map_alo, k2 * BK, row0, P->site);
              }
            }
          }
        }
        for (int q = g > STAGES ? g - STAGES : 0; q < g; ++q)
          mbar_wait(&full_a[q % STAGES], (q / STAGES) & 1, abort_p, false);
      }
    } else if (warp == 1) {
      if (lane == 0 && rank == 0) {
        // ---------------- MMA issuer (even CTA) ----------------
        int g = 0, t = 0;
        bool ok = true, any = false;
        for (int tile = pair; tile < tiles && ok; tile += npairs) {
          const FTile T = fused_tile(tile, NGT, NT, Lx, Ly, act, sweep);
          if (!T.active) continue;
          const int buf = t % NBUF;
          if (t >= NBUF && !mbar_wait_cluster(&acc_empty[buf], ((t / NBUF) - 1) & 1, abort_p)) break;
          ++t;
          tc_fence_after();
          for (int kb = 0; kb < KB; ++kb, ++g) {
            const int s = g % STAGES;
            if (!mbar_wait_cluster(&full[s], (g / STAGES) & 1, abort_p)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t st = smem_u32(stage_ptr(s));
            const uint32_t x_hi = st + GT * F_A_GROUP, x_lo = x_hi + PX_TILE;
#pragma unroll
            for (int k8 = 0; k8 < BK / 8; ++k8) {
              const uint32_t off = k8 * 32;
              const uint64_t dxh = sdesc_sw128(x_hi + off), dxl = sdesc_sw128(x_lo + off);
#pragma unroll
              for (int gi = 0; gi < GT; ++gi) {
                const uint32_t a_hi = st + gi * F_A_GROUP, a_lo = a_hi + A_TILE;
                const uint64_t dah = sdesc_sw128(a_hi + off), dal = sdesc_sw128(a_lo + off);
                const uint32_t dacc = tmem + (uint32_t)((buf * GT + gi) * BN);
                mma_pair_tf32(dacc, dah, dxh, P_IDESC, (kb | k8) ? 1u : 0u);
                mma_pair_tf32(dacc, dah, dxl, P_IDESC, 1u);
                mma_pair_tf32(dacc, dal, dxh, P_IDESC, 1u);
              }
            }
            mma_commit_pair_mc(&empty[s], 0x3);
            any = true;
          }
          if (ok) mma_commit_pair_mc(&acc_full[buf], 0x3);
        }
        if (any) {
          mma_commit_pair_mc(&drain, 0x1);
          mbar_wait(&drain, 0, abort_p, false);
        }
      }
    } else if (warp == F_RELAY_W) {
      if (lane == 0) {
        // ---------------- relay: this CTA's stage complete -> even CTA's stage barrier ----------------
        const uint32_t full_bar0 = mapa(smem_u32(&full[0]), 0);
        int g = 0;
        bool ok = true;
        for (int tile = pair; tile < tiles && ok; tile += npairs) {
          const FTile T = fused_tile(tile, NGT, NT, Lx, Ly, act, sweep);
          if (!T.active) continue;
          for (int kb = 0; kb < KB; ++kb, ++g) {
            const int s = g % STAGES;
            if (!mbar_wait(&full_a[s], (g / STAGES) & 1, abort_p) || !mbar_wait(&xready[s], (g / STAGES) & 1, abort_p)) {
              ok = false;
              break;
            }
            mbar_arrive_remote(full_bar0 + (uint32_t)(s * 8));
          }
        }
      }
    }
  } else if (warp < F_EPI_W0) {
    reg_budget<F_REG_PROD, F_REGS_AT_LAUNCH>();
    // ---------------- gather producers (both CTAs) ----------------
    // thread pt: 16-byte chunk j of the k-block row (k = 32 kb + 4 j .. + 3) for the
    // tile columns c0 + 32 i, i = 0..3, of this CTA's half
    const int pt = threadIdx.x - F_PROD_W0 * 32;
    const int j = pt & 7, c0 = pt >> 3;
    int g = 0;
    int ok = 1;
    for (int tile = pair; tile < tiles && ok; tile += npairs) {
      const FTile T = fused_tile(tile, NGT, NT, Lx, Ly, act, sweep);
      if (!T.active) continue;
      int nb[4], bd[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        nb[q] = __ldg(nbr + T.site * 4 + q);
        bd[q] = nb[q] >= 0 ? __ldg(nbond + T.site * 4 + q) : 0;
      }
      const int col0 = T.nt * BN + (int)rank * (BN / 2);
      // this thread's columns col0 + c0 + 32 i, i < ni, lie before the end
      const int ni = max(0, min(4, (ncol - col0 - c0 + 31) / 32));
      // row of neighbour q at the first column (a valid address also where the neighbour is missing)
      const float* nbp[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        nbp[q] = din + (nb[q] >= 0 && ni > 0 ? ((size_t)nb[q] * ncol + col0 + c0) * N2 : 0) + 4 * j;
      const size_t cstride = (size_t)32 * N2;            // 32 columns further
      // sixteen neighbour loads and four hopping loads per k-block, issued back to back
      // (no load behind a branch) one k-block ahead of their sums, so that their latency
      // overlaps the previous k-block's stage wait and shared-memory stores
      float4 v[4][4], jv[4];
      auto issue = [&](int kb) {
        const int k = kb * BK + 4 * j;
        const int kz = k < Nc ? k : k - Nc;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          jv[q] = __ldg(reinterpret_cast<const float4*>(Jz + (size_t)bd[q] * Nc + kz));
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const bool ok_qi = nb[q] >= 0 && i < ni;
            v[q][i] = __ldg(reinterpret_cast<const float4*>(ok_qi ? nbp[q] + i * cstride + kb * BK : nbp[q]));
          }
        }
      };
      issue(0);
      for (int kb = 0; kb < KB; ++kb, ++g) {
        const int s = g % STAGES;
        float4 acc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc[i] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (nb[q] >= 0 && i < ni) {
              acc[i].x = fmaf(jv[q].x, v[q][i].x, acc[i].x);
              acc[i].y = fmaf(jv[q].y, v[q][i].y, acc[i].y);
              acc[i].z = fmaf(jv[q].z, v[q][i].z, acc[i].z);
              acc[i].w = fmaf(jv[q].w, v[q][i].w, acc[i].w);
            }
          }
        }
        if (kb + 1 < KB) issue(kb + 1);
        if (g >= STAGES && !mbar_wait(&empty[s], ((g / STAGES) - 1) & 1, abort_p)) ok = 0;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        uint8_t* xs = stage_ptr(s) + GT * F_A_GROUP;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = c0 + 32 * i;
          const int off = c * 128 + ((j ^ (c & 7)) << 4);
          float4 h, l;
          h.x = to_tf32(acc[i].x); l.x = to_tf32(acc[i].x - h.x);
          h.y = to_tf32(acc[i].y); l.y = to_tf32(acc[i].y - h.y);
          h.z = to_tf32(acc[i].z); l.z = to_tf32(acc[i].z - h.z);
          h.w = to_tf32(acc[i].w); l.w = to_tf32(acc[i].w - h.w);
          *reinterpret_cast<float4*>(xs + off) = h;
          *reinterpret_cast<float4*>(xs + PX_TILE + off) = l;
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&xready[s]);
      }
    }
  } else {
    reg_budget<F_REG_EPI, F_REGS_AT_LAUNCH>();
    // ---------------- epilogue (both CTAs, own 128 rows of each group) ----------------
    const int q4 = warp - F_EPI_W0;
    const uint32_t empty_bar0 = mapa(smem_u32(&acc_empty[0]), 0);
    int t = 0;
    for (int tile = pair; tile < tiles; tile += npairs) {
      const FTile T = fused_tile(tile, NGT, NT, Lx, Ly, act, sweep);
      if (!T.active) continue;
      const int buf = t % NBUF;
      bool go = mbar_wait(&acc_full[buf], (t / NBUF) & 1, abort_p);
      ++t;
      go = __all_sync(0xffffffffu, go);
      if (!go) break;
      tc_fence_after();
      // r = 0 (a matvec), or r non-zero only on the rows of each column's source site
      // (the first right-hand side Lambda delta_s) and no column of the tile has its
      // source here: its loads are skipped
      bool rz = r == nullptr;
      if (!rz && rsrc) {
        bool here = false;
        for (int n = T.nt * BN + lane; n < min(ncol, T.nt * BN + BN); n += 32) here |= __ldg(rsrc + n) == T.site;
        rz = !__any_sync(0xffffffffu, here);
      }
#pragma unroll
      for (int gi = 0; gi < GT; ++gi) {
        const uint32_t tacc = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)((buf * GT + gi) * BN);
        const int mg = (T.gt * GT + gi) * PM + (int)rank * BM + q4 * 32 + lane;
        if (rz)
          epilogue_rows<16, true>(tacc, mg, T.nt * BN, T.site, ncol, gs, (size_t)N2, r, din, dout, norm, lane);
        else
          epilogue_rows<16, false>(tacc, mg, T.nt * BN, T.site, ncol, gs, (size_t)N2, r, din, dout, norm, lane);
      }
      tc_fence_before();
      mbar_arrive_remote(empty_bar0 + (uint32_t)(buf * sizeof(uint64_t)));
    }
  }

  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc_pair(tmem, TMEM_COLS);
  }
  if (threadIdx.x == 0 && wctl.abort) atomicExch(err, 1);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
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

// 3D map over an fp32 array [d2][d1][d0] with a (32 x box1 x 1) box, 128-byte swizzle
bool make_map(CUtensorMap* m, const float* base, uint64_t d0, uint64_t d1, uint64_t d2, uint32_t box1) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {d0, d1, d2};
  cuuint64_t strides[2] = {d0 * 4, d0 * d1 * 4};
  cuuint32_t box[3] = {(cuuint32_t)BK, box1, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

TcState* state(dyson_ctx* c) {
  if (!c->tc) c->tc = new TcState();
  return static_cast<TcState*>(c->tc);
}

// co-resident CTA pairs of k_tc_gemm_pair on this device (0: the pair kernel cannot run)
int pair_clusters(dyson_ctx* c, TcState* st) {
  if (st->pair_clusters >= 0) return st->pair_clusters;
  st->pair_clusters = 0;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) sms = 0;
  if (sms >= 2 &&
      cudaFuncSetAttribute(k_tc_gemm_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM_BYTES) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (unsigned)(sms / 2));
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = P_SMEM_BYTES;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_tc_gemm_pair, &cfg) == cudaSuccess) st->pair_clusters = ncl;
  }
  cudaGetLastError();
  return st->pair_clusters;
}

// co-resident CTA pairs of k_tc_fused<GT> on this device (0: it cannot run)
template <int GT>
int fused_clusters(dyson_ctx* c, TcState* st) {
  int& n = st->fused_clusters[GT - 1];
  if (n >= 0) return n;
  n = 0;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) sms = 0;
  // the warpgroups' register shares add up to exactly F_REGS_AT_LAUNCH per thread: with
  // any other count at launch the producers' increase could not be met, so the kernel is
  // not offered
  cudaFuncAttributes fa = {};
  if (cudaFuncGetAttributes(&fa, k_tc_fused<GT>) != cudaSuccess || fa.numRegs != F_REGS_AT_LAUNCH) sms = 0;
  if (sms >= 2 && cudaFuncSetAttribute(k_tc_fused<GT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       FusedCfg<GT>::SMEM) == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (unsigned)(sms / 2));
    cfg.blockDim = dim3(F_THREADS);
    cfg.dynamicSmemBytes = FusedCfg<GT>::SMEM;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_tc_fused<GT>, &cfg) == cudaSuccess) n = ncl;
  }
  cudaGetLastError();
  return n;
}

// row groups per fused tile for the context's variant (0: the fused kernel does not serve it)
int fused_gt(dyson_ctx* c) {
  if (c->Nc % 128 != 0 || c->Lx * c->Ly != c->Nr) return 0;
  if (c->tc_variant == DYSON_SWEEP_FUSED_PAIR) return fused_clusters<1>(c, state(c)) > 0 ? 1 : 0;
  if (c->tc_variant == DYSON_SWEEP_FUSED_PAIR_WIDE && c->Nc % 256 == 0)
    return fused_clusters<2>(c, state(c)) > 0 ? 2 : 0;
  return 0;
}

}  // namespace

bool tc_uses_fused(dyson_ctx* c) { return fused_gt(c) > 0; }

bool tc_uses_pair(dyson_ctx* c) {
  return c->tc_variant == DYSON_SWEEP_CTA_PAIR && c->Nc % 128 == 0 && pair_clusters(c, state(c)) > 0;
}

bool tc_supported(dyson_ctx* c, int Nc) {
  (void)c;
  return Nc % 64 == 0 && encode_fn() != nullptr;
}

namespace {

// tensor maps of Lambda and the gather buffer of context c for ncol columns
int tc_prepare(dyson_ctx* c, int ncol, bool need_x = true) {
  TcState* st = state(c);
  const int Nc = c->Nc, N2 = 2 * Nc, Nr = c->Nr;
  if (!st->d_err) {
    DY_CUDA(c, cudaMalloc(&st->d_err, sizeof(int)));
    DY_CUDA(c, cudaMemsetAsync(st->d_err, 0, sizeof(int), c->stream));
    DY_CUDA(c, cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  }
  if (st->a_hi_ptr != c->d_lam_hi || st->a_lo_ptr != c->d_lam_lo || st->a_Nr != Nr || st->a_Nc != Nc) {
    if (!make_map(&st->a_hi, c->d_lam_hi, N2, N2, Nr, BM) || !make_map(&st->a_lo, c->d_lam_lo, N2, N2, Nr, BM))
      return ctx_fail(c, DYSON_ERR_CUDA, "cuTensorMapEncodeTiled failed for Lambda");
    st->a_hi_ptr = c->d_lam_hi;
    st->a_lo_ptr = c->d_lam_lo;
    st->a_Nr = Nr;
    st->a_Nc = Nc;
    st->inst_valid = false;
  }
  if (!st->smem_set) {
    DY_CUDA(c, cudaFuncSetAttribute(k_tc_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    DY_CUDA(c, cudaFuncSetAttribute(k_tc_gemm<TC_MAX_INSTANCES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    SMEM_BYTES));
    st->smem_set = true;
  }
  if (!need_x) return DYSON_OK;                          // the fused sweep gathers in shared memory
  size_t xbytes = (size_t)Nr * ncol * N2 * sizeof(float);
  if (st->xbuf_bytes < xbytes) {
    if (st->xbuf) cudaFree(st->xbuf);
    st->xbuf = nullptr;
    st->xbuf_bytes = 0;
    cudaError_t e = cudaMalloc(&st->xbuf, xbytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return ctx_fail(c, DYSON_ERR_OOM, "tensor-core gather buffer");
    }
    st->xbuf_bytes = xbytes;
    st->x_ptr = nullptr;
  }
  if (st->x_ptr != st->xbuf || st->x_ncol != ncol) {
    if (!make_map(&st->x, st->xbuf, N2, ncol, Nr, BN))
      return ctx_fail(c, DYSON_ERR_CUDA, "cuTensorMapEncodeTiled failed for X");
    st->x_ptr = st->xbuf;
    st->x_ncol = ncol;
    st->inst_valid = false;
  }
  return DYSON_OK;
}

template <int GT>
int launch_fused(dyson_ctx* c, int ncol, int gs, const float* r, const float* din, float* dout, const int* act,
                 int sweep, const int* rsrc) {
  TcState* st = state(c);
  const long long tiles = (long long)c->Nr * ((ncol + BN - 1) / BN) * ((2 * c->Nc) / (PM * GT));
  const int pairs = (int)std::min<long long>(tiles, fused_clusters<GT>(c, st));
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3(2 * (unsigned)pairs);
  cfg.blockDim = dim3(F_THREADS);
  cfg.dynamicSmemBytes = FusedCfg<GT>::SMEM;
  cfg.stream = c->stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  DY_CUDA(c, cudaLaunchKernelEx(&cfg, k_tc_fused<GT>, st->a_hi, st->a_lo, r, din, dout, rsrc,
                                (const float*)c->d_Jz,
                                (const int*)c->d_nbr, (const int*)c->d_nbond, c->Lx, c->Ly, c->Nc, ncol, gs,
                                c->d_norm, st->d_err, act, sweep, c->sweep_run, c->sweep_count));
  DY_CUDA(c, cudaGetLastError());
  c->launches += 1;
  return DYSON_OK;
}

}  // namespace

int tc_prepare_sweep(dyson_ctx* c, int ncol) { return tc_prepare(c, ncol, fused_gt(c) == 0); }

int tc_fill_instance(dyson_ctx* c, int ncol, int gs, const float* r, float* buf0, float* buf1,
                     unsigned long long* norm, const int* active, TcInst* e, CUtensorMap* a_hi, CUtensorMap* a_lo,
                     CUtensorMap* x) {
  int rc = tc_prepare(c, ncol);
  if (rc) return rc;
  TcState* st = state(c);
  std::memset(static_cast<void*>(e), 0, sizeof(TcInst));
  *a_hi = st->a_hi;
  *a_lo = st->a_lo;
  *x = st->x;
  e->r = r;
  e->buf[0] = buf0;
  e->buf[1] = buf1;
  e->X = st->xbuf;
  e->Jz = c->d_Jz;
  e->nbr = c->d_nbr;
  e->nbond = c->d_nbond;
  e->norm = norm;
  e->active = active;
  e->Nr = c->Nr;
  e->Nc = c->Nc;
  e->ncol = ncol;
  e->gs = gs;
  return DYSON_OK;
}

int tc_instance_tiles(const TcInst& e) { return (2 * e.Nc / BM) * ((e.ncol + BN - 1) / BN) * e.Nr; }
int tc_instance_gather_blocks(const TcInst& e) { return e.Nr * ((e.ncol + GATHER_COLS - 1) / GATHER_COLS); }

namespace {

template <int MAXI>
int launch_gemm(dyson_ctx* c, const CUtensorMap* a_hi, const CUtensorMap* a_lo, const CUtensorMap* x,
                const TcInst* d_tab, int ninst, int tiles, int parity, cudaStream_t stream, const int* act,
                int sweep) {
  TcState* st = state(c);
  static_assert(sizeof(TcMaps<MAXI>) <= 30000, "tensor maps exceed the kernel-parameter space");
  TcMaps<MAXI> maps;
  for (int k = 0; k < ninst; ++k) {
    maps.a_hi[k] = a_hi[k];
    maps.a_lo[k] = a_lo[k];
    maps.x[k] = x[k];
  }
  const int grid = std::min(tiles, st->num_sms > 0 ? st->num_sms : 148);
  k_tc_gemm<MAXI><<<grid, THREADS, SMEM_BYTES, stream>>>(maps, d_tab, ninst, tiles, parity, st->d_err, act,
                                                         sweep);
  return DYSON_OK;
}

}  // namespace

int tc_launch_table(dyson_ctx* c, const TcInst* d_tab, int ninst, int tiles, int gblocks, int parity, int phases,
                    cudaStream_t stream, const CUtensorMap* a_hi, const CUtensorMap* a_lo, const CUtensorMap* x,
                    const TcInst* h_one, const int* act, int sweep) {
  if (ninst < 1 || ninst > TC_MAX_INSTANCES)
    return ctx_fail(c, DYSON_ERR_INVALID_ARG, "instance table of 1.." + std::to_string(TC_MAX_INSTANCES) + " entries");
  if (act && !(ninst == 1 && h_one))
    return ctx_fail(c, DYSON_ERR_INVALID_ARG, "support truncation needs a one-entry table with its host copy");
  TcState* st = state(c);
  if (phases & TC_GATHER) {
    if (h_one && ninst == 1)
      k_tc_gather_one<<<gblocks, 256, 0, stream>>>(h_one->buf[parity], h_one->Jz, h_one->nbr, h_one->nbond, h_one->X,
                                                   h_one->Nr, h_one->Nc, h_one->ncol, act, sweep);
    else
      k_tc_gather<<<gblocks, 256, 0, stream>>>(d_tab, ninst, parity);
    DY_CUDA(c, cudaGetLastError());
    c->launches += 1;
  }
  if (phases & TC_GEMM) {
    int rc = ninst == 1 ? launch_gemm<1>(c, a_hi, a_lo, x, d_tab, ninst, tiles, parity, stream, act, sweep)
                        : launch_gemm<TC_MAX_INSTANCES>(c, a_hi, a_lo, x, d_tab, ninst, tiles, parity, stream,
                                                        nullptr, 0);
    if (rc) return rc;
    DY_CUDA(c, cudaGetLastError());
    c->launches += 1;
  }
  return DYSON_OK;
}

int tc_sweep(dyson_ctx* c, int ncol, int gs, const float* r, const float* din, float* dout, int phases,
             const int* act, int sweep, int rform) {
  const int gt = (phases & TC_TABLE_ONLY) ? 0 : fused_gt(c);
  int rc = tc_prepare(c, ncol, gt == 0);
  if (rc) return rc;
  if (gt > 0) {
    // one launch gathers and multiplies: the gather phase alone launches nothing
    if (!(phases & TC_GEMM)) return DYSON_OK;
    const float* rr = rform == TC_R_ZERO ? nullptr : r;
    const int* rsrc = rform == TC_R_ON_SOURCES ? c->d_src_site : nullptr;
    return gt == 1 ? launch_fused<1>(c, ncol, gs, rr, din, dout, act, sweep, rsrc)
                   : launch_fused<2>(c, ncol, gs, rr, din, dout, act, sweep, rsrc);
  }
  TcState* st = state(c);
  const int Nc = c->Nc, N2 = 2 * Nc, Nr = c->Nr;
  // truncated sweeps run on the single-CTA kernel, which skips tiles
  if (!(phases & TC_TABLE_ONLY) && !act && tc_uses_pair(c)) {
    if (phases & TC_GATHER) {
      // the one-entry table serves the gather of the pair form too
      if ((rc = tc_sweep(c, ncol, gs, r, din, dout, TC_GATHER | TC_TABLE_ONLY))) return rc;
    }
    if (!(phases & TC_GEMM)) return DYSON_OK;
    if (st->xh_ptr != st->xbuf || st->xh_ncol != ncol) {
      if (!make_map(&st->xh, st->xbuf, N2, ncol, Nr, BN / 2))
        return ctx_fail(c, DYSON_ERR_CUDA, "cuTensorMapEncodeTiled failed for X halves");
      st->xh_ptr = st->xbuf;
      st->xh_ncol = ncol;
    }
    const long long tiles = (long long)(N2 / PM) * ((ncol + BN - 1) / BN) * Nr;
    const int pairs = (int)std::min<long long>(tiles, st->pair_clusters);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(2 * (unsigned)pairs);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = P_SMEM_BYTES;
    cfg.stream = c->stream;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    DY_CUDA(c, cudaLaunchKernelEx(&cfg, k_tc_gemm_pair, st->a_hi, st->a_lo, st->xh, r, din, dout, Nr, Nc, ncol, gs,
                                  c->d_norm, st->d_err));
    DY_CUDA(c, cudaGetLastError());
    c->launches += 1;
    return DYSON_OK;
  }
  // one-entry table; the two states keep their slots, the parity says which is d_in
  if (!st->h_inst) {
    DY_CUDA(c, cudaMallocHost((void**)&st->h_inst, sizeof(TcInst)));
    DY_CUDA(c, cudaMalloc((void**)&st->d_inst, sizeof(TcInst)));
    st->inst_valid = false;
  }
  TcInst* h = st->h_inst;
  int parity = -1;
  if (st->inst_valid && h->r == r && h->ncol == ncol && h->gs == gs && h->norm == c->d_norm) {
    if (h->buf[0] == din && h->buf[1] == dout) parity = 0;
    else if (h->buf[1] == din && h->buf[0] == dout) parity = 1;
  }
  if (parity < 0) {
    // the previous launches may still read the table: refill it behind them on the stream
    DY_CUDA(c, cudaStreamSynchronize(c->stream));
    CUtensorMap m0, m1, m2;
    if ((rc = tc_fill_instance(c, ncol, gs, r, const_cast<float*>(din), dout, c->d_norm, nullptr, h, &m0, &m1, &m2)))
      return rc;
    DY_CUDA(c, cudaMemcpyAsync(st->d_inst, h, sizeof(TcInst), cudaMemcpyHostToDevice, c->stream));
    st->inst_valid = true;
    parity = 0;
  }
  return tc_launch_table(c, st->d_inst, 1, tc_instance_tiles(*h), tc_instance_gather_blocks(*h), parity,
                         phases & (TC_GATHER | TC_GEMM), c->stream, &st->a_hi, &st->a_lo, &st->x, h, act, sweep);
}

int tc_set_wait_limit(dyson_ctx* c, unsigned long long ns) {
  DY_CUDA(c, cudaMemcpyToSymbolAsync(ptx::g_wait_limit_ns, &ns, sizeof ns, 0, cudaMemcpyHostToDevice, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  return DYSON_OK;
}

int tc_error_enqueue(dyson_ctx* c) {
  TcState* st = static_cast<TcState*>(c->tc);
  if (!st || !st->d_err) return DYSON_OK;
  if (!st->h_err) {
    DY_CUDA(c, cudaMallocHost((void**)&st->h_err, sizeof(int)));
    *st->h_err = 0;
  }
  DY_CUDA(c, cudaMemcpyAsync(st->h_err, st->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  return DYSON_OK;
}

int tc_error_status(dyson_ctx* c) {
  TcState* st = static_cast<TcState*>(c->tc);
  if (!st || !st->h_err || !*st->h_err) return DYSON_OK;
  *st->h_err = 0;
  cudaMemsetAsync(st->d_err, 0, sizeof(int), c->stream);
  return ctx_fail(c, DYSON_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its time limit");
}

int tc_check_error(dyson_ctx* c) {
  int rc = tc_error_enqueue(c);
  if (rc) return rc;
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  return tc_error_status(c);
}

void tc_release(dyson_ctx* c) {
  TcState* st = static_cast<TcState*>(c->tc);
  if (!st) return;
  if (st->xbuf) cudaFree(st->xbuf);
  if (st->d_err) cudaFree(st->d_err);
  if (st->h_err) cudaFreeHost(st->h_err);
  if (st->h_inst) cudaFreeHost(st->h_inst);
  if (st->d_inst) cudaFree(st->d_inst);
  delete st;
  c->tc = nullptr;
}
