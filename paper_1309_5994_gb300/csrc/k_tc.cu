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
//   k_tc_gemm    per CTA one 128 x 256 output tile of one site:
//                warp 0 issues TMA loads (A_hi, A_lo, X tiles, 128-byte swizzle),
//                warps 4-7 split X into TF32 hi/lo in place in shared memory,
//                warp 1 (one thread) issues tcgen05.mma into a TMEM accumulator,
//                warps 4-7 then read TMEM, add r, store d_out and reduce the
//                per-block-column update norm.
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the CTA
// raises an error flag, lets in-flight copies and MMAs land, frees TMEM and
// exits, and the host returns DYSON_ERR_TIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc.cuh"

namespace {

constexpr int BM = 128, BN = 256, BK = 32, STAGES = 2;
constexpr int A_TILE = BM * BK * 4;                    // 16 KB
constexpr int X_TILE = BN * BK * 4;                    // 32 KB
constexpr int STAGE_BYTES = 2 * A_TILE + 2 * X_TILE;   // A_hi, A_lo, X (-> X_hi), X_lo
constexpr int TMA_BYTES = 2 * A_TILE + X_TILE;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024;
constexpr int THREADS = 256;
constexpr uint32_t TMEM_COLS = 256;
constexpr unsigned long long WAIT_NS = 2000000000ull;

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
  bool smem_set = false;
};

// ---------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait.  Returns false if the CTA abort flag is (or gets) raised or the
// wait exceeds WAIT_NS; with honour_abort = false only the time limit applies.
__device__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag, bool honour_abort = true) {
  unsigned long long t0 = gtimer();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try(b, parity)) return true;
    if (honour_abort && *abort_flag) return false;
    if ((it & 63) == 63 && gtimer() - t0 > WAIT_NS) {
      *abort_flag = 1;
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: kind::tf32, D = F32, A = B = TF32, both K-major, M = 128, N = 256
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float to_tf32(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

__device__ __forceinline__ unsigned long long nonneg_bits(float v) {
  double d = (v == v) ? (double)v : __longlong_as_double(0x7ff0000000000000ULL);
  return (unsigned long long)__double_as_longlong(d);
}

// ---------------------------------------------------------------------------
// gather: X[i][n][k] = sum_j J_ij(k mod Nc) d_j[n][k]
// grid: one CTA per (block of 16 vector columns, site), column block outermost
// ---------------------------------------------------------------------------
constexpr int GATHER_COLS = 16;

__global__ __launch_bounds__(256) void k_tc_gather(const float* __restrict__ din, const float* __restrict__ Jz,
                                                   const int* __restrict__ nbr, const int* __restrict__ nbond,
                                                   float* __restrict__ X, int Nr, int Nc, int ncol) {
  const int i = blockIdx.x % Nr;
  const int nblk = blockIdx.x / Nr;
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

// ---------------------------------------------------------------------------
// GEMM + epilogue
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap map_ahi, const __grid_constant__ CUtensorMap map_alo,
              const __grid_constant__ CUtensorMap map_x, const float* __restrict__ r, const float* __restrict__ din,
              float* __restrict__ dout, int Nc, int ncol, unsigned long long* __restrict__ norm,
              int* __restrict__ err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_tma[STAGES], full_split[STAGES], empty[STAGES], acc_full;
  __shared__ uint32_t tmem_holder;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int mt = blockIdx.x, nt = blockIdx.y, site = blockIdx.z;
  const int KB = (2 * Nc) / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_tma[s], 1);
      mbar_init(&full_split[s], 128);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&acc_full, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_holder;
  volatile int* abort_p = &abort_flag;

  auto stage_ptr = [&](int s) { return smem + (size_t)s * STAGE_BYTES; };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      int issued = 0;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) - 1) & 1, abort_p)) break;
        uint8_t* st = stage_ptr(s);
        mbar_expect_tx(&full_tma[s], TMA_BYTES);
        tma_load_3d(st, &map_ahi, &full_tma[s], kb * BK, mt * BM, site);
        tma_load_3d(st + A_TILE, &map_alo, &full_tma[s], kb * BK, mt * BM, site);
        tma_load_3d(st + 2 * A_TILE, &map_x, &full_tma[s], kb * BK, nt * BN, site);
        issued = kb + 1;
      }
      // let every copy this thread issued land before the CTA can exit
      for (int kb = issued > STAGES ? issued - STAGES : 0; kb < issued; ++kb)
        mbar_wait(&full_tma[kb % STAGES], (kb / STAGES) & 1, abort_p, false);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      bool any = false;
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % STAGES;
        if (!mbar_wait(&full_split[s], (kb / STAGES) & 1, abort_p)) break;
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
          mma_tf32(tmem, dah, dxh, (kb | k8) ? 1u : 0u);
          mma_tf32(tmem, dah, dxl, 1u);
          mma_tf32(tmem, dal, dxh, 1u);
        }
        mma_commit(&empty[s]);
        any = true;
      }
      if (any) {
        mma_commit(&acc_full);
        mbar_wait(&acc_full, 0, abort_p, false);   // the MMAs this thread issued have completed
      }
    }
  } else if (warp >= 4) {
    const int t = threadIdx.x - 128;
    // ---------------- split X into TF32 hi / lo ----------------
    bool ok = true;
    for (int kb = 0; kb < KB && ok; ++kb) {
      const int s = kb % STAGES;
      if (!mbar_wait(&full_tma[s], (kb / STAGES) & 1, abort_p)) {
        ok = false;
        break;
      }
      float4* xh = reinterpret_cast<float4*>(stage_ptr(s) + 2 * A_TILE);
      float4* xl = reinterpret_cast<float4*>(stage_ptr(s) + 2 * A_TILE + X_TILE);
#pragma unroll 4
      for (int e = t; e < X_TILE / 16; e += 128) {
        float4 v = xh[e], h, l;
        h.x = to_tf32(v.x); l.x = to_tf32(v.x - h.x);
        h.y = to_tf32(v.y); l.y = to_tf32(v.y - h.y);
        h.z = to_tf32(v.z); l.z = to_tf32(v.z - h.z);
        h.w = to_tf32(v.w); l.w = to_tf32(v.w - h.w);
        xh[e] = h;
        xl[e] = l;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&full_split[s]);
    }
    // ---------------- epilogue ----------------
    bool go = ok && mbar_wait(&acc_full, 0, abort_p);
    go = __all_sync(0xffffffffu, go);               // tcgen05.ld below is warp-collective
    if (go) {
      tc_fence_after();
      const int q4 = warp - 4;                      // TMEM lane quarter of this warp
      const int mg = mt * BM + q4 * 32 + lane;      // row of the 2Nc planar vector
      const size_t N2 = 2 * (size_t)Nc;
      const int n_first = nt * BN;
      int qcur = n_first / Nc;
      float runmax = 0.f;
      // Nc is a multiple of 64, so a chunk of 32 columns lies in one block column
      // and ncol is a multiple of 32: no per-column branch inside a chunk.
      for (int c = 0; c < BN / 32; ++c) {
        const int n0 = n_first + c * 32;
        if (n0 >= ncol) break;                      // uniform across the warp
        const int q = n0 / Nc;
        if (q != qcur) {
          float m = runmax;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
          if (lane == 0) atomicMax(norm + qcur, nonneg_bits(m));
          qcur = q;
          runmax = 0.f;
        }
        float v[32], rv[32], dv[32];
        const size_t base = ((size_t)site * ncol + n0) * N2 + mg;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          rv[j] = __ldcs(r + base + (size_t)j * N2);
          dv[j] = __ldcs(din + base + (size_t)j * N2);
        }
        tmem_ld32(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(c * 32), v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float y = rv[j] + v[j];
          float d = fabsf(y - dv[j]);
          d = (d == d) ? d : __int_as_float(0x7f800000);
          dout[base + (size_t)j * N2] = y;
          runmax = fmaxf(runmax, d);
        }
      }
      float m = runmax;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) atomicMax(norm + qcur, nonneg_bits(m));
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
  if (threadIdx.x == 0 && abort_flag) atomicExch(err, 1);
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

}  // namespace

bool tc_supported(dyson_ctx* c, int Nc) {
  (void)c;
  return Nc % 64 == 0 && encode_fn() != nullptr;
}

int tc_sweep(dyson_ctx* c, int nq, const float* r, const float* din, float* dout) {
  TcState* st = state(c);
  const int Nc = c->Nc, N2 = 2 * Nc, Nr = c->Nr;
  const int ncol = nq * Nc;
  if (!st->d_err) {
    DY_CUDA(c, cudaMalloc(&st->d_err, sizeof(int)));
    DY_CUDA(c, cudaMemsetAsync(st->d_err, 0, sizeof(int), c->stream));
  }
  if (st->a_hi_ptr != c->d_lam_hi || st->a_lo_ptr != c->d_lam_lo || st->a_Nr != Nr || st->a_Nc != Nc) {
    if (!make_map(&st->a_hi, c->d_lam_hi, N2, N2, Nr, BM) || !make_map(&st->a_lo, c->d_lam_lo, N2, N2, Nr, BM))
      return ctx_fail(c, DYSON_ERR_CUDA, "cuTensorMapEncodeTiled failed for Lambda");
    st->a_hi_ptr = c->d_lam_hi;
    st->a_lo_ptr = c->d_lam_lo;
    st->a_Nr = Nr;
    st->a_Nc = Nc;
  }
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
  }
  if (!st->smem_set) {
    DY_CUDA(c, cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES));
    st->smem_set = true;
  }
  int gblocks = Nr * ((ncol + GATHER_COLS - 1) / GATHER_COLS);
  k_tc_gather<<<gblocks, 256, 0, c->stream>>>(din, c->d_Jz, c->d_nbr, c->d_nbond, st->xbuf, Nr, Nc, ncol);
  dim3 grid(N2 / BM, (ncol + BN - 1) / BN, Nr);
  k_tc_gemm<<<grid, THREADS, SMEM_BYTES, c->stream>>>(st->a_hi, st->a_lo, st->x, r, din, dout, Nc, ncol, c->d_norm,
                                                       st->d_err);
  DY_CUDA(c, cudaGetLastError());
  c->launches += 2;
  return DYSON_OK;
}

int tc_check_error(dyson_ctx* c) {
  TcState* st = static_cast<TcState*>(c->tc);
  if (!st || !st->d_err) return DYSON_OK;
  int h = 0;
  DY_CUDA(c, cudaMemcpyAsync(&h, st->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DY_CUDA(c, cudaStreamSynchronize(c->stream));
  if (h) {
    cudaMemsetAsync(st->d_err, 0, sizeof(int), c->stream);
    return ctx_fail(c, DYSON_ERR_TIMEOUT, "a tensor-core pipeline wait exceeded its time limit");
  }
  return DYSON_OK;
}

void tc_release(dyson_ctx* c) {
  TcState* st = static_cast<TcState*>(c->tc);
  if (!st) return;
  if (st->xbuf) cudaFree(st->xbuf);
  if (st->d_err) cudaFree(st->d_err);
  delete st;
  c->tc = nullptr;
}
