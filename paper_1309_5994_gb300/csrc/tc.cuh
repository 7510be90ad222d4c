// Tensor-core (tcgen05) sweep: interface used by the host driver.
#pragma once
#include <cuda.h>

#include "common.cuh"

// Most instances one tensor-core launch serves.  Their TMA maps travel as
// __grid_constant__ kernel parameters (3 x 128 bytes each, 24 KB for 64), not in
// global memory, where a map written at a recycled address could meet a stale
// descriptor in the TMA unit's cache.
constexpr int TC_MAX_INSTANCES = 64;
template <int MAXI>
struct TcMaps {
  CUtensorMap a_hi[MAXI], a_lo[MAXI], x[MAXI];
};

// One problem instance of a (batched) tensor-core sweep: a device table entry.
// The state of the series alternates between buf[0] and buf[1]: a sweep of
// parity p reads d_in = buf[p] and writes d_out = buf[p ^ 1].
struct TcInst {
  const float* r;                    // right-hand side of the series [Nr][ncol][2Nc]
  float* buf[2];                     // the two FP32 states
  float* X;                          // gather output, the GEMM's B operand
  const float* Jz;                   // [Nb][Nc] hopping on the contour
  const int* nbr;                    // [Nr][4] neighbour sites (-1: none)
  const int* nbond;                  // [Nr][4] bond of each neighbour slot
  unsigned long long* norm;          // update max-norm per group of gs columns
  const int* active;                 // nullptr, or a device flag: 0 skips the instance
  int Nr, Nc, ncol, gs;
  int tile0;                         // first global GEMM tile of this instance
  int gblk0;                         // first global gather block of this instance
};


// true when the 3xTF32 tcgen05 sweep supports this contour length
bool tc_supported(dyson_ctx* c, int Nc);
// true when tc_sweep runs the CTA-pair (cta_group::2) kernel for this context
bool tc_uses_pair(dyson_ctx* c);
// true when tc_sweep runs the fused gather + GEMM kernel (k_tc_fused) for this context:
// the context's variant is DYSON_SWEEP_FUSED_PAIR (Nc % 128 == 0) or
// DYSON_SWEEP_FUSED_PAIR_WIDE (Nc % 256 == 0); TC_GATHER alone then launches nothing
bool tc_uses_fused(dyson_ctx* c);
// tensor maps and buffers of tc_sweep for ncol columns, set up ahead of a stream capture
int tc_prepare_sweep(dyson_ctx* c, int ncol);
// one sweep d_out = r + K d_in over the FP32 planar chunk state of ncol vector columns;
// writes c->d_norm[q] for groups of gs columns (gs a multiple of 32, Nc a multiple of 64).
// phases: TC_GATHER launches X = J d_in, TC_GEMM launches the tensor-core product and
// epilogue (in that order; both = one whole sweep).
// act (optional, device [Nr][ceil(ncol / 256)]): support truncation (App. C, Sec. IV.D):
// the first sweep at which each (site, 256-column tile) can be non-zero; tiles with
// act > sweep are skipped, so their d_out must already hold zeros.
// rform: what the caller knows of r, for the fused kernel to skip loads of zeros:
// TC_R_DENSE (general), TC_R_ZERO (r = 0: a matvec), TC_R_ON_SOURCES (r non-zero only
// on the rows of each column's source site, c->d_src_site: the first right-hand side)
enum { TC_GATHER = 1, TC_GEMM = 2, TC_TABLE_ONLY = 4 };
enum { TC_R_DENSE = 0, TC_R_ZERO = 1, TC_R_ON_SOURCES = 2 };
constexpr int TC_TILE_COLS = 256;
int tc_sweep(dyson_ctx* c, int ncol, int gs, const float* r, const float* d_in, float* d_out, int phases,
             const int* act = nullptr, int sweep = 0, int rform = TC_R_DENSE);
// DYSON_ERR_TIMEOUT if a bounded pipeline wait of an earlier sweep expired (clears the flag);
// synchronises the context's stream
int tc_check_error(dyson_ctx* c);
// the same in two halves around a synchronisation the caller makes anyway: enqueue the
// copy of the flag to pinned host memory, then, after the stream has synchronised, read it
int tc_error_enqueue(dyson_ctx* c);
// time limit (ns) of the pipeline waits of this file's kernels on the context's device
int tc_set_wait_limit(dyson_ctx* c, unsigned long long ns);
int tc_error_status(dyson_ctx* c);
// free tensor-core module state
void tc_release(dyson_ctx* c);

// Fill one instance-table entry for context c (gather buffer, the state buffers
// buf0/buf1, norm words and an optional device activity flag) and return its
// three TMA maps; tile0 and gblk0 are left 0 for the caller to set.
int tc_fill_instance(dyson_ctx* c, int ncol, int gs, const float* r, float* buf0, float* buf1,
                     unsigned long long* norm, const int* active, TcInst* e, CUtensorMap* a_hi, CUtensorMap* a_lo,
                     CUtensorMap* x);
int tc_instance_tiles(const TcInst& e);           // 128 x 256 GEMM tiles of the entry
int tc_instance_gather_blocks(const TcInst& e);   // gather blocks of the entry
// Launch the gather and/or the GEMM of one sweep of parity `parity` over a device
// table of ninst entries (tiles, gblocks: totals); errors and the launch count
// are recorded on context c.  a_hi, a_lo, x: the entries' maps (host arrays of
// ninst <= TC_MAX_INSTANCES).  h_one: for a one-entry table, its host copy (the
// gather then takes the entry's pointers as kernel parameters), else nullptr.
int tc_launch_table(dyson_ctx* c, const TcInst* d_tab, int ninst, int tiles, int gblocks, int parity, int phases,
                    cudaStream_t stream, const CUtensorMap* a_hi, const CUtensorMap* a_lo, const CUtensorMap* x,
                    const TcInst* h_one = nullptr, const int* act = nullptr, int sweep = 0);
