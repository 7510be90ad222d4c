// Tensor-core (tcgen05) sweep: interface used by the host driver.
#pragma once
#include "common.cuh"

// true when the 3xTF32 tcgen05 sweep supports this contour length
bool tc_supported(dyson_ctx* c, int Nc);
// true when tc_sweep runs the CTA-pair (cta_group::2) kernel for this context
bool tc_uses_pair(dyson_ctx* c);
// one sweep d_out = r + K d_in over the FP32 planar chunk state of ncol vector columns;
// writes c->d_norm[q] for groups of gs columns (gs a multiple of 32, Nc a multiple of 64).
// phases: TC_GATHER launches X = J d_in, TC_GEMM launches the tensor-core product and
// epilogue (in that order; both = one whole sweep)
enum { TC_GATHER = 1, TC_GEMM = 2 };
int tc_sweep(dyson_ctx* c, int ncol, int gs, const float* r, const float* d_in, float* d_out, int phases);
// DYSON_ERR_TIMEOUT if a bounded pipeline wait of an earlier sweep expired (clears the flag)
int tc_check_error(dyson_ctx* c);
// free tensor-core module state
void tc_release(dyson_ctx* c);
