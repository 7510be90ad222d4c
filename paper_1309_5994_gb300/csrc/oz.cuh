// FP64-accurate Dyson residual on the BF16 tensor cores (slice-split products).
#pragma once
#include "common.cuh"

// true when the split-product residual supports this contour (Nc % 64 == 0, 2Nc <= 512)
bool oz_supported(dyson_ctx* c);
// device bytes of X slices per complex state element
size_t oz_bytes_per_element();
// forget the Lambda slices (after dyson_build_sigma)
void oz_invalidate(dyson_ctx* c);
// r32 = B + K G - G (FP32 planar output, values accurate to ~2^-43 of |K||G|, ~2^-33 when tol >= 1e-8,
// where the first five of the seven slices are used); c->d_norm[q] = max |r|
int oz_residual(dyson_ctx* c, int ncol, int gs, const double2* G, float* r32, double tol);
// DYSON_ERR_TIMEOUT if a bounded pipeline wait expired (clears the flag); synchronises
int oz_check_error(dyson_ctx* c);
// the same in two halves around a synchronisation of the caller's: enqueue the flag's
// copy to pinned memory, then (after the stream synchronised) read it
int oz_error_enqueue(dyson_ctx* c);
int oz_error_status(dyson_ctx* c);
// time limit (ns) of the pipeline waits of the residual kernels on the context's device
int oz_set_wait_limit(dyson_ctx* c, unsigned long long ns);
void oz_release(dyson_ctx* c);
