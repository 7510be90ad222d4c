// GMRES inner solver (k_gmres.cu): interface used by the host driver.
#pragma once
#include <functional>

#include "common.cuh"

// out = zero + K in over the FP32 planar chunk state (one series sweep with a zero
// right-hand side); returns a DYSON_ERR_* code
using MatvecFn = std::function<int(const float* zero, const float* in, float* out)>;

// Restart length that fits the free device memory for ncol columns (0: none fits).
int gmres_restart_length(dyson_ctx* c, int ncol);
// Solve (I - K) x = r per vector column of the chunk by restarted GMRES, starting
// from x = r (the preconditioned right-hand side of App. C), until the largest
// relative residual estimate is <= tol or max_iters matvecs have run.
int gmres_inner_solve(dyson_ctx* c, int ncol, const float* r, float* x, int max_iters, double tol,
                      dyson_report* rep, const MatvecFn& matvec);
// free the GMRES buffers of a context
void gmres_release(dyson_ctx* c);
