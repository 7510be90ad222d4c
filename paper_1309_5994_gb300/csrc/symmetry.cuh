// C4v irreducible-wedge solves (symmetry.cu): interface used by the host driver.
#pragma once
#include "common.cuh"

// dyson_solve_columns for a context with DYSON_SYMMETRY_C4V: solves one source
// per symmetry orbit and fills the others' observables (and G) by the symmetry
int solve_columns_c4v(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                      int32_t max_sweeps, double* g_out, dyson_report* rep_out);
