// C4v irreducible-wedge solves (symmetry.cu): interface used by the host driver.
#pragma once
#include "common.cuh"

// dyson_solve_columns for a context with DYSON_SYMMETRY_C4V: solves one source
// per symmetry orbit and fills the others' observables (and G) by the symmetry
int solve_columns_c4v(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                      int32_t max_sweeps, double* g_out, dyson_report* rep_out);

// dyson_local_greens for a context with DYSON_SYMMETRY_C4V: solves one site per
// orbit; the diagonal block of every other requested site is that of its
// representative (G_{g(r), g(r)} = G_{r, r})
int local_greens_c4v(dyson_ctx* c, const int32_t* src, int64_t n_src, int precision, double tol,
                     int32_t max_sweeps, double* gloc, dyson_report* rep_out);
