// Team solver kernels for 256-thread blocks (with and without staged entry
// values), compiled in a translation unit of their own so that the library's
// kernels build in parallel.
#include "fct_solver.cuh"

template __global__ void fct_solve_kernel<256, false, 0>(const SolveArgs a);
template __global__ void fct_solve_kernel<256, true, 0>(const SolveArgs a);
