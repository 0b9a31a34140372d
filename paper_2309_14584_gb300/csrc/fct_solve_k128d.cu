// Team solver kernel for 128-thread blocks in its deep-gather variant (plans
// with long rows or many grids), compiled in a translation unit of its own so
// that the library's kernels build in parallel.
#include "fct_solver.cuh"

template __global__ void fct_solve_kernel<128, false, 1>(const SolveArgs a);
