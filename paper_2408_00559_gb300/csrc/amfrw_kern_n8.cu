// Solver kernels for N = 8 axes (7 forward rate(s) and V).
#include "amfrw_solver.cuh"
AMFRW_INSTANTIATE(8)
