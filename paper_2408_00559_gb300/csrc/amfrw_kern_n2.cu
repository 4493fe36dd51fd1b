// Solver kernels for N = 2 axes (1 forward rate(s) and V).
#include "amfrw_solver.cuh"
AMFRW_INSTANTIATE(2)
