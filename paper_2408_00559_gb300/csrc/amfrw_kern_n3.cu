// Solver kernels for N = 3 axes (2 forward rate(s) and V).
#include "amfrw_solver.cuh"
AMFRW_INSTANTIATE(3)
