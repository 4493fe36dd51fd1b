// Solver kernels for N = 4 axes (3 forward rate(s) and V).
#include "amfrw_solver.cuh"
AMFRW_INSTANTIATE(4)
