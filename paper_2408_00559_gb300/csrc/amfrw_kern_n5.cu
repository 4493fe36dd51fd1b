// Solver kernels for N = 5 axes (4 forward rate(s) and V).
#include "amfrw_solver.cuh"
AMFRW_INSTANTIATE(5)
