// Solver kernels for N = 6 axes (5 forward rate(s) and V).
#include "amfrw_solver.cuh"
AMFRW_INSTANTIATE(6)
