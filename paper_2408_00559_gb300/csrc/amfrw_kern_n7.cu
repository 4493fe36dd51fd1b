// Solver kernels for N = 7 axes (6 forward rate(s) and V).
#include "amfrw_solver.cuh"
AMFRW_INSTANTIATE(7)
