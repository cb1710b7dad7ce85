// stage_sym_o10.cu -- stage kernels with mirrored neighbour loads (symmetry
// boundaries) for central differences of order 10 (radius 5).
#include "stage.cuh"

OSB_DEFINE_ORDER_SYM(10)
