// stage_sym_o2.cu -- stage kernels with mirrored neighbour loads (symmetry
// boundaries) for central differences of order 2 (radius 1).
#include "stage.cuh"

OSB_DEFINE_ORDER_SYM(2)
