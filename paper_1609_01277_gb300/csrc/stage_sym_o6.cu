// stage_sym_o6.cu -- stage kernels with mirrored neighbour loads (symmetry
// boundaries) for central differences of order 6 (radius 3).
#include "stage.cuh"

OSB_DEFINE_ORDER_SYM(6)
