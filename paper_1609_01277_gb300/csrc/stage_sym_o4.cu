// stage_sym_o4.cu -- stage kernels with mirrored neighbour loads (symmetry
// boundaries) for central differences of order 4 (radius 2).
#include "stage.cuh"

OSB_DEFINE_ORDER_SYM(4)
