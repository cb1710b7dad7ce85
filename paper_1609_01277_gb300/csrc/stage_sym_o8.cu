// stage_sym_o8.cu -- stage kernels with mirrored neighbour loads (symmetry
// boundaries) for central differences of order 8 (radius 4).
#include "stage.cuh"

OSB_DEFINE_ORDER_SYM(8)
