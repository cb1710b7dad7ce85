// stage_sym_o12.cu -- stage kernels with mirrored neighbour loads (symmetry
// boundaries) for central differences of order 12 (radius 6).
#include "stage.cuh"

OSB_DEFINE_ORDER_SYM(12)
