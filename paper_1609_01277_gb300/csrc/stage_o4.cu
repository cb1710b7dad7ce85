// stage_o4.cu -- stage kernels for central differences of order 4 (radius 2).
#include "zmarch.cuh"

OSB_DEFINE_ORDER(4)
