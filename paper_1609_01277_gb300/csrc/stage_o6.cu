// stage_o6.cu -- stage kernels for central differences of order 6 (radius 3).
#include "zmarch.cuh"

OSB_DEFINE_ORDER(6)
