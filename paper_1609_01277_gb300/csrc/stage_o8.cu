// stage_o8.cu -- stage kernels for central differences of order 8 (radius 4).
#include "zmarch.cuh"

OSB_DEFINE_ORDER(8)
