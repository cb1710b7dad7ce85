// stage_o2.cu -- stage kernels for central differences of order 2 (radius 1).
#include "zmarch.cuh"

OSB_DEFINE_ORDER(2)
