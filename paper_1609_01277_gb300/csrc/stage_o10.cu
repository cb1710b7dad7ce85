// stage_o10.cu -- stage kernels for central differences of order 10 (radius 5).
#include "zmarch.cuh"

OSB_DEFINE_ORDER(10)
