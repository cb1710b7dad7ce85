// stage_o12.cu -- stage kernels for central differences of order 12 (radius 6).
#include "zmarch.cuh"

OSB_DEFINE_ORDER(12)
