// Per-phase ensemble launches (batch_phase.cuh), radii 3 and 4.
#include "batch_phase.cuh"

OSB_DEFINE_BATCH_PHASE(3)
OSB_DEFINE_BATCH_PHASE(4)
