// Per-phase ensemble launches (batch_phase.cuh), radii 5 and 6.
#include "batch_phase.cuh"

OSB_DEFINE_BATCH_PHASE(5)
OSB_DEFINE_BATCH_PHASE(6)
