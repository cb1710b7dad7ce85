// Per-phase ensemble launches (batch_phase.cuh), radii 1 and 2.
#include "batch_phase.cuh"

OSB_DEFINE_BATCH_PHASE(1)
OSB_DEFINE_BATCH_PHASE(2)
