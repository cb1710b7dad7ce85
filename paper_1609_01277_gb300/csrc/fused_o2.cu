// fused_o2.cu -- the fused FP32 stage kernel for central differences of order 2
// (radius 1), in its own translation unit so the orders compile in parallel.
#include "fused.cuh"

namespace osb {
namespace fz {
cudaError_t launch_fused_r1(const StageArgs &a) { return launch_fused<1>(a); }
}  // namespace fz
}  // namespace osb
