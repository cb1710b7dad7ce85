// fused_o4.cu -- the fused FP32 stage kernel for central differences of order 4
// (radius 2), in its own translation unit so the orders compile in parallel.
#include "fused.cuh"

namespace osb {
namespace fz {
cudaError_t launch_fused_r2(const StageArgs &a) { return launch_fused<2>(a); }
}  // namespace fz
}  // namespace osb
