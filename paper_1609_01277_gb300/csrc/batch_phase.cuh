// batch_phase.cuh -- an ensemble of periodic grids advanced phase by phase:
// each of the 9 sub-steps of an RK3 step (primitives, gradient fluxes,
// residual + update, per stage) is ONE launch over the tiles of every
// instance, and stream order stands in for the persistent kernel's
// per-instance completion counters.  Each sub-step then runs with its own
// register budget (the per-grid kernels' launch bounds), where the persistent
// kernel carries the largest phase's registers for all of them: the
// double-float ensemble's residual phase runs at four CTAs per SM here, at
// two in the persistent kernel.  Included by batch_phase_*.cu, two radii per
// translation unit.
#pragma once

#include "stage.cuh"

namespace osb {
namespace bp {

// resident CTAs per SM the per-grid kernels target, by sub-step
template <typename T, int R, int SUB>
constexpr int min_blocks() {
    if constexpr (SUB == 2 && is_dd<T>) return R <= 2 ? 4 : (R <= 4 ? 2 : 1);
    return 1;
}

// z planes per CTA: the stage-argument copy and the instance search are paid
// once per PHASE_ZP planes
constexpr int PHASE_ZP = kPhaseZP;

// One CTA: one BX x BY tile of PHASE_ZP z planes of one instance.  Blocks are
// numbered instance by instance (P.pprefix: prefix sums of tiles_x * tiles_y
// * ceil(nz / PHASE_ZP)); the instance's stage arguments for this step's
// parity go to shared memory first.
template <typename T, int R, bool VB, int SUB>
__global__ void __launch_bounds__(BX *BY, (min_blocks<T, R, SUB>())) k_phase(const BatchParams P) {
    __shared__ StageArgs sa;
    const long long blk = blockIdx.x;
    int lo = 0, hi = P.n;  // P.pprefix[lo] <= blk < P.pprefix[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (blk >= P.pprefix[mid])
            lo = mid;
        else
            hi = mid;
    }
    const int inst = lo;
    const BatchInst *B = P.rec[inst];
    const int par = (P.p0[inst] + P.step) & 1;
    {
        const int *src = reinterpret_cast<const int *>(&B->st[par][P.stage]);
        int *dst = reinterpret_cast<int *>(&sa);
        const int tid = threadIdx.y * BX + threadIdx.x;
        for (int w = tid; w < (int)(sizeof(StageArgs) / sizeof(int)); w += BX * BY) dst[w] = __ldg(src + w);
    }
    __syncthreads();
    const int t = (int)(blk - P.pprefix[inst]);
    const int txi = t % B->tiles_x, tyi = (t / B->tiles_x) % B->tiles_y, zb = t / (B->tiles_x * B->tiles_y) * PHASE_ZP;
    const int x = txi * BX + threadIdx.x, y = tyi * BY + threadIdx.y;
    if (x >= sa.d.nx || y >= sa.d.ny) return;
    const int ze = min(zb + PHASE_ZP, sa.d.nz);
    for (int z = zb; z < ze; ++z) {
        if constexpr (SUB == 0)
            prim_point<LD_NC, T, T>(sa, x, y, z);
        else if constexpr (SUB == 1)
            grad_point<LD_NC, T, T, R, VB>(sa, x, y, z);
        else
            resid_point<LD_NC, T, T, R, 0, VB>(sa, x, y, z);
    }
}

template <typename T, int R, bool VB>
cudaError_t launch_phase_t(const BatchParams &P, cudaStream_t st) {
    const unsigned blocks = (unsigned)P.pprefix[P.n];
    if (blocks == 0) return cudaSuccess;
    const dim3 blk(BX, BY, 1);
    k_phase<T, R, VB, 0><<<blocks, blk, 0, st>>>(P);
    k_phase<T, R, VB, 1><<<blocks, blk, 0, st>>>(P);
    k_phase<T, R, VB, 2><<<blocks, blk, 0, st>>>(P);
    return cudaGetLastError();
}

// the three sub-steps of RK stage P.stage of step P.step, double-float items
template <int R>
cudaError_t launch_phase_r(const BatchParams &P, int visc_form, cudaStream_t st) {
    return visc_form == OSB_VISC_B ? launch_phase_t<dd, R, true>(P, st) : launch_phase_t<dd, R, false>(P, st);
}

}  // namespace bp
}  // namespace osb

#define OSB_DEFINE_BATCH_PHASE(R)                                                                        \
    namespace osb {                                                                                      \
    cudaError_t launch_batch_phase_r##R(const BatchParams &P, int visc_form, cudaStream_t st) {          \
        return bp::launch_phase_r<R>(P, visc_form, st);                                                  \
    }                                                                                                    \
    }
