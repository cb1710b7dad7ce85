// batch.cu -- an ensemble of independent periodic grids (uneven sizes and
// parameters) advanced by ONE persistent kernel launch for many RK3 steps.
//
// Work items are (step, phase, instance, tile), phase = 3 RK stages x 3
// sub-steps (primitives, gradient fluxes, residual + update).  CTAs take items
// in order from a global counter.  Each instance keeps a count of its
// completed items; an item of sequence s = 9*step + phase of instance i starts
// only when that count reaches s * tiles_i, i.e. when every item of the
// instance's previous phases is done (a per-instance barrier).  Waits only ever
// target items that running CTAs took earlier, so the scheme cannot deadlock;
// each wait is still bounded by a time limit (%globaltimer), after which the
// kernel raises an error flag that every CTA observes and exits.  While one
// instance waits, CTAs keep taking items of the others: small and large grids
// share the GPU without per-instance launches.
//
// Intermediate data written by other CTAs during the launch is read through
// L2 (ld.global.cg), never through the non-coherent per-SM L1.
#include "zmarch.cuh"

namespace osb {

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T, int R, bool VB>
__device__ __forceinline__ void batch_loop(const BatchParams &P);

template <typename T, int R, bool VB>
__global__ void __launch_bounds__(BX *BY) k_batch(const BatchParams P) {
    batch_loop<T, R, VB>(P);
}
// double-float items: bounded to two CTAs per SM (128 registers, no spills;
// three, with about 100 bytes spilled at order 4, measured the same within
// run-to-run spread)
template <int R, bool VB>
__global__ void __launch_bounds__(BX *BY, 2) k_batch_dd(const BatchParams P) {
    batch_loop<dd, R, VB>(P);
}

template <typename T, int R, bool VB>
__device__ __forceinline__ void batch_loop(const BatchParams &P) {
    __shared__ StageArgs sa;
    __shared__ long long item_s;
    __shared__ int stop_s;
    const int tid = threadIdx.y * BX + threadIdx.x;
    while (true) {
        if (tid == 0) {
            item_s = (long long)atomicAdd(P.counter, 1ull);
            stop_s = ld_volatile_i32(P.err) != 0;
        }
        __syncthreads();
        const long long k = item_s;
        if (k >= P.total_items || stop_s) break;
        const long long seq = k / P.tiles_total;
        const int rem = (int)(k - seq * P.tiles_total);
        int inst = 0;
        while (rem >= P.prefix[inst + 1]) ++inst;
        const int tile = rem - P.prefix[inst];
        const int tiles_i = P.prefix[inst + 1] - P.prefix[inst];
        const BatchInst *B = P.rec[inst];
        const int step = (int)(seq / P.phases), phase = (int)(seq % P.phases), stage = phase / 3, sub = phase % 3;
        if (tid == 0) {
            const unsigned target = P.inject_stall ? 0xffffffffu : (unsigned)(seq * tiles_i);
            if (ld_acquire_u32(P.done + inst) < target) {
                const unsigned long long t0 = globaltimer();
                unsigned nap = 32;  // exponential backoff: many CTAs poll one counter
                while (true) {
                    if (ld_volatile_i32(P.err)) {
                        stop_s = 1;
                        break;
                    }
                    if (ld_acquire_u32(P.done + inst) >= target) break;
                    if (globaltimer() - t0 > (unsigned long long)P.timeout_ns) {
                        atomicExch(P.err, 1);
                        stop_s = 1;
                        break;
                    }
                    __nanosleep(nap);
                    nap = nap < 2048 ? 2 * nap : 2048;
                }
            }
        }
        // stage arguments of this instance and step parity into shared memory
        {
            const int par = (P.p0[inst] + step) & 1;
            const int *src = reinterpret_cast<const int *>(&B->st[par][stage]);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int w = tid; w < (int)(sizeof(StageArgs) / sizeof(int)); w += BX * BY) dst[w] = src[w];
        }
        __syncthreads();
        if (stop_s) break;
        const int txi = tile % B->tiles_x, tyi = (tile / B->tiles_x) % B->tiles_y, tzi = tile / (B->tiles_x * B->tiles_y);
        const int x = txi * BX + threadIdx.x, y = tyi * BY + threadIdx.y;
        const int zb = tzi * B->tz, ze = min(zb + B->tz, sa.d.nz);
        if (x < sa.d.nx && y < sa.d.ny) {
            for (int z = zb; z < ze; ++z) {
                if (sub == 0)
                    prim_point<LD_CG, T, T>(sa, x, y, z);
                else if (sub == 1)
                    grad_point<LD_CG, T, T, R, VB>(sa, x, y, z);
                else
                    resid_point<LD_CG, T, T, R, 0, VB>(sa, x, y, z);
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(P.done + inst, 1u);
        }
    }
}

// FP32 ensembles: the same work-item scheme over the z-march stage (items:
// instance x column tile x z chunk, phases: flux then residual per RK stage,
// 6 per step).  Each CTA keeps its shared-memory plane ring and mbarriers for
// the whole launch; the barrier phase bits carry over from item to item.
template <int R>
__global__ void __launch_bounds__(zm::NT, (R <= 2) ? 2 : 1) k_batch_z(const BatchParams P) {
    using G = zm::Geo<R>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ StageArgs sa;
    __shared__ long long item_s;
    __shared__ int stop_s;
    __shared__ __align__(8) unsigned long long bars[G::NS];
    zm::FluxSmem<R> &SF = *reinterpret_cast<zm::FluxSmem<R> *>(smem_raw);
    zm::RhsSmem<R> &SR = *reinterpret_cast<zm::RhsSmem<R> *>(smem_raw);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < G::NS; ++s) zm::bar_init(zm::smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;
    while (true) {
        if (tid == 0) {
            item_s = (long long)atomicAdd(P.counter, 1ull);
            stop_s = ld_volatile_i32(P.err) != 0;
        }
        __syncthreads();
        const long long k = item_s;
        if (k >= P.total_items || stop_s) break;
        const long long seq = k / P.tiles_total;
        const int rem = (int)(k - seq * P.tiles_total);
        int inst = 0;
        while (rem >= P.prefix[inst + 1]) ++inst;
        const int tile = rem - P.prefix[inst];
        const int tiles_i = P.prefix[inst + 1] - P.prefix[inst];
        const BatchInst *B = P.rec[inst];
        const int step = (int)(seq / 6), ph = (int)(seq % 6), stage = ph / 2, sub = ph % 2;
        if (tid == 0) {
            const unsigned target = P.inject_stall ? 0xffffffffu : (unsigned)(seq * tiles_i);
            if (ld_acquire_u32(P.done + inst) < target) {
                const unsigned long long t0 = globaltimer();
                unsigned nap = 32;  // exponential backoff: many CTAs poll one counter
                while (true) {
                    if (ld_volatile_i32(P.err)) {
                        stop_s = 1;
                        break;
                    }
                    if (ld_acquire_u32(P.done + inst) >= target) break;
                    if (globaltimer() - t0 > (unsigned long long)P.timeout_ns) {
                        atomicExch(P.err, 1);
                        stop_s = 1;
                        break;
                    }
                    __nanosleep(nap);
                    nap = nap < 2048 ? 2 * nap : 2048;
                }
            }
        }
        const int par = (P.p0[inst] + step) & 1;
        {
            const int *src = reinterpret_cast<const int *>(&B->st[par][stage]);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int w = tid; w < (int)(sizeof(StageArgs) / sizeof(int)); w += zm::NT) dst[w] = src[w];
        }
        __syncthreads();
        if (stop_s) break;
        // the TMA loads below (async proxy) read planes that other CTAs wrote
        // with ordinary stores before the acquire above
        if (tid == 0) asm volatile("fence.proxy.async.global;" ::: "memory");
        const int txi = tile % B->tiles_x, tyi = (tile / B->tiles_x) % B->tiles_y, tzi = tile / (B->tiles_x * B->tiles_y);
        const int x0 = txi * zm::TX, y0 = tyi * zm::TY, z0 = tzi * B->tz, z1 = min(z0 + B->tz, sa.d.nz);
        const zm::ZTma &tm = B->tma[B->zsrc[par][stage]][sub];
        if (sub == 0)
            zm::zflux_body<R, true>(sa, tm, x0, y0, z0, z1, SF, bars, phase);
        else
            zm::zrhs_body<R, true>(sa, tm, x0, y0, z0, z1, SR, bars, phase);
        if (tid == 0) {
            __threadfence();
            atomicAdd(P.done + inst, 1u);
        }
    }
}

template <int R>
static cudaError_t launch_batch_z(const BatchParams &P, cudaStream_t st) {
    constexpr size_t sm = zm::rhs_smem<R>() > zm::flux_smem<R>() ? zm::rhs_smem<R>() : zm::flux_smem<R>();
    int per_sm = 0, sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_batch_z<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_z<R>, zm::NT, sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)per_sm * sms;
    if (blocks > P.total_items) blocks = P.total_items > 0 ? P.total_items : 1;
    k_batch_z<R><<<(unsigned)blocks, zm::NT, sm, st>>>(P);
    return cudaGetLastError();
}

template <typename T, int R, bool VB>
static cudaError_t launch_batch_t(const BatchParams &P, cudaStream_t st) {
    int per_sm = 0, sms = 0, dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    if constexpr (is_dd<T>)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_dd<R, VB>, BX * BY, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<T, R, VB>, BX * BY, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    long long blocks = (long long)per_sm * sms;
    if (blocks > P.total_items) blocks = P.total_items > 0 ? P.total_items : 1;
    if constexpr (is_dd<T>)
        k_batch_dd<R, VB><<<(unsigned)blocks, dim3(BX, BY, 1), 0, st>>>(P);
    else
        k_batch<T, R, VB><<<(unsigned)blocks, dim3(BX, BY, 1), 0, st>>>(P);
    return cudaGetLastError();
}

template <int R>
static cudaError_t launch_batch_r(const BatchParams &P, int precision, int visc_form, int zmode, cudaStream_t st) {
    if constexpr (R <= 4) {
        if (zmode) return launch_batch_z<R>(P, st);
    }
    if (precision == OSB_FP64)
        return visc_form == OSB_VISC_B ? launch_batch_t<double, R, true>(P, st) : launch_batch_t<double, R, false>(P, st);
    if (precision == OSB_DF64)
        return visc_form == OSB_VISC_B ? launch_batch_t<dd, R, true>(P, st) : launch_batch_t<dd, R, false>(P, st);
    return visc_form == OSB_VISC_B ? launch_batch_t<float, R, true>(P, st) : launch_batch_t<float, R, false>(P, st);
}

cudaError_t launch_batch(const BatchParams &P, int order, int precision, int visc_form, int zmode, cudaStream_t st) {
    switch (order / 2) {
        case 1: return launch_batch_r<1>(P, precision, visc_form, zmode, st);
        case 2: return launch_batch_r<2>(P, precision, visc_form, zmode, st);
        case 3: return launch_batch_r<3>(P, precision, visc_form, zmode, st);
        case 4: return launch_batch_r<4>(P, precision, visc_form, zmode, st);
        case 5: return launch_batch_r<5>(P, precision, visc_form, zmode, st);
        case 6: return launch_batch_r<6>(P, precision, visc_form, zmode, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace osb
