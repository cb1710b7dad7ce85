// closure.cu -- learned residual correction for coarse grids: a 3-layer
// 3x3x3 periodic convolution network (5 -> H -> H -> 5, ReLU, H = 32) whose
// output is added to the residual R in every RK stage, and the kernels that
// train it: forward, backward (data and weight gradients), MSE loss, Adam.
//
// Arithmetic: BF16 weights and activations, FP32 accumulation on the tensor
// cores (mma.m16n8k16 BF16 tiles, implicit GEMM: M = grid points, N = output
// channels, K = 27 taps x input channels).  Activations are channels-last,
// channel counts padded to multiples of 8/16 with zeros.
//
// Also here: the box filter that maps a fine grid onto a coarse one (the
// training data), and the per-channel normalisation of inputs and targets.
#include <cuda_bf16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "osb_internal.cuh"

namespace osb {
namespace cl {

// brick of points handled by one CTA of the convolution kernels
constexpr int PX = 8, PY = 4, PZ = 4, NP = PX * PY * PZ;  // 128 points
constexpr int HX = PX + 2, HY = PY + 2, HZ = PZ + 2, NH = HX * HY * HZ;

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint16_t bf16_bits(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
__device__ __forceinline__ float bf16_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// ---------------------------------------------------------------------------
// Convolution y[p][co] = sum_k sum_ci W[k][co][ci] in[p + off(k)][ci]
//   EPI_RELU : + bias, ReLU, store BF16            (hidden layers)
//   EPI_LIN  : + bias, store FP32                  (output layer)
//   EPI_MASK : * [mask[p][co] > 0], store BF16     (data gradient through ReLU)
// in: BF16 [N][CI]; W: BF16 [27][CO][CI] (tap k = (dz+1)*9 + (dy+1)*3 + dx+1).
// ---------------------------------------------------------------------------
enum { EPI_RELU = 0, EPI_LIN = 1, EPI_MASK = 2 };

// 16-byte global -> shared copy that skips the registers (and L1).
__device__ __forceinline__ void tc_cp_async16(void *smem, const void *gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(256) k_conv(int nx, int ny, int nz, const uint16_t *__restrict__ in,
                                              const uint16_t *__restrict__ W, const float *__restrict__ bias,
                                              const uint16_t *__restrict__ mask, void *__restrict__ out) {
    constexpr int SI = CI + 8;  // padded per-point stride (bank-conflict free fragments)
    constexpr int SW = CI + 8;
    extern __shared__ __align__(16) uint16_t smem[];
    uint16_t *in_s = smem;             // [NH][SI]
    uint16_t *w_s = smem + NH * SI;    // [27][CO][SW]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bx = nx / PX, by = ny / PY;
    const int brick = blockIdx.x;
    const int x0 = (brick % bx) * PX, y0 = ((brick / bx) % by) * PY, z0 = (brick / (bx * by)) * PZ;

    // halo tile of the input (16-byte chunks, periodic wrap)
    constexpr int CH = CI / 8;  // 16-byte chunks per point
    for (int e = tid; e < NH * CH; e += 256) {
        const int hp = e / CH, ch = e - hp * CH;
        const int hx = hp % HX, hy = (hp / HX) % HY, hz = hp / (HX * HY);
        const int gx = wrapi(x0 + hx - 1, nx), gy = wrapi(y0 + hy - 1, ny), gz = wrapi(z0 + hz - 1, nz);
        const size_t gp = ((size_t)gz * ny + gy) * nx + gx;
        tc_cp_async16(in_s + hp * SI + ch * 8, in + gp * CI + ch * 8);
    }
    for (int e = tid; e < 27 * CO * CH; e += 256) {
        const int row = e / CH, ch = e - row * CH;  // row = k*CO + co
        tc_cp_async16(w_s + row * SW + ch * 8, W + row * CI + ch * 8);
    }
    cp_async_wait_all();
    __syncthreads();

    const int g = lane >> 2, tg = lane & 3;
    const int p0 = warp * 16 + g, p1 = p0 + 8;
    const int px0 = p0 % PX, py0 = (p0 / PX) % PY, pz0 = p0 / (PX * PY);
    const int px1 = p1 % PX, py1 = (p1 / PX) % PY, pz1 = p1 / (PX * PY);
    constexpr int NT = CO / 8;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;

#pragma unroll 1
    for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        const int h0 = ((pz0 + 1 + dz) * HY + (py0 + 1 + dy)) * HX + (px0 + 1 + dx);
        const int h1 = ((pz1 + 1 + dz) * HY + (py1 + 1 + dy)) * HX + (px1 + 1 + dx);
#pragma unroll
        for (int s = 0; s < CI / 16; ++s) {
            uint32_t a[4];
            a[0] = *reinterpret_cast<const uint32_t *>(in_s + h0 * SI + s * 16 + tg * 2);
            a[1] = *reinterpret_cast<const uint32_t *>(in_s + h1 * SI + s * 16 + tg * 2);
            a[2] = *reinterpret_cast<const uint32_t *>(in_s + h0 * SI + s * 16 + 8 + tg * 2);
            a[3] = *reinterpret_cast<const uint32_t *>(in_s + h1 * SI + s * 16 + 8 + tg * 2);
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const uint16_t *wr = w_s + (k * CO + j * 8 + g) * SW + s * 16 + tg * 2;
                uint32_t b[2];
                b[0] = *reinterpret_cast<const uint32_t *>(wr);
                b[1] = *reinterpret_cast<const uint32_t *>(wr + 8);
                mma_bf16(acc[j], a, b);
            }
        }
    }

    // epilogue
    const size_t gp0 = ((size_t)(z0 + pz0) * ny + (y0 + py0)) * nx + (x0 + px0);
    const size_t gp1 = ((size_t)(z0 + pz1) * ny + (y0 + py1)) * nx + (x0 + px1);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        const int c0 = j * 8 + tg * 2;
        float v[4] = {acc[j][0], acc[j][1], acc[j][2], acc[j][3]};
        if (EPI != EPI_MASK) {
            v[0] += bias[c0];
            v[1] += bias[c0 + 1];
            v[2] += bias[c0];
            v[3] += bias[c0 + 1];
        }
        if (EPI == EPI_RELU) {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = fmaxf(v[q], 0.f);
        }
        if (EPI == EPI_MASK) {
            if (!(bf16_val(mask[gp0 * CO + c0]) > 0.f)) v[0] = 0.f;
            if (!(bf16_val(mask[gp0 * CO + c0 + 1]) > 0.f)) v[1] = 0.f;
            if (!(bf16_val(mask[gp1 * CO + c0]) > 0.f)) v[2] = 0.f;
            if (!(bf16_val(mask[gp1 * CO + c0 + 1]) > 0.f)) v[3] = 0.f;
        }
        if (EPI == EPI_LIN) {
            float *o = static_cast<float *>(out);
            o[gp0 * CO + c0] = v[0];
            o[gp0 * CO + c0 + 1] = v[1];
            o[gp1 * CO + c0] = v[2];
            o[gp1 * CO + c0 + 1] = v[3];
        } else {
            uint16_t *o = static_cast<uint16_t *>(out);
            *reinterpret_cast<uint32_t *>(o + gp0 * CO + c0) = (uint32_t)bf16_bits(v[0]) | ((uint32_t)bf16_bits(v[1]) << 16);
            *reinterpret_cast<uint32_t *>(o + gp1 * CO + c0) = (uint32_t)bf16_bits(v[2]) | ((uint32_t)bf16_bits(v[3]) << 16);
        }
    }
}

// ---------------------------------------------------------------------------
// The same convolution on the 5th-generation tensor cores (tcgen05): one CTA
// of 128 threads per brick of 8 x 16 x 1 points (M = 128 rows of the GEMM),
// N = CO = 32 output channels, K = 27 taps x CI.  Operands in shared memory in
// the K-major, no-swizzle core-matrix layout (8 rows x 16 bytes):
//   A (input halo 10 x 18 x 3): [CI/8 chunks][540 positions][8 ch]; the 8 rows
//     of a core matrix are 8 consecutive x positions of one halo row, so for a
//     tap the descriptor strides are constant: 160 B between core matrices along
//     M (next y row), 8640 B along K (next channel chunk);
//   B (weights): [27 taps][CI/8 chunks][CO][8 ch]; 128 B along N, CO*16 B along K.
// One thread issues the 27*CI/16 MMAs into an FP32 accumulator of 32 TMEM
// columns; tcgen05.commit signals an mbarrier; each warp then reads its 32
// rows (points) with tcgen05.ld and applies the epilogue.
// ---------------------------------------------------------------------------
constexpr int TBX = 8, TBY = 16, THX = TBX + 2, THY = TBY + 2, THZ = 3, THN = THX * THY * THZ;  // 540
constexpr unsigned TC_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

template <int CO>
__host__ __device__ constexpr uint32_t tc_idesc() {
    // D FP32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), both K-major,
    // N >> 3 at bits 17-22, M >> 4 at bits 24-28 (M = 128)
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(CO >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

template <int CI, int CO>
constexpr size_t tc_smem_used() {
    return (size_t)THN * CI * 2 + (size_t)27 * CI * CO * 2;
}

template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(128) k_conv_tc(int nx, int ny, int nz, const uint16_t *__restrict__ in,
                                                 const uint16_t *__restrict__ W, const float *__restrict__ bias,
                                                 const uint16_t *__restrict__ mask, void *__restrict__ out,
                                                 int *__restrict__ err) {
    static_assert(CO == 32, "tensor-core path built for 32 output channels");
    constexpr int NCH = CI / 8;
    extern __shared__ __align__(128) uint8_t tsm[];
    uint8_t *A = tsm;
    uint8_t *B = tsm + THN * CI * 2;
    __shared__ uint32_t taddr_s;
    __shared__ __align__(8) uint64_t bar;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bx = nx / TBX, by = ny / TBY;
    const int brick = blockIdx.x;
    const int x0 = (brick % bx) * TBX, y0 = ((brick / bx) % by) * TBY, z0 = brick / (bx * by);

    if (warp == 0) {
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(&taddr_s);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(sa));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    const uint32_t bar_a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // halo tile -> A (chunk-major core-matrix rows of 16 bytes)
    for (int e = tid; e < THN * NCH; e += 128) {
        const int pos = e / NCH, ch = e - pos * NCH;
        const int hx = pos % THX, hy = (pos / THX) % THY, hz = pos / (THX * THY);
        const int gx = wrapi(x0 + hx - 1, nx), gy = wrapi(y0 + hy - 1, ny), gz = wrapi(z0 + hz - 1, nz);
        const size_t gp = ((size_t)gz * ny + gy) * nx + gx;
        tc_cp_async16(A + ((size_t)ch * THN + pos) * 16, in + gp * CI + ch * 8);
    }
    // weights [27][CO][CI] -> B [27][NCH][CO][8]
    for (int e = tid; e < 27 * CO * NCH; e += 128) {
        const int k = e / (CO * NCH), n = (e / NCH) % CO, ch = e % NCH;
        tc_cp_async16(B + (((size_t)k * NCH + ch) * CO + n) * 16, W + ((size_t)k * CO + n) * CI + ch * 8);
    }
    // all of this thread's copies in flight at once, then one wait
    cp_async_wait_all();
    // make the shared-memory writes visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = taddr_s;

    if (tid == 0) {
        const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(A), b0 = (uint32_t)__cvta_generic_to_shared(B);
        constexpr uint32_t idesc = tc_idesc<CO>();
        for (int k = 0; k < 27; ++k) {
            const int dx = k % 3, dy = (k / 3) % 3, dz = k / 9;  // halo offsets of brick point (0, 0)
            const uint32_t pos0 = (uint32_t)((dz * THY + dy) * THX + dx);
#pragma unroll
            for (int s = 0; s < CI / 16; ++s) {
                const uint64_t ad = tc_desc(a0 + ((uint32_t)(2 * s) * THN + pos0) * 16, THN * 16, THX * 16);
                const uint64_t bd = tc_desc(b0 + ((uint32_t)(k * NCH + 2 * s) * CO) * 16, CO * 16, 128);
                const uint32_t acc = (k | s) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(taddr),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                     : "memory");
    }
    // bounded wait for the accumulator (phase 0 of the mbarrier)
    {
        uint32_t done = 0;
        for (unsigned it = 0; it < TC_WAIT_LIMIT && !done; ++it) {
            asm volatile(
                "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                : "=r"(done)
                : "r"(bar_a), "r"(0u)
                : "memory");
            if (!done) __nanosleep(64);
        }
        if (!done && lane == 0) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr + ((uint32_t)(warp * 32) << 16)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");

    // epilogue: this thread's point is row 32*warp + lane of the brick
    const int p = warp * 32 + lane, px = p % TBX, py = p / TBX;
    const size_t gp = ((size_t)z0 * ny + (y0 + py)) * nx + (x0 + px);
    float v[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
    if (EPI != EPI_MASK) {
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] += bias[c];
    }
    if (EPI == EPI_RELU) {
#pragma unroll
        for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c], 0.f);
    }
    if (EPI == EPI_MASK) {
        const uint4 *mk = reinterpret_cast<const uint4 *>(mask + gp * CO);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 m4 = mk[q];
            const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const uint16_t mb = (uint16_t)(mw[h / 2] >> (16 * (h & 1)));
                if (!(bf16_val(mb) > 0.f)) v[q * 8 + h] = 0.f;
            }
        }
    }
    uint4 *o = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(out) + gp * CO);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t w[4];
#pragma unroll
        for (int h = 0; h < 4; ++h)
            w[h] = (uint32_t)bf16_bits(v[q * 8 + 2 * h]) | ((uint32_t)bf16_bits(v[q * 8 + 2 * h + 1]) << 16);
        o[q] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(taddr));
}

// ---------------------------------------------------------------------------
// The tcgen05 convolution as a z-march: one CTA owns a column of 8 x 16 bricks
// and a chunk of z planes.  The weights stay in shared memory for the whole
// chunk; input planes (the 10 x 18 haloed tile of one z, CI channels) stream
// through a ring of TC_SLOTS slots two planes ahead of use (cp.async, wrapped
// periodically); two TMEM accumulators alternate between planes, so one
// thread of a fifth warp issues the 27 * CI/16 MMAs of output plane z while
// warps 0-3 read the accumulator of plane z-1 and write it out (a thread that
// queues many MMAs can stall at issue: kept apart, that stall does not hold
// back an epilogue).  Per output plane:
//   (a) every thread waits for its copies of plane z+1, fences them to the
//       async proxy, block barrier (which also means the epilogue of plane z-2
//       has read accumulator z&1);
//   (b) warp 4 issues plane z's MMAs (taps dz = -1, 0, +1 read the slots of
//       planes z-1, z, z+1) and commits them to mbarrier z&1, then goes on to
//       the next barrier;
//   (c) warps 0-3 wait for plane z-1's commit (bounded), which also frees the
//       slot of plane z-2 (its last reader was plane z-1's MMAs);
//   (d) copies of plane z+3 go into that slot;
//   (e) epilogue of plane z-1.
// Shared memory at CI = 32: weights 55.3 KB + ring 5 x 11.5 KB: two CTAs per SM.
// The output layer (CO = 8, FP32 out) runs as N = 16 MMAs against weights
// padded with zero rows.
// ---------------------------------------------------------------------------
constexpr int TC_SLOTS = 5;
constexpr int TC_THREADS = 160;  // warps 0-3: copies and epilogue (one TMEM lane quarter each); warp 4: MMA issue
constexpr int TPP = THX * THY;  // 180 haloed positions of one plane

// z planes per CTA: the chunk count c minimising (CTA rounds of two per SM)
// x (planes per CTA + 3 for the ring start); OSB_TC_ZCHUNK overrides.
inline int tc_zchunk(int cols, int nz) {
    if (const char *e = getenv("OSB_TC_ZCHUNK")) {
        const int v = atoi(e);
        if (v > 0) return v < nz ? v : nz;
    }
    constexpr long long slots = 2 * 152;
    long long best = -1;
    int bz = nz;
    for (int c = 1; c <= nz; ++c) {
        const int zc = (nz + c - 1) / c;
        const int cc = (nz + zc - 1) / zc;
        const long long rounds = ((long long)cols * cc + slots - 1) / slots;
        const long long cost = rounds * (zc + 3);
        if (best < 0 || cost < best) best = cost, bz = zc;
    }
    return bz;
}

// MMA width N for CO output channels: M = 128 takes N in multiples of 16
template <int CO>
__host__ __device__ constexpr int tc_n() {
    return CO < 16 ? 16 : CO;
}

template <int CI, int CO>
constexpr size_t tcp_smem() {
    return (size_t)27 * CI * tc_n<CO>() * 2 + (size_t)TC_SLOTS * TPP * CI * 2;
}

// TMEM -> registers: this warp's 32 lanes (points), NC consecutive columns
template <int NC>
__device__ __forceinline__ void tm_ld(uint32_t taddr, uint32_t (&r)[NC]) {
    static_assert(NC == 8 || NC == 32, "8 or 32 columns");
    if constexpr (NC == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc, bool accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc), "r"((uint32_t)accumulate));
}

__device__ __forceinline__ bool tc_bar_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    for (unsigned it = 0; it < TC_WAIT_LIMIT && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (!done && it > 16) __nanosleep(32);
    }
    return done != 0;
}

template <int CI, int CO, int EPI>
__global__ void __launch_bounds__(TC_THREADS) k_conv_tcp(int nx, int ny, int nz, int zchunk, const uint16_t *__restrict__ in,
                                                  const uint16_t *__restrict__ W, const float *__restrict__ bias,
                                                  const uint16_t *__restrict__ mask, void *__restrict__ out,
                                                  int *__restrict__ err) {
    static_assert((CO == 32 && EPI != EPI_LIN) || (CO == 8 && EPI == EPI_LIN), "hidden or output layer");
    constexpr int NCH = CI / 8;
    constexpr int NT = tc_n<CO>();          // MMA N and TMEM columns per accumulator
    constexpr uint32_t TCOLS = 2 * NT < 32 ? 32 : 2 * NT;  // allocation: a power of two >= 32
    constexpr uint32_t SLOT = (uint32_t)TPP * CI * 2;  // bytes of one ring slot: [NCH][180][8 ch]
    extern __shared__ __align__(128) uint8_t tsm[];
    uint8_t *Bw = tsm;                          // weights [27][NCH][NT][8 ch], rows >= CO zero
    uint8_t *A = tsm + (size_t)27 * CI * NT * 2;  // ring
    __shared__ uint32_t taddr_s;
    __shared__ __align__(8) uint64_t bars[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bx = nx / TBX, by = ny / TBY;
    const int colx = blockIdx.x % (bx * by), chunk = blockIdx.x / (bx * by);
    const int x0 = (colx % bx) * TBX, y0 = (colx / bx) * TBY;
    const int z0 = chunk * zchunk, z1 = min(z0 + zchunk, nz);

    if (warp == 0) {
        const uint32_t sa = (uint32_t)__cvta_generic_to_shared(&taddr_s);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sa), "n"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[0]);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // weights [27][CO][CI] -> [27][NCH][NT][8], with the first plane's copies
    for (int e = tid; e < 27 * NT * NCH && warp < 4; e += 128) {
        const int k = e / (NT * NCH), n = (e / NCH) % NT, ch = e % NCH;
        uint8_t *dst = Bw + (((size_t)k * NCH + ch) * NT + n) * 16;
        if (n < CO)
            tc_cp_async16(dst, W + ((size_t)k * CO + n) * CI + ch * 8);
        else
            *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    // input plane zp (any integer, wrapped) -> its ring slot; one commit group per plane
    auto load_plane = [&](int zp) {
        const int slot = ((zp - z0 + 1) % TC_SLOTS + TC_SLOTS) % TC_SLOTS;  // plane z0-1 in slot 0
        const int gz = wrapi(wrapi(zp, nz), nz);
        uint8_t *As = A + (size_t)slot * SLOT;
        for (int e = tid; e < TPP * NCH && warp < 4; e += 128) {
            const int pos = e / NCH, ch = e - pos * NCH;
            const int hx = pos % THX, hy = pos / THX;
            const int gx = wrapi(x0 + hx - 1, nx), gy = wrapi(y0 + hy - 1, ny);
            const size_t gp = ((size_t)gz * ny + gy) * nx + gx;
            tc_cp_async16(As + ((size_t)ch * TPP + pos) * 16, in + gp * CI + ch * 8);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    load_plane(z0 - 1);
    load_plane(z0);
    load_plane(z0 + 1);
    load_plane(z0 + 2);
    __syncthreads();  // TMEM address and barrier initialisation visible
    const uint32_t taddr = taddr_s;
    const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(A), b0 = (uint32_t)__cvta_generic_to_shared(Bw);
    constexpr uint32_t idesc = tc_idesc<NT>();
    const uint64_t adesc0 = tc_desc(a0, TPP * 16, THX * 16), bdesc0 = tc_desc(b0, NT * 16, 128);
    const int p = warp * 32 + lane, px = p % TBX, py = p / TBX;  // this thread's row of the brick

    auto epilogue = [&](int j) {  // output plane z0 + j from accumulator j & 1
        uint32_t r[CO];
        tm_ld<CO>(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j & 1) * NT, r);
        const size_t gp = ((size_t)(z0 + j) * ny + (y0 + py)) * nx + (x0 + px);
        float v[CO];
#pragma unroll
        for (int c = 0; c < CO; ++c) v[c] = __uint_as_float(r[c]);
        if (EPI != EPI_MASK) {
#pragma unroll
            for (int c = 0; c < CO; ++c) v[c] += bias[c];
        }
        if (EPI == EPI_RELU) {
#pragma unroll
            for (int c = 0; c < CO; ++c) v[c] = fmaxf(v[c], 0.f);
        }
        if (EPI == EPI_MASK) {
            const uint4 *mk = reinterpret_cast<const uint4 *>(mask + gp * CO);
#pragma unroll
            for (int q = 0; q < CO / 8; ++q) {
                const uint4 m4 = mk[q];
                const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
#pragma unroll
                for (int h = 0; h < 8; ++h) {
                    const uint16_t mb = (uint16_t)(mw[h / 2] >> (16 * (h & 1)));
                    if (!(bf16_val(mb) > 0.f)) v[q * 8 + h] = 0.f;
                }
            }
        }
        if (EPI == EPI_LIN) {  // FP32 out
            float4 *o = reinterpret_cast<float4 *>(static_cast<float *>(out) + gp * CO);
#pragma unroll
            for (int q = 0; q < CO / 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {  // BF16 out
            uint4 *o = reinterpret_cast<uint4 *>(static_cast<uint16_t *>(out) + gp * CO);
#pragma unroll
            for (int q = 0; q < CO / 8; ++q) {
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h)
                    w[h] = (uint32_t)bf16_bits(v[q * 8 + 2 * h]) | ((uint32_t)bf16_bits(v[q * 8 + 2 * h + 1]) << 16);
                o[q] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    };

    bool ok = true;
#pragma unroll 1
    for (int j = 0; j < z1 - z0; ++j) {
        // (a) planes up to z+1 in shared memory, visible to the tensor cores
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // (b) plane z's MMAs into accumulator j & 1.  Descriptors are the base
        // descriptors plus constant offsets (the 14-bit address field holds
        // the whole shared window, so the sums never carry out of it).
        if (tid == 128) {
            const uint32_t acc_addr = taddr + (uint32_t)(j & 1) * NT;
            uint64_t adz[3];
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)  // plane z - 1 + dz lives in slot (j + dz) % TC_SLOTS
                adz[dz] = adesc0 + (uint64_t)((((j + dz) % TC_SLOTS) * SLOT) >> 4);
#pragma unroll
            for (int k = 0; k < 27; ++k) {
                const int dx = k % 3, dy = (k / 3) % 3, dz = k / 9;
#pragma unroll
                for (int s = 0; s < CI / 16; ++s) {
                    const uint64_t ad = adz[dz] + (uint64_t)((((2 * s) * TPP + dy * THX + dx) * 16) >> 4);
                    const uint64_t bd = bdesc0 + (uint64_t)((((k * NCH + 2 * s) * NT) * 16) >> 4);
                    tc_mma(acc_addr, ad, bd, idesc, (k | s) != 0);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar0 + 8u * (uint32_t)(j & 1))
                         : "memory");
        }
        if (warp == 4) continue;  // the MMA warp: on to the next plane's barrier
        // (c) plane z-1's MMAs done: its accumulator is ready, the slot of plane z-2 free
        if (j >= 1) {
            if (!tc_bar_wait(bar0 + 8u * (uint32_t)((j - 1) & 1), (uint32_t)(((j - 1) >> 1) & 1))) ok = false;
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below is warp-collective
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        // (d) plane z+3 into the slot of plane z-2
        if (z0 + j + 3 <= z1)
            load_plane(z0 + j + 3);
        else
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        // (e) epilogue of plane z-1
        if (j >= 1 && ok) epilogue(j - 1);
    }
    const int last = z1 - z0 - 1;
    if (last >= 0 && warp < 4) {
        if (!tc_bar_wait(bar0 + 8u * (uint32_t)(last & 1), (uint32_t)((last >> 1) & 1))) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (ok) epilogue(last);
    }
    if (!ok && lane == 0) atomicExch(err, 1);
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(TCOLS));
}

template <int CI, int CO>
constexpr size_t conv_smem() {
    return (size_t)(NH * (CI + 8) + 27 * CO * (CI + 8)) * sizeof(uint16_t);
}

// ---------------------------------------------------------------------------
// Weight gradient dW[k][co][ci] = sum_p dz[p][co] h[p + off(k)][ci] and bias
// gradient db[co] = sum_p dz[p][co].  GEMM with M = co (16-row tiles), N = ci
// (8), K = points of a brick; CTAs loop over bricks and write one partial each,
// reduced in fixed order by k_wgrad_reduce (deterministic).
// dz: BF16 [N][CO]; h: BF16 [N][CI].  CO multiple of 16, CI multiple of 8.
// ---------------------------------------------------------------------------
template <int CI, int CO>
__global__ void __launch_bounds__(256) k_wgrad(int nx, int ny, int nz, const uint16_t *__restrict__ dz,
                                               const uint16_t *__restrict__ h, float *__restrict__ partial) {
    constexpr int SD = CO + 8, SH = CI + 8;
    constexpr int MT = CO / 16, NTL = CI / 8, TILES = 27 * MT * NTL;
    constexpr int TPW = (TILES + 7) / 8;
    extern __shared__ __align__(16) uint16_t smem[];
    uint16_t *dz_s = smem;               // [NP][SD]
    uint16_t *h_s = smem + NP * SD;      // [NH][SH]
    __shared__ float db_s[CO];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tg = lane & 3;
    const int bx = nx / PX, by = ny / PY, nbricks = bx * by * (nz / PZ);
    float acc[TPW][4];
#pragma unroll
    for (int t = 0; t < TPW; ++t) acc[t][0] = acc[t][1] = acc[t][2] = acc[t][3] = 0.f;
    float dbacc = 0.f;

    for (int brick = blockIdx.x; brick < nbricks; brick += gridDim.x) {
        const int x0 = (brick % bx) * PX, y0 = ((brick / bx) % by) * PY, z0 = (brick / (bx * by)) * PZ;
        __syncthreads();
        for (int e = tid; e < NP * (CO / 8); e += 256) {
            const int p = e / (CO / 8), ch = e - p * (CO / 8);
            const int gx = x0 + p % PX, gy = y0 + (p / PX) % PY, gz = z0 + p / (PX * PY);
            const size_t gp = ((size_t)gz * ny + gy) * nx + gx;
            tc_cp_async16(dz_s + p * SD + ch * 8, dz + gp * CO + ch * 8);
        }
        for (int e = tid; e < NH * (CI / 8); e += 256) {
            const int hp = e / (CI / 8), ch = e - hp * (CI / 8);
            const int hx = hp % HX, hy = (hp / HX) % HY, hz = hp / (HX * HY);
            const int gx = wrapi(x0 + hx - 1, nx), gy = wrapi(y0 + hy - 1, ny), gz = wrapi(z0 + hz - 1, nz);
            const size_t gp = ((size_t)gz * ny + gy) * nx + gx;
            tc_cp_async16(h_s + hp * SH + ch * 8, h + gp * CI + ch * 8);
        }
        cp_async_wait_all();
        __syncthreads();
        if (tid < CO)
            for (int p = 0; p < NP; ++p) dbacc += bf16_val(dz_s[p * SD + tid]);
#pragma unroll
        for (int t = 0; t < TPW; ++t) {
            const int tile = warp + 8 * t;
            if (tile >= TILES) break;
            const int k = tile / (MT * NTL), mt = (tile / NTL) % MT, nt = tile % NTL;
            const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dzo = k / 9 - 1;
#pragma unroll
            for (int s = 0; s < NP / 16; ++s) {
                // A[m = co][kk = point], B[kk = point][n = ci]
                const int pa = s * 16 + tg * 2;
                uint32_t a[4], b[2];
                const int co0 = mt * 16 + g, co1 = co0 + 8;
                a[0] = (uint32_t)dz_s[pa * SD + co0] | ((uint32_t)dz_s[(pa + 1) * SD + co0] << 16);
                a[1] = (uint32_t)dz_s[pa * SD + co1] | ((uint32_t)dz_s[(pa + 1) * SD + co1] << 16);
                a[2] = (uint32_t)dz_s[(pa + 8) * SD + co0] | ((uint32_t)dz_s[(pa + 9) * SD + co0] << 16);
                a[3] = (uint32_t)dz_s[(pa + 8) * SD + co1] | ((uint32_t)dz_s[(pa + 9) * SD + co1] << 16);
                const int ci = nt * 8 + g;
                int hq[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int p = pa + (q & 1) + (q >> 1) * 8;
                    const int px = p % PX, py = (p / PX) % PY, pz = p / (PX * PY);
                    hq[q] = ((pz + 1 + dzo) * HY + (py + 1 + dy)) * HX + (px + 1 + dx);
                }
                b[0] = (uint32_t)h_s[hq[0] * SH + ci] | ((uint32_t)h_s[hq[1] * SH + ci] << 16);
                b[1] = (uint32_t)h_s[hq[2] * SH + ci] | ((uint32_t)h_s[hq[3] * SH + ci] << 16);
                mma_bf16(acc[t], a, b);
            }
        }
    }
    // write this CTA's partial: [tile][16 x 8] in (row, col) order, then db
    float *pp = partial + (size_t)blockIdx.x * (TILES * 128 + CO);
#pragma unroll
    for (int t = 0; t < TPW; ++t) {
        const int tile = warp + 8 * t;
        if (tile >= TILES) break;
        float *o = pp + tile * 128;
        o[g * 8 + tg * 2] = acc[t][0];
        o[g * 8 + tg * 2 + 1] = acc[t][1];
        o[(g + 8) * 8 + tg * 2] = acc[t][2];
        o[(g + 8) * 8 + tg * 2 + 1] = acc[t][3];
    }
    if (tid < CO) db_s[tid] = dbacc;
    __syncthreads();
    if (tid < CO) pp[TILES * 128 + tid] = db_s[tid];
}

// Sums the per-CTA partials in index order into the FP32 master layout
// dW[co][ci][k] (real channels only) and db[co].
template <int CI, int CO>
__global__ void k_wgrad_reduce(const float *__restrict__ partial, int nparts, int co_real, int ci_real,
                               float *__restrict__ dW, float *__restrict__ db) {
    constexpr int MT = CO / 16, NTL = CI / 8, TILES = 27 * MT * NTL, STRIDE = TILES * 128 + CO;
    const int nw = co_real * ci_real * 27;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nw + co_real; e += gridDim.x * blockDim.x) {
        int src;
        if (e < nw) {
            const int co = e / (ci_real * 27), ci = (e / 27) % ci_real, k = e % 27;
            const int mt = co / 16, r = co % 16, nt = ci / 8, c = ci % 8;
            src = ((k * MT + mt) * NTL + nt) * 128 + r * 8 + c;
        } else {
            src = TILES * 128 + (e - nw);
        }
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += partial[(size_t)b * STRIDE + src];
        if (e < nw)
            dW[e] = (float)s;
        else
            db[e - nw] = (float)s;
    }
}

template <int CI, int CO>
constexpr size_t wgrad_smem() {
    return (size_t)(NP * (CO + 8) + NH * (CI + 8)) * sizeof(uint16_t);
}
template <int CI, int CO>
constexpr int wgrad_stride() {
    return 27 * (CO / 16) * (CI / 8) * 128 + CO;
}

// ---------------------------------------------------------------------------
// Point-wise kernels
// ---------------------------------------------------------------------------
// Normalised BF16 features x[p][c] = (Q_c - mean_c) * inv_std_c, c < 5, zero pad to 16.
template <typename S>
__global__ void k_features(int n, const S *__restrict__ Q, size_t qs, const float *__restrict__ nrm,
                           uint16_t *__restrict__ x) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        uint32_t w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) w[c] = 0;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float v = (float(Q[c * qs + p]) - nrm[c]) * nrm[5 + c];
            w[c / 2] |= (uint32_t)bf16_bits(v) << (16 * (c & 1));
        }
        uint4 *o = reinterpret_cast<uint4 *>(x + (size_t)p * 16);
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(0, 0, 0, 0);
    }
}

// Normalised FP32 targets t[p][c] = C*_c / out_std_c (c < 5), zero pad to 8.
__global__ void k_targets(int n, const double *__restrict__ C, size_t cs, const float *__restrict__ nrm,
                          float *__restrict__ t) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 8; ++c) t[(size_t)p * 8 + c] = c < 5 ? float(C[c * cs + p]) / nrm[10 + c] : 0.f;
    }
}

// MSE on the normalised output: loss partials and dy = 2 (y - t) / (5 N) (BF16, 16 channels).
__global__ void __launch_bounds__(256) k_mse(int n, const float *__restrict__ y, const float *__restrict__ t,
                                             uint16_t *__restrict__ dy, float *__restrict__ partial, float weight) {
    const float sc = 2.f * weight / (5.f * n);
    double s = 0.0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        uint32_t w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) w[c] = 0;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float d = y[(size_t)p * 8 + c] - t[(size_t)p * 8 + c];
            s += (double)d * d;
            w[c / 2] |= (uint32_t)bf16_bits(sc * d) << (16 * (c & 1));
        }
        uint4 *o = reinterpret_cast<uint4 *>(dy + (size_t)p * 16);
        o[0] = make_uint4(w[0], w[1], w[2], w[3]);
        o[1] = make_uint4(0, 0, 0, 0);
    }
    __shared__ double sm[256];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = (float)sm[0];
}

__global__ void k_sum_partials(const float *__restrict__ partial, int nparts, float scale, float *__restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += partial[b];
        *out = (float)(s * scale);
    }
}

// Correction added to R: C_m(p) = apply_m * out_std_m * y[p][m], in SoA (stride n).
// With the dissipative option (nrm[21] = 1) the momentum part never feeds
// kinetic energy at a point: where u . C_m > 0 its component along u is
// removed (C_m -= (u . C_m / |u|^2) u), the backscatter clipping of
// eddy-viscosity subgrid models.  u = rho u_i / rho from the stencil source.
template <typename S>
__global__ void k_closure_out(int n, const float *__restrict__ y, const float *__restrict__ nrm, float *__restrict__ C,
                              const S *__restrict__ Q, size_t qs) {
    const bool dissipative = nrm[21] > 0.5f;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        float c[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) c[k] = nrm[16 + k] * nrm[10 + k] * y[(size_t)p * 8 + k];
        if (dissipative) {
            const float ri = 1.f / float(Q[p]);
            const float u = float(Q[qs + p]) * ri, v = float(Q[2 * qs + p]) * ri, w = float(Q[3 * qs + p]) * ri;
            const float d = u * c[1] + v * c[2] + w * c[3], uu = u * u + v * v + w * w;
            if (d > 0.f && uu > 0.f) {
                const float s = d / uu;
                c[1] -= s * u;
                c[2] -= s * v;
                c[3] -= s * w;
            }
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) C[(size_t)k * n + p] = c[k];
    }
}

// FP32 master parameters -> BF16 forward weights Wf[k][co][ci] (padded) and
// data-gradient weights Wd[k][ci][co] = W[co][ci][26 - k] (flipped taps).
__global__ void k_prep_weights(const float *__restrict__ W, int co_real, int ci_real, int co_pad, int ci_pad,
                               uint16_t *__restrict__ Wf, uint16_t *__restrict__ Wd, int wd_ci_pad, int wd_co_pad) {
    const int total = 27 * co_pad * ci_pad;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int k = e / (co_pad * ci_pad), co = (e / ci_pad) % co_pad, ci = e % ci_pad;
        const float v = (co < co_real && ci < ci_real) ? W[(co * ci_real + ci) * 27 + k] : 0.f;
        Wf[e] = bf16_bits(v);
        if (Wd && ci < wd_ci_pad && co < wd_co_pad) Wd[((26 - k) * wd_ci_pad + ci) * wd_co_pad + co] = bf16_bits(v);
    }
}

__global__ void k_adam(int n, float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// Box filter: coarse[Z][Y][X] = mean of the f^3 fine points of the block.
__global__ void k_box_filter(const double *__restrict__ fine, size_t fs, int fnx, int fny, int f, int cnx, int cny,
                             int cnz, double *__restrict__ coarse, size_t cs) {
    const int nc = cnx * cny * cnz;
    const double inv = 1.0 / ((double)f * f * f);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 5 * nc; i += gridDim.x * blockDim.x) {
        const int m = i / nc, p = i - m * nc;
        const int X = p % cnx, Y = (p / cnx) % cny, Z = p / (cnx * cny);
        double s = 0.0;
        for (int dz = 0; dz < f; ++dz)
            for (int dy = 0; dy < f; ++dy) {
                const double *row = fine + m * fs + ((size_t)(Z * f + dz) * fny + (Y * f + dy)) * fnx + X * f;
                for (int dx = 0; dx < f; ++dx) s += row[dx];
            }
        coarse[m * cs + p] = s * inv;
    }
}

}  // namespace cl
}  // namespace osb

// ===========================================================================
// Host side
// ===========================================================================
namespace osb {
namespace cl {

constexpr int H = 32;  // hidden channels
// FP32 master parameters: W1[H][5][27] b1[H] W2[H][H][27] b2[H] W3[5][H][27] b3[5]
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * 5 * 27, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H * 27,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + 5 * H * 27, NPARAM = OFF_B3 + 5;
constexpr int NPART = 152 * 2;  // weight-gradient partials (CTAs of k_wgrad)

struct Buffers {
    uint16_t *x0, *h1, *h2, *dy, *dz2, *dz1;
    float *y, *t, *C, *part, *lpart, *nrm, *b3pad;
    int *tcerr;  // set when a tensor-core accumulator wait ran out
    uint16_t *wf1, *wf2, *wf3, *wd2, *wd3;
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Carves the workspace; returns the bytes needed (buffers set when base != nullptr).
size_t carve(char *base, int n, Buffers *B) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    Buffers b;
    b.x0 = (uint16_t *)take((size_t)n * 16 * 2);
    b.h1 = (uint16_t *)take((size_t)n * H * 2);
    b.h2 = (uint16_t *)take((size_t)n * H * 2);
    b.dy = (uint16_t *)take((size_t)n * 16 * 2);
    b.dz2 = (uint16_t *)take((size_t)n * H * 2);
    b.dz1 = (uint16_t *)take((size_t)n * H * 2);
    b.y = (float *)take((size_t)n * 8 * 4);
    b.t = (float *)take((size_t)n * 8 * 4);
    b.C = (float *)take((size_t)n * 5 * 4);
    b.part = (float *)take((size_t)NPART * wgrad_stride<32, 32>() * 4);
    b.lpart = (float *)take(NPART * 4);
    b.nrm = (float *)take(24 * 4);  // mean[5], 1/std[5], out_std[5], -, apply[5]
    b.b3pad = (float *)take(8 * 4);
    b.tcerr = (int *)take(16);
    b.wf1 = (uint16_t *)take(27 * H * 16 * 2);
    b.wf2 = (uint16_t *)take(27 * H * H * 2);
    b.wf3 = (uint16_t *)take(27 * 8 * H * 2);
    b.wd2 = (uint16_t *)take(27 * H * H * 2);
    b.wd3 = (uint16_t *)take(27 * H * 16 * 2);
    if (B) *B = b;
    return off;
}


// 1: tensor-core (tcgen05) z-marching convolutions where applicable; 2: the
// same MMAs one brick per CTA (k_conv_tc); 0: mma.sync only.  OSB_CLOSURE_MMA
// = "sync" | "brick" selects the others.
int g_tc_mode = -1;

template <int CI, int CO, int EPI>
cudaError_t conv(int nx, int ny, int nz, const uint16_t *in, const uint16_t *W, const float *bias, const uint16_t *mask,
                 void *out, int *tcerr, cudaStream_t st) {
    {
        const char *env = getenv("OSB_CLOSURE_MMA");
        g_tc_mode = !env ? 1 : strcmp(env, "sync") == 0 ? 0 : strcmp(env, "brick") == 0 ? 2 : 1;
    }
    if constexpr ((CO == 32 && EPI != EPI_LIN) || (CO == 8 && EPI == EPI_LIN)) {
        if constexpr (CO == 32) {
            if (g_tc_mode == 2 && ny % TBY == 0 && nx % TBX == 0 && tcerr) {
                constexpr size_t sm = tc_smem_used<CI, CO>();
                cudaError_t e = cudaFuncSetAttribute(k_conv_tc<CI, CO, EPI>,
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                if (e != cudaSuccess) return e;
                const int bricks = (nx / TBX) * (ny / TBY) * nz;
                k_conv_tc<CI, CO, EPI><<<bricks, 128, sm, st>>>(nx, ny, nz, in, W, bias, mask, out, tcerr);
                return cudaGetLastError();
            }
        }
        if (g_tc_mode == 1 && ny % TBY == 0 && nx % TBX == 0 && tcerr) {
            constexpr size_t sm = tcp_smem<CI, CO>();
            cudaError_t e = cudaFuncSetAttribute(k_conv_tcp<CI, CO, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)sm);
            if (e != cudaSuccess) return e;
            const int cols = (nx / TBX) * (ny / TBY);
            const int zc = tc_zchunk(cols, nz);
            const int ctas = cols * ((nz + zc - 1) / zc);
            k_conv_tcp<CI, CO, EPI><<<ctas, TC_THREADS, sm, st>>>(nx, ny, nz, zc, in, W, bias, mask, out, tcerr);
            return cudaGetLastError();
        }
    }
    const size_t sm = conv_smem<CI, CO>();
    cudaError_t e = cudaFuncSetAttribute(k_conv<CI, CO, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int bricks = (nx / PX) * (ny / PY) * (nz / PZ);
    k_conv<CI, CO, EPI><<<bricks, 256, sm, st>>>(nx, ny, nz, in, W, bias, mask, out);
    return cudaGetLastError();
}

template <int CI, int CO>
cudaError_t wgrad(int nx, int ny, int nz, const uint16_t *dz, const uint16_t *h, float *part, int co_real,
                  int ci_real, float *dW, float *db, cudaStream_t st) {
    const size_t sm = wgrad_smem<CI, CO>();
    cudaError_t e = cudaFuncSetAttribute(k_wgrad<CI, CO>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_wgrad<CI, CO><<<NPART, 256, sm, st>>>(nx, ny, nz, dz, h, part);
    k_wgrad_reduce<CI, CO><<<64, 256, 0, st>>>(part, NPART, co_real, ci_real, dW, db);
    return cudaGetLastError();
}

}  // namespace cl
}  // namespace osb

struct osb_closure {
    int nx, ny, nz, n;
    float *params;  // NPARAM params, then Adam m, then Adam v
    char *ws;
    osb::cl::Buffers B;
    cudaStream_t st;
    float nrm_h[24];
    float loss_weight;  // multiplies the loss and its gradient (per-sample weighting)
};

namespace osb {
namespace cl {

// Forward pass into cl->B.y (normalised output) from a stage source.
cudaError_t forward_y(osb_closure *c, const void *src, int src_is_f64, size_t stride) {
    const int n = c->n;
    const int blocks = (n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216;
    if (src_is_f64)
        k_features<double><<<blocks, 256, 0, c->st>>>(n, (const double *)src, stride, c->B.nrm, c->B.x0);
    else
        k_features<float><<<blocks, 256, 0, c->st>>>(n, (const float *)src, stride, c->B.nrm, c->B.x0);
    cudaError_t e = conv<16, 32, EPI_RELU>(c->nx, c->ny, c->nz, c->B.x0, c->B.wf1, c->params + OFF_B1, nullptr, c->B.h1,
                                           c->B.tcerr, c->st);
    if (e != cudaSuccess) return e;
    e = conv<32, 32, EPI_RELU>(c->nx, c->ny, c->nz, c->B.h1, c->B.wf2, c->params + OFF_B2, nullptr, c->B.h2, c->B.tcerr,
                               c->st);
    if (e != cudaSuccess) return e;
    return conv<32, 8, EPI_LIN>(c->nx, c->ny, c->nz, c->B.h2, c->B.wf3, c->B.b3pad, nullptr, c->B.y, c->B.tcerr, c->st);
}

cudaError_t closure_correction(osb_closure *c, const void *src, int src_is_f64, size_t stride, const float **C) {
    cudaError_t e = forward_y(c, src, src_is_f64, stride);
    if (e != cudaSuccess) return e;
    const int blocks = (c->n + 255) / 256 < 1216 ? (c->n + 255) / 256 : 1216;
    if (src_is_f64)
        k_closure_out<double><<<blocks, 256, 0, c->st>>>(c->n, c->B.y, c->B.nrm, c->B.C, (const double *)src, stride);
    else
        k_closure_out<float><<<blocks, 256, 0, c->st>>>(c->n, c->B.y, c->B.nrm, c->B.C, (const float *)src, stride);
    *C = c->B.C;
    return cudaGetLastError();
}

int closure_points(const osb_closure *c) { return c->n; }

}  // namespace cl
}  // namespace osb

using namespace osb;

extern "C" {

size_t osb_closure_param_count(void) { return cl::NPARAM; }

size_t osb_closure_workspace_bytes(int nx, int ny, int nz) {
    if (nx < cl::PX || ny < cl::PY || nz < cl::PZ || nx % cl::PX || ny % cl::PY || nz % cl::PZ) return 0;
    if ((long long)nx * ny * nz > (1LL << 28)) return 0;
    return cl::carve(nullptr, nx * ny * nz, nullptr);
}

osb_status osb_closure_create(int nx, int ny, int nz, float *params_dev, void *ws_dev, size_t ws_bytes, void *stream,
                              osb_closure **out) {
    if (!out) return OSB_ERR_INVALID_ARG;
    *out = nullptr;
    const size_t need = osb_closure_workspace_bytes(nx, ny, nz);
    if (need == 0) {
        set_last_error("closure: grid sizes must be multiples of (8, 4, 4), at most 2^28 points");
        return OSB_ERR_UNSUPPORTED;
    }
    if (!params_dev || !ws_dev) {
        set_last_error("closure: NULL buffer");
        return OSB_ERR_INVALID_ARG;
    }
    if (((uintptr_t)params_dev & 15) || ((uintptr_t)ws_dev & 255) || ws_bytes < need) {
        set_last_error("closure: params must be 16-byte aligned, workspace 256-byte aligned and large enough");
        return OSB_ERR_BUFFER;
    }
    osb_closure *c = new (std::nothrow) osb_closure;
    if (!c) return OSB_ERR_INVALID_ARG;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->n = nx * ny * nz;
    c->params = params_dev;
    c->ws = (char *)ws_dev;
    c->st = (cudaStream_t)stream;
    cl::carve(c->ws, c->n, &c->B);
    for (int i = 0; i < 24; ++i) c->nrm_h[i] = ((i >= 5 && i < 15) || (i >= 16 && i < 21)) ? 1.f : 0.f;
    c->loss_weight = 1.f;
    // zero the padded BF16 weight buffers once (padding entries stay zero)
    cudaError_t e = cudaMemsetAsync(c->B.tcerr, 0, (char *)c->ws + need - (char *)c->B.tcerr, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->B.nrm, c->nrm_h, sizeof(c->nrm_h), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        delete c;
        set_last_error("closure: initial copies failed");
        return OSB_ERR_CUDA;
    }
    *out = c;
    return OSB_OK;
}

osb_status osb_closure_destroy(osb_closure *c) {
    if (!c) return OSB_ERR_INVALID_ARG;
    delete c;
    return OSB_OK;
}

osb_status osb_closure_set_normalization(osb_closure *c, const float *in_mean, const float *in_std,
                                         const float *out_std) {
    if (!c || !in_mean || !in_std || !out_std) return OSB_ERR_INVALID_ARG;
    for (int i = 0; i < 5; ++i) {
        if (!(in_std[i] > 0) || !(out_std[i] > 0) || !isfinite(in_mean[i])) {
            set_last_error("closure: standard deviations must be > 0");
            return OSB_ERR_INVALID_ARG;
        }
        c->nrm_h[i] = in_mean[i];
        c->nrm_h[5 + i] = 1.f / in_std[i];
        c->nrm_h[10 + i] = out_std[i];
    }
    cudaError_t e = cudaMemcpyAsync(c->B.nrm, c->nrm_h, sizeof(c->nrm_h), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        set_last_error("closure: normalisation copy failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

osb_status osb_closure_set_channels(osb_closure *c, const int *apply) {
    if (!c || !apply) return OSB_ERR_INVALID_ARG;
    for (int i = 0; i < 5; ++i) c->nrm_h[16 + i] = apply[i] ? 1.f : 0.f;
    cudaError_t e = cudaMemcpyAsync(c->B.nrm, c->nrm_h, sizeof(c->nrm_h), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        set_last_error("closure: channel mask copy failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

osb_status osb_closure_set_loss_weight(osb_closure *c, float w) {
    if (!c || !(w > 0) || !isfinite(w)) return OSB_ERR_INVALID_ARG;
    c->loss_weight = w;
    return OSB_OK;
}

osb_status osb_closure_set_dissipative(osb_closure *c, int on) {
    if (!c) return OSB_ERR_INVALID_ARG;
    c->nrm_h[21] = on ? 1.f : 0.f;
    cudaError_t e = cudaMemcpyAsync(c->B.nrm, c->nrm_h, sizeof(c->nrm_h), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        set_last_error("closure: option copy failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

osb_status osb_closure_sync_weights(osb_closure *c) {
    if (!c) return OSB_ERR_INVALID_ARG;
    const float *P = c->params;
    cl::k_prep_weights<<<64, 256, 0, c->st>>>(P + cl::OFF_W1, cl::H, 5, cl::H, 16, c->B.wf1, nullptr, 0, 0);
    cl::k_prep_weights<<<128, 256, 0, c->st>>>(P + cl::OFF_W2, cl::H, cl::H, cl::H, cl::H, c->B.wf2, c->B.wd2, cl::H, cl::H);
    cl::k_prep_weights<<<32, 256, 0, c->st>>>(P + cl::OFF_W3, 5, cl::H, 8, cl::H, c->B.wf3, c->B.wd3, cl::H, 16);
    cudaError_t e = cudaMemsetAsync(c->B.b3pad, 0, 8 * sizeof(float), c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->B.b3pad, P + cl::OFF_B3, 5 * sizeof(float), cudaMemcpyDeviceToDevice, c->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error("closure: weight preparation failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

osb_status osb_closure_forward(osb_closure *c, const double *Q_dev, size_t field_stride, float *C_dev) {
    if (!c || !Q_dev || !C_dev || field_stride < (size_t)c->n) return OSB_ERR_INVALID_ARG;
    const float *C = nullptr;
    cudaError_t e = cl::closure_correction(c, Q_dev, 1, field_stride, &C);
    if (e == cudaSuccess) e = cudaMemcpyAsync(C_dev, C, (size_t)c->n * 5 * sizeof(float), cudaMemcpyDeviceToDevice, c->st);
    if (e != cudaSuccess) {
        set_last_error("closure: forward failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

osb_status osb_closure_loss_grad(osb_closure *c, const double *X_dev, size_t xs, const double *Cstar_dev, size_t cs,
                                 float *grad_dev, float *loss_dev) {
    if (!c || !X_dev || !Cstar_dev || !grad_dev || !loss_dev || xs < (size_t)c->n || cs < (size_t)c->n)
        return OSB_ERR_INVALID_ARG;
    using namespace cl;
    const int n = c->n, nx = c->nx, ny = c->ny, nz = c->nz;
    cudaError_t e = forward_y(c, X_dev, 1, xs);
    const int blocks = (n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216;
    if (e == cudaSuccess) {
        k_targets<<<blocks, 256, 0, c->st>>>(n, Cstar_dev, cs, c->B.nrm, c->B.t);
        k_mse<<<NPART, 256, 0, c->st>>>(n, c->B.y, c->B.t, c->B.dy, c->B.lpart, c->loss_weight);
        k_sum_partials<<<1, 32, 0, c->st>>>(c->B.lpart, NPART, c->loss_weight / (5.f * n), loss_dev);
        e = cudaGetLastError();
    }
    // layer 3: dW3, db3; then dz2 = (W3^T dy) * [h2 > 0]
    if (e == cudaSuccess)
        e = wgrad<32, 16>(nx, ny, nz, c->B.dy, c->B.h2, c->B.part, 5, H, grad_dev + OFF_W3, grad_dev + OFF_B3, c->st);
    if (e == cudaSuccess)
        e = conv<16, 32, EPI_MASK>(nx, ny, nz, c->B.dy, c->B.wd3, nullptr, c->B.h2, c->B.dz2, c->B.tcerr, c->st);
    // layer 2
    if (e == cudaSuccess)
        e = wgrad<32, 32>(nx, ny, nz, c->B.dz2, c->B.h1, c->B.part, H, H, grad_dev + OFF_W2, grad_dev + OFF_B2, c->st);
    if (e == cudaSuccess)
        e = conv<32, 32, EPI_MASK>(nx, ny, nz, c->B.dz2, c->B.wd2, nullptr, c->B.h1, c->B.dz1, c->B.tcerr, c->st);
    // layer 1
    if (e == cudaSuccess)
        e = wgrad<16, 32>(nx, ny, nz, c->B.dz1, c->B.x0, c->B.part, H, 5, grad_dev + OFF_W1, grad_dev + OFF_B1, c->st);
    if (e != cudaSuccess) {
        set_last_error("closure: loss/gradient launch failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

osb_status osb_closure_adam_step(osb_closure *c, const float *grad_dev, float lr, int step) {
    if (!c || !grad_dev || !(lr > 0) || step < 1) return OSB_ERR_INVALID_ARG;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f / (1.f - powf(b1, (float)step)), c2 = 1.f / (1.f - powf(b2, (float)step));
    const int np = cl::NPARAM;
    cl::k_adam<<<(np + 255) / 256, 256, 0, c->st>>>(np, c->params, c->params + np, c->params + 2 * np, grad_dev, lr,
                                                    b1, b2, eps, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error("closure: Adam launch failed");
        return OSB_ERR_CUDA;
    }
    return osb_closure_sync_weights(c);
}

osb_status osb_closure_status(osb_closure *c) {
    if (!c) return OSB_ERR_INVALID_ARG;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, c->B.tcerr, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) {
        set_last_error("closure: status read failed");
        return OSB_ERR_CUDA;
    }
    if (h) {
        set_last_error("closure: a tensor-core accumulator wait ran out");
        return OSB_ERR_TIMEOUT;
    }
    return OSB_OK;
}

osb_status osb_box_filter(const double *fine_dev, int fnx, int fny, int fnz, int factor, double *coarse_dev,
                          void *stream) {
    if (!fine_dev || !coarse_dev || factor < 1 || fnx < 1 || fny < 1 || fnz < 1 || fnx % factor || fny % factor ||
        fnz % factor) {
        set_last_error("box filter: sizes must be positive multiples of the factor");
        return OSB_ERR_INVALID_ARG;
    }
    const int cnx = fnx / factor, cny = fny / factor, cnz = fnz / factor;
    const long long nc = (long long)cnx * cny * cnz;
    int blocks = (int)((5 * nc + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    cl::k_box_filter<<<blocks, 256, 0, (cudaStream_t)stream>>>(fine_dev, (size_t)fnx * fny * fnz, fnx, fny, factor,
                                                                cnx, cny, cnz, coarse_dev, (size_t)nc);
    if (cudaGetLastError() != cudaSuccess) {
        set_last_error("box filter launch failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

}  // extern "C"
