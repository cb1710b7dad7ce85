// zmarch.cuh -- FP32 stage as two z-marching kernels (orders 2..8, viscous
// work form A), the memory-lean form of the three kernels in stage.cuh.
//
// Each CTA owns a TX x TY column tile of the grid and a chunk of z planes.
// Planes stream through a shared-memory ring one or two planes ahead of their use,
// over the tile plus a halo (R rows in y; 4 columns in x, so that every row
// starts on a 16-byte boundary).  Tiles away from the periodic boundary load
// each field's plane with one TMA box copy (cp.async.bulk.tensor.3d) that
// completes on the slot's mbarrier; tiles touching the boundary use 4-byte
// cp.async copies at wrapped addresses (TMA fills out-of-range boxes with zeros
// instead of wrapping).  Along z every thread keeps its own column in register
// queues of 2R+1 values; x/y stencils read the ring, z stencils the queues.
//
//   k_zflux: velocity gradient -> energy flux F_j (with the viscous work
//            u_i tau_ij), g_i = (div u - D_i u_i)/Re, div u     (7 FP32 fields)
//   k_zrhs : residual of all equations + RK update, reading Q, F_j, g_i, div u
//
// HBM traffic per point and stage (FP32 q, FP64 U): k_zflux reads q (20 B)
// and writes 28 B; k_zrhs reads q, F, g, div (48 B) and U (40 B), writes q
// (20 B) and U (40 B), plus the 20 B FP32 copy of U in the last stage.
#pragma once

#include <cuda.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>

#include "stage.cuh"

namespace osb {
namespace zm {

constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int CX = 4;   // ring column of the tile's first x (row start x0 - 4 is 16-byte aligned)
constexpr unsigned ZM_WAIT_LIMIT = 1u << 24;

template <int R>
struct Geo {
    static constexpr int RW = TX + 2 * CX, RH = TY + 2 * R, RA = RW * RH;
    static constexpr int RAP = (RA + 31) / 32 * 32;  // ring plane stride: TMA destinations need 128-byte alignment
    // planes in flight ahead of the lead plane: two, except at radius 2, where
    // the second ring slot would leave room for one CTA per SM instead of two
    // (measured at 256^3: radius 1, 3, 4 gain 3-4% with two; radius 2 loses 40%)
    static constexpr int PF = (R == 2) ? 1 : 2;
    static constexpr int NS = R + 1 + PF;            // ring slots
};


__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void bar_init(uint32_t bar, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the given phase parity; false if the limit ran out.
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    for (unsigned it = 0; it < ZM_WAIT_LIMIT; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_cg(void *smem, const void *gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ int wrapz(int z, int nz) {
    z %= nz;
    return z < 0 ? z + nz : z;
}

// In-plane offsets of the tile rectangle (tile + R halo, periodic wrap).
template <int R>
__device__ __forceinline__ void make_offsets(int *off, int x0, int y0, const Dims &d) {
    using G = Geo<R>;
    for (int e = threadIdx.x; e < G::RA; e += NT) {
        const int ry = e / G::RW, rx = e - ry * G::RW;
        off[e] = wrapc(y0 + ry - R, d.ny) * d.nx + wrapc(x0 + rx - CX, d.nx);
    }
}

template <int N>
__device__ __forceinline__ void qpush(float (&q)[N], float v) {
#pragma unroll
    for (int k = 0; k < N - 1; ++k) q[k] = q[k + 1];
    q[N - 1] = v;
}

// z first derivative from a register queue centred at index R.
template <int R>
__device__ __forceinline__ float qd1(const float (&q)[2 * R + 1], const float *c) {
    float s = 0.f;
#pragma unroll
    for (int k = R; k >= 1; --k) s = fmaf(c[k], q[R + k] - q[R - k], s);
    return s;
}
// x / y first derivatives from a shared-memory plane (rectangle layout).
template <int R>
__device__ __forceinline__ float sdx1(const float *p, int ce, const float *c) {
    float s = 0.f;
#pragma unroll
    for (int k = R; k >= 1; --k) s = fmaf(c[k], p[ce + k] - p[ce - k], s);
    return s;
}
template <int R>
__device__ __forceinline__ float sdy1(const float *p, int ce, const float *c) {
    constexpr int W = Geo<R>::RW;
    float s = 0.f;
#pragma unroll
    for (int k = R; k >= 1; --k) s = fmaf(c[k], p[ce + k * W] - p[ce - k * W], s);
    return s;
}

// Tap-by-tap accumulation into a sum: acc + sum_k w_k (f_{+k} -+ f_{-k}) along
// x or y of a shared-memory plane, or along z of a register queue (w indexed
// by k = 1..R; the centre tap of a second derivative is the caller's).
template <int R, int STRIDE>
__device__ __forceinline__ float acc_s1(float acc, const float *p, int ce, const float *w, bool neg = false) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fmaf(neg ? -w[k] : w[k], p[ce + k * STRIDE] - p[ce - k * STRIDE], acc);
    return acc;
}
template <int R, int STRIDE>
__device__ __forceinline__ float acc_s2(float acc, const float *p, int ce, const float *w) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fmaf(w[k], p[ce + k * STRIDE] + p[ce - k * STRIDE], acc);
    return acc;
}
template <int R>
__device__ __forceinline__ float acc_q1(float acc, const float (&q)[2 * R + 1], const float *w, bool neg = false) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fmaf(neg ? -w[k] : w[k], q[R + k] - q[R - k], acc);
    return acc;
}
template <int R>
__device__ __forceinline__ float acc_q2(float acc, const float (&q)[2 * R + 1], const float *w) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fmaf(w[k], q[R + k] + q[R - k], acc);
    return acc;
}

// ---------------------------------------------------------------------------
// k_zflux
// ---------------------------------------------------------------------------
template <int R>
struct FluxSmem {
    using G = Geo<R>;
    float ring[G::NS][4][G::RAP];  // rho, m0, m1, m2 over the rectangle (TMA destinations first)
    float ering[G::NS][NT];       // rho E at the tile points
    float vel[3][G::RA];          // u_i of the output plane
    int off[G::RA];
    unsigned long long bars[G::NS];
};

// One column tile (x0, y0) over planes [z0, z1) of k_zflux.  PERSIST: called
// from the persistent ensemble kernel -- data written earlier in the same
// launch is read through L2 only (TMA, 16-byte cp.async.cg, ld.global.cg).
// bars: the NS ring-slot mbarriers (initialised by the caller); phase: their
// parity bits, carried across calls.
// DIAG: also sum the first-stage diagnostics into the block's record.
template <int R, bool PERSIST, bool DIAG = false>
__device__ __forceinline__ void zflux_body(const StageArgs &a, const ZTma &tm, int x0, int y0, int z0, int z1,
                                           FluxSmem<R> &S, unsigned long long *bars, uint32_t &phase) {
    using G = Geo<R>;
    const Dims d = a.d;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int ce = (ty + R) * G::RW + tx + CX;
    const bool active = (x0 + tx < d.nx) && (y0 + ty < d.ny);
    const int plane = d.nx * d.ny;
    const float *Q = static_cast<const float *>(a.src);
    const size_t qs = a.src_stride, as = a.aux_stride;
    float *aux = static_cast<float *>(a.aux);
    const bool use_tma = tm.use && x0 >= CX && x0 - CX + G::RW <= d.nx && y0 >= R && y0 + TY + R <= d.ny;
    const bool vec16 = (d.nx % 4) == 0;  // 16-byte chunks of a row never straddle the wrap

    make_offsets<R>(S.off, x0, y0, d);
    __syncthreads();
    const int coff = S.off[ce];

    auto issue = [&](int L) {
        const int s = ((L % G::NS) + G::NS) % G::NS;
        const int zc = wrapz(L, d.nz);
        if (use_tma) {
            if (tid == 0) {
                const uint32_t bar = smem_u32(&bars[s]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect(bar, (uint32_t)((4 * G::RA + NT) * sizeof(float)));
#pragma unroll
                for (int f = 0; f < 4; ++f) tma_load3(&S.ring[s][f][0], &tm.rect[f], x0 - CX, y0 - R, zc, bar);
                tma_load3(&S.ering[s][0], &tm.col[0], x0, y0, zc, bar);
            }
        } else {
            const size_t zb = (size_t)zc * plane;
            if (PERSIST || vec16) {
                for (int ch = tid; ch < G::RA / 4; ch += NT) {
                    const int e = ch * 4;
                    const size_t g = zb + S.off[e];
#pragma unroll
                    for (int f = 0; f < 4; ++f) cp_async16_cg(&S.ring[s][f][e], Q + f * qs + g);
                }
                if (tid < NT / 4) {
                    const int row = tid / (TX / 4), j = tid % (TX / 4);
                    cp_async16_cg(&S.ering[s][row * TX + 4 * j],
                                  Q + 4 * qs + zb + S.off[(row + R) * G::RW + CX + 4 * j]);
                }
            } else {
                for (int e = tid; e < G::RA; e += NT) {
                    const size_t g = zb + S.off[e];
#pragma unroll
                    for (int f = 0; f < 4; ++f) cp_async4(&S.ring[s][f][e], Q + f * qs + g);
                }
                cp_async4(&S.ering[s][tid], Q + 4 * qs + zb + coff);
            }
            cp_commit();
        }
    };
    auto wait_plane = [&](int L) {
        if (use_tma) {
            const int s = ((L % G::NS) + G::NS) % G::NS;
            if (!bar_wait(smem_u32(&bars[s]), (phase >> s) & 1u) && tid == 0 && a.kerr) atomicOr(a.kerr, KERR_WAIT);
            phase ^= 1u << s;
        } else {
            cp_wait<G::PF - 1>();
        }
    };

    float qu[2 * R + 1], qv[2 * R + 1], qw[2 * R + 1];
#pragma unroll
    for (int k = 0; k < 2 * R + 1; ++k) qu[k] = qv[k] = qw[k] = 0.f;

    const int Lbeg = z0 - R, Lend = z1 + R;  // lead planes [Lbeg, Lend)
#pragma unroll 1
    for (int p = 0; p < G::PF; ++p) issue(Lbeg + p);
    const FoldW<float> &fw = a.f32;
    // first-stage diagnostics: this thread's sums of (1/2) rho u.u and
    // (1/2) rho |omega|^2 over its column, in FP64
    double dg_ke = 0.0, dg_ens = 0.0;
    const float gm1 = float(a.ph.gm1);
#pragma unroll 1
    for (int L = Lbeg; L < Lend; ++L) {
        wait_plane(L);
        __syncthreads();
        if (L + G::PF < Lend)
            issue(L + G::PF);
        else if (!use_tma)
            cp_commit();  // keep the group count uniform
        const int sL = ((L % G::NS) + G::NS) % G::NS;
        {
            const float rho = S.ring[sL][0][ce];
            const float ri = __fdividef(1.f, rho);
            qpush(qu, S.ring[sL][1][ce] * ri);
            qpush(qv, S.ring[sL][2][ce] * ri);
            qpush(qw, S.ring[sL][3][ce] * ri);
        }
        const int zo = L - R;
        if (zo < z0) continue;
        const int so = ((zo % G::NS) + G::NS) % G::NS;
        for (int e = tid; e < G::RA; e += NT) {
            const float ri = __fdividef(1.f, S.ring[so][0][e]);
            S.vel[0][e] = S.ring[so][1][e] * ri;
            S.vel[1][e] = S.ring[so][2][e] * ri;
            S.vel[2][e] = S.ring[so][3][e] * ri;
        }
        __syncthreads();
        // s_ij = (1/Re) d_j u_i, the 1/Re of tau folded into the weights
        const float gxx = sdx1<R>(S.vel[0], ce, fw.d1ir[0]), gxy = sdy1<R>(S.vel[0], ce, fw.d1ir[1]),
                    gxz = qd1<R>(qu, fw.d1ir[2]);
        const float gyx = sdx1<R>(S.vel[1], ce, fw.d1ir[0]), gyy = sdy1<R>(S.vel[1], ce, fw.d1ir[1]),
                    gyz = qd1<R>(qv, fw.d1ir[2]);
        const float gzx = sdx1<R>(S.vel[2], ce, fw.d1ir[0]), gzy = sdy1<R>(S.vel[2], ce, fw.d1ir[1]),
                    gzz = qd1<R>(qw, fw.d1ir[2]);
        const float divs = gxx + gyy + gzz;  // (1/Re) div u
        const float tdiv = (2.f / 3.f) * divs;
        const float txx = fmaf(2.f, gxx, -tdiv), tyy = fmaf(2.f, gyy, -tdiv), tzz = fmaf(2.f, gzz, -tdiv);
        const float txy = gxy + gyx, txz = gxz + gzx, tyz = gyz + gzy;
        const float u = qu[R], v = qv[R], w = qw[R];
        const float rho = S.ring[so][0][ce], e = S.ering[so][tid];
        const float p = gm1 * (e - 0.5f * rho * (u * u + v * v + w * w));
        const float hE = fmaf(0.5f, e, p);
        if (DIAG && active) {
            const float o0 = gzy - gyz, o1 = gxz - gzx, o2 = gyx - gxy;  // omega / Re
            dg_ke += double(0.5f * rho * fmaf(u, u, fmaf(v, v, w * w)));
            dg_ens += double(0.5f * rho * fmaf(o0, o0, fmaf(o1, o1, o2 * o2)));
        }
        if (active) {
            size_t i = (size_t)zo * plane + coff;
            if (!OSB_BC_OK(zo >= 0 && zo < d.nz && coff >= 0 && coff < plane, a.kerr)) i = 0;
            aux[A_FX * as + i] = hE * u - (u * txx + v * txy + w * txz);
            aux[A_FY * as + i] = hE * v - (u * txy + v * tyy + w * tyz);
            aux[A_FZ * as + i] = hE * w - (u * txz + v * tyz + w * tzz);
            aux[A_GX * as + i] = gyy + gzz;  // g_i / Re
            aux[A_GY * as + i] = gxx + gzz;
            aux[A_GZ * as + i] = gxx + gyy;
            aux[A_DIV * as + i] = fw.Re * divs;
        }
    }
    cp_wait<0>();
    __syncthreads();  // the ring may be refilled by the caller's next tile
    if constexpr (DIAG) {
        const double Re = double(fw.Re);
        block_record2(dg_ke, dg_ens * (Re * Re), a.diag_rec);
    }
}

template <int R, bool DIAG>
__global__ void __launch_bounds__(NT, 2) k_zflux(const StageArgs a, int zchunk, const __grid_constant__ ZTma tm) {
    using G = Geo<R>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FluxSmem<R> &S = *reinterpret_cast<FluxSmem<R> *>(smem_raw);
    if (threadIdx.x == 0) {
        for (int s = 0; s < G::NS; ++s) bar_init(smem_u32(&S.bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;
    const int z0 = blockIdx.z * zchunk;
    zflux_body<R, false, DIAG>(a, tm, blockIdx.x * TX, blockIdx.y * TY, z0, min(z0 + zchunk, a.d.nz), S, S.bars,
                               phase);
}

// ---------------------------------------------------------------------------
// k_zrhs
// ---------------------------------------------------------------------------
enum RingField { RF_RHO = 0, RF_M0, RF_M1, RF_M2, RF_E, RF_FX, RF_FY, RF_GX, RF_GY, RF_N };
enum DerField { DF_U = 0, DF_V, DF_W, DF_T, DF_PXX, DF_PYY, DF_PXY, DF_PXZ, DF_PYZ, DF_N };

template <int R>
struct RhsSmem {
    using G = Geo<R>;
    float ring[G::NS][RF_N][G::RAP];  // TMA destinations first
    float cring[G::NS][2][NT];       // F_z, g_z at the tile points
    float der[DF_N][G::RA];
    int off[G::RA];
    unsigned long long bars[G::NS];
};

// One column tile of k_zrhs (see zflux_body for PERSIST, bars and phase).
template <int R, bool PERSIST>
__device__ __forceinline__ void zrhs_body(const StageArgs &a, const ZTma &tm, int x0, int y0, int z0, int z1,
                                          RhsSmem<R> &S, unsigned long long *bars, uint32_t &phase) {
    using G = Geo<R>;
    constexpr int Q = 2 * R + 1;
    const Dims d = a.d;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int ce = (ty + R) * G::RW + tx + CX;
    const bool active = (x0 + tx < d.nx) && (y0 + ty < d.ny);
    const int plane = d.nx * d.ny;
    const float *Qg = static_cast<const float *>(a.src);
    const size_t qs = a.src_stride, as = a.aux_stride;
    const float *aux = static_cast<const float *>(a.aux);
    const Coef<float> &c = a.c32;
    const bool use_tma = tm.use && x0 >= CX && x0 - CX + G::RW <= d.nx && y0 >= R && y0 + TY + R <= d.ny;
    const bool vec16 = (d.nx % 4) == 0;

    make_offsets<R>(S.off, x0, y0, d);
    __syncthreads();
    const int coff = S.off[ce];

    auto issue = [&](int L) {
        const int s = ((L % G::NS) + G::NS) % G::NS;
        const int zc = wrapz(L, d.nz);
        if (use_tma) {
            if (tid == 0) {
                const uint32_t bar = smem_u32(&bars[s]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect(bar, (uint32_t)((RF_N * G::RA + 2 * NT) * sizeof(float)));
#pragma unroll
                for (int f = 0; f < RF_N; ++f) tma_load3(&S.ring[s][f][0], &tm.rect[f], x0 - CX, y0 - R, zc, bar);
                tma_load3(&S.cring[s][0][0], &tm.col[0], x0, y0, zc, bar);
                tma_load3(&S.cring[s][1][0], &tm.col[1], x0, y0, zc, bar);
            }
        } else {
            const size_t zb = (size_t)zc * plane;
            const float *src[RF_N] = {Qg, Qg + qs, Qg + 2 * qs, Qg + 3 * qs, Qg + 4 * qs,
                                      aux + A_FX * as, aux + A_FY * as, aux + A_GX * as, aux + A_GY * as};
            if (PERSIST || vec16) {
                for (int ch = tid; ch < G::RA / 4; ch += NT) {
                    const int e = ch * 4;
                    const size_t g = zb + S.off[e];
#pragma unroll
                    for (int f = 0; f < RF_N; ++f) cp_async16_cg(&S.ring[s][f][e], src[f] + g);
                }
                if (tid < NT / 2) {
                    const int cf = tid / (NT / 4), t4 = tid % (NT / 4);
                    const int row = t4 / (TX / 4), j = t4 % (TX / 4);
                    cp_async16_cg(&S.cring[s][cf][row * TX + 4 * j],
                                  aux + (cf ? A_GZ : A_FZ) * as + zb + S.off[(row + R) * G::RW + CX + 4 * j]);
                }
            } else {
                for (int e = tid; e < G::RA; e += NT) {
                    const size_t g = zb + S.off[e];
#pragma unroll
                    for (int f = 0; f < RF_N; ++f) cp_async4(&S.ring[s][f][e], src[f] + g);
                }
                cp_async4(&S.cring[s][0][tid], aux + A_FZ * as + zb + coff);
                cp_async4(&S.cring[s][1][tid], aux + A_GZ * as + zb + coff);
            }
            cp_commit();
        }
    };
    auto wait_plane = [&](int L) {
        if (use_tma) {
            const int s = ((L % G::NS) + G::NS) % G::NS;
            if (!bar_wait(smem_u32(&bars[s]), (phase >> s) & 1u) && tid == 0 && a.kerr) atomicOr(a.kerr, KERR_WAIT);
            phase ^= 1u << s;
        } else {
            cp_wait<G::PF - 1>();
        }
    };

    // register queues along z (planes zo-R .. zo+R once full)
    float qQ[5][Q], qPxz[Q], qPyz[Q], qPzz[Q], qFz[Q], qU[Q], qV[Q], qW[Q], qT[Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
#pragma unroll
        for (int m = 0; m < 5; ++m) qQ[m][k] = 0.f;
        qPxz[k] = qPyz[k] = qPzz[k] = qFz[k] = qU[k] = qV[k] = qW[k] = qT[k] = 0.f;
    }
    // g_i arrive scaled by 1/Re from k_zflux
    const float third = 1.f / 3.f, gm1 = float(a.ph.gm1), gM2 = float(a.ph.gM2);
    const float bdt = float(a.beta_dt), adt = float(a.alpha_dt);
    float *qo = static_cast<float *>(a.q_out);
    float *cp = static_cast<float *>(a.u32_out);

    const int Lbeg = z0 - R, Lend = z1 + R;
#pragma unroll 1
    for (int p = 0; p < G::PF; ++p) issue(Lbeg + p);
#pragma unroll 1
    for (int L = Lbeg; L < Lend; ++L) {
        wait_plane(L);
        __syncthreads();
        if (L + G::PF < Lend)
            issue(L + G::PF);
        else if (!use_tma)
            cp_commit();
        const int sL = ((L % G::NS) + G::NS) % G::NS;
        {   // lead plane: point-wise quantities of this thread's column
            const float rho = S.ring[sL][RF_RHO][ce], m0 = S.ring[sL][RF_M0][ce], m1 = S.ring[sL][RF_M1][ce],
                        m2 = S.ring[sL][RF_M2][ce], e = S.ring[sL][RF_E][ce];
            const float ri = __fdividef(1.f, rho);
            const float u = m0 * ri, v = m1 * ri, w = m2 * ri;
            const float p = gm1 * (e - 0.5f * (m0 * u + m1 * v + m2 * w));
            qpush(qQ[0], rho);
            qpush(qQ[1], m0);
            qpush(qQ[2], m1);
            qpush(qQ[3], m2);
            qpush(qQ[4], e);
            qpush(qU, u);
            qpush(qV, v);
            qpush(qW, w);
            qpush(qT, gM2 * p * ri);
            qpush(qPxz, 0.5f * m0 * w);
            qpush(qPyz, 0.5f * m1 * w);
            qpush(qPzz, fmaf(-third, S.cring[sL][1][tid], fmaf(0.5f * m2, w, p)));
            qpush(qFz, S.cring[sL][0][tid]);
        }
        const int zo = L - R;
        if (zo < z0) continue;
        const int so = ((zo % G::NS) + G::NS) % G::NS;
        size_t i = (size_t)zo * plane + coff;
        if (!OSB_BC_OK(!active || (zo >= 0 && zo < d.nz && coff >= 0 && coff < plane), a.kerr)) i = 0;
        // FP64 accumulator of this point: issue the loads before the plane work
        double Ui[5];
        float divc;
        if (PERSIST) {
#pragma unroll
            for (int m = 0; m < 5; ++m) Ui[m] = __ldcg(a.U_in + m * a.u_stride + i);
            divc = __ldcg(aux + A_DIV * as + i);
        } else {
#pragma unroll
            for (int m = 0; m < 5; ++m) Ui[m] = a.U_in[m * a.u_stride + i];
            divc = aux[A_DIV * as + i];
        }
        // point-wise fields of the output plane over the rectangle
        for (int e = tid; e < G::RA; e += NT) {
            const float rho = S.ring[so][RF_RHO][e], m0 = S.ring[so][RF_M0][e], m1 = S.ring[so][RF_M1][e],
                        m2 = S.ring[so][RF_M2][e], en = S.ring[so][RF_E][e];
            const float ri = __fdividef(1.f, rho);
            const float u = m0 * ri, v = m1 * ri, w = m2 * ri;
            const float p = gm1 * (en - 0.5f * (m0 * u + m1 * v + m2 * w));
            S.der[DF_U][e] = u;
            S.der[DF_V][e] = v;
            S.der[DF_W][e] = w;
            S.der[DF_T][e] = gM2 * p * ri;
            S.der[DF_PXX][e] = fmaf(-third, S.ring[so][RF_GX][e], fmaf(0.5f * m0, u, p));
            S.der[DF_PYY][e] = fmaf(-third, S.ring[so][RF_GY][e], fmaf(0.5f * m1, v, p));
            S.der[DF_PXY][e] = 0.5f * m0 * v;
            S.der[DF_PXZ][e] = 0.5f * m0 * w;
            S.der[DF_PYZ][e] = 0.5f * m1 * w;
        }
        __syncthreads();
        const float u = qU[R], v = qV[R], w = qW[R];
        constexpr int W = G::RW;
        float res[5];
        // advective half of the skew-symmetric form and dilatation,
        // res_m = -(1/2)(q_m div u + u_j D_j q_m): -u_j/2 folded into the
        // weights of axis j (radius <= 3), except for rho u_j along j, whose
        // derivative the mass flux -(1/2) D_j (rho u_j) shares
        {
            const float hdiv = -0.5f * divc, hu = -0.5f * u, hv = -0.5f * v, hw = -0.5f * w;
            float wx[R + 1], wy[R + 1], wz[R + 1];
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                wx[k] = hu * c.d1[0][k];
                wy[k] = hv * c.d1[1][k];
                wz[k] = hw * c.d1[2][k];
            }
#pragma unroll
            for (int m = 0; m < 5; ++m) res[m] = hdiv * qQ[m][R];
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const float *f = S.ring[so][RF_RHO + m];
                if (m == 1 || R > 3) {
                    const float dx = sdx1<R>(f, ce, c.d1[0]);
                    res[m] = fmaf(hu, dx, res[m]);
                    if (m == 1) res[0] = fmaf(-0.5f, dx, res[0]);
                } else {
                    res[m] = acc_s1<R, 1>(res[m], f, ce, wx);
                }
                if (m == 2 || R > 3) {
                    const float dy = sdy1<R>(f, ce, c.d1[1]);
                    res[m] = fmaf(hv, dy, res[m]);
                    if (m == 2) res[0] = fmaf(-0.5f, dy, res[0]);
                } else {
                    res[m] = acc_s1<R, W>(res[m], f, ce, wy);
                }
                if (m == 3 || R > 3) {
                    const float dz = qd1<R>(qQ[m], c.d1[2]);
                    res[m] = fmaf(hw, dz, res[m]);
                    if (m == 3) res[0] = fmaf(-0.5f, dz, res[0]);
                } else {
                    res[m] = acc_q1<R>(res[m], qQ[m], wz);
                }
            }
        }
        // momentum and energy flux divergences, tap by tap
        res[1] = acc_s1<R, 1>(res[1], S.der[DF_PXX], ce, c.d1[0], true);
        res[1] = acc_s1<R, W>(res[1], S.der[DF_PXY], ce, c.d1[1], true);
        res[1] = acc_q1<R>(res[1], qPxz, c.d1[2], true);
        res[2] = acc_s1<R, 1>(res[2], S.der[DF_PXY], ce, c.d1[0], true);
        res[2] = acc_s1<R, W>(res[2], S.der[DF_PYY], ce, c.d1[1], true);
        res[2] = acc_q1<R>(res[2], qPyz, c.d1[2], true);
        res[3] = acc_s1<R, 1>(res[3], S.der[DF_PXZ], ce, c.d1[0], true);
        res[3] = acc_s1<R, W>(res[3], S.der[DF_PYZ], ce, c.d1[1], true);
        res[3] = acc_q1<R>(res[3], qPzz, c.d1[2], true);
        res[4] = acc_s1<R, 1>(res[4], S.ring[so][RF_FX], ce, c.d1[0], true);
        res[4] = acc_s1<R, W>(res[4], S.ring[so][RF_FY], ce, c.d1[1], true);
        res[4] = acc_q1<R>(res[4], qFz, c.d1[2], true);
        // viscous Laplacians and heat flux with 1/Re, 4/(3 Re), kappa folded
        // into the weights and one centre weight per equation
        const FoldW<float> &fw = a.f32;
        res[1] = fmaf(fw.c_u, u, res[1]);
        res[1] = acc_s2<R, 1>(res[1], S.der[DF_U], ce, fw.vis43[0]);
        res[1] = acc_s2<R, W>(res[1], S.der[DF_U], ce, fw.vis[1]);
        res[1] = acc_q2<R>(res[1], qU, fw.vis[2]);
        res[2] = fmaf(fw.c_v, v, res[2]);
        res[2] = acc_s2<R, 1>(res[2], S.der[DF_V], ce, fw.vis[0]);
        res[2] = acc_s2<R, W>(res[2], S.der[DF_V], ce, fw.vis43[1]);
        res[2] = acc_q2<R>(res[2], qV, fw.vis[2]);
        res[3] = fmaf(fw.c_w, w, res[3]);
        res[3] = acc_s2<R, 1>(res[3], S.der[DF_W], ce, fw.vis[0]);
        res[3] = acc_s2<R, W>(res[3], S.der[DF_W], ce, fw.vis[1]);
        res[3] = acc_q2<R>(res[3], qW, fw.vis43[2]);
        res[4] = fmaf(fw.c_T, qT[R], res[4]);
        res[4] = acc_s2<R, 1>(res[4], S.der[DF_T], ce, fw.heat[0]);
        res[4] = acc_s2<R, W>(res[4], S.der[DF_T], ce, fw.heat[1]);
        res[4] = acc_q2<R>(res[4], qT, fw.heat[2]);
        if (a.closure) {
#pragma unroll
            for (int m = 0; m < 5; ++m) res[m] += a.closure[(size_t)m * d.n + i];
        }
        if (active) {
            // stage value q = float(U_in) + alpha dt R; in the first stage the
            // stencil source is the FP32 copy of U_in, so float(U_in) is the
            // queue centre and needs no conversion
            auto update = [&](auto from_src) {
#pragma unroll
                for (int m = 0; m < 5; ++m) {
                    const double Un = Ui[m] + f2d_bits(bdt * res[m]);
                    a.U_out[m * a.u_stride + i] = Un;
                    if (qo) qo[m * a.q_stride + i] = fmaf(adt, res[m], decltype(from_src)::value ? qQ[m][R] : d2f_bits(Ui[m]));
                    if (cp) cp[m * a.q_stride + i] = d2f_bits(Un);
                }
            };
            if (a.src_is_u32)
                update(std::true_type{});
            else
                update(std::false_type{});
        }
    }
    cp_wait<0>();
    __syncthreads();  // the ring may be refilled by the caller's next tile
}

template <int R>
__global__ void __launch_bounds__(NT, (R <= 2) ? 2 : 1) k_zrhs(const StageArgs a, int zchunk,
                                                                const __grid_constant__ ZTma tm) {
    using G = Geo<R>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RhsSmem<R> &S = *reinterpret_cast<RhsSmem<R> *>(smem_raw);
    if (threadIdx.x == 0) {
        for (int s = 0; s < G::NS; ++s) bar_init(smem_u32(&S.bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    uint32_t phase = 0;
    const int z0 = blockIdx.z * zchunk;
    zrhs_body<R, false>(a, tm, blockIdx.x * TX, blockIdx.y * TY, z0, min(z0 + zchunk, a.d.nz), S, S.bars, phase);
}

template <int R>
constexpr size_t flux_smem() {
    static_assert(Geo<R>::RAP * sizeof(float) % 128 == 0 && offsetof(FluxSmem<R>, ering) % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
    return sizeof(FluxSmem<R>);
}
template <int R>
constexpr size_t rhs_smem() {
    static_assert(Geo<R>::RAP * sizeof(float) % 128 == 0 && offsetof(RhsSmem<R>, cring) % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
    return sizeof(RhsSmem<R>);
}

}  // namespace zm
}  // namespace osb

#include "zrhs_narrow.cuh"

namespace osb {
namespace zm {

// The narrow residual kernel for radius 3 and 4 (OSB_FP32_ZRHS=wide: k_zrhs).
inline bool use_narrow_rhs() {
    const char *e = getenv("OSB_FP32_ZRHS");
    return !(e && strcmp(e, "wide") == 0);
}

// Launches k_zflux then the residual kernel for one RK stage of the FP32
// path: k_zrhs up to radius 2, k_zrhs_n at radius 3 and 4.
template <int R>
cudaError_t launch_zstage(const StageArgs &a) {
    static_assert(R <= 4, "z-march kernels are built for orders up to 8");
    // z planes per CTA: long chunks amortise the 2R-plane warm-up of the z
    // queues; short chunks give small grids enough CTAs (about four per SM)
    const int tiles_xy = ((a.d.nx + TX - 1) / TX) * ((a.d.ny + TY - 1) / TY);
    int zchunk = (int)(((long long)a.d.nz * tiles_xy + 4 * 152 - 1) / (4 * 152));
    zchunk = zchunk < 4 ? 4 : (zchunk > 32 ? 32 : zchunk);
    dim3 grd((a.d.nx + TX - 1) / TX, (a.d.ny + TY - 1) / TY, (a.d.nz + zchunk - 1) / zchunk);
    const size_t sf = flux_smem<R>(), sr = rhs_smem<R>();
    auto kflux = a.diag_rec ? k_zflux<R, true> : k_zflux<R, false>;
    cudaError_t e = cudaFuncSetAttribute(kflux, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sf);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_zrhs<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
    if (e != cudaSuccess) return e;
    static const ZTma none = {};
    const ZTma &tf = a.ztma_flux ? *static_cast<const ZTma *>(a.ztma_flux) : none;
    const ZTma &tr = a.ztma_rhs ? *static_cast<const ZTma *>(a.ztma_rhs) : none;
    if (a.ev) cudaEventRecord(a.ev[0], a.stream);
    if (a.ev) cudaEventRecord(a.ev[1], a.stream);  // no separate primitive kernel
    kflux<<<grd, NT, sf, a.stream>>>(a, zchunk, tf);
    if (a.ev) cudaEventRecord(a.ev[2], a.stream);
    if constexpr (R >= 3) {
        if (use_narrow_rhs()) {
            using GN = GeoN<R>;
            const size_t sn = rhs_smem_n<R>();
            e = cudaFuncSetAttribute(k_zrhs_n<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sn);
            if (e != cudaSuccess) return e;
            // narrow tiles: z chunks for about four CTA rounds of three per SM
            const int tiles_n = ((a.d.nx + TX - 1) / TX) * ((a.d.ny + GN::TYN - 1) / GN::TYN);
            int zc = (int)(((long long)a.d.nz * tiles_n + 12 * 152 - 1) / (12 * 152));
            zc = zc < 4 ? 4 : (zc > 32 ? 32 : zc);
            dim3 gn((a.d.nx + TX - 1) / TX, (a.d.ny + GN::TYN - 1) / GN::TYN, (a.d.nz + zc - 1) / zc);
            static const ZTmaN none_n = {};
            const ZTmaN &tn = a.ztma_rhs_n ? *static_cast<const ZTmaN *>(a.ztma_rhs_n) : none_n;
            k_zrhs_n<R><<<gn, GN::NTN, sn, a.stream>>>(a, zc, tn);
            if (a.ev) cudaEventRecord(a.ev[3], a.stream);
            return cudaGetLastError();
        }
    }
    k_zrhs<R><<<grd, NT, sr, a.stream>>>(a, zchunk, tr);
    if (a.ev) cudaEventRecord(a.ev[3], a.stream);
    return cudaGetLastError();
}

}  // namespace zm

// Per-order stage entry: the fused stage kernel (FP32 increment form, orders
// 2 and 4) when the stage arguments ask for it, the two z-march kernels for
// the FP32 path (form A, orders <= 8), the three-kernel stage otherwise.
template <int R>
cudaError_t stage_entry_z(const StageArgs &a) {
    if constexpr (R <= 2) {
        if (a.fz_mode) return R == 1 ? fz::launch_fused_r1(a) : fz::launch_fused_r2(a);
    }
    if constexpr (R <= 4) {
        if (a.precision == OSB_FP32 && a.visc_form == OSB_VISC_A && !a.src_is_f64 && a.zmarch)
            return zm::launch_zstage<R>(a);
    }
    return launch_stage<R>(a, 0);
}

}  // namespace osb

#undef OSB_DEFINE_ORDER
#define OSB_DEFINE_ORDER(ORDER)                                                          \
    namespace osb {                                                                      \
    OrderKernels kernels_o##ORDER() {                                                    \
        return OrderKernels{ORDER, &stage_entry_z<ORDER / 2>, &residual_entry<ORDER / 2>}; \
    }                                                                                    \
    }
