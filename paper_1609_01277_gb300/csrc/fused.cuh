// fused.cuh -- the FP32 RK stage as ONE z-marching kernel per stage (orders 2
// and 4, viscous work form A, periodic grids).  Included by fused_o2.cu and
// fused_o4.cu, one radius per translation unit.
//
// Residual (Section 3.3, regrouped by linearity as in stage.cuh), with
// Q = (rho, m_i, e), D_j / L_j the first / second-derivative stencils along j,
// A(a) = (u_j D_j a + a div u) / 2:
//   R_rho = -sum_j D_j(m_j/2) - A(rho)
//   R_mi  = -sum_j D_j Phi_ij - A(m_i) + (1/Re)[sum_j L_j u_i + L_i u_i/3]
//   R_e   = -sum_j D_j F_j    - A(e)   + kappa sum_j L_j T
//   Phi_ij = m_i u_j/2 + delta_ij (p - g_i/(3 Re)),  g_i = div u - D_i u_i,
//   F_j    = (e/2 + p) u_j - u_i tau_ij.
//
// Work decomposition.  A CTA owns a TX x TY column tile (32 x 8 points) and a
// chunk of z planes; each of its 128 threads owns an x-PAIR of points and does
// all arithmetic on pairs with the packed FP32x2 instructions of sm_100-class
// GPUs (add/mul/fma .f32x2), so every issued FP32 instruction does two points'
// work and every shared-memory stencil tap is one 64-bit load.  Lead plane L:
//   A  conserved planes arrive in a 4-slot shared-memory ring over the tile
//      plus a 2R halo (TMA box copies away from the periodic boundary, wrapped
//      cp.async at it); the velocity of the whole haloed plane goes into a
//      (2R+1)-plane ring; the column values of Q and T go into register
//      queues of 2R+1 pairs (plane mod 2R+1).
//   B  gradient plane g = L - R: velocity gradient over the tile and its R
//      halo in x and y (z derivatives from the velocity ring) -> tau, g_i and
//      the in-plane fluxes Phi_xx, Phi_yy, Phi_xy, Phi_xz, Phi_yz, F_x, F_y and T
//      on the halo strips, in shared memory: nothing goes through HBM.  At the
//      tile pair the z stencils of the point-wise fluxes Phi_iz, (e/2 + p) w
//      and of the velocity Laplacians are formed from the queues and the ring
//      taps the gradient loads.
//   C  residual of plane g: all x/y stencils from shared memory, the z
//      stencils of Q and T from the register queues.  rho, m_x, m_y
//      are complete and their RK update is written at plane g.  m_z and e still
//      miss D_z of the gradient-dependent parts of Phi_zz (-g_z/(3 Re)) and
//      F_z (-u_i tau_iz), known one plane at a time: those are scattered into
//      2R+1 pending accumulators, and the update of m_z, e is written at plane
//      g - R once the last contribution (from plane g) has arrived.
// The register queues and accumulators are shifted by one pair per plane
// (fixed register positions; unrolling the plane loop instead would let the
// positions rotate for free, but the 2R+1 copies of the plane body do not fit
// the instruction cache: ncu showed warps stalled on instruction fetch).
//
// RK registers of the FP32 form (low-storage scheme alpha, beta of Section
// 2.4; Uf = FP32 copy of the FP64 accumulator U at the step start):
//   stage 1: q1 = Uf + alpha_1 dt R0;          d1 = beta_1 dt R0
//   stage 2: q2 = Uf + (d1 + alpha_2 dt R1);   d2 = d1 + beta_2 dt R1
//   stage 3: U' = U + (double)(d2 + beta_3 dt R2);  Uf' = float(U')
// i.e. U_k = U_{k-1} + beta_k dt R_{k-1} and q_k = U_{k-1} + alpha_k dt R_{k-1}
// exactly as in the FP64 scheme, with the two FP32 increments of a step summed
// in FP32 and added to the FP64 accumulator once per step.  HBM traffic per
// point and step: stage 1 reads Uf, writes q1, d1 (60 B); stage 2 reads q1,
// Uf, d1, writes q2, d2 (100 B); stage 3 reads q2, d2, U, writes U, Uf'
// (140 B): 300 B, i.e. 100 B per point-stage.
#pragma once

#include "zmarch.cuh"

namespace osb {
namespace fz {

using zm::bar_expect;
using zm::bar_init;
using zm::bar_wait;
using zm::cp_async16_cg;
using zm::cp_async4;
using zm::cp_commit;
using zm::cp_wait;
using zm::smem_u32;
using zm::tma_load3;
using zm::wrapz;

constexpr int NPX = TX / 2;      // x-pairs per tile row
constexpr int NT = NPX * TY;     // 128 threads
constexpr int CX = 4;            // x halo columns (>= 2R; row starts stay 16-byte aligned)

template <int R>
struct Geo {
    static_assert(R == 1 || R == 2, "the fused stage is built for orders 2 and 4");
    static constexpr int EW = TX + 2 * CX;        // haloed plane width
    static constexpr int EH = TY + 4 * R;         // haloed plane height (2R halo rows)
    static constexpr int EP = EW * EH;            // floats per haloed plane
    static_assert(EP % 32 == 0, "ring planes must stay 128-byte aligned (TMA destinations)");
    static constexpr int NQ = R + 2;              // conserved-plane ring: planes L-R..L and L+1 in flight
    static constexpr int P = 2 * R + 1;           // velocity ring, queue and accumulator period
    static constexpr int XROW = 2 * R;            // x-strip fields hold rows [2R, 2R+TY)
    static constexpr int YROW = R;                // cross fields hold rows [R, 3R+TY)
    static constexpr int XS = EW * TY;
    static constexpr int YS = EW * (TY + 2 * R);
    static constexpr int NE2 = EP / 2;            // pairs of the haloed plane
    static constexpr int NEH = NE2 - NT;          // pairs outside the tile
    static constexpr int NEA = (NEH + NT - 1) / NT;  // halo pairs per thread (phase A)
    static constexpr int NHY = 2 * R * NPX;       // y-strip halo pairs (phase B)
    static constexpr int NHX = 2 * TY;            // x-strip halo pairs (phase B)
};

// Kernel arguments: FP32 weights duplicated into pairs, so packed FMAs take
// them straight from the parameter bank.
struct FArgs {
    Dims d;
    int zchunk;                // z planes per segment
    float2 c1[3][MAXR + 1];    // c_k / h_a
    float2 nc1[3][MAXR + 1];   // -c_k / h_a (flux divergences, tap by tap)
    float2 d1ir[3][MAXR + 1];  // c_k / (h_a Re): the gradient in units of 1/Re
    float2 vis[3][MAXR + 1], vis43[3][MAXR + 1], heat[3][MAXR + 1];  // (k >= 1)
    float2 c13z[MAXR + 1], nc13z[MAXR + 1];  // +-c_k / (3 h_z)
    float2 cu, cv, cw, cT;     // centre weights of the Laplacians
    float2 gm1, gM2, hal, nhal, nthird, Re2, ntwo3, two;
    float2 adt, bdt;           // alpha_k dt, beta_k dt
    float gm1s, Res;
    const float *src;          // stencil source, 5 fields
    const float *ufc;          // stage 2: Uf at the point
    float *dinc;               // increments d (read in stages 2-3, written in 1-2)
    float *q_out;              // stages 1-2: next stage value (stage 2: in place over Uf)
    const double *U_in;        // stage 3
    double *U_out;
    float *copy_out;           // stage 3: float(U_out)
    const float *closure;      // learned correction (5 fields, stride d.n) or nullptr
    double *diag_rec;          // first-stage diagnostics block records, or nullptr
    int *kerr;
    size_t qs, us, ds;         // field strides of the FP32 registers, FP64 registers, increments
    int has_d;                 // stage 3: 0 = forward Euler (no increment to read)
};

// ---------------------------------------------------------------------------
// Packed FP32x2 arithmetic (PTX add/mul/fma .f32x2, round to nearest)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 A, B, D;\nmov.b64 A, {%2, %3};\nmov.b64 B, {%4, %5};\n"
        "add.rn.f32x2 D, A, B;\nmov.b64 {%0, %1}, D;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 A, B, D;\nmov.b64 A, {%2, %3};\nmov.b64 B, {%4, %5};\n"
        "sub.rn.f32x2 D, A, B;\nmov.b64 {%0, %1}, D;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
    float2 d;
    asm("{\n.reg .b64 A, B, D;\nmov.b64 A, {%2, %3};\nmov.b64 B, {%4, %5};\n"
        "mul.rn.f32x2 D, A, B;\nmov.b64 {%0, %1}, D;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
    float2 d;
    asm("{\n.reg .b64 A, B, C, D;\nmov.b64 A, {%2, %3};\nmov.b64 B, {%4, %5};\nmov.b64 C, {%6, %7};\n"
        "fma.rn.f32x2 D, A, B, C;\nmov.b64 {%0, %1}, D;\n}"
        : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__device__ __forceinline__ float2 rcp2(float2 a) { return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y)); }
__device__ __forceinline__ float2 ld2(const float *p) { return *reinterpret_cast<const float2 *>(p); }
__device__ __forceinline__ void st2(float *p, float2 v) { *reinterpret_cast<float2 *>(p) = v; }
__device__ __forceinline__ float2 zero2() { return make_float2(0.f, 0.f); }

// Stencil taps of a pair at the even shared-memory index c (points c, c+1).
// Along x the pair needs f[c-R .. c+1+R]: aligned 64-bit loads A[j] =
// (f[c+2j], f[c+2j+1]), j = -H..H; an odd offset k pairs halves of two loads.
template <int R>
struct XT {
    static constexpr int H = (R + 1) / 2;
    float2 a[2 * H + 1];
    __device__ __forceinline__ void load(const float *f, int c) {
#pragma unroll
        for (int j = -H; j <= H; ++j) a[j + H] = ld2(f + c + 2 * j);
    }
    __device__ __forceinline__ float2 at(int j) const { return a[j + H]; }
    __device__ __forceinline__ float2 centre() const { return a[H]; }
    // (f[+k] - f[-k]) per lane
    __device__ __forceinline__ float2 diff(int k) const {
        if ((k & 1) == 0) return sub2(at(k / 2), at(-k / 2));
        return make_float2(at((k - 1) / 2).y - at((-k - 1) / 2).y, at((k + 1) / 2).x - at((1 - k) / 2).x);
    }
    // (f[+k] + f[-k]) per lane
    __device__ __forceinline__ float2 sum(int k) const {
        if ((k & 1) == 0) return add2(at(k / 2), at(-k / 2));
        return make_float2(at((k - 1) / 2).y + at((-k - 1) / 2).y, at((k + 1) / 2).x + at((1 - k) / 2).x);
    }
    // acc + sum_k w_k (f[+k] -+ f[-k])
    __device__ __forceinline__ float2 d1(float2 acc, const float2 *w) const {
#pragma unroll
        for (int k = R; k >= 1; --k) acc = fma2(w[k], diff(k), acc);
        return acc;
    }
    __device__ __forceinline__ float2 d2(float2 acc, const float2 *w) const {
#pragma unroll
        for (int k = R; k >= 1; --k) acc = fma2(w[k], sum(k), acc);
        return acc;
    }
};

// Along y of a shared-memory plane (row stride W) and along z of a queue.
template <int R, int W>
__device__ __forceinline__ float2 yd1(float2 acc, const float *f, int c, const float2 *w) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fma2(w[k], sub2(ld2(f + c + k * W), ld2(f + c - k * W)), acc);
    return acc;
}
template <int R, int W>
__device__ __forceinline__ float2 yd2(float2 acc, const float *f, int c, const float2 *w) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fma2(w[k], add2(ld2(f + c + k * W), ld2(f + c - k * W)), acc);
    return acc;
}


template <int R>
struct Smem {
    using G = Geo<R>;
    float rq[G::NQ][5][G::EP];     // conserved planes (TMA destinations first)
    float ve[G::P][3][G::EP];      // velocity ring
    float dx[3][G::XS];            // Phi_xx, Phi_xz, F_x on the x strip
    float dy[5][G::YS];            // Phi_yy, Phi_yz, F_y, T, Phi_xy on the cross rows
    int off[G::EP];                // wrapped in-plane offsets (boundary tiles)
    unsigned long long bars[G::NQ];
};
enum { DX_PXX = 0, DX_PXZ, DX_FX };
enum { DY_PYY = 0, DY_PYZ, DY_FY, DY_T, DY_PXY };
enum { QQ_RHO = 0, QQ_M0, QQ_M1, QQ_M2, QQ_E, QQ_T, QQ_N };

// Register state of a thread across planes.
template <int R>
struct Regs {
    float2 q[QQ_N][2 * R + 1];   // column queues: position i holds plane L - 2R + i
    float2 acc[2][2 * R + 1];    // pending m_z, e residuals: position i holds plane g - R + i
    double ke, ens;              // first-stage diagnostics sums
};

// Per-CTA constants of the march.
struct Ctx {
    int x0, y0, z0, z1, Lbeg, Lend;
    int ce, cx, cy;          // thread pair: haloed-plane index, x-strip index, cross index
    int eA[4];               // haloed-plane pairs of phase A outside the tile
    int chy, chx;            // phase B halo pair (haloed-plane index) or -1
    size_t gidx;             // in-plane index of the pair's first point
    bool act0, act1, vec;    // lanes inside the grid; 64-bit global accesses allowed
    bool use_tma, vec16;
    int rs;                  // ring slot of the lead plane
    int vs;                  // velocity ring slot of the lead plane
    uint32_t phase;          // mbarrier parities of the ring slots
};

// ---------------------------------------------------------------------------
// Plane loads into the conserved-plane ring
// ---------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void issue_plane(Smem<R> &S, const FArgs &a, const FTma &tm, const Ctx &c, int L,
                                            int slot) {
    using G = Geo<R>;
    const int zc = wrapz(L, a.d.nz);
    if (c.use_tma) {
        if (threadIdx.x == 0) {
            const uint32_t bar = smem_u32(&S.bars[slot]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bar_expect(bar, (uint32_t)(5 * G::EP * sizeof(float)));
#pragma unroll
            for (int f = 0; f < 5; ++f) tma_load3(&S.rq[slot][f][0], &tm.q[f], c.x0 - CX, c.y0 - 2 * R, zc, bar);
        }
    } else {
        const size_t zb = (size_t)zc * a.d.nx * a.d.ny;
        if (c.vec16) {
            for (int ch = threadIdx.x; ch < G::EP / 4; ch += NT) {
                const int e = 4 * ch;
                const size_t gi = zb + S.off[e];
#pragma unroll
                for (int f = 0; f < 5; ++f) cp_async16_cg(&S.rq[slot][f][e], a.src + f * a.qs + gi);
            }
        } else {
            for (int e = threadIdx.x; e < G::EP; e += NT) {
                const size_t gi = zb + S.off[e];
#pragma unroll
                for (int f = 0; f < 5; ++f) cp_async4(&S.rq[slot][f][e], a.src + f * a.qs + gi);
            }
        }
        cp_commit();
    }
}

template <int R>
__device__ __forceinline__ void wait_plane(Smem<R> &S, const FArgs &a, Ctx &c, int slot) {
    if (c.use_tma) {
        if (!bar_wait(smem_u32(&S.bars[slot]), (c.phase >> slot) & 1u) && threadIdx.x == 0 && a.kerr)
            atomicOr(a.kerr, KERR_WAIT);
        c.phase ^= 1u << slot;
    } else {
        cp_wait<0>();
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Point-wise quantities (the same expressions wherever a value is formed, so
// a field computed in two phases is bitwise the same)
// ---------------------------------------------------------------------------
struct PW {
    float2 rho, m0, m1, m2, e, u, v, w, ri, p;
};
__device__ __forceinline__ PW pw_load(const float *Q, int ep, int c) {
    PW q;
    q.rho = ld2(Q + c);
    q.m0 = ld2(Q + ep + c);
    q.m1 = ld2(Q + 2 * ep + c);
    q.m2 = ld2(Q + 3 * ep + c);
    q.e = ld2(Q + 4 * ep + c);
    return q;
}
__device__ __forceinline__ void pw_vel(PW &q) {
    q.ri = rcp2(q.rho);
    q.u = mul2(q.m0, q.ri);
    q.v = mul2(q.m1, q.ri);
    q.w = mul2(q.m2, q.ri);
}
// p = (gamma - 1)(e - (m0 u + m1 v + m2 w)/2)
__device__ __forceinline__ void pw_p(const FArgs &a, PW &q) {
    const float2 k = fma2(q.m0, q.u, fma2(q.m1, q.v, mul2(q.m2, q.w)));
    q.p = mul2(a.gm1, fma2(a.nhal, k, q.e));
}
__device__ __forceinline__ float2 pw_T(const FArgs &a, const PW &q) { return mul2(mul2(a.gM2, q.p), q.ri); }
__device__ __forceinline__ float2 pw_pxz(const FArgs &a, const PW &q) { return mul2(mul2(a.hal, q.m0), q.w); }
__device__ __forceinline__ float2 pw_pyz(const FArgs &a, const PW &q) { return mul2(mul2(a.hal, q.m1), q.w); }
__device__ __forceinline__ float2 pw_pxy(const FArgs &a, const PW &q) { return mul2(mul2(a.hal, q.m0), q.v); }
__device__ __forceinline__ float2 pw_hE(const FArgs &a, const PW &q) { return fma2(a.hal, q.e, q.p); }

// z stencils of a register queue centred at position R (planes g - R .. g + R),
// and of the velocity ring (vk[i]: the slot of plane g - R + i)
template <int R>
__device__ __forceinline__ float2 qz1(float2 acc, const float2 (&q)[2 * R + 1], const float2 *w) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fma2(w[k], sub2(q[R + k], q[R - k]), acc);
    return acc;
}
template <int R>
__device__ __forceinline__ float2 qz2(float2 acc, const float2 (&q)[2 * R + 1], const float2 *w) {
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fma2(w[k], add2(q[R + k], q[R - k]), acc);
    return acc;
}
template <int R>
__device__ __forceinline__ float2 vz1(float2 acc, const float *const *vk, int f, int c, const float2 *w) {
    constexpr int EP = Geo<R>::EP;
#pragma unroll
    for (int k = R; k >= 1; --k) acc = fma2(w[k], sub2(ld2(vk[R + k] + f * EP + c), ld2(vk[R - k] + f * EP + c)), acc);
    return acc;
}

// ---------------------------------------------------------------------------
// Phase B at one pair of the gradient plane: KIND 0 tile pair (everything),
// 1 y-strip halo pair (what D_y of Phi_yy, F_y, Phi_xy, Phi_yz, T needs),
// 2 x-strip halo pair (what D_x of Phi_xx, F_x, Phi_xy, Phi_xz, T needs).
// The velocity gradient s_ij = (1/Re) D_j u_i (1/Re folded into the weights).
// ---------------------------------------------------------------------------
struct GradOut {
    float2 divRe, gzs, ftz;   // div u; g_z/Re; u_i tau_iz (tile pairs)
    float2 u, v, w;
    float2 o0, o1, o2, rho;   // vorticity / Re and density (diagnostics)
    float2 zf[4];             // -D_z of Phi_xz, Phi_yz, m_z w/2 + p, (e/2 + p) w
    float2 lz[3];             // z parts of the viscous Laplacians of u, v, w
};

// Phase B at the thread's tile pair: the full velocity gradient, the in-plane
// fluxes of the tile points, and (when plane g gets its residual) every z
// stencil of a point-wise flux: Phi_xz, Phi_yz, m_z w/2 + p and (e/2 + p) w at
// the planes g +- k are formed from the column queues of Q and the velocity
// ring taps that the gradient loads anyway, and the z parts of the viscous
// Laplacians come from the same taps.
template <int R>
__device__ __forceinline__ void tile_pair(Smem<R> &S, const FArgs &a, const Regs<R> &rg, const float *Qg,
                                          const float *const *vk, int c, int cxs, int cys, bool doC, GradOut &go) {
    using G = Geo<R>;
    constexpr int W = G::EW, EP = G::EP;
    const float *vu = vk[R], *vv = vk[R] + EP, *vw = vk[R] + 2 * EP;
    const float2 z2 = zero2();
    XT<R> tu, tv, tw;
    tu.load(vu, c);
    tv.load(vv, c);
    tw.load(vw, c);
    float2 zu[2 * R + 1], zv[2 * R + 1], zw[2 * R + 1];  // velocity at planes g + k, index k + R
#pragma unroll
    for (int k = 1; k <= R; ++k) {
        zu[R + k] = ld2(vk[R + k] + c);
        zv[R + k] = ld2(vk[R + k] + EP + c);
        zw[R + k] = ld2(vk[R + k] + 2 * EP + c);
        zu[R - k] = ld2(vk[R - k] + c);
        zv[R - k] = ld2(vk[R - k] + EP + c);
        zw[R - k] = ld2(vk[R - k] + 2 * EP + c);
    }
    PW q = pw_load(Qg, G::EP, c);
    q.u = tu.centre();
    q.v = tv.centre();
    q.w = tw.centre();
    const float2 gxx = tu.d1(z2, a.d1ir[0]), gyx = tv.d1(z2, a.d1ir[0]), gzx = tw.d1(z2, a.d1ir[0]);
    const float2 gxy = yd1<R, W>(z2, vu, c, a.d1ir[1]), gyy = yd1<R, W>(z2, vv, c, a.d1ir[1]),
                 gzy = yd1<R, W>(z2, vw, c, a.d1ir[1]);
    float2 gxz = z2, gyz = z2, gzz = z2;
#pragma unroll
    for (int k = R; k >= 1; --k) {
        gxz = fma2(a.d1ir[2][k], sub2(zu[R + k], zu[R - k]), gxz);
        gyz = fma2(a.d1ir[2][k], sub2(zv[R + k], zv[R - k]), gyz);
        gzz = fma2(a.d1ir[2][k], sub2(zw[R + k], zw[R - k]), gzz);
    }
    q.ri = rcp2(q.rho);
    pw_p(a, q);
    const float2 hE = pw_hE(a, q);
    const float2 divs = add2(add2(gxx, gyy), gzz);
    const float2 ntdiv = mul2(a.ntwo3, divs);
    const float2 txx = fma2(a.two, gxx, ntdiv), tyy = fma2(a.two, gyy, ntdiv), tzz = fma2(a.two, gzz, ntdiv);
    const float2 txy = add2(gxy, gyx), txz = add2(gxz, gzx), tyz = add2(gyz, gzy);
    const float2 fx = fma2(q.u, txx, fma2(q.v, txy, mul2(q.w, txz)));
    const float2 fy = fma2(q.u, txy, fma2(q.v, tyy, mul2(q.w, tyz)));
    go.ftz = fma2(q.u, txz, fma2(q.v, tyz, mul2(q.w, tzz)));
    const float2 gx = add2(gyy, gzz), gy = add2(gxx, gzz);
    go.gzs = add2(gxx, gyy);
    go.divRe = mul2(a.Re2, divs);
    go.u = q.u;
    go.v = q.v;
    go.w = q.w;
    go.rho = q.rho;
    go.o0 = sub2(gzy, gyz);
    go.o1 = sub2(gxz, gzx);
    go.o2 = sub2(gyx, gxy);
    st2(&S.dx[DX_PXX][cxs], fma2(a.nthird, gx, fma2(mul2(a.hal, q.m0), q.u, q.p)));
    st2(&S.dx[DX_PXZ][cxs], pw_pxz(a, q));
    st2(&S.dx[DX_FX][cxs], sub2(mul2(hE, q.u), fx));
    st2(&S.dy[DY_PYY][cys], fma2(a.nthird, gy, fma2(mul2(a.hal, q.m1), q.v, q.p)));
    st2(&S.dy[DY_PYZ][cys], pw_pyz(a, q));
    st2(&S.dy[DY_FY][cys], sub2(mul2(hE, q.v), fy));
    st2(&S.dy[DY_T][cys], pw_T(a, q));
    st2(&S.dy[DY_PXY][cys], pw_pxy(a, q));
    if (doC) {
        go.lz[0] = go.lz[1] = go.lz[2] = z2;
        go.zf[0] = go.zf[1] = go.zf[2] = go.zf[3] = z2;
#pragma unroll
        for (int k = R; k >= 1; --k) {
            go.lz[0] = fma2(a.vis[2][k], add2(zu[R + k], zu[R - k]), go.lz[0]);
            go.lz[1] = fma2(a.vis[2][k], add2(zv[R + k], zv[R - k]), go.lz[1]);
            go.lz[2] = fma2(a.vis43[2][k], add2(zw[R + k], zw[R - k]), go.lz[2]);
            PW hp, hm;  // planes g + k, g - k
            hp.rho = rg.q[QQ_RHO][R + k];
            hp.m0 = rg.q[QQ_M0][R + k];
            hp.m1 = rg.q[QQ_M1][R + k];
            hp.m2 = rg.q[QQ_M2][R + k];
            hp.e = rg.q[QQ_E][R + k];
            hp.u = zu[R + k];
            hp.v = zv[R + k];
            hp.w = zw[R + k];
            hm.rho = rg.q[QQ_RHO][R - k];
            hm.m0 = rg.q[QQ_M0][R - k];
            hm.m1 = rg.q[QQ_M1][R - k];
            hm.m2 = rg.q[QQ_M2][R - k];
            hm.e = rg.q[QQ_E][R - k];
            hm.u = zu[R - k];
            hm.v = zv[R - k];
            hm.w = zw[R - k];
            pw_p(a, hp);
            pw_p(a, hm);
            const float2 nc = a.nc1[2][k];
            go.zf[0] = fma2(nc, sub2(pw_pxz(a, hp), pw_pxz(a, hm)), go.zf[0]);
            go.zf[1] = fma2(nc, sub2(pw_pyz(a, hp), pw_pyz(a, hm)), go.zf[1]);
            go.zf[2] = fma2(nc, sub2(fma2(mul2(a.hal, hp.m2), hp.w, hp.p), fma2(mul2(a.hal, hm.m2), hm.w, hm.p)),
                            go.zf[2]);
            go.zf[3] = fma2(nc, sub2(mul2(pw_hE(a, hp), hp.w), mul2(pw_hE(a, hm), hm.w)), go.zf[3]);
        }
    }
}

template <int R, int KIND>
__device__ __forceinline__ void grad_pair(Smem<R> &S, const FArgs &a, const float *Qg, const float *const *vk, int c,
                                          int cxs, int cys) {
    using G = Geo<R>;
    constexpr int W = G::EW;
    const float *vu = vk[R], *vv = vk[R] + G::EP, *vw = vk[R] + 2 * G::EP;
    const float2 z2 = zero2();
    XT<R> tu, tv;
    tu.load(vu, c);
    tv.load(vv, c);
    const float2 u = tu.centre(), v = tv.centre();
    const float2 gxx = tu.d1(z2, a.d1ir[0]);               // D_x u
    const float2 gyy = yd1<R, W>(z2, vv, c, a.d1ir[1]);     // D_y v
    const float2 gzz = vz1<R>(z2, vk, 2, c, a.d1ir[2]);  // D_z w
    const float2 gxy = yd1<R, W>(z2, vu, c, a.d1ir[1]);     // D_y u
    const float2 gyx = tv.d1(z2, a.d1ir[0]);               // D_x v
    PW q = pw_load(Qg, G::EP, c);
    q.u = u;
    q.v = v;
    const float2 divs = add2(add2(gxx, gyy), gzz);
    const float2 ntdiv = mul2(a.ntwo3, divs);  // -(2/3) div u / Re
    const float2 txy = add2(gxy, gyx);
    if constexpr (KIND == 1) {
        q.w = ld2(vw + c);
        const float2 gzy = yd1<R, W>(z2, vw, c, a.d1ir[1]);     // D_y w
        const float2 gyz = vz1<R>(z2, vk, 1, c, a.d1ir[2]);  // D_z v
        q.ri = rcp2(q.rho);
        pw_p(a, q);
        const float2 hE = pw_hE(a, q);
        const float2 tyy = fma2(a.two, gyy, ntdiv);
        const float2 tyz = add2(gyz, gzy);
        const float2 fy = fma2(q.u, txy, fma2(q.v, tyy, mul2(q.w, tyz)));
        const float2 gy = add2(gxx, gzz);
        st2(&S.dy[DY_PYY][cys], fma2(a.nthird, gy, fma2(mul2(a.hal, q.m1), q.v, q.p)));
        st2(&S.dy[DY_PYZ][cys], pw_pyz(a, q));
        st2(&S.dy[DY_FY][cys], sub2(mul2(hE, q.v), fy));
        st2(&S.dy[DY_T][cys], pw_T(a, q));
        st2(&S.dy[DY_PXY][cys], pw_pxy(a, q));
    } else {
        XT<R> tw;
        tw.load(vw, c);
        q.w = tw.centre();
        const float2 gzx = tw.d1(z2, a.d1ir[0]);               // D_x w
        const float2 gxz = vz1<R>(z2, vk, 0, c, a.d1ir[2]);  // D_z u
        q.ri = rcp2(q.rho);
        pw_p(a, q);
        const float2 hE = pw_hE(a, q);
        const float2 txx = fma2(a.two, gxx, ntdiv);
        const float2 txz = add2(gxz, gzx);
        const float2 fx = fma2(q.u, txx, fma2(q.v, txy, mul2(q.w, txz)));
        const float2 gx = add2(gyy, gzz);
        st2(&S.dx[DX_PXX][cxs], fma2(a.nthird, gx, fma2(mul2(a.hal, q.m0), q.u, q.p)));
        st2(&S.dx[DX_PXZ][cxs], pw_pxz(a, q));
        st2(&S.dx[DX_FX][cxs], sub2(mul2(hE, q.u), fx));
        st2(&S.dy[DY_T][cys], pw_T(a, q));
        st2(&S.dy[DY_PXY][cys], pw_pxy(a, q));
    }
}
// ---------------------------------------------------------------------------
// Global point data of the RK update (prefetched at the start of phase B)
// ---------------------------------------------------------------------------
// Lanes outside the grid (ragged tiles) touch no global memory: their index
// may lie past the last plane.
__device__ __forceinline__ float2 gld2(const float *p, const Ctx &c) {
    if (c.vec) return c.act0 ? *reinterpret_cast<const float2 *>(p) : zero2();
    return make_float2(c.act0 ? p[0] : 0.f, c.act1 ? p[1] : 0.f);
}
__device__ __forceinline__ void gst2(float *p, float2 v, const Ctx &c) {
    if (c.vec) {
        if (c.act0) *reinterpret_cast<float2 *>(p) = v;
    } else {
        if (c.act0) p[0] = v.x;
        if (c.act1) p[1] = v.y;
    }
}
__device__ __forceinline__ double2 gldd2(const double *p, const Ctx &c) {
    if (c.vec) return c.act0 ? *reinterpret_cast<const double2 *>(p) : make_double2(0.0, 0.0);
    return make_double2(c.act0 ? p[0] : 0.0, c.act1 ? p[1] : 0.0);
}
__device__ __forceinline__ void gstd2(double *p, double2 v, const Ctx &c) {
    if (c.vec) {
        if (c.act0) *reinterpret_cast<double2 *>(p) = v;
    } else {
        if (c.act0) p[0] = v.x;
        if (c.act1) p[1] = v.y;
    }
}

template <int MODE>
struct Pre {
    float2 uf[5], d[5];
    double2 U[5];
};

template <int MODE>
__device__ __forceinline__ void prefetch(const FArgs &a, const Ctx &c, int m, size_t i, Pre<MODE> &pr) {
    if constexpr (MODE == 2) {
        pr.uf[m] = gld2(a.ufc + m * a.qs + i, c);
        pr.d[m] = gld2(a.dinc + m * a.ds + i, c);
    } else if constexpr (MODE == 3) {
        pr.U[m] = gldd2(a.U_in + m * a.us + i, c);
        pr.d[m] = a.has_d ? gld2(a.dinc + m * a.ds + i, c) : zero2();
    }
}

// RK update of field m at global index i (see the register scheme above).
template <int MODE>
__device__ __forceinline__ void emit(const FArgs &a, const Ctx &c, int m, size_t i, float2 res, float2 srcc,
                                     const Pre<MODE> &pr) {
    if (!OSB_BC_OK(!c.act0 || i + (c.act1 ? 1 : 0) < (size_t)a.d.n, a.kerr)) return;
    if (a.closure) res = add2(res, gld2(a.closure + (size_t)m * a.d.n + i, c));
    if constexpr (MODE == 1) {
        gst2(a.q_out + m * a.qs + i, fma2(a.adt, res, srcc), c);
        gst2(a.dinc + m * a.ds + i, mul2(a.bdt, res), c);
    } else if constexpr (MODE == 2) {
        gst2(a.q_out + m * a.qs + i, add2(pr.uf[m], fma2(a.adt, res, pr.d[m])), c);
        gst2(a.dinc + m * a.ds + i, fma2(a.bdt, res, pr.d[m]), c);
    } else {
        const float2 inc = fma2(a.bdt, res, pr.d[m]);
        double2 Un = pr.U[m];
        Un.x += f2d_bits(inc.x);
        Un.y += f2d_bits(inc.y);
        gstd2(a.U_out + m * a.us + i, Un, c);
        gst2(a.copy_out + m * a.qs + i, make_float2(d2f_bits(Un.x), d2f_bits(Un.y)), c);
    }
}

// ---------------------------------------------------------------------------
// One lead plane L (slot J of the queues and the velocity ring)
// ---------------------------------------------------------------------------
template <int R, int MODE, bool DIAG>
__device__ __forceinline__ void plane_step(Smem<R> &S, const FArgs &a, const FTma &tm, Ctx &c, Regs<R> &rg,
                                           int L) {
    using G = Geo<R>;
    constexpr int P = G::P, W = G::EW, EP = G::EP;
    const int g = L - R, o = L - 2 * R;   // gradient / residual plane, plane whose m_z, e complete
    // velocity ring slots of planes g - R .. g + R (= L)
    const float *vk[P];
#pragma unroll
    for (int i = 0; i < P; ++i) {
        int s = c.vs - 2 * R + i;
        s = s < 0 ? s + P : s;
        vk[i] = &S.ve[s][0][0];
    }
    const int rsL = c.rs;
    const int rsG = (c.rs + 2 >= G::NQ) ? c.rs + 2 - G::NQ : c.rs + 2;  // slot of plane L - R (NQ = R + 2)
    const int rsN = (c.rs + 1 == G::NQ) ? 0 : c.rs + 1;

    const bool doB = L >= c.z0;                 // g in [z0 - R, z1 + R)
    const bool doC = g >= c.z0 && g < c.z1;     // residual and update of rho, m_x, m_y at g
    const bool doO = o >= c.z0 && o < c.z1;     // update of m_z, e at o
    const size_t plane = (size_t)a.d.nx * a.d.ny;
    const size_t ig = (size_t)g * plane + c.gidx, io = (size_t)o * plane + c.gidx;
    Pre<MODE> pr;
    if constexpr (MODE != 1) {
        if (doO) {
#pragma unroll
            for (int m = 3; m < 5; ++m) prefetch<MODE>(a, c, m, io, pr);
        }
    }
    wait_plane<R>(S, a, c, rsL);
    // ---- A: velocity of the haloed lead plane, column queues
    {
        const float *Q = &S.rq[rsL][0][0];
        float *vL = &S.ve[c.vs][0][0];
        PW q = pw_load(Q, EP, c.ce);
        pw_vel(q);
        st2(vL + c.ce, q.u);
        st2(vL + EP + c.ce, q.v);
        st2(vL + 2 * EP + c.ce, q.w);
        pw_p(a, q);
#pragma unroll
        for (int f = 0; f < QQ_N; ++f)
#pragma unroll
            for (int i = 0; i < P - 1; ++i) rg.q[f][i] = rg.q[f][i + 1];
        rg.q[QQ_RHO][P - 1] = q.rho;
        rg.q[QQ_M0][P - 1] = q.m0;
        rg.q[QQ_M1][P - 1] = q.m1;
        rg.q[QQ_M2][P - 1] = q.m2;
        rg.q[QQ_E][P - 1] = q.e;
        rg.q[QQ_T][P - 1] = pw_T(a, q);
#pragma unroll
        for (int t = 0; t < G::NEA; ++t) {
            const int e = c.eA[t];
            if (e >= 0) {
                PW h;
                h.rho = ld2(Q + e);
                h.m0 = ld2(Q + EP + e);
                h.m1 = ld2(Q + 2 * EP + e);
                h.m2 = ld2(Q + 3 * EP + e);
                pw_vel(h);
                st2(vL + e, h.u);
                st2(vL + EP + e, h.v);
                st2(vL + 2 * EP + e, h.w);
            }
        }
    }
    __syncthreads();
    if (L + 1 < c.Lend) issue_plane<R>(S, a, tm, c, L + 1, rsN);

    if constexpr (MODE != 1) {
        if (doC) {
#pragma unroll
            for (int m = 0; m < 3; ++m) prefetch<MODE>(a, c, m, ig, pr);
        }
    }
    // ---- B: gradient plane g over the tile and its R halo strips
    GradOut go;
    if (doB) {
        const float *Qg = &S.rq[rsG][0][0];
        tile_pair<R>(S, a, rg, Qg, vk, c.ce, c.cx, c.cy, doC, go);
        // D_z of the gradient parts: -D_z(-g_z/(3 Re)) into m_z, -D_z(-u_i tau_iz)
        // into e, scattered to the planes g -+ k; plane g - R is then complete
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            rg.acc[0][R - k] = fma2(a.c13z[k], go.gzs, rg.acc[0][R - k]);
            rg.acc[0][R + k] = fma2(a.nc13z[k], go.gzs, rg.acc[0][R + k]);
            rg.acc[1][R - k] = fma2(a.c1[2][k], go.ftz, rg.acc[1][R - k]);
            rg.acc[1][R + k] = fma2(a.nc1[2][k], go.ftz, rg.acc[1][R + k]);
        }
        if (doO) {
            emit<MODE>(a, c, 3, io, rg.acc[0][0], rg.q[QQ_M2][0], pr);
            emit<MODE>(a, c, 4, io, rg.acc[1][0], rg.q[QQ_E][0], pr);
        }
        if (c.chy >= 0) grad_pair<R, 1>(S, a, Qg, vk, c.chy, 0, c.chy - G::YROW * W);
        if (c.chx >= 0) grad_pair<R, 2>(S, a, Qg, vk, c.chx, c.chx - G::XROW * W, c.chx - G::YROW * W);
        if (doC) {
            if (DIAG) {
                const float kx = 0.5f * go.rho.x * fmaf(go.u.x, go.u.x, fmaf(go.v.x, go.v.x, go.w.x * go.w.x));
                const float ky = 0.5f * go.rho.y * fmaf(go.u.y, go.u.y, fmaf(go.v.y, go.v.y, go.w.y * go.w.y));
                const float ex = 0.5f * go.rho.x * fmaf(go.o0.x, go.o0.x, fmaf(go.o1.x, go.o1.x, go.o2.x * go.o2.x));
                const float ey = 0.5f * go.rho.y * fmaf(go.o0.y, go.o0.y, fmaf(go.o1.y, go.o1.y, go.o2.y * go.o2.y));
                if (c.act0) {
                    rg.ke += double(kx);
                    rg.ens += double(ex);
                }
                if (c.act1) {
                    rg.ke += double(ky);
                    rg.ens += double(ey);
                }
            }
        }
    }
    __syncthreads();
    // ---- C: residual of plane g
    if (doC) {
        const float *Qg = &S.rq[rsG][0][0];
        const float *vu = vk[R], *vv = vk[R] + EP, *vw = vk[R] + 2 * EP;
        const int ce = c.ce, cxs = c.cx, cys = c.cy;
        const float2 z2 = zero2();
        const float2 uc = ld2(vu + ce), vc = ld2(vv + ce), wc = ld2(vw + ce);
        float2 res[5];
        {
            const float2 hdiv = mul2(a.nhal, go.divRe);
#pragma unroll
            for (int m = 0; m < 5; ++m) res[m] = mul2(hdiv, rg.q[m][R]);
        }
        // advective half of the skew-symmetric form, -u_j/2 folded into the
        // weights of axis j, except for m_j along j, whose derivative the mass
        // flux -(1/2) D_j m_j shares
        const float2 hu = mul2(a.nhal, uc), hv = mul2(a.nhal, vc), hw = mul2(a.nhal, wc);
        float2 wx[R + 1], wy[R + 1], wz[R + 1];
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            wx[k] = mul2(hu, a.c1[0][k]);
            wy[k] = mul2(hv, a.c1[1][k]);
            wz[k] = mul2(hw, a.c1[2][k]);
        }
        {
            XT<R> t;
            t.load(Qg, ce);
            res[0] = t.d1(res[0], wx);
            res[0] = yd1<R, W>(res[0], Qg, ce, wy);
            res[0] = qz1<R>(res[0], rg.q[QQ_RHO], wz);
        }
        {
            const float *f = Qg + EP;
            XT<R> t;
            t.load(f, ce);
            const float2 dx = t.d1(z2, a.c1[0]);
            res[1] = fma2(hu, dx, res[1]);
            res[0] = fma2(a.nhal, dx, res[0]);
            res[1] = yd1<R, W>(res[1], f, ce, wy);
            res[1] = qz1<R>(res[1], rg.q[QQ_M0], wz);
        }
        {
            const float *f = Qg + 2 * EP;
            XT<R> t;
            t.load(f, ce);
            res[2] = t.d1(res[2], wx);
            const float2 dy = yd1<R, W>(z2, f, ce, a.c1[1]);
            res[2] = fma2(hv, dy, res[2]);
            res[0] = fma2(a.nhal, dy, res[0]);
            res[2] = qz1<R>(res[2], rg.q[QQ_M1], wz);
        }
        {
            const float *f = Qg + 3 * EP;
            XT<R> t;
            t.load(f, ce);
            res[3] = t.d1(res[3], wx);
            res[3] = yd1<R, W>(res[3], f, ce, wy);
            const float2 dz = qz1<R>(z2, rg.q[QQ_M2], a.c1[2]);
            res[3] = fma2(hw, dz, res[3]);
            res[0] = fma2(a.nhal, dz, res[0]);
        }
        {
            const float *f = Qg + 4 * EP;
            XT<R> t;
            t.load(f, ce);
            res[4] = t.d1(res[4], wx);
            res[4] = yd1<R, W>(res[4], f, ce, wy);
            res[4] = qz1<R>(res[4], rg.q[QQ_E], wz);
        }
        // momentum and energy flux divergences, tap by tap
        {
            XT<R> t;
            t.load(S.dx[DX_PXX], cxs);
            res[1] = t.d1(res[1], a.nc1[0]);
        }
        res[1] = yd1<R, W>(res[1], S.dy[DY_PXY], cys, a.nc1[1]);
        res[1] = add2(res[1], go.zf[0]);
        {
            XT<R> t;
            t.load(S.dy[DY_PXY], cys);
            res[2] = t.d1(res[2], a.nc1[0]);
        }
        res[2] = yd1<R, W>(res[2], S.dy[DY_PYY], cys, a.nc1[1]);
        res[2] = add2(res[2], go.zf[1]);
        {
            XT<R> t;
            t.load(S.dx[DX_PXZ], cxs);
            res[3] = t.d1(res[3], a.nc1[0]);
        }
        res[3] = yd1<R, W>(res[3], S.dy[DY_PYZ], cys, a.nc1[1]);
        res[3] = add2(res[3], go.zf[2]);
        {
            XT<R> t;
            t.load(S.dx[DX_FX], cxs);
            res[4] = t.d1(res[4], a.nc1[0]);
        }
        res[4] = yd1<R, W>(res[4], S.dy[DY_FY], cys, a.nc1[1]);
        res[4] = add2(res[4], go.zf[3]);
        // viscous Laplacians and heat flux, 1/Re, 4/(3 Re), kappa folded into
        // the weights, one centre weight per equation
        res[1] = fma2(a.cu, uc, res[1]);
        {
            XT<R> t;
            t.load(vu, ce);
            res[1] = t.d2(res[1], a.vis43[0]);
        }
        res[1] = yd2<R, W>(res[1], vu, ce, a.vis[1]);
        res[1] = add2(res[1], go.lz[0]);
        res[2] = fma2(a.cv, vc, res[2]);
        {
            XT<R> t;
            t.load(vv, ce);
            res[2] = t.d2(res[2], a.vis[0]);
        }
        res[2] = yd2<R, W>(res[2], vv, ce, a.vis43[1]);
        res[2] = add2(res[2], go.lz[1]);
        res[3] = fma2(a.cw, wc, res[3]);
        {
            XT<R> t;
            t.load(vw, ce);
            res[3] = t.d2(res[3], a.vis[0]);
        }
        res[3] = yd2<R, W>(res[3], vw, ce, a.vis[1]);
        res[3] = add2(res[3], go.lz[2]);
        {
            XT<R> t;
            t.load(S.dy[DY_T], cys);
            res[4] = fma2(a.cT, rg.q[QQ_T][R], res[4]);
            res[4] = t.d2(res[4], a.heat[0]);
        }
        res[4] = yd2<R, W>(res[4], S.dy[DY_T], cys, a.heat[1]);
        res[4] = qz2<R>(res[4], rg.q[QQ_T], a.heat[2]);
#pragma unroll
        for (int m = 0; m < 3; ++m) emit<MODE>(a, c, m, ig, res[m], rg.q[m][R], pr);
        rg.acc[0][R] = add2(rg.acc[0][R], res[3]);
        rg.acc[1][R] = add2(rg.acc[1][R], res[4]);
    }
    // the pending residuals move one plane on (plane g - R is done)
#pragma unroll
    for (int i = 0; i < P - 1; ++i) {
        rg.acc[0][i] = rg.acc[0][i + 1];
        rg.acc[1][i] = rg.acc[1][i + 1];
    }
    rg.acc[0][P - 1] = rg.acc[1][P - 1] = zero2();
    c.vs = (c.vs + 1 == P) ? 0 : c.vs + 1;
    c.rs = rsN;
}


template <int R, int MODE, bool DIAG>
__global__ void __launch_bounds__(NT, NT <= 128 ? 2 : 1) k_fused(const __grid_constant__ FArgs a, const __grid_constant__ FTma tm) {
    using G = Geo<R>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Smem<R> &S = *reinterpret_cast<Smem<R> *>(smem_raw);
    const int tid = threadIdx.x, px = tid % NPX, ty = tid / NPX;
    const Dims &d = a.d;
    Ctx c;
    c.ce = (ty + 2 * R) * G::EW + CX + 2 * px;
    c.cx = c.ce - G::XROW * G::EW;
    c.cy = c.ce - G::YROW * G::EW;
    c.vec = (d.nx & 1) == 0;
    c.vec16 = (d.nx % 4) == 0;
    // phase A: the haloed-plane pairs outside the tile, h = tid, tid + NT, ...
#pragma unroll
    for (int t = 0; t < 4; ++t) c.eA[t] = -1;
#pragma unroll
    for (int t = 0; t < G::NEA; ++t) {
        const int h = tid + t * NT;
        if (h < G::NEH) {
            constexpr int PR = G::EW / 2;        // pairs per haloed row
            constexpr int TOP = 2 * R * PR;      // pairs in the 2R rows above the tile
            constexpr int SIDE = TY * (PR - NPX);
            int ey, ex2;
            if (h < TOP) {
                ey = h / PR;
                ex2 = h % PR;
            } else if (h < TOP + SIDE) {
                const int t2 = h - TOP, side = PR - NPX;  // CX/2 pairs each side
                ey = 2 * R + t2 / side;
                const int j = t2 % side;
                ex2 = j < side / 2 ? j : NPX + j;
            } else {
                const int t2 = h - TOP - SIDE;
                ey = 2 * R + TY + t2 / PR;
                ex2 = t2 % PR;
            }
            c.eA[t] = ey * G::EW + 2 * ex2;
        }
    }
    (void)OSB_BC_OK(c.ce >= 0 && c.ce + 1 < G::EP && c.cx >= 0 && c.cx + 1 < G::XS && c.cy >= 0 && c.cy + 1 < G::YS,
                    a.kerr);
    // phase B halo pairs: the y strips on the first NHY threads (whole warps), then the x strips
    c.chy = c.chx = -1;
    if (tid < G::NHY) {
        const int hr = tid / NPX, p2 = tid % NPX;
        const int ey = hr < R ? R + hr : TY + R + hr;
        c.chy = ey * G::EW + CX + 2 * p2;
    } else if (tid < G::NHY + G::NHX) {
        const int j = tid - G::NHY, side = j / TY, row = j % TY;
        c.chx = (2 * R + row) * G::EW + (side ? CX + TX : CX - 2);
    }
    c.phase = 0;
    c.rs = 0;
    if (tid == 0) {
        for (int s = 0; s < G::NQ; ++s) bar_init(smem_u32(&S.bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    Regs<R> rg;
#pragma unroll
    for (int f = 0; f < QQ_N; ++f)
#pragma unroll
        for (int k = 0; k < 2 * R + 1; ++k) rg.q[f][k] = zero2();
    rg.ke = rg.ens = 0.0;
    // Work: z chunks of a.zchunk planes of every tile, ordered tile-fastest then
    // chunk, so that the CTAs resident at any time cover a narrow band of z
    // planes whose haloed loads the L2 serves; CTA b takes the b-th of
    // gridDim.x equal runs of that order, one march (with its 4R warm-up
    // planes) per (tile, chunk) segment the run touches.
    const int tiles_x = (d.nx + TX - 1) / TX, tiles = tiles_x * ((d.ny + TY - 1) / TY);
    const int nchunk = (d.nz + a.zchunk - 1) / a.zchunk;
    const long long total = (long long)tiles * nchunk;  // segments
    long long pos = total * blockIdx.x / gridDim.x;
    const long long stop = total * (blockIdx.x + 1) / gridDim.x;
#pragma unroll 1
    for (; pos < stop; ++pos) {
        const int chunk = (int)(pos / tiles), tile = (int)(pos - (long long)chunk * tiles);
        c.z0 = chunk * a.zchunk;
        c.z1 = min(d.nz, c.z0 + a.zchunk);
        c.x0 = (tile % tiles_x) * TX;
        c.y0 = (tile / tiles_x) * TY;
        c.Lbeg = c.z0 - 2 * R;
        c.Lend = c.z1 + 2 * R;
        const int xg = c.x0 + 2 * px, yg = c.y0 + ty;
        c.act0 = xg < d.nx && yg < d.ny;
        c.act1 = xg + 1 < d.nx && yg < d.ny;
        c.gidx = (size_t)yg * d.nx + xg;
        if (!OSB_BC_OK(!c.act0 || c.gidx + (c.act1 ? 1 : 0) < (size_t)d.nx * d.ny, a.kerr)) c.act0 = c.act1 = false;
        (void)OSB_BC_OK(c.z0 >= 0 && c.z1 <= d.nz && c.z0 < c.z1 && ((c.x0 - CX) & 3) == 0, a.kerr);
        c.use_tma = tm.use && c.x0 >= CX && c.x0 - CX + G::EW <= d.nx && c.y0 >= 2 * R &&
                    c.y0 - 2 * R + G::EH <= d.ny;
        c.vs = 0;
        __syncthreads();  // the previous march is done with the offset table
        if (!c.use_tma) {
            for (int e = tid; e < G::EP; e += NT) {
                const int ey = e / G::EW, ex = e - ey * G::EW;
                const int v = wrapc(c.y0 + ey - 2 * R, d.ny) * d.nx + wrapc(c.x0 + ex - CX, d.nx);
                S.off[e] = OSB_BC_OK(v >= 0 && v < d.nx * d.ny, a.kerr) ? v : 0;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 2 * R + 1; ++k) rg.acc[0][k] = rg.acc[1][k] = zero2();
        issue_plane<R>(S, a, tm, c, c.Lbeg, c.rs);
#pragma unroll 1
        for (int L = c.Lbeg; L < c.Lend; ++L) plane_step<R, MODE, DIAG>(S, a, tm, c, rg, L);
        if (!c.use_tma) cp_wait<0>();
    }
    if constexpr (DIAG) {
        const double Re = double(a.Res);
        block_record2(rg.ke, rg.ens * (Re * Re), a.diag_rec);
    }
}

template <int R>
constexpr size_t fused_smem() {
    static_assert(offsetof(Smem<R>, rq) == 0 && (Geo<R>::EP * sizeof(float)) % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
    return sizeof(Smem<R>);
}

// Host: kernel arguments from the stage arguments, then one launch.
// z planes per segment: short enough that the resident CTAs cover a narrow
// band of planes (L2 hits for the haloed loads), long enough to amortise the
// 4R warm-up planes of a march.
constexpr int FUSED_ZCHUNK = 32;

template <int R>
cudaError_t launch_fused(const StageArgs &s) {
    const size_t sm = fused_smem<R>();
    FArgs a;
    memset(&a, 0, sizeof(a));
    a.d = s.d;
    auto pr = [](double v) { return make_float2((float)v, (float)v); };
    auto pf = [](float v) { return make_float2(v, v); };
    for (int ax = 0; ax < 3; ++ax)
        for (int k = 0; k <= MAXR; ++k) {
            a.c1[ax][k] = pf(s.c32.d1[ax][k]);
            a.nc1[ax][k] = pf(-s.c32.d1[ax][k]);
            a.d1ir[ax][k] = pf(s.f32.d1ir[ax][k]);
            a.vis[ax][k] = pf(s.f32.vis[ax][k]);
            a.vis43[ax][k] = pf(s.f32.vis43[ax][k]);
            a.heat[ax][k] = pf(s.f32.heat[ax][k]);
        }
    for (int k = 0; k <= MAXR; ++k) {
        a.c13z[k] = pr(s.c64.d1[2][k] / 3.0);
        a.nc13z[k] = pr(-s.c64.d1[2][k] / 3.0);
    }
    a.cu = pf(s.f32.c_u);
    a.cv = pf(s.f32.c_v);
    a.cw = pf(s.f32.c_w);
    a.cT = pf(s.f32.c_T);
    a.gm1 = pr(s.ph.gm1);
    a.gM2 = pr(s.ph.gM2);
    a.hal = pf(0.5f);
    a.nhal = pf(-0.5f);
    a.nthird = pf(-(1.f / 3.f));
    a.Re2 = pf(s.f32.Re);
    a.ntwo3 = pf(-(2.f / 3.f));
    a.two = pf(2.f);
    a.adt = pr(s.alpha_dt);
    a.bdt = pr(s.beta_dt);
    a.gm1s = (float)s.ph.gm1;
    a.Res = s.f32.Re;
    a.src = static_cast<const float *>(s.src);
    a.ufc = s.fz_ufc;
    a.dinc = s.fz_dinc;
    a.q_out = static_cast<float *>(s.q_out);
    a.U_in = s.U_in;
    a.U_out = s.U_out;
    a.copy_out = static_cast<float *>(s.u32_out);
    a.closure = s.closure;
    a.diag_rec = s.diag_rec;
    a.kerr = s.kerr;
    a.qs = s.q_stride;
    a.us = s.u_stride;
    a.ds = s.fz_dstride;
    a.has_d = s.fz_has_d;
    int zc = FUSED_ZCHUNK;
    if (const char *env = getenv("OSB_FUSED_ZCHUNK")) {
        const int v = atoi(env);
        if (v >= 1) zc = v;
    }
    a.zchunk = zc;
    const long long segs = (long long)((s.d.nx + TX - 1) / TX) * ((s.d.ny + TY - 1) / TY) * ((s.d.nz + zc - 1) / zc);
    long long ctas = segs;  // one segment per CTA; the hardware hands segments to SMs in order
    if (const char *env = getenv("OSB_FUSED_CTAS")) {
        const long long v = atoll(env);
        if (v >= 1) ctas = v;
    }
    if (ctas > segs) ctas = segs;
    const dim3 grid((unsigned)ctas);
    static const FTma none = {};
    const FTma &tm = s.fz_tma ? *static_cast<const FTma *>(s.fz_tma) : none;
    void (*k)(const FArgs, const FTma) = nullptr;
    const bool diag = s.diag_rec != nullptr;
    switch (s.fz_mode) {
        case 1: k = diag ? k_fused<R, 1, true> : k_fused<R, 1, false>; break;
        case 2: k = k_fused<R, 2, false>; break;
        case 3: k = diag ? k_fused<R, 3, true> : k_fused<R, 3, false>; break;
        default: return cudaErrorInvalidValue;
    }
    if (s.fz_mode == 2 && diag) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if (s.ev) {
        cudaEventRecord(s.ev[0], s.stream);
        cudaEventRecord(s.ev[1], s.stream);
        cudaEventRecord(s.ev[2], s.stream);
    }
    k<<<grid, NT, sm, s.stream>>>(a, tm);
    if (s.ev) cudaEventRecord(s.ev[3], s.stream);
    return cudaGetLastError();
}

}  // namespace fz
}  // namespace osb
