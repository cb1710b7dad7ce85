// stage.cuh -- one stage of the low-storage RK3 step for the compressible
// Navier-Stokes equations (OpenSBLI paper, Section 3.3), templated on the
// stencil radius R (order 2R), the stencil source type S and the arithmetic
// type T.  Included once per order by stage_o<2R>.cu.
//
// A stage is three kernels, each visiting every point once:
//   k_prim : point-wise primitives and momentum fluxes           (reads Q)
//   k_grad : velocity gradient -> tau, energy flux, div u       (stencils on u)
//   k_resid: all remaining derivatives, the residual R and the RK update
// Each FP64 operation of the residual is executed once per point: on GB300
// FP64 issues at 1/64 of the FP32 rate, so re-computing intermediates in
// stencil halos costs more than writing and re-reading them (HBM and L2 have
// ample headroom at FP64 arithmetic rates).
//
// Residual, with Q = (rho, m_i = rho u_i, e = rho E), D_j / L_j the first /
// second-derivative stencils along j, g_i = div u - D_i u_i:
//   R_rho = -sum_j D_j(m_j/2)     - A(rho)
//   R_mi  = -sum_j D_j Phi_ij     - A(m_i) + (1/Re)[sum_j L_j u_i + L_i u_i/3]
//   R_e   = -sum_j D_j F_j        - A(e)   + kappa sum_j L_j T
//   A(a)  = (sum_j u_j D_j a + a div u)/2
//   Phi_ij = m_i u_j/2 + delta_ij (p - g_i/(3 Re)),
//   F_j    = (e/2 + p) u_j - u_i tau_ij.
// This is the skew-symmetric convective form, the pressure terms, d_j tau_ij
// (Laplacian by L, mixed terms as D_i(D_k u_k)) and the conservative viscous
// work and heat flux, regrouped by linearity of D_j.
// Viscous work form B (template VB) instead keeps F_j = (e/2 + p) u_j and
// Phi_ii = m_i u_i/2 + p, and adds u_i V_i + tau_ij D_j u_i to R_e, where
// V_i = (1/Re)[sum_j L_j u_i + L_i u_i/3 + D_i g_i/3] is the viscous momentum
// term (the product rule applied to d_j(u_i tau_ij)).
#pragma once

#include <string.h>

#include <type_traits>

#include "osb_internal.cuh"

namespace osb {

template <typename T>
struct CoefPick;
template <>
struct CoefPick<double> {
    static __device__ __forceinline__ const Coef<double> &get(const StageArgs &a) { return a.c64; }
};
template <>
struct CoefPick<float> {
    static __device__ __forceinline__ const Coef<float> &get(const StageArgs &a) { return a.c32; }
};
template <>
struct CoefPick<dd> {
    static __device__ __forceinline__ const Coef<dd> &get(const StageArgs &a) { return a.cdd; }
};
template <typename T>
constexpr bool is_dd = std::is_same<T, dd>::value;

template <typename T>
struct FoldPick;
template <>
struct FoldPick<double> {
    static __device__ __forceinline__ const FoldW<double> &get(const StageArgs &a) { return a.f64; }
};
template <>
struct FoldPick<float> {
    static __device__ __forceinline__ const FoldW<float> &get(const StageArgs &a) { return a.f32; }
};

// Physical constants in the arithmetic type (double-float ones precomputed on
// the host, so no kernel converts them).
template <typename T>
__device__ __forceinline__ T k_gm1(const StageArgs &a) {
    if constexpr (is_dd<T>) return a.kdd.gm1; else return T(a.ph.gm1);
}
template <typename T>
__device__ __forceinline__ T k_gM2(const StageArgs &a) {
    if constexpr (is_dd<T>) return a.kdd.gM2; else return T(a.ph.gM2);
}

__device__ __forceinline__ int wrapc(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

// Index of grid point j (any integer) on an axis of n points between two
// symmetry planes (Section 2.6): the halo beyond the plane after the last
// point mirrors the points before it, x_{n+k} -> x_{n-1-k}, and likewise
// x_{-1-k} -> x_k at the first point, which makes the field the restriction
// of a 2n-periodic, mirror-symmetric one.  refl: an odd number of mirrorings,
// so a field that is odd in this axis changes sign.
__device__ __forceinline__ int mirrorc(int j, int n, bool &refl) {
    const int n2 = 2 * n;
    int m = j % n2;
    m = m < 0 ? m + n2 : m;
    refl = m >= n;
    return refl ? n2 - 1 - m : m;
}

// Neighbour offsets of one point, per axis, k = -R..R: wrapped on periodic
// axes; with SYM, mirrored on the axes of Dims::sym, with a bit per k that
// records the sign change of odd fields.
template <bool SYM>
struct NbrMask {
    uint32_t rx = 0, ry = 0, rz = 0;  // bit k + R set where the neighbour is a mirror image
};
template <>
struct NbrMask<false> {};

template <int R, bool SYM = false>
struct Nbr : NbrMask<SYM> {
    int x[2 * R + 1];  // x + k
    int y[2 * R + 1];  // (y + k) * nx
    int z[2 * R + 1];  // (z + k) * nx * ny
    __device__ __forceinline__ void init(int px, int py, int pz, const Dims &d, int *kerr = nullptr) {
#pragma unroll
        for (int k = -R; k <= R; ++k) {
            if constexpr (SYM) {
                bool fx = false, fy = false, fz = false;
                x[k + R] = (d.sym & 1) ? mirrorc(px + k, d.nx, fx) : wrapc(px + k, d.nx);
                y[k + R] = ((d.sym & 2) ? mirrorc(py + k, d.ny, fy) : wrapc(py + k, d.ny)) * d.nx;
                z[k + R] = ((d.sym & 4) ? mirrorc(pz + k, d.nz, fz) : wrapc(pz + k, d.nz)) * d.nx * d.ny;
                this->rx |= (uint32_t)fx << (k + R);
                this->ry |= (uint32_t)fy << (k + R);
                this->rz |= (uint32_t)fz << (k + R);
            } else {
                x[k + R] = wrapc(px + k, d.nx);
                y[k + R] = wrapc(py + k, d.ny) * d.nx;
                z[k + R] = wrapc(pz + k, d.nz) * d.nx * d.ny;
            }
        }
#ifdef OSB_BOUNDS_CHECK
        check(px, py, pz, d, kerr);
#else
        (void)kerr;
#endif
    }
#ifdef OSB_BOUNDS_CHECK
    // every neighbour inside the field: x in [0, nx), y a row start, z a plane start
    __device__ __forceinline__ void check(int px, int py, int pz, const Dims &d, int *kerr) {
        bool ok = px >= 0 && px < d.nx && py >= 0 && py < d.ny && pz >= 0 && pz < d.nz;
        const int plane = d.nx * d.ny;
#pragma unroll
        for (int k = 0; k < 2 * R + 1; ++k)
            ok = ok && x[k] >= 0 && x[k] < d.nx && y[k] >= 0 && y[k] < plane && y[k] % d.nx == 0 && z[k] >= 0 &&
                 z[k] < d.n && z[k] % plane == 0;
        if (!OSB_BC_OK(ok, kerr))
#pragma unroll
            for (int k = 0; k < 2 * R + 1; ++k) x[k] = y[k] = z[k] = 0;
    }
#endif
    template <int AX>
    __device__ __forceinline__ int at(int k) const {
        if (AX == 0) return z[R] + y[R] + x[R + k];
        if (AX == 1) return z[R] + y[R + k] + x[R];
        return z[R + k] + y[R] + x[R];
    }
    __device__ __forceinline__ int center() const { return z[R] + y[R] + x[R]; }
    // the neighbour at offset k along AX of a field with parity bits par
    // (bit a: odd in axis a) carries a sign change
    template <int AX>
    __device__ __forceinline__ bool flip(int k, int par) const {
        if constexpr (!SYM) {
            return false;
        } else {
            if (!((par >> AX) & 1)) return false;
            const uint32_t m = AX == 0 ? this->rx : (AX == 1 ? this->ry : this->rz);
            return (m >> (k + R)) & 1u;
        }
    }
};

// Parity bits of the fields under the symmetry planes (Section 2.6: scalars
// even, the i-th component of a vector odd along axis i); a product takes the
// exclusive or of its factors' bits.
enum Parity : int { PAR_EVEN = 0, PAR_X = 1, PAR_Y = 2, PAR_Z = 4, PAR_XY = 3, PAR_XZ = 5, PAR_YZ = 6 };

template <typename T>
__device__ __forceinline__ T neg_if(bool b, const T &v) {
    return b ? -v : v;
}

// Global-load policy.  LD_NC: read-only path (data written before the launch).
// LD_CG: L2 only, for data that other CTAs of the same (persistent) launch
// wrote -- the per-SM L1 is not coherent with those writes.
enum LoadPolicy { LD_NC = 0, LD_CG = 1 };

template <int POL, typename T, typename P>
__device__ __forceinline__ T ld(const P *p) {
    if constexpr (is_dd<P>) {
        const float2 v = (POL == LD_CG) ? __ldcg(reinterpret_cast<const float2 *>(p))
                                         : __ldg(reinterpret_cast<const float2 *>(p));
        return dd(v.x, v.y);
    } else if constexpr (POL == LD_CG) {
        return T(__ldcg(p));
    } else {
        return T(__ldg(p));
    }
}

// First derivative along AX of field f at the point (weights already / h).
// par: parity bits of f (mirrored neighbours of a field odd along AX change sign).
template <int R, int AX, int POL = LD_NC, typename T, typename P, bool SYM>
__device__ __forceinline__ T D1(const P *__restrict__ f, const Nbr<R, SYM> &nb, const Coef<T> &c, int par = 0) {
    T s = T(0);
#pragma unroll
    for (int k = R; k >= 1; --k) {
        const T fp = neg_if(nb.template flip<AX>(k, par), ld<POL, T>(f + nb.template at<AX>(k)));
        const T fm = neg_if(nb.template flip<AX>(-k, par), ld<POL, T>(f + nb.template at<AX>(-k)));
        s = fma(c.d1[AX][k], fp - fm, s);
    }
    return s;
}

// Second derivative along AX (weights already / h^2).
template <int R, int AX, int POL = LD_NC, typename T, typename P, bool SYM>
__device__ __forceinline__ T D2(const P *__restrict__ f, const Nbr<R, SYM> &nb, const Coef<T> &c, int par = 0) {
    T s = c.d2[AX][0] * ld<POL, T>(f + nb.center());
#pragma unroll
    for (int k = R; k >= 1; --k) {
        const T fp = neg_if(nb.template flip<AX>(k, par), ld<POL, T>(f + nb.template at<AX>(k)));
        const T fm = neg_if(nb.template flip<AX>(-k, par), ld<POL, T>(f + nb.template at<AX>(-k)));
        s = fma(c.d2[AX][k], fp + fm, s);
    }
    return s;
}


// acc + sum_k w_k (f_{+k} - f_{-k}) (w: weights indexed by k = 1..R; a
// negative sign is folded into the FMA); acc + sum_k w_k (f_{+k} + f_{-k})
// (the centre tap is the caller's).
template <int R, int AX, int POL, typename T, typename P, bool SYM>
__device__ __forceinline__ T add_d1(T acc, const P *__restrict__ f, const Nbr<R, SYM> &nb, const T *w, int par,
                                    bool negate = false) {
#pragma unroll
    for (int k = R; k >= 1; --k) {
        const T fp = neg_if(nb.template flip<AX>(k, par), ld<POL, T>(f + nb.template at<AX>(k)));
        const T fm = neg_if(nb.template flip<AX>(-k, par), ld<POL, T>(f + nb.template at<AX>(-k)));
        acc = fma(negate ? -w[k] : w[k], fp - fm, acc);
    }
    return acc;
}
template <int R, int AX, int POL, typename T, typename P, bool SYM>
__device__ __forceinline__ T add_d2(T acc, const P *__restrict__ f, const Nbr<R, SYM> &nb, const T *w, int par) {
#pragma unroll
    for (int k = R; k >= 1; --k) {
        const T fp = neg_if(nb.template flip<AX>(k, par), ld<POL, T>(f + nb.template at<AX>(k)));
        const T fm = neg_if(nb.template flip<AX>(-k, par), ld<POL, T>(f + nb.template at<AX>(-k)));
        acc = fma(w[k], fp + fm, acc);
    }
    return acc;
}

// Double-float stencils: differences (sums) of the neighbours are formed with
// exact head arithmetic and weighted into a compensated accumulator,
// normalised once at the end (dd_acc).
template <int R, int AX, int POL, typename P, bool SYM>
__device__ __forceinline__ dd nb_ld(const P *__restrict__ f, const Nbr<R, SYM> &nb, int k, int par) {
    return neg_if(nb.template flip<AX>(k, par), ld<POL, dd>(f + nb.template at<AX>(k)));
}
template <int R, int AX, int POL = LD_NC, typename P, bool SYM>
__device__ __forceinline__ dd D1(const P *__restrict__ f, const Nbr<R, SYM> &nb, const Coef<dd> &c, int par = 0) {
    dd_acc s;
#pragma unroll
    for (int k = R; k >= 1; --k)
        s.add_wdiff(c.d1[AX][k], nb_ld<R, AX, POL>(f, nb, k, par), nb_ld<R, AX, POL>(f, nb, -k, par));
    return s.get();
}
template <int R, int AX, int POL = LD_NC, typename P, bool SYM>
__device__ __forceinline__ dd D2(const P *__restrict__ f, const Nbr<R, SYM> &nb, const Coef<dd> &c, int par = 0) {
    dd_acc s;
    const dd f0 = ld<POL, dd>(f + nb.center());
    s.add_prod(c.d2[AX][0], f0.hi, f0.lo);
#pragma unroll
    for (int k = R; k >= 1; --k)
        s.add_wsum(c.d2[AX][k], nb_ld<R, AX, POL>(f, nb, k, par), nb_ld<R, AX, POL>(f, nb, -k, par));
    return s.get();
}

// Exact float -> double and round-to-nearest-even double -> float, on the
// integer pipes (GB300 issues FP64 instructions, conversions included, at
// 1/64 of the FP32 rate).  Values below the smallest normal float are flushed
// to signed zero; infinities and NaNs are kept.  Branch-free:
// the special cases are selects, so a warp never diverges here.
__host__ __device__ __forceinline__ uint32_t fbits(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float bitsf(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

__host__ __device__ __forceinline__ double f2d_bits(float f) {
    const uint32_t b = fbits(f), sign = b & 0x80000000u, a = b & 0x7fffffffu;
    // exponent rebias 127 -> 1023 is + (896 << 20) on the high word; for
    // infinities and NaNs the exponent field goes from 0xff to 0x7ff instead
    uint32_t hi = (a >> 3) + (a >= 0x7f800000u ? 0x70000000u : 0x38000000u);
    uint32_t lo = b << 29;
    const bool tiny = a < 0x00800000u;  // zero or denormal
    hi = tiny ? 0u : hi;
    lo = tiny ? 0u : lo;
    const uint64_t r = ((uint64_t)(sign | hi) << 32) | lo;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)r);
#else
    double d;
    memcpy(&d, &r, 8);
    return d;
#endif
}

__host__ __device__ __forceinline__ float d2f_bits(double d) {
#ifdef __CUDA_ARCH__
    const uint64_t b = (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    memcpy(&b, &d, 8);
#endif
    const uint32_t hw = (uint32_t)(b >> 32), lw = (uint32_t)b;
    const uint32_t sign = hw & 0x80000000u, ah = hw & 0x7fffffffu;
    // normal range: exponent 1023 -> 127 and the top 23 mantissa bits
    const uint32_t f = ((ah - 0x38000000u) << 3) | (lw >> 29);
    // round to nearest, ties to even, on the 29 dropped bits (a carry into
    // the exponent is correct, up to infinity)
    const uint32_t inc = ((lw & 0x1fffffffu) + (f & 1u) + 0x0fffffffu) >> 29;
    uint32_t r = sign | (f + inc);
    r = ah < 0x38100000u ? sign : r;  // below the smallest normal float
    const uint32_t nan = (ah > 0x7ff00000u || (ah == 0x7ff00000u && lw != 0u)) ? 0x400000u : 0u;
    r = ah >= 0x47f00000u ? (sign | 0x7f800000u | nan) : r;  // overflow, infinity, NaN
    return bitsf(r);
}

// Sums (a, b) over the thread block in a fixed order -- warp shuffles, then
// thread 0 over the per-warp sums -- and writes the block's record of the
// first-stage diagnostics (layout at StageArgs::diag_rec).  Every thread of
// the block must call it.
__device__ __forceinline__ void block_record2(double a, double b, double *rec) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, off);
        b += __shfl_down_sync(0xffffffffu, b, off);
    }
    __shared__ double part[2][32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nw = (blockDim.x * blockDim.y * blockDim.z + 31) >> 5;
    if ((tid & 31) == 0) {
        part[0][tid >> 5] = a;
        part[1][tid >> 5] = b;
    }
    __syncthreads();
    if (tid == 0) {
        double s0 = 0.0, s1 = 0.0;
        for (int w = 0; w < nw; ++w) {
            s0 += part[0][w];
            s1 += part[1][w];
        }
        const long long blk = blockIdx.x + (long long)gridDim.x * (blockIdx.y + (long long)gridDim.y * blockIdx.z);
        rec[2 + 2 * blk] = s0;
        rec[3 + 2 * blk] = s1;
        if (blk == 0) rec[0] = (double)gridDim.x * gridDim.y * gridDim.z;
    }
}

// ---------------------------------------------------------------------------
// k_prim: primitives and the point-wise momentum fluxes
// ---------------------------------------------------------------------------
template <int POL, typename S, typename T>
__device__ __forceinline__ void prim_point(const StageArgs &a, int x, int y, int z) {
    int i = (z * a.d.ny + y) * a.d.nx + x;
    if (!OSB_BC_OK(x >= 0 && x < a.d.nx && y >= 0 && y < a.d.ny && z >= 0 && z < a.d.nz, a.kerr)) i = 0;
    const S *Q = static_cast<const S *>(a.src);
    const size_t qs = a.src_stride;
    T *aux = static_cast<T *>(a.aux);
    const size_t as = a.aux_stride;

    const T rho = ld<POL, T>(Q + i), mx = ld<POL, T>(Q + qs + i), my = ld<POL, T>(Q + 2 * qs + i);
    const T mz = ld<POL, T>(Q + 3 * qs + i), e = ld<POL, T>(Q + 4 * qs + i);
    const T rinv = T(1) / rho;
    const T u = mx * rinv, v = my * rinv, w = mz * rinv;
    const T ke = T(0.5) * (mx * u + my * v + mz * w);
    // double-float: e holds rho E - e_ref, so p holds p - p_ref
    const T p = k_gm1<T>(a) * (e - ke);
    T temp;
    if constexpr (is_dd<T>)
        temp = k_gM2<T>(a) * (p + a.kdd.p_ref) * rinv;
    else
        temp = T(a.ph.gM2) * p * rinv;
    const T hmx = T(0.5) * mx, hmy = T(0.5) * my;
    aux[A_U * as + i] = u;
    aux[A_V * as + i] = v;
    aux[A_W * as + i] = w;
    aux[A_P * as + i] = p;
    aux[A_T * as + i] = temp;
    aux[A_PXX * as + i] = fma(hmx, u, p);
    aux[A_PYY * as + i] = fma(hmy, v, p);
    aux[A_PZZ * as + i] = fma(T(0.5) * mz, w, p);
    aux[A_PXY * as + i] = hmx * v;
    aux[A_PXZ * as + i] = hmx * w;
    aux[A_PYZ * as + i] = hmy * w;
}

template <typename S, typename T>
__global__ void __launch_bounds__(BX *BY) k_prim(const StageArgs a) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= a.d.nx || y >= a.d.ny) return;
    prim_point<LD_NC, S, T>(a, x, y, z);
}

// ---------------------------------------------------------------------------
// k_grad: velocity gradient -> div u, tau_ij, energy flux, viscous g-term
// ---------------------------------------------------------------------------
template <int POL, typename S, int R, bool SYM>
__device__ __forceinline__ void grad_point_dd(const StageArgs &a, int x, int y, int z, double *dg);

// Double-float, viscous form B: the gradient, tau, F_j, g_i and tau : grad u
// in double-float operations (g_i unscaled; the residual's weights for D_i g_i
// carry 1/(3 Re)).
// (1/2) rho u.u and (1/2) rho |omega|^2 at a point (Section 3.3), from
// double-float values, in FP64
__device__ __forceinline__ void point_diag_dd(double *dg, const dd &rho, const dd &u, const dd &v, const dd &w,
                                              const dd &w0, const dd &w1, const dd &w2) {
    const double r = double(rho), uu = double(u), vv = double(v), ww = double(w);
    const double o0 = double(w0), o1 = double(w1), o2 = double(w2);
    dg[0] = 0.5 * r * (uu * uu + vv * vv + ww * ww);
    dg[1] = 0.5 * r * (o0 * o0 + o1 * o1 + o2 * o2);
}

template <int POL, typename S, int R, bool SYM>
__device__ __forceinline__ void grad_point_dd_b(const StageArgs &a, int x, int y, int z, double *dg) {
    Nbr<R, SYM> nb;
    nb.init(x, y, z, a.d, a.kerr);
    const int i = nb.center();
    const Coef<dd> &c = a.cdd;
    dd *aux = static_cast<dd *>(a.aux);
    const size_t as = a.aux_stride;
    const dd *U = aux + A_U * as, *V = aux + A_V * as, *W = aux + A_W * as;
    const dd gxx = D1<R, 0, POL>(U, nb, c, PAR_X), gxy = D1<R, 1, POL>(U, nb, c, PAR_X), gxz = D1<R, 2, POL>(U, nb, c, PAR_X);
    const dd gyx = D1<R, 0, POL>(V, nb, c, PAR_Y), gyy = D1<R, 1, POL>(V, nb, c, PAR_Y), gyz = D1<R, 2, POL>(V, nb, c, PAR_Y);
    const dd gzx = D1<R, 0, POL>(W, nb, c, PAR_Z), gzy = D1<R, 1, POL>(W, nb, c, PAR_Z), gzz = D1<R, 2, POL>(W, nb, c, PAR_Z);
    const dd div = gxx + gyy + gzz;
    const dd ir = a.kdd.inv_re;
    const dd tdiv = dd(2.0 / 3.0) * div;
    const dd txx = ir * (gxx + gxx - tdiv), tyy = ir * (gyy + gyy - tdiv), tzz = ir * (gzz + gzz - tdiv);
    const dd txy = ir * (gxy + gyx), txz = ir * (gxz + gzx), tyz = ir * (gyz + gzy);
    const dd u = ld<POL, dd>(aux + A_U * as + i), v = ld<POL, dd>(aux + A_V * as + i);
    const dd w = ld<POL, dd>(aux + A_W * as + i), p = ld<POL, dd>(aux + A_P * as + i);
    const S *Q = static_cast<const S *>(a.src);
    const dd hE = fma(dd(0.5f, 0.f), ld<POL, dd>(Q + 4 * a.src_stride + i), p);
    aux[A_DIV * as + i] = div;
    aux[A_FX * as + i] = hE * u;
    aux[A_FY * as + i] = hE * v;
    aux[A_FZ * as + i] = hE * w;
    aux[A_GX * as + i] = gyy + gzz;
    aux[A_GY * as + i] = gxx + gzz;
    aux[A_GZ * as + i] = gxx + gyy;
    aux[A_TG * as + i] = txx * gxx + tyy * gyy + tzz * gzz + txy * (gxy + gyx) + txz * (gxz + gzx) +
                         tyz * (gyz + gzy);
    if (dg) point_diag_dd(dg, ld<POL, dd>(Q + i), u, v, w, gzy - gyz, gxz - gzx, gyx - gxy);
}

// dg (or nullptr): receives (1/2) rho u.u and (1/2) rho |omega|^2 of the point,
// omega_i = eps_ijk D_j u_k, for the first-stage diagnostics.
template <int POL, typename S, typename T, int R, bool VB, bool SYM = false>
__device__ __forceinline__ void grad_point(const StageArgs &a, int x, int y, int z, double *dg = nullptr) {
    if constexpr (is_dd<T> && !VB) {
        grad_point_dd<POL, S, R, SYM>(a, x, y, z, dg);
        return;
    } else if constexpr (is_dd<T>) {
        grad_point_dd_b<POL, S, R, SYM>(a, x, y, z, dg);
        return;
    } else {
    Nbr<R, SYM> nb;
    nb.init(x, y, z, a.d, a.kerr);
    const int i = nb.center();
    const FoldW<T> &fw = FoldPick<T>::get(a);
    T *aux = static_cast<T *>(a.aux);
    const size_t as = a.aux_stride;
    const T *U = aux + A_U * as, *V = aux + A_V * as, *W = aux + A_W * as;

    // s_ij = (1/Re) d_j u_i: the 1/Re of tau folded into the stencil weights
    const T sxx = add_d1<R, 0, POL>(T(0), U, nb, fw.d1ir[0], PAR_X), sxy = add_d1<R, 1, POL>(T(0), U, nb, fw.d1ir[1], PAR_X);
    const T sxz = add_d1<R, 2, POL>(T(0), U, nb, fw.d1ir[2], PAR_X), syx = add_d1<R, 0, POL>(T(0), V, nb, fw.d1ir[0], PAR_Y);
    const T syy = add_d1<R, 1, POL>(T(0), V, nb, fw.d1ir[1], PAR_Y), syz = add_d1<R, 2, POL>(T(0), V, nb, fw.d1ir[2], PAR_Y);
    const T szx = add_d1<R, 0, POL>(T(0), W, nb, fw.d1ir[0], PAR_Z), szy = add_d1<R, 1, POL>(T(0), W, nb, fw.d1ir[1], PAR_Z);
    const T szz = add_d1<R, 2, POL>(T(0), W, nb, fw.d1ir[2], PAR_Z);
    const T divs = sxx + syy + szz;  // (1/Re) div u
    const T tdivs = T(2.0 / 3.0) * divs;
    // tau_ij = (1/Re)(d_j u_i + d_i u_j - (2/3) div u delta_ij)
    const T txx = fma(T(2), sxx, -tdivs), tyy = fma(T(2), syy, -tdivs), tzz = fma(T(2), szz, -tdivs);
    const T txy = sxy + syx, txz = sxz + szx, tyz = syz + szy;
    const T u = ld<POL, T>(aux + A_U * as + i), v = ld<POL, T>(aux + A_V * as + i);
    const T w = ld<POL, T>(aux + A_W * as + i), p = ld<POL, T>(aux + A_P * as + i);
    const S *Q = static_cast<const S *>(a.src);
    const T hE = fma(T(0.5), ld<POL, T>(Q + 4 * a.src_stride + i), p);
    aux[A_DIV * as + i] = fw.Re * divs;
    if (!VB) {
        aux[A_FX * as + i] = hE * u - (u * txx + v * txy + w * txz);
        aux[A_FY * as + i] = hE * v - (u * txy + v * tyy + w * tyz);
        aux[A_FZ * as + i] = hE * w - (u * txz + v * tyz + w * tzz);
        // Phi_ii - (1/(3 Re)) sum_{k != i} d_k u_k
        const T third = T(1.0 / 3.0);
        aux[A_PXX * as + i] = fma(-third, syy + szz, ld<POL, T>(aux + A_PXX * as + i));
        aux[A_PYY * as + i] = fma(-third, sxx + szz, ld<POL, T>(aux + A_PYY * as + i));
        aux[A_PZZ * as + i] = fma(-third, sxx + syy, ld<POL, T>(aux + A_PZZ * as + i));
    } else {
        aux[A_FX * as + i] = hE * u;
        aux[A_FY * as + i] = hE * v;
        aux[A_FZ * as + i] = hE * w;
        // g_i scaled by 1/Re (the residual's weights for D_i g_i carry 1/3 only)
        aux[A_GX * as + i] = syy + szz;
        aux[A_GY * as + i] = sxx + szz;
        aux[A_GZ * as + i] = sxx + syy;
        // tau : grad u = Re sum_ij tau_ij s_ij, with s_ij + s_ji = tau_ij off the diagonal
        aux[A_TG * as + i] = fw.Re * fma(txx, sxx, fma(tyy, syy, fma(tzz, szz,
                                         fma(txy, txy, fma(txz, txz, tyz * tyz)))));
    }
    if (dg) {
        // omega = Re (s_zy - s_yz, s_xz - s_zx, s_yx - s_xy)
        const T rho = ld<POL, T>(Q + i);
        const T o0 = szy - syz, o1 = sxz - szx, o2 = syx - sxy;
        const double Re = double(fw.Re);
        dg[0] = double(T(0.5) * rho * fma(u, u, fma(v, v, w * w)));
        dg[1] = double(T(0.5) * rho * fma(o0, o0, fma(o1, o1, o2 * o2))) * (Re * Re);
    }
    }
}

// Double-float gradient kernel (viscous form A): the energy flux
// F_j = hE u_j - u_i tau_ij is expanded into products of a velocity with one
// gradient entry, tau_ij = (1/Re)(g_ij + g_ji - (2/3) div u delta_ij), and
// accumulated compensated; likewise Phi_ii - (1/(3Re)) sum_{k != i} g_kk.
__device__ __forceinline__ void acc_add(dd_acc &acc, const dd &w, const dd &x) { acc.add_prod(w, x.hi, x.lo); }

template <int POL, typename S, int R, bool SYM>
__device__ __forceinline__ void grad_point_dd(const StageArgs &a, int x, int y, int z, double *dg) {
    Nbr<R, SYM> nb;
    nb.init(x, y, z, a.d, a.kerr);
    const int i = nb.center();
    const Coef<dd> &c = a.cdd;
    dd *aux = static_cast<dd *>(a.aux);
    const size_t as = a.aux_stride;
    const dd *U = aux + A_U * as, *V = aux + A_V * as, *W = aux + A_W * as;
    const dd gxx = D1<R, 0, POL>(U, nb, c, PAR_X), gxy = D1<R, 1, POL>(U, nb, c, PAR_X), gxz = D1<R, 2, POL>(U, nb, c, PAR_X);
    const dd gyx = D1<R, 0, POL>(V, nb, c, PAR_Y), gyy = D1<R, 1, POL>(V, nb, c, PAR_Y), gyz = D1<R, 2, POL>(V, nb, c, PAR_Y);
    const dd gzx = D1<R, 0, POL>(W, nb, c, PAR_Z), gzy = D1<R, 1, POL>(W, nb, c, PAR_Z), gzz = D1<R, 2, POL>(W, nb, c, PAR_Z);
    dd_acc dv;
    const dd one(1.f, 0.f);
    acc_add(dv, one, gxx);
    acc_add(dv, one, gyy);
    acc_add(dv, one, gzz);
    const dd div = dv.get();
    const dd u = ld<POL, dd>(aux + A_U * as + i), v = ld<POL, dd>(aux + A_V * as + i);
    const dd w = ld<POL, dd>(aux + A_W * as + i), p = ld<POL, dd>(aux + A_P * as + i);
    const S *Q = static_cast<const S *>(a.src);
    const dd hE = dd_scale(ld<POL, dd>(Q + 4 * a.src_stride + i), 0.5f) + p;
    aux[A_DIV * as + i] = div;
    const dd ir = a.kdd.inv_re;
    const dd iru = ir * u, irv = ir * v, irw = ir * w;
    const dd m2u = dd_scale(iru, -2.f), m2v = dd_scale(irv, -2.f), m2w = dd_scale(irw, -2.f);
    const dd two3 = dd(2.0 / 3.0);
    const dd tdiv = two3 * div;  // (2/3) div u
    const dd niru = -iru, nirv = -irv, nirw = -irw;
    dd_acc fx, fy, fz;
    acc_add(fx, hE, u);
    acc_add(fx, m2u, gxx);
    acc_add(fx, iru, tdiv);
    acc_add(fx, nirv, gxy);
    acc_add(fx, nirv, gyx);
    acc_add(fx, nirw, gxz);
    acc_add(fx, nirw, gzx);
    acc_add(fy, hE, v);
    acc_add(fy, niru, gxy);
    acc_add(fy, niru, gyx);
    acc_add(fy, m2v, gyy);
    acc_add(fy, irv, tdiv);
    acc_add(fy, nirw, gyz);
    acc_add(fy, nirw, gzy);
    acc_add(fz, hE, w);
    acc_add(fz, niru, gxz);
    acc_add(fz, niru, gzx);
    acc_add(fz, nirv, gyz);
    acc_add(fz, nirv, gzy);
    acc_add(fz, m2w, gzz);
    acc_add(fz, irw, tdiv);
    aux[A_FX * as + i] = fx.get();
    aux[A_FY * as + i] = fy.get();
    aux[A_FZ * as + i] = fz.get();
    const dd nir3 = -(ir * dd(1.0 / 3.0));
    dd_acc px, py, pz;
    acc_add(px, one, ld<POL, dd>(aux + A_PXX * as + i));
    acc_add(px, nir3, gyy);
    acc_add(px, nir3, gzz);
    acc_add(py, one, ld<POL, dd>(aux + A_PYY * as + i));
    acc_add(py, nir3, gxx);
    acc_add(py, nir3, gzz);
    acc_add(pz, one, ld<POL, dd>(aux + A_PZZ * as + i));
    acc_add(pz, nir3, gxx);
    acc_add(pz, nir3, gyy);
    aux[A_PXX * as + i] = px.get();
    aux[A_PYY * as + i] = py.get();
    aux[A_PZZ * as + i] = pz.get();
    if (dg) point_diag_dd(dg, ld<POL, dd>(Q + i), u, v, w, gzy - gyz, gxz - gzx, gyx - gxy);
}

template <typename S, typename T, int R, bool VB, bool SYM>
__global__ void __launch_bounds__(BX *BY) k_grad(const StageArgs a) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (!a.diag_rec) {
        if (x >= a.d.nx || y >= a.d.ny) return;
        grad_point<LD_NC, S, T, R, VB, SYM>(a, x, y, z);
        return;
    }
    double dg[2] = {0.0, 0.0};
    if (x < a.d.nx && y < a.d.ny) grad_point<LD_NC, S, T, R, VB, SYM>(a, x, y, z, dg);
    block_record2(dg[0], dg[1], a.diag_rec);
}

// ---------------------------------------------------------------------------
// Double-float residual: every term of an equation goes into one compensated
// accumulator (dd_acc) -- the flux divergences, Laplacians and heat flux with
// their constant factors folded into the stencil weights, the advective
// products as products -- normalised once per equation.
// ---------------------------------------------------------------------------
template <int R, int AX, int POL, typename P, bool SYM>
__device__ __forceinline__ void acc_d1(dd_acc &acc, const P *__restrict__ f, const Nbr<R, SYM> &nb, const Coef<dd> &w,
                                       bool negate, int par) {
#pragma unroll
    for (int k = R; k >= 1; --k) {
        const dd wk = negate ? -w.d1[AX][k] : w.d1[AX][k];
        acc.add_wdiff(wk, nb_ld<R, AX, POL>(f, nb, k, par), nb_ld<R, AX, POL>(f, nb, -k, par));
    }
}
template <int R, int AX, int POL, typename P, bool SYM>
__device__ __forceinline__ void acc_d2(dd_acc &acc, const P *__restrict__ f, const Nbr<R, SYM> &nb, const Coef<dd> &w,
                                       const dd &f0, int par) {
    acc.add_prod(w.d2[AX][0], f0.hi, f0.lo);
#pragma unroll
    for (int k = R; k >= 1; --k)
        acc.add_wsum(w.d2[AX][k], nb_ld<R, AX, POL>(f, nb, k, par), nb_ld<R, AX, POL>(f, nb, -k, par));
}

// parity bits of the conserved fields rho, rho u, rho v, rho w, rho E
__device__ __forceinline__ constexpr int q_parity(int m) { return m == 1 ? PAR_X : (m == 2 ? PAR_Y : (m == 3 ? PAR_Z : PAR_EVEN)); }

// One axis of the advective half (double-float): acc_m += h D_AX q_m, and the
// mass flux -(1/2) D_AX (rho u_AX).
template <int R, int AX, int POL, typename S, bool SYM>
__device__ __forceinline__ void adv_axis_dd(dd_acc (&acc)[5], const S *Q, size_t qs, const Nbr<R, SYM> &nb,
                                            const Coef<dd> &c, const dd &h) {
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const dd d = D1<R, AX, POL>(Q + m * qs, nb, c, q_parity(m));
        acc[m].add_prod(h, d.hi, d.lo);
        if (m == 1 + AX) acc[0].add_prod(dd(-0.5f, 0.f), d.hi, d.lo);
    }
}

template <int POL, typename S, int R, bool VB, bool SYM>
__device__ __forceinline__ void resid_terms_dd(const StageArgs &a, const Nbr<R, SYM> &nb, int i, dd (&res)[5]) {
    const Coef<dd> &c = a.cdd;
    const S *Q = static_cast<const S *>(a.src);
    const size_t qs = a.src_stride;
    const dd *aux = static_cast<const dd *>(a.aux);
    const size_t as = a.aux_stride;
    const dd u = ld<POL, dd>(aux + A_U * as + i), v = ld<POL, dd>(aux + A_V * as + i);
    const dd w = ld<POL, dd>(aux + A_W * as + i), div = ld<POL, dd>(aux + A_DIV * as + i);
    const dd hu = dd_scale(u, -0.5f), hv = dd_scale(v, -0.5f), hw = dd_scale(w, -0.5f), hdiv = dd_scale(div, -0.5f);
    dd_acc acc[5];
    // advective + dilatation half of the skew-symmetric form; mass flux
    // (axis by axis: one derivative live at a time)
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        dd qc = ld<POL, dd>(Q + m * qs + i);
        if (m == 4) qc = qc + a.kdd.e_ref;  // the full rho E multiplies div u
        acc[m].add_prod(hdiv, qc.hi, qc.lo);
    }
    adv_axis_dd<R, 0, POL>(acc, Q, qs, nb, c, hu);
    adv_axis_dd<R, 1, POL>(acc, Q, qs, nb, c, hv);
    adv_axis_dd<R, 2, POL>(acc, Q, qs, nb, c, hw);
    // momentum fluxes -D_j Phi_ij and energy flux -D_j F'_j - c_ref div u
    const dd *Pxx = aux + A_PXX * as, *Pyy = aux + A_PYY * as, *Pzz = aux + A_PZZ * as;
    const dd *Pxy = aux + A_PXY * as, *Pxz = aux + A_PXZ * as, *Pyz = aux + A_PYZ * as;
    acc_d1<R, 0, POL>(acc[1], Pxx, nb, c, true, PAR_EVEN);
    acc_d1<R, 1, POL>(acc[1], Pxy, nb, c, true, PAR_XY);
    acc_d1<R, 2, POL>(acc[1], Pxz, nb, c, true, PAR_XZ);
    acc_d1<R, 0, POL>(acc[2], Pxy, nb, c, true, PAR_XY);
    acc_d1<R, 1, POL>(acc[2], Pyy, nb, c, true, PAR_EVEN);
    acc_d1<R, 2, POL>(acc[2], Pyz, nb, c, true, PAR_YZ);
    acc_d1<R, 0, POL>(acc[3], Pxz, nb, c, true, PAR_XZ);
    acc_d1<R, 1, POL>(acc[3], Pyz, nb, c, true, PAR_YZ);
    acc_d1<R, 2, POL>(acc[3], Pzz, nb, c, true, PAR_EVEN);
    acc_d1<R, 0, POL>(acc[4], aux + A_FX * as, nb, c, true, PAR_X);
    acc_d1<R, 1, POL>(acc[4], aux + A_FY * as, nb, c, true, PAR_Y);
    acc_d1<R, 2, POL>(acc[4], aux + A_FZ * as, nb, c, true, PAR_Z);
    acc[4].add_prod(-a.kdd.c_ref, div.hi, div.lo);
    // viscous Laplacians (1/Re)[sum_j L_j u_i + L_i u_i / 3]
    const dd *Uf = aux + A_U * as, *Vf = aux + A_V * as, *Wf = aux + A_W * as;
    if (!VB) {
        acc_d2<R, 0, POL>(acc[1], Uf, nb, a.cdd_vis43, u, PAR_X);
        acc_d2<R, 1, POL>(acc[1], Uf, nb, a.cdd_vis, u, PAR_X);
        acc_d2<R, 2, POL>(acc[1], Uf, nb, a.cdd_vis, u, PAR_X);
        acc_d2<R, 0, POL>(acc[2], Vf, nb, a.cdd_vis, v, PAR_Y);
        acc_d2<R, 1, POL>(acc[2], Vf, nb, a.cdd_vis43, v, PAR_Y);
        acc_d2<R, 2, POL>(acc[2], Vf, nb, a.cdd_vis, v, PAR_Y);
        acc_d2<R, 0, POL>(acc[3], Wf, nb, a.cdd_vis, w, PAR_Z);
        acc_d2<R, 1, POL>(acc[3], Wf, nb, a.cdd_vis, w, PAR_Z);
        acc_d2<R, 2, POL>(acc[3], Wf, nb, a.cdd_vis43, w, PAR_Z);
    } else {
        // form B: the viscous momentum term (with D_i g_i / 3) is also needed
        // as a value for the work u_i (viscous term) + tau : grad u
        dd_acc vx, vy, vz;
        acc_d2<R, 0, POL>(vx, Uf, nb, a.cdd_vis43, u, PAR_X);
        acc_d2<R, 1, POL>(vx, Uf, nb, a.cdd_vis, u, PAR_X);
        acc_d2<R, 2, POL>(vx, Uf, nb, a.cdd_vis, u, PAR_X);
        acc_d1<R, 0, POL>(vx, aux + A_GX * as, nb, a.cdd_g, false, PAR_EVEN);
        acc_d2<R, 0, POL>(vy, Vf, nb, a.cdd_vis, v, PAR_Y);
        acc_d2<R, 1, POL>(vy, Vf, nb, a.cdd_vis43, v, PAR_Y);
        acc_d2<R, 2, POL>(vy, Vf, nb, a.cdd_vis, v, PAR_Y);
        acc_d1<R, 1, POL>(vy, aux + A_GY * as, nb, a.cdd_g, false, PAR_EVEN);
        acc_d2<R, 0, POL>(vz, Wf, nb, a.cdd_vis, w, PAR_Z);
        acc_d2<R, 1, POL>(vz, Wf, nb, a.cdd_vis, w, PAR_Z);
        acc_d2<R, 2, POL>(vz, Wf, nb, a.cdd_vis43, w, PAR_Z);
        acc_d1<R, 2, POL>(vz, aux + A_GZ * as, nb, a.cdd_g, false, PAR_EVEN);
        const dd VX = vx.get(), VY = vy.get(), VZ = vz.get();
        acc[1].add_prod(dd(1.f, 0.f), VX.hi, VX.lo);
        acc[2].add_prod(dd(1.f, 0.f), VY.hi, VY.lo);
        acc[3].add_prod(dd(1.f, 0.f), VZ.hi, VZ.lo);
        acc[4].add_prod(u, VX.hi, VX.lo);
        acc[4].add_prod(v, VY.hi, VY.lo);
        acc[4].add_prod(w, VZ.hi, VZ.lo);
        const dd tg = ld<POL, dd>(aux + A_TG * as + i);
        acc[4].add_prod(dd(1.f, 0.f), tg.hi, tg.lo);
    }
    // heat flux kappa sum_j L_j T
    const dd *Tf = aux + A_T * as;
    const dd T0 = ld<POL, dd>(Tf + i);
    acc_d2<R, 0, POL>(acc[4], Tf, nb, a.cdd_heat, T0, PAR_EVEN);
    acc_d2<R, 1, POL>(acc[4], Tf, nb, a.cdd_heat, T0, PAR_EVEN);
    acc_d2<R, 2, POL>(acc[4], Tf, nb, a.cdd_heat, T0, PAR_EVEN);
#pragma unroll
    for (int m = 0; m < 5; ++m) res[m] = acc[m].get();
}

// One axis of the advective half of the skew-symmetric form (FP64 / FP32):
// res_m += -(1/2) u_AX D_AX q_m.  The momentum component along AX keeps its
// derivative, which the mass flux -(1/2) D_AX (rho u_AX) shares; for the other
// fields, up to radius 3, -(1/2) u_AX is folded into the R weights once and
// each tap goes straight into the sum (beyond radius 3 the R extra products
// cost more than the one multiply per field they save).
template <int R, int AX, int POL, typename S, typename T, bool SYM>
__device__ __forceinline__ void adv_axis(T (&res)[5], const S *Q, size_t qs, const Nbr<R, SYM> &nb, const Coef<T> &c,
                                         T vel) {
    const T hv = T(-0.5) * vel;
    T wk[R + 1];
#pragma unroll
    for (int k = 0; k <= R; ++k) wk[k] = (R <= 3 && k > 0) ? hv * c.d1[AX][k] : T(0);
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const S *f = Q + m * qs;
        if (m == 1 + AX || R > 3) {
            const T d = D1<R, AX, POL>(f, nb, c, q_parity(m));
            res[m] = fma(hv, d, res[m]);
            if (m == 1 + AX) res[0] = fma(T(-0.5), d, res[0]);
        } else {
            res[m] = add_d1<R, AX, POL>(res[m], f, nb, wk, q_parity(m));
        }
    }
}

// ---------------------------------------------------------------------------
// k_resid: residual and RK update (MODE 0) or residual only (MODE 1)
// ---------------------------------------------------------------------------
template <int POL, typename S, typename T, int R, int MODE, bool VB, bool SYM = false>
__device__ __forceinline__ void resid_point(const StageArgs &a, int x, int y, int z) {
    Nbr<R, SYM> nb;
    nb.init(x, y, z, a.d, a.kerr);
    const int i = nb.center();
    const Coef<T> &c = CoefPick<T>::get(a);
    const S *Q = static_cast<const S *>(a.src);
    const size_t qs = a.src_stride;
    const T *aux = static_cast<const T *>(a.aux);
    const size_t as = a.aux_stride;

    T res[5];
    if constexpr (is_dd<T>) {
        resid_terms_dd<POL, S, R, VB, SYM>(a, nb, i, res);
    } else {
    const T u = ld<POL, T>(aux + A_U * as + i), v = ld<POL, T>(aux + A_V * as + i);
    const T w = ld<POL, T>(aux + A_W * as + i), div = ld<POL, T>(aux + A_DIV * as + i);

    // advective + dilatation half of the skew-symmetric form,
    // res_m = -(1/2)(q_m div u + u_j D_j q_m), axis by axis
    const T hdiv = T(-0.5) * div;
#pragma unroll
    for (int m = 0; m < 5; ++m) res[m] = hdiv * ld<POL, T>(Q + m * qs + i);
    adv_axis<R, 0, POL>(res, Q, qs, nb, c, u);
    adv_axis<R, 1, POL>(res, Q, qs, nb, c, v);
    adv_axis<R, 2, POL>(res, Q, qs, nb, c, w);
    // momentum fluxes -D_j Phi_ij and energy flux -D_j F_j, tap by tap into
    // the equation's sum
    const T *Pxx = aux + A_PXX * as, *Pyy = aux + A_PYY * as, *Pzz = aux + A_PZZ * as;
    const T *Pxy = aux + A_PXY * as, *Pxz = aux + A_PXZ * as, *Pyz = aux + A_PYZ * as;
    res[1] = add_d1<R, 0, POL>(res[1], Pxx, nb, c.d1[0], PAR_EVEN, true);
    res[1] = add_d1<R, 1, POL>(res[1], Pxy, nb, c.d1[1], PAR_XY, true);
    res[1] = add_d1<R, 2, POL>(res[1], Pxz, nb, c.d1[2], PAR_XZ, true);
    res[2] = add_d1<R, 0, POL>(res[2], Pxy, nb, c.d1[0], PAR_XY, true);
    res[2] = add_d1<R, 1, POL>(res[2], Pyy, nb, c.d1[1], PAR_EVEN, true);
    res[2] = add_d1<R, 2, POL>(res[2], Pyz, nb, c.d1[2], PAR_YZ, true);
    res[3] = add_d1<R, 0, POL>(res[3], Pxz, nb, c.d1[0], PAR_XZ, true);
    res[3] = add_d1<R, 1, POL>(res[3], Pyz, nb, c.d1[1], PAR_YZ, true);
    res[3] = add_d1<R, 2, POL>(res[3], Pzz, nb, c.d1[2], PAR_EVEN, true);
    res[4] = add_d1<R, 0, POL>(res[4], aux + A_FX * as, nb, c.d1[0], PAR_X, true);
    res[4] = add_d1<R, 1, POL>(res[4], aux + A_FY * as, nb, c.d1[1], PAR_Y, true);
    res[4] = add_d1<R, 2, POL>(res[4], aux + A_FZ * as, nb, c.d1[2], PAR_Z, true);
    // viscous Laplacians (1/Re)[sum_j L_j u_i + L_i u_i / 3] and the heat flux
    // kappa sum_j L_j T, with 1/Re, 4/(3 Re) and kappa folded into the weights
    const FoldW<T> &fw = FoldPick<T>::get(a);
    {
        const T *Uf = aux + A_U * as, *Vf = aux + A_V * as, *Wf = aux + A_W * as, *Tf = aux + A_T * as;
        T vx = VB ? T(0) : res[1], vy = VB ? T(0) : res[2], vz = VB ? T(0) : res[3];
        vx = fma(fw.c_u, u, vx);
        vx = add_d2<R, 0, POL>(vx, Uf, nb, fw.vis43[0], PAR_X);
        vx = add_d2<R, 1, POL>(vx, Uf, nb, fw.vis[1], PAR_X);
        vx = add_d2<R, 2, POL>(vx, Uf, nb, fw.vis[2], PAR_X);
        vy = fma(fw.c_v, v, vy);
        vy = add_d2<R, 0, POL>(vy, Vf, nb, fw.vis[0], PAR_Y);
        vy = add_d2<R, 1, POL>(vy, Vf, nb, fw.vis43[1], PAR_Y);
        vy = add_d2<R, 2, POL>(vy, Vf, nb, fw.vis[2], PAR_Y);
        vz = fma(fw.c_w, w, vz);
        vz = add_d2<R, 0, POL>(vz, Wf, nb, fw.vis[0], PAR_Z);
        vz = add_d2<R, 1, POL>(vz, Wf, nb, fw.vis[1], PAR_Z);
        vz = add_d2<R, 2, POL>(vz, Wf, nb, fw.vis43[2], PAR_Z);
        if (VB) {
            // form B: the viscous momentum term (with D_i g_i / 3) is also
            // needed as a value, for the work u_i (viscous term) + tau : grad u
            vx = add_d1<R, 0, POL>(vx, aux + A_GX * as, nb, fw.g[0], PAR_EVEN);
            vy = add_d1<R, 1, POL>(vy, aux + A_GY * as, nb, fw.g[1], PAR_EVEN);
            vz = add_d1<R, 2, POL>(vz, aux + A_GZ * as, nb, fw.g[2], PAR_EVEN);
            res[4] += fma(u, vx, fma(v, vy, fma(w, vz, ld<POL, T>(aux + A_TG * as + i))));
            res[1] += vx;
            res[2] += vy;
            res[3] += vz;
        } else {
            res[1] = vx;
            res[2] = vy;
            res[3] = vz;
        }
        res[4] = fma(fw.c_T, ld<POL, T>(Tf + i), res[4]);
        res[4] = add_d2<R, 0, POL>(res[4], Tf, nb, fw.heat[0], PAR_EVEN);
        res[4] = add_d2<R, 1, POL>(res[4], Tf, nb, fw.heat[1], PAR_EVEN);
        res[4] = add_d2<R, 2, POL>(res[4], Tf, nb, fw.heat[2], PAR_EVEN);
    }
    }

    if (a.closure) {
#pragma unroll
        for (int m = 0; m < 5; ++m) res[m] += T(ld<POL, float>(a.closure + (size_t)m * a.d.n + i));
    }
    if (MODE == 0) {
        T *qo = static_cast<T *>(a.q_out);
        if constexpr (sizeof(T) == 8) {
            // FP64 and double-float: the accumulator update in FP64; the
            // double-float path also writes the next step's double-float
            // copy of the accumulator in the last stage
            T *cp = static_cast<T *>(a.u32_out);
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const double Ui = ld<POL, double>(a.U_in + m * a.u_stride + i);
                const double Rm = double(res[m]);
                const double Un = fma(a.beta_dt, Rm, Ui);
                a.U_out[m * a.u_stride + i] = Un;
                const double off = (is_dd<T> && m == 4) ? a.e_ref : 0.0;  // double-float registers: rho E - e_ref
                if (qo) qo[m * a.q_stride + i] = T(fma(a.alpha_dt, Rm, Ui) - off);
                if (cp) cp[m * a.q_stride + i] = T(Un - off);
            }
        } else {
            // FP32 path: the FP64 accumulator takes one DADD per field; the
            // increment and the stage value are formed in FP32 and converted
            // on the integer pipes.
            float *cp = static_cast<float *>(a.u32_out);
            const float bdt = float(a.beta_dt), adt = float(a.alpha_dt);
#pragma unroll
            for (int m = 0; m < 5; ++m) {
                const double Ui = ld<POL, double>(a.U_in + m * a.u_stride + i);
                const double Un = Ui + f2d_bits(bdt * float(res[m]));
                a.U_out[m * a.u_stride + i] = Un;
                if (qo) qo[m * a.q_stride + i] = T(fmaf(adt, float(res[m]), d2f_bits(Ui)));
                if (cp) cp[m * a.q_stride + i] = d2f_bits(Un);
            }
        }
    } else {
#pragma unroll
        for (int m = 0; m < 5; ++m) a.R_out[m * a.R_stride + i] = double(res[m]);
    }
}

template <typename S, typename T, int R, int MODE, bool VB, bool SYM>
__global__ void __launch_bounds__(BX *BY) k_resid(const StageArgs a) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= a.d.nx || y >= a.d.ny) return;
    resid_point<LD_NC, S, T, R, MODE, VB, SYM>(a, x, y, z);
}

// Double-float residual kernel with explicit occupancy targets: four CTAs per
// SM up to order 4 (64 registers, a few bytes spilled, 32 resident warps to
// hide the neighbour-load latency this kernel waits on), two for orders 6 and
// 8 (three spill hundreds of bytes and measured slower at order 8), one (all
// registers, no spills) for orders 10 and 12.
template <typename S, int R, int MODE, bool VB, bool SYM>
__global__ void __launch_bounds__(BX *BY, R <= 2 ? 4 : (R <= 4 ? 2 : 1)) k_resid_dd(const StageArgs a) {
    const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y, z = blockIdx.z;
    if (x >= a.d.nx || y >= a.d.ny) return;
    resid_point<LD_NC, S, dd, R, MODE, VB, SYM>(a, x, y, z);
}

// SYM: the mirrored-stencil kernels for grids with symmetry boundaries.
template <typename S, typename T, int R, bool VB, bool SYM>
cudaError_t launch_stage_typed(const StageArgs &a, int mode) {
    dim3 blk(BX, BY, 1), grd((a.d.nx + BX - 1) / BX, (a.d.ny + BY - 1) / BY, a.d.nz);
    if (a.ev) cudaEventRecord(a.ev[0], a.stream);
    k_prim<S, T><<<grd, blk, 0, a.stream>>>(a);
    if (a.ev) cudaEventRecord(a.ev[1], a.stream);
    k_grad<S, T, R, VB, SYM><<<grd, blk, 0, a.stream>>>(a);
    if (a.ev) cudaEventRecord(a.ev[2], a.stream);
    if constexpr (is_dd<T>) {
        if (mode == 0)
            k_resid_dd<S, R, 0, VB, SYM><<<grd, blk, 0, a.stream>>>(a);
        else
            k_resid_dd<S, R, 1, VB, SYM><<<grd, blk, 0, a.stream>>>(a);
    } else {
        if (mode == 0)
            k_resid<S, T, R, 0, VB, SYM><<<grd, blk, 0, a.stream>>>(a);
        else
            k_resid<S, T, R, 1, VB, SYM><<<grd, blk, 0, a.stream>>>(a);
    }
    if (a.ev) cudaEventRecord(a.ev[3], a.stream);
    return cudaGetLastError();
}

template <typename S, typename T, int R, bool SYM>
cudaError_t launch_stage_form(const StageArgs &a, int mode) {
    if (a.visc_form == OSB_VISC_B) return launch_stage_typed<S, T, R, true, SYM>(a, mode);
    return launch_stage_typed<S, T, R, false, SYM>(a, mode);
}

template <int R, bool SYM = false>
cudaError_t launch_stage(const StageArgs &a, int mode) {
    if (a.precision == OSB_FP64) return launch_stage_form<double, double, R, SYM>(a, mode);
    if (a.precision == OSB_DF64)
        return a.src_is_f64 ? launch_stage_form<double, dd, R, SYM>(a, mode) : launch_stage_form<dd, dd, R, SYM>(a, mode);
    if (a.src_is_f64) return launch_stage_form<double, float, R, SYM>(a, mode);
    return launch_stage_form<float, float, R, SYM>(a, mode);
}

template <int R, bool SYM = false>
cudaError_t stage_entry(const StageArgs &a) {
    return launch_stage<R, SYM>(a, 0);
}
template <int R, bool SYM = false>
cudaError_t residual_entry(const StageArgs &a) {
    return launch_stage<R, SYM>(a, 1);
}

}  // namespace osb

#define OSB_DEFINE_ORDER(ORDER)                                                 \
    namespace osb {                                                            \
    OrderKernels kernels_o##ORDER() {                                          \
        return OrderKernels{ORDER, &stage_entry<ORDER / 2>, &residual_entry<ORDER / 2>}; \
    }                                                                          \
    }

// Grids with symmetry boundaries: the three-kernel stage with mirrored
// neighbour loads, in every precision.
#define OSB_DEFINE_ORDER_SYM(ORDER)                                                         \
    namespace osb {                                                                        \
    OrderKernels kernels_sym_o##ORDER() {                                                  \
        return OrderKernels{ORDER, &stage_entry<ORDER / 2, true>, &residual_entry<ORDER / 2, true>}; \
    }                                                                                      \
    }
