// zrhs_narrow.cuh -- the z-march residual kernel of the FP32 stage at orders 6
// and 8 (radius 3, 4), on narrow 32 x 4 tiles, three CTAs of 128 threads per
// SM.  Included by zmarch.cuh after k_zrhs, whose work it does at those radii.
//
// At radius 3-4 k_zrhs holds a ring of 2R+3 haloed planes of nine fields
// (201 KB of shared memory at radius 4) and thirteen register queues of 2R+1
// values (195 registers): one CTA of eight warps per SM, whose dependent
// floating-point chains leave issue at ~43%.  Here:
//   * the ring holds the output plane's haloed rectangle only (re-read from
//     L2 R planes after its columns first arrived as the lead plane) and the
//     lead plane's tile columns, two slots each (one in use, one in flight);
//   * the z derivatives of the conserved fields keep their register queues
//     (the advective terms multiply them by the centre velocity), while the
//     z-derivative and z-Laplacian parts of the four flux and viscous sums are
//     SCATTERED: each lead value adds its taps to 2R+1 pending sums, one per
//     plane that its stencil reaches, and the output plane's sum is complete
//     when the lead reaches it + R;
//   * 61 KB of shared memory and under 170 registers give three resident CTAs
//     (twelve warps per SM).
// Residual, stencils and update are those of k_zrhs (Section 3.3 equations,
// regrouped as in stage.cuh); only the summation order of the z taps differs.
#pragma once

namespace osb {
namespace zm {

template <int R>
struct GeoN {
    static constexpr int TYN = 4, NTN = TX * TYN;  // 32 x 4 tile, 128 threads
    static constexpr int RW = TX + 2 * CX, RH = TYN + 2 * R, RA = RW * RH;
    static constexpr int RAP = (RA + 31) / 32 * 32;  // ring plane stride (TMA destinations: 128-byte aligned)
};

enum ColFieldN { CN_RHO = 0, CN_M0, CN_M1, CN_M2, CN_E, CN_FZ, CN_GZ, CN_N };

static_assert(sizeof(ZTmaN::rect) / sizeof(CUtensorMap) == RF_N && sizeof(ZTmaN::col) / sizeof(CUtensorMap) == CN_N,
              "descriptor counts follow the ring and column fields");

template <int R>
struct RhsSmemN {
    using G = GeoN<R>;
    float ring[2][RF_N][G::RAP];   // output-plane rectangles (TMA destinations first)
    float col[2][CN_N][G::NTN];    // lead-plane columns
    float der[DF_N][G::RA];
    int off[G::RA];
    unsigned long long bars[2];
};


// In-plane offsets of the narrow rectangle (tile + R halo, periodic wrap).
template <int R>
__device__ __forceinline__ void make_offsets_n(int *off, int x0, int y0, const Dims &d, int *kerr) {
    using G = GeoN<R>;
    for (int e = threadIdx.x; e < G::RA; e += G::NTN) {
        const int ry = e / G::RW, rx = e - ry * G::RW;
        const int v = wrapc(y0 + ry - R, d.ny) * d.nx + wrapc(x0 + rx - CX, d.nx);
        off[e] = OSB_BC_OK(v >= 0 && v < d.nx * d.ny, kerr) ? v : 0;
    }
}

template <int R>
__global__ void __launch_bounds__(GeoN<R>::NTN, 3) k_zrhs_n(const StageArgs a, int zchunk,
                                                             const __grid_constant__ ZTmaN tm) {
    using G = GeoN<R>;
    constexpr int Q = 2 * R + 1, NTN = G::NTN, W = G::RW;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    RhsSmemN<R> &S = *reinterpret_cast<RhsSmemN<R> *>(smem_raw);
    const Dims d = a.d;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * G::TYN;
    const int z0 = blockIdx.z * zchunk, z1 = min(z0 + zchunk, d.nz);
    const int ce = (ty + R) * W + tx + CX;
    const bool active = (x0 + tx < d.nx) && (y0 + ty < d.ny);
    const int plane = d.nx * d.ny;
    const float *Qg = static_cast<const float *>(a.src);
    const size_t qs = a.src_stride, as = a.aux_stride;
    const float *aux = static_cast<const float *>(a.aux);
    const Coef<float> &c = a.c32;
    const FoldW<float> &fw = a.f32;
    const bool use_tma = tm.use && x0 >= CX && x0 - CX + W <= d.nx && y0 >= R && y0 + G::TYN + R <= d.ny;
    const bool vec16 = (d.nx % 4) == 0;  // 16-byte chunks of a row never straddle the wrap

    if (tid == 0) {
        for (int s = 0; s < 2; ++s) bar_init(smem_u32(&S.bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    make_offsets_n<R>(S.off, x0, y0, d, a.kerr);
    __syncthreads();
    const int coff = S.off[ce];
    uint32_t phase = 0;

    const float *rsrc[RF_N] = {Qg, Qg + qs, Qg + 2 * qs, Qg + 3 * qs, Qg + 4 * qs,
                               aux + A_FX * as, aux + A_FY * as, aux + A_GX * as, aux + A_GY * as};
    const float *csrc[CN_N] = {Qg, Qg + qs, Qg + 2 * qs, Qg + 3 * qs, Qg + 4 * qs, aux + A_FZ * as, aux + A_GZ * as};
    const int Lbeg = z0 - R, Lend = z1 + R;  // lead planes [Lbeg, Lend); output plane zo = L - R
    // Step L loads the lead plane's tile columns and, once zo = L - R is an
    // output plane of this chunk, zo's haloed rectangle, into slot L mod 2.
    auto issue = [&](int L) {
        const int s = L & 1;
        const bool rect = L - R >= z0;
        const int zl = wrapz(L, d.nz), zr = wrapz(L - R, d.nz);
        if (use_tma) {
            if (tid == 0) {
                const uint32_t bar = smem_u32(&S.bars[s]);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect(bar, (uint32_t)((CN_N * NTN + (rect ? RF_N * G::RA : 0)) * sizeof(float)));
#pragma unroll
                for (int f = 0; f < CN_N; ++f) tma_load3(&S.col[s][f][0], &tm.col[f], x0, y0, zl, bar);
                if (rect) {
#pragma unroll
                    for (int f = 0; f < RF_N; ++f) tma_load3(&S.ring[s][f][0], &tm.rect[f], x0 - CX, y0 - R, zr, bar);
                }
            }
        } else {
            const size_t zbl = (size_t)zl * plane, zbr = (size_t)zr * plane;
            if (vec16) {
                // columns: TYN rows of TX points, 16-byte chunks
                for (int ch = tid; ch < CN_N * NTN / 4; ch += NTN) {
                    const int f = ch / (NTN / 4), t4 = ch % (NTN / 4);
                    const int row = t4 / (TX / 4), j = t4 % (TX / 4);
                    cp_async16_cg(&S.col[s][f][row * TX + 4 * j], csrc[f] + zbl + S.off[(row + R) * W + CX + 4 * j]);
                }
                if (rect) {
                    for (int ch = tid; ch < G::RA / 4; ch += NTN) {
                        const int e = ch * 4;
                        const size_t g = zbr + S.off[e];
#pragma unroll
                        for (int f = 0; f < RF_N; ++f) cp_async16_cg(&S.ring[s][f][e], rsrc[f] + g);
                    }
                }
            } else {
#pragma unroll
                for (int f = 0; f < CN_N; ++f) cp_async4(&S.col[s][f][tid], csrc[f] + zbl + coff);
                if (rect) {
                    for (int e = tid; e < G::RA; e += NTN) {
                        const size_t g = zbr + S.off[e];
#pragma unroll
                        for (int f = 0; f < RF_N; ++f) cp_async4(&S.ring[s][f][e], rsrc[f] + g);
                    }
                }
            }
            cp_commit();
        }
    };
    auto wait_step = [&](int L) {
        if (use_tma) {
            const int s = L & 1;
            if (!bar_wait(smem_u32(&S.bars[s]), (phase >> s) & 1u) && tid == 0 && a.kerr) atomicOr(a.kerr, KERR_WAIT);
            phase ^= 1u << s;
        } else {
            cp_wait<0>();
        }
    };

    // conserved fields along z (planes L-2R .. L), for the advective z terms
    float qQ[5][Q];
    // pending z sums of the four flux and viscous equations: position i holds
    // plane L - R + i; -D_z(Phi_xz, Phi_yz, Phi_zz, F_z) plus the off-centre
    // taps of the z Laplacians of u, v, w, T (centre weights at the output)
    float zs[4][Q];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
#pragma unroll
        for (int m = 0; m < 5; ++m) qQ[m][k] = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) zs[m][k] = 0.f;
    }
    const float third = 1.f / 3.f, gm1 = float(a.ph.gm1), gM2 = float(a.ph.gM2);
    const float bdt = float(a.beta_dt), adt = float(a.alpha_dt);
    float *qo = static_cast<float *>(a.q_out);
    float *cp = static_cast<float *>(a.u32_out);

    issue(Lbeg);
#pragma unroll 1
    for (int L = Lbeg; L < Lend; ++L) {
        wait_step(L);
        __syncthreads();  // everyone is done with slot (L + 1) mod 2 from step L - 1
        if (L + 1 < Lend) issue(L + 1);
        const int s = L & 1;
        {   // lead plane: this thread's column
            const float rho = S.col[s][CN_RHO][tid], m0 = S.col[s][CN_M0][tid], m1 = S.col[s][CN_M1][tid],
                        m2 = S.col[s][CN_M2][tid], e = S.col[s][CN_E][tid];
            const float ri = __fdividef(1.f, rho);
            const float u = m0 * ri, v = m1 * ri, w = m2 * ri;
            const float p = gm1 * (e - 0.5f * (m0 * u + m1 * v + m2 * w));
            const float T = gM2 * p * ri;
            const float pf[4] = {0.5f * m0 * w, 0.5f * m1 * w, fmaf(-third, S.col[s][CN_GZ][tid], fmaf(0.5f * m2, w, p)),
                                 S.col[s][CN_FZ][tid]};
            const float vf[4] = {u, v, w, T};
            const float *wl[4] = {fw.vis[2], fw.vis[2], fw.vis43[2], fw.heat[2]};
            qpush(qQ[0], rho);
            qpush(qQ[1], m0);
            qpush(qQ[2], m1);
            qpush(qQ[3], m2);
            qpush(qQ[4], e);
            // this plane's taps into the sums of planes L -+ k: -c_k f and
            // +c_k f for the flux divergence, w_k f on both sides for the
            // Laplacian
#pragma unroll
            for (int m = 0; m < 4; ++m) {
#pragma unroll
                for (int k = 1; k <= R; ++k) {
                    const float lap = wl[m][k] * vf[m];
                    zs[m][R - k] = fmaf(-c.d1[2][k], pf[m], zs[m][R - k] + lap);
                    zs[m][R + k] = fmaf(c.d1[2][k], pf[m], zs[m][R + k] + lap);
                }
            }
        }
        const int zo = L - R;
        if (zo >= z0) {
            size_t i = (size_t)zo * plane + coff;
            if (!OSB_BC_OK(!active || (zo >= 0 && zo < d.nz && coff >= 0 && coff < plane), a.kerr)) i = 0;
            double Ui[5];
#pragma unroll
            for (int m = 0; m < 5; ++m) Ui[m] = a.U_in[m * a.u_stride + i];
            const float divc = aux[A_DIV * as + i];
            const float(*rg)[G::RAP] = S.ring[s];
            // point-wise fields of the output plane over the rectangle
            for (int e = tid; e < G::RA; e += NTN) {
                const float rho = rg[RF_RHO][e], m0 = rg[RF_M0][e], m1 = rg[RF_M1][e], m2 = rg[RF_M2][e],
                            en = rg[RF_E][e];
                const float ri = __fdividef(1.f, rho);
                const float u = m0 * ri, v = m1 * ri, w = m2 * ri;
                const float p = gm1 * (en - 0.5f * (m0 * u + m1 * v + m2 * w));
                S.der[DF_U][e] = u;
                S.der[DF_V][e] = v;
                S.der[DF_W][e] = w;
                S.der[DF_T][e] = gM2 * p * ri;
                S.der[DF_PXX][e] = fmaf(-third, rg[RF_GX][e], fmaf(0.5f * m0, u, p));
                S.der[DF_PYY][e] = fmaf(-third, rg[RF_GY][e], fmaf(0.5f * m1, v, p));
                S.der[DF_PXY][e] = 0.5f * m0 * v;
                S.der[DF_PXZ][e] = 0.5f * m0 * w;
                S.der[DF_PYZ][e] = 0.5f * m1 * w;
            }
            __syncthreads();
            const float u = S.der[DF_U][ce], v = S.der[DF_V][ce], w = S.der[DF_W][ce], T = S.der[DF_T][ce];
            float res[5];
            {   // advective half of the skew-symmetric form and dilatation (as in k_zrhs)
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
                    const float *f = rg[RF_RHO + m];
                    if (m == 1 || R > 3) {
                        const float dx = sdx1<R>(f, ce, c.d1[0]);
                        res[m] = fmaf(hu, dx, res[m]);
                        if (m == 1) res[0] = fmaf(-0.5f, dx, res[0]);
                    } else {
                        res[m] = acc_s1<R, 1>(res[m], f, ce, wx);
                    }
                    if (m == 2 || R > 3) {
                        const float dy = acc_s1<R, W>(0.f, f, ce, c.d1[1]);
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
            // in-plane momentum and energy flux divergences, tap by tap
            res[1] = acc_s1<R, 1>(res[1], S.der[DF_PXX], ce, c.d1[0], true);
            res[1] = acc_s1<R, W>(res[1], S.der[DF_PXY], ce, c.d1[1], true);
            res[2] = acc_s1<R, 1>(res[2], S.der[DF_PXY], ce, c.d1[0], true);
            res[2] = acc_s1<R, W>(res[2], S.der[DF_PYY], ce, c.d1[1], true);
            res[3] = acc_s1<R, 1>(res[3], S.der[DF_PXZ], ce, c.d1[0], true);
            res[3] = acc_s1<R, W>(res[3], S.der[DF_PYZ], ce, c.d1[1], true);
            res[4] = acc_s1<R, 1>(res[4], rg[RF_FX], ce, c.d1[0], true);
            res[4] = acc_s1<R, W>(res[4], rg[RF_FY], ce, c.d1[1], true);
            // in-plane viscous Laplacians and heat flux, centre weights of all axes
            res[1] = fmaf(fw.c_u, u, res[1]);
            res[1] = acc_s2<R, 1>(res[1], S.der[DF_U], ce, fw.vis43[0]);
            res[1] = acc_s2<R, W>(res[1], S.der[DF_U], ce, fw.vis[1]);
            res[2] = fmaf(fw.c_v, v, res[2]);
            res[2] = acc_s2<R, 1>(res[2], S.der[DF_V], ce, fw.vis[0]);
            res[2] = acc_s2<R, W>(res[2], S.der[DF_V], ce, fw.vis43[1]);
            res[3] = fmaf(fw.c_w, w, res[3]);
            res[3] = acc_s2<R, 1>(res[3], S.der[DF_W], ce, fw.vis[0]);
            res[3] = acc_s2<R, W>(res[3], S.der[DF_W], ce, fw.vis[1]);
            res[4] = fmaf(fw.c_T, T, res[4]);
            res[4] = acc_s2<R, 1>(res[4], S.der[DF_T], ce, fw.heat[0]);
            res[4] = acc_s2<R, W>(res[4], S.der[DF_T], ce, fw.heat[1]);
            // the z parts, complete now that the lead is R planes past zo
#pragma unroll
            for (int m = 0; m < 4; ++m) res[m + 1] += zs[m][0];
            if (a.closure) {
#pragma unroll
                for (int m = 0; m < 5; ++m) res[m] += a.closure[(size_t)m * d.n + i];
            }
            if (active) {
                auto update = [&](auto from_src) {
#pragma unroll
                    for (int m = 0; m < 5; ++m) {
                        const double Un = Ui[m] + f2d_bits(bdt * res[m]);
                        a.U_out[m * a.u_stride + i] = Un;
                        if (qo)
                            qo[m * a.q_stride + i] =
                                fmaf(adt, res[m], decltype(from_src)::value ? qQ[m][R] : d2f_bits(Ui[m]));
                        if (cp) cp[m * a.q_stride + i] = d2f_bits(Un);
                    }
                };
                if (a.src_is_u32)
                    update(std::true_type{});
                else
                    update(std::false_type{});
            }
        }
        // the pending sums move one plane on
#pragma unroll
        for (int m = 0; m < 4; ++m) {
#pragma unroll
            for (int k = 0; k < Q - 1; ++k) zs[m][k] = zs[m][k + 1];
            zs[m][Q - 1] = 0.f;
        }
    }
    if (!use_tma) cp_wait<0>();
}

template <int R>
constexpr size_t rhs_smem_n() {
    static_assert(GeoN<R>::RAP * sizeof(float) % 128 == 0 && offsetof(RhsSmemN<R>, ring) == 0 &&
                      offsetof(RhsSmemN<R>, col) % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
    return sizeof(RhsSmemN<R>);
}

}  // namespace zm
}  // namespace osb
