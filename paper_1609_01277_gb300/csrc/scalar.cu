// scalar.cu -- scalar advection-diffusion on the periodic box [0, 2 pi)^3, the
// equation of the paper's wave-propagation (Section 3.1) and
// manufactured-solution (Section 3.2) tests:
//
//   d phi/dt + d_j(phi a_j - k d_j phi) + S = 0,   a_j, k constant,
//   R(phi) = - sum_j a_j D_j phi + k sum_j L_j phi - S,
//
// advanced by the same low-storage RK3 scheme as the flow solver (Section
// 2.4), in FP64.  The work is FP64-arithmetic bound on GB300 (two FP64
// operations per stencil tap against 40 B of HBM traffic per point-stage),
// so along each axis the two stencils are applied as one: with
// c_k, d_k the first/second-derivative weights (already / h, / h^2),
//   -a D f + k L f = k d_0 f_0 + sum_k [(k d_k - a c_k) f_{+k} + (k d_k + a c_k) f_{-k}],
// one DFMA per tap instead of two operations per tap per operator.  The
// centre weights of all axes are summed into one multiply.  An axis with one
// point carries no derivative.
#include <cstring>

#include "osb_internal.cuh"

namespace osb {
namespace {

struct ScalarW {
    double wp[3][MAXR + 1];  // weight of f_{+k} along each axis
    double wm[3][MAXR + 1];  // weight of f_{-k}
    double w0;               // sum of the centre weights
    int active[3];           // axis has more than one point
};

struct ScalarStage {
    const double *src;  // stencil source q_{k-1}
    const double *U_in; // accumulator at the point
    double *U_out;
    double *q_out;      // next stencil source, or nullptr (last stage)
    const double *S;    // source, or nullptr
    double adt, bdt;    // alpha_k dt, beta_k dt
    int nx, ny, nz;
};

constexpr int SX = 32, SY = 8;

__device__ __forceinline__ int wrapi(int i, int n) {
    i %= n;
    return i < 0 ? i + n : i;
}

template <int R>
__global__ void __launch_bounds__(SX *SY) k_scalar_stage(const ScalarStage s, const ScalarW w) {
    const int x = blockIdx.x * SX + threadIdx.x, y = blockIdx.y * SY + threadIdx.y, z = blockIdx.z;
    if (x >= s.nx || y >= s.ny) return;
    const size_t plane = (size_t)s.nx * s.ny;
    const size_t row = (size_t)y * s.nx, zoff = (size_t)z * plane;
    const size_t i = zoff + row + x;
    const double *f = s.src;
    double r = w.w0 * __ldg(f + i);
    if (w.active[0]) {
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            r = fma(w.wp[0][k], __ldg(f + zoff + row + wrapi(x + k, s.nx)), r);
            r = fma(w.wm[0][k], __ldg(f + zoff + row + wrapi(x - k, s.nx)), r);
        }
    }
    if (w.active[1]) {
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            r = fma(w.wp[1][k], __ldg(f + zoff + (size_t)wrapi(y + k, s.ny) * s.nx + x), r);
            r = fma(w.wm[1][k], __ldg(f + zoff + (size_t)wrapi(y - k, s.ny) * s.nx + x), r);
        }
    }
    if (w.active[2]) {
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            r = fma(w.wp[2][k], __ldg(f + (size_t)wrapi(z + k, s.nz) * plane + row + x), r);
            r = fma(w.wm[2][k], __ldg(f + (size_t)wrapi(z - k, s.nz) * plane + row + x), r);
        }
    }
    if (s.S) r -= __ldg(s.S + i);
    const double u = s.U_in[i];
    if (s.q_out) s.q_out[i] = fma(s.adt, r, u);
    s.U_out[i] = fma(s.bdt, r, u);
}

template <int R>
cudaError_t launch_scalar_stage(const ScalarStage &s, const ScalarW &w, cudaStream_t st) {
    dim3 blk(SX, SY, 1), grd((s.nx + SX - 1) / SX, (s.ny + SY - 1) / SY, s.nz);
    k_scalar_stage<R><<<grd, blk, 0, st>>>(s, w);
    return cudaGetLastError();
}

cudaError_t scalar_stage(int order, const ScalarStage &s, const ScalarW &w, cudaStream_t st) {
    switch (order / 2) {
        case 1: return launch_scalar_stage<1>(s, w, st);
        case 2: return launch_scalar_stage<2>(s, w, st);
        case 3: return launch_scalar_stage<3>(s, w, st);
        case 4: return launch_scalar_stage<4>(s, w, st);
        case 5: return launch_scalar_stage<5>(s, w, st);
        case 6: return launch_scalar_stage<6>(s, w, st);
    }
    return cudaErrorInvalidValue;
}

// RK3 coefficients of the flow solver's low-storage scheme (Section 2.4).
const double SC_ALPHA[3] = {2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0};
const double SC_BETA[3] = {1.0 / 4.0, 3.0 / 20.0, 3.0 / 5.0};

osb_status sc_fail(osb_status s, const char *msg) {
    set_last_error(msg);
    return s;
}

}  // namespace
}  // namespace osb

extern "C" osb_status osb_scalar_rk3(double *phi_dev, double *work_dev, const double *src_dev, int nx, int ny,
                                     int nz, int order, const double *adv, double diff, double dt, int nsteps,
                                     void *cuda_stream) {
    using namespace osb;
    if (!phi_dev || !work_dev || !adv) return sc_fail(OSB_ERR_INVALID_ARG, "scalar: NULL pointer");
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > 0x7fffffffLL)
        return sc_fail(OSB_ERR_INVALID_ARG, "scalar: bad grid size");
    if (order < 2 || order > 2 * MAXR || order % 2) return sc_fail(OSB_ERR_INVALID_ARG, "scalar: order must be 2..12, even");
    if (nsteps < 0 || !(dt > 0) || !(diff >= 0)) return sc_fail(OSB_ERR_INVALID_ARG, "scalar: bad dt, diffusivity or step count");
    if (((uintptr_t)phi_dev | (uintptr_t)work_dev | (uintptr_t)src_dev) & 7)
        return sc_fail(OSB_ERR_BUFFER, "scalar: buffers must be 8-byte aligned");
    if (nsteps == 0) return OSB_OK;
    Coef<double> c64;
    Coef<float> c32;
    make_coefs(order, nx, ny, nz, &c64, &c32);
    const int dims[3] = {nx, ny, nz};
    ScalarW w;
    memset(&w, 0, sizeof(w));
    for (int a = 0; a < 3; ++a) {
        w.active[a] = dims[a] > 1;
        if (!w.active[a]) continue;
        w.w0 += diff * c64.d2[a][0];
        for (int k = 1; k <= order / 2; ++k) {
            w.wp[a][k] = diff * c64.d2[a][k] - adv[a] * c64.d1[a][k];
            w.wm[a][k] = diff * c64.d2[a][k] + adv[a] * c64.d1[a][k];
        }
    }
    const size_t n = (size_t)nx * ny * nz;
    double *A = work_dev, *B = work_dev + n;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    // registers per step: even steps start from phi and end in A, odd steps
    // start from A and end in phi; no stage writes its own stencil source
    for (int step = 0; step < nsteps; ++step) {
        double *U0 = (step & 1) ? A : phi_dev, *U1 = (step & 1) ? phi_dev : A;
        // stage 1: source U0, q_1 -> B, U_1 -> U1; stage 2: q_2 -> U0 (free once
        // stage 1 has read it); stage 3: source q_2, U_3 -> U1
        const double *srcs[3] = {U0, B, U0};
        double *qouts[3] = {B, U0, nullptr};
        for (int k = 0; k < 3; ++k) {
            ScalarStage s;
            s.src = srcs[k];
            s.U_in = (k == 0) ? U0 : U1;
            s.U_out = U1;
            s.q_out = qouts[k];
            s.S = src_dev;
            s.adt = SC_ALPHA[k] * dt;
            s.bdt = SC_BETA[k] * dt;
            s.nx = nx, s.ny = ny, s.nz = nz;
            cudaError_t e = scalar_stage(order, s, w, st);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                return sc_fail(OSB_ERR_CUDA, "scalar: stage launch failed");
            }
        }
    }
    if (nsteps & 1) {
        cudaError_t e = cudaMemcpyAsync(phi_dev, A, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return sc_fail(OSB_ERR_CUDA, "scalar: result copy failed");
        }
    }
    return OSB_OK;
}
