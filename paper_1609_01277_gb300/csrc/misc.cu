// misc.cu -- Taylor-Green initial state and FP64 diagnostics reductions.
#include <math.h>

#include "stage.cuh"

namespace osb {

// ---------------------------------------------------------------------------
// Taylor-Green vortex initial state (OpenSBLI paper, Section 3.3), L = 1:
//   u0 = sin x cos y cos z, u1 = -cos x sin y cos z, u2 = 0,
//   p  = 1/(gamma M^2) + (cos 2x + cos 2y)(2 + cos 2z)/16,  T = 1 -> rho = gamma M^2 p;
// optional u_i += amp * noise[i] at fixed rho and p.
// Periodic axis: x_i = i h, h = 2 pi / n.  Axis between symmetry planes at 0
// and pi (two of the vortex's own mirror planes): x_i = (i + 1/2) h, h = pi / n.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double axis_coord(int i, int n, bool sym) {
    const double pi = 3.141592653589793238462643383279;
    return sym ? (i + 0.5) * (pi / n) : i * (2.0 * pi / n);
}

__global__ void k_init_tgv(const Dims d, const Phys ph, double *__restrict__ U, size_t s,
                           const double *__restrict__ noise, double amp) {
    // 64-bit index: i + stride must not overflow for grids near 2^31 points
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < d.n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % d.nx), y = (int)((i / d.nx) % d.ny), z = (int)(i / ((long long)d.nx * d.ny));
        const double X = axis_coord(x, d.nx, d.sym & 1), Y = axis_coord(y, d.ny, d.sym & 2);
        const double Z = axis_coord(z, d.nz, d.sym & 4);
        double sx, cx, sy, cy, sz, cz;
        sincos(X, &sx, &cx);
        sincos(Y, &sy, &cy);
        sincos(Z, &sz, &cz);
        double u0 = sx * cy * cz, u1 = -cx * sy * cz, u2 = 0.0;
        const double p = 1.0 / ph.gM2 + (cos(2.0 * X) + cos(2.0 * Y)) * (2.0 + cos(2.0 * Z)) / 16.0;
        const double rho = ph.gM2 * p;
        if (noise) {
            u0 += amp * noise[i];
            u1 += amp * noise[d.n + i];
            u2 += amp * noise[2 * (size_t)d.n + i];
        }
        U[i] = rho;
        U[s + i] = rho * u0;
        U[2 * s + i] = rho * u1;
        U[3 * s + i] = rho * u2;
        U[4 * s + i] = p / ph.gm1 + 0.5 * rho * (u0 * u0 + u1 * u1 + u2 * u2);
    }
}

cudaError_t launch_init_tgv(const Dims &d, const Phys &ph, double *U, size_t stride, const double *noise,
                            double amp, cudaStream_t st) {
    int blocks = (d.n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_init_tgv<<<blocks, 256, 0, st>>>(d, ph, U, stride, noise, amp);
    return cudaGetLastError();
}

// FP32 copy of the FP64 accumulator (round to nearest), the stage-1 stencil
// source of the FP32 path.
__global__ void k_to_f32(const double *__restrict__ U, size_t us, float *__restrict__ q, size_t qs, int n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int m = 0; m < 5; ++m) q[m * qs + i] = d2f_bits(U[m * us + i]);
}

// Double-float copy of the accumulator; the energy field as rho E - e_ref.
__global__ void k_to_dd(const double *__restrict__ U, size_t us, dd *__restrict__ q, size_t qs, int n, double e_ref) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int m = 0; m < 4; ++m) q[m * qs + i] = dd(U[m * us + i]);
        q[4 * qs + i] = dd(U[4 * us + i] - e_ref);
    }
}

cudaError_t launch_to_dd(const double *U, size_t u_stride, dd *q, size_t q_stride, int n, double e_ref,
                         cudaStream_t st) {
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_to_dd<<<blocks, 256, 0, st>>>(U, u_stride, q, q_stride, n, e_ref);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double *U, size_t u_stride, float *q, size_t q_stride, int n, cudaStream_t st) {
    int blocks = (n + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_to_f32<<<blocks, 256, 0, st>>>(U, u_stride, q, q_stride, n);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-step diagnostics series: one block sums the first stage's block records
// in index order (fixed per thread, then a fixed-order combine), divides by
// the number of points and appends the two means to the ring `series`.
// ---------------------------------------------------------------------------
constexpr int SERIES_THREADS = 256;

__global__ void __launch_bounds__(SERIES_THREADS)
    k_series_final(const double *__restrict__ rec, double inv_n, double *__restrict__ series, int capacity,
                   int *__restrict__ count) {
    const long long nrec = (long long)rec[0];
    double a = 0.0, b = 0.0;
    for (long long r = threadIdx.x; r < nrec; r += SERIES_THREADS) {
        a += rec[2 + 2 * r];
        b += rec[3 + 2 * r];
    }
    __shared__ double part[2][SERIES_THREADS];
    part[0][threadIdx.x] = a;
    part[1][threadIdx.x] = b;
    __syncthreads();
    for (int h = SERIES_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            part[0][threadIdx.x] += part[0][threadIdx.x + h];
            part[1][threadIdx.x] += part[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int k = *count;
        const int slot = k % capacity;
        series[2 * slot] = part[0][0] * inv_n;
        series[2 * slot + 1] = part[1][0] * inv_n;
        *count = k + 1;
    }
}

cudaError_t launch_series_final(const double *rec, double inv_n, double *series, int capacity, int *count,
                                cudaStream_t st) {
    k_series_final<<<1, SERIES_THREADS, 0, st>>>(rec, inv_n, series, capacity, count);
    return cudaGetLastError();
}

long long series_max_records(const Dims &d) {
    return (long long)((d.nx + BX - 1) / BX) * ((d.ny + BY - 1) / BY) * d.nz;
}

// ---------------------------------------------------------------------------
// Diagnostics (Section 3.3): grid sums of (1/2) rho u_j u_j, (1/2) rho |omega|^2
// with omega_i = eps_ijk D_j u_k, the conserved fields, the non-finite count
// and the max of dt sum_j (|u_j| + c)/h_j.  FP64 from the FP64 accumulator.
// Deterministic: a fixed grid-stride split, warp shuffles, a fixed-order
// block combine, then one block combines the partials in index order.
// ---------------------------------------------------------------------------
constexpr int DIAG_THREADS = 256;
constexpr int DIAG_MAX_BLOCKS = 152 * 8;

int diag_num_partials(const Dims &d) {
    int b = (d.n + DIAG_THREADS - 1) / DIAG_THREADS;
    return b < DIAG_MAX_BLOCKS ? b : DIAG_MAX_BLOCKS;
}

__device__ __forceinline__ void diag_block_combine(double v[NDIAG], double *out) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
#pragma unroll
        for (int q = 0; q < NDIAG; ++q) {
            const double o = __shfl_down_sync(0xffffffffu, v[q], off);
            v[q] = (q == NDIAG - 1) ? fmax(v[q], o) : v[q] + o;
        }
    }
    __shared__ double sm[DIAG_THREADS / 32][NDIAG];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int q = 0; q < NDIAG; ++q) sm[warp][q] = v[q];
    __syncthreads();
    if (threadIdx.x < NDIAG) {
        const int q = threadIdx.x;
        double acc = sm[0][q];
        for (int w = 1; w < DIAG_THREADS / 32; ++w) acc = (q == NDIAG - 1) ? fmax(acc, sm[w][q]) : acc + sm[w][q];
        out[q] = acc;
    }
}

template <int R>
__device__ __forceinline__ double vel_d1(const double *__restrict__ rho, const double *__restrict__ m,
                                         const int *off, const double *c) {
    double s = 0.0;
#pragma unroll
    for (int k = R; k >= 1; --k) {
        const int ip = off[R + k], im = off[R - k];
        s = fma(c[k], __ldg(m + ip) / __ldg(rho + ip) - __ldg(m + im) / __ldg(rho + im), s);
    }
    return s;
}

// Planes [zlo, zhi) of the array are reduced (a z-slab's own planes); nzd is
// the number of planes of the whole periodic box along z (its spacing).
template <int R>
__global__ void __launch_bounds__(DIAG_THREADS)
    k_diag(const Dims d, const Phys ph, const Coef<double> c, double dt, const double *__restrict__ U,
           size_t s, double *__restrict__ partials, int zlo, int zhi, int nzd) {
    double v[NDIAG];
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) v[q] = 0.0;
    const double two_pi = 6.283185307179586476925286766559, pi = 0.5 * two_pi;
    const double ih[3] = {d.nx / ((d.sym & 1) ? pi : two_pi), d.ny / ((d.sym & 2) ? pi : two_pi),
                          nzd / ((d.sym & 4) ? pi : two_pi)};
    const double *rho = U, *m0 = U + s, *m1 = U + 2 * s, *m2 = U + 3 * s, *e = U + 4 * s;
    const long long plane = (long long)d.nx * d.ny, i_end = zhi * plane;
    for (long long i = zlo * plane + (long long)blockIdx.x * blockDim.x + threadIdx.x; i < i_end;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % d.nx), y = (int)((i / d.nx) % d.ny), z = (int)(i / plane);
        const double r = rho[i];
        const double u0 = m0[i] / r, u1 = m1[i] / r, u2 = m2[i] / r;
        const double uu = u0 * u0 + u1 * u1 + u2 * u2;
        v[0] += 0.5 * r * uu;
        int ox[2 * R + 1], oy[2 * R + 1], oz[2 * R + 1];
#pragma unroll
        for (int k = -R; k <= R; ++k) {
            bool f;  // no sign: each vorticity term differentiates a velocity component even along that axis
            const int xk = (d.sym & 1) ? mirrorc(x + k, d.nx, f) : wrapc(x + k, d.nx);
            const int yk = (d.sym & 2) ? mirrorc(y + k, d.ny, f) : wrapc(y + k, d.ny);
            const int zk = (d.sym & 4) ? mirrorc(z + k, d.nz, f) : wrapc(z + k, d.nz);
            ox[k + R] = (z * d.ny + y) * d.nx + xk;
            oy[k + R] = (z * d.ny + yk) * d.nx + x;
            oz[k + R] = (zk * d.ny + y) * d.nx + x;
        }
        // omega = (D_y u2 - D_z u1, D_z u0 - D_x u2, D_x u1 - D_y u0)
        const double w0 = vel_d1<R>(rho, m2, oy, c.d1[1]) - vel_d1<R>(rho, m1, oz, c.d1[2]);
        const double w1 = vel_d1<R>(rho, m0, oz, c.d1[2]) - vel_d1<R>(rho, m2, ox, c.d1[0]);
        const double w2 = vel_d1<R>(rho, m1, ox, c.d1[0]) - vel_d1<R>(rho, m0, oy, c.d1[1]);
        v[1] += 0.5 * r * (w0 * w0 + w1 * w1 + w2 * w2);
        const double q0 = r, q1 = m0[i], q2 = m1[i], q3 = m2[i], q4 = e[i];
        v[2] += q0;
        v[3] += q1;
        v[4] += q2;
        v[5] += q3;
        v[6] += q4;
        const bool bad = !(isfinite(q0) && isfinite(q1) && isfinite(q2) && isfinite(q3) && isfinite(q4));
        v[7] += bad ? 1.0 : 0.0;
        const double p = ph.gm1 * (q4 - 0.5 * r * uu);
        const double cs = sqrt(ph.gamma * p / r);
        const double sum = (fabs(u0) + cs) * ih[0] + (fabs(u1) + cs) * ih[1] + (fabs(u2) + cs) * ih[2];
        v[8] = fmax(v[8], sum * dt);
    }
    diag_block_combine(v, partials + (size_t)blockIdx.x * DIAG_STRIDE);
}

__global__ void __launch_bounds__(DIAG_THREADS)
    k_diag_final(const double *__restrict__ partials, int nparts, double inv_n, double *__restrict__ result) {
    double v[NDIAG];
#pragma unroll
    for (int q = 0; q < NDIAG; ++q) v[q] = 0.0;
    for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
#pragma unroll
        for (int q = 0; q < NDIAG; ++q) {
            const double o = partials[(size_t)b * DIAG_STRIDE + q];
            v[q] = (q == NDIAG - 1) ? fmax(v[q], o) : v[q] + o;
        }
    }
    __shared__ double out[NDIAG];
    diag_block_combine(v, out);
    __syncthreads();
    if (threadIdx.x < NDIAG) {
        const int q = threadIdx.x;
        // means for the sums, raw count / max for the last two
        result[q] = (q < 7) ? out[q] * inv_n : out[q];
    }
}

cudaError_t launch_diagnostics(const Dims &d, const Phys &ph, int order, const Coef<double> &c, double dt,
                               const double *U, size_t stride, double *partials, int max_partials,
                               double *result, cudaStream_t st, int zlo, int zhi, int nzd) {
    const int blocks = diag_num_partials(d);
    if (blocks > max_partials) return cudaErrorInvalidValue;
    if (zhi < 0) zhi = d.nz;
    if (nzd <= 0) nzd = d.nz;
    if (zlo < 0 || zhi > d.nz || zlo >= zhi) return cudaErrorInvalidValue;
    switch (order / 2) {
        case 1: k_diag<1><<<blocks, DIAG_THREADS, 0, st>>>(d, ph, c, dt, U, stride, partials, zlo, zhi, nzd); break;
        case 2: k_diag<2><<<blocks, DIAG_THREADS, 0, st>>>(d, ph, c, dt, U, stride, partials, zlo, zhi, nzd); break;
        case 3: k_diag<3><<<blocks, DIAG_THREADS, 0, st>>>(d, ph, c, dt, U, stride, partials, zlo, zhi, nzd); break;
        case 4: k_diag<4><<<blocks, DIAG_THREADS, 0, st>>>(d, ph, c, dt, U, stride, partials, zlo, zhi, nzd); break;
        case 5: k_diag<5><<<blocks, DIAG_THREADS, 0, st>>>(d, ph, c, dt, U, stride, partials, zlo, zhi, nzd); break;
        case 6: k_diag<6><<<blocks, DIAG_THREADS, 0, st>>>(d, ph, c, dt, U, stride, partials, zlo, zhi, nzd); break;
        default: return cudaErrorInvalidValue;
    }
    const double n = (double)(zhi - zlo) * d.nx * d.ny;
    k_diag_final<<<1, DIAG_THREADS, 0, st>>>(partials, blocks, 1.0 / n, result);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// z-slab halo exchange (the decomposition of a periodic box into slabs of
// planes, one per GPU): the H planes next to each face of a slab's own planes
// are packed into two contiguous staging buffers, [field][plane][y][x], and
// the buffers received from the neighbours are unpacked into the H ghost
// planes at each end of the slab array.  Words of 4 or 8 bytes.
// ---------------------------------------------------------------------------
template <typename W>
__global__ void k_halo(W *__restrict__ field, size_t stride, int nz, int H, long long plane, W *__restrict__ lo,
                       W *__restrict__ hi, int unpack, int *kerr) {
    const long long per = (long long)H * plane;  // words per field and face
    const long long total = 2 * 5 * per;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int face = (int)(i / (5 * per));
        const long long r = i - face * 5 * per;
        const int m = (int)(r / per);
        const long long j = r - m * per;
        // own planes next to the face (pack) or the ghost planes beyond it (unpack)
        const long long z0 = unpack ? (face ? (long long)(nz - H) : 0) : (face ? (long long)(nz - 2 * H) : (long long)H);
        if (!OSB_BC_OK(z0 >= 0 && z0 + H <= nz && j < per && m < 5, kerr)) continue;
        W *f = field + m * stride + z0 * plane + j;
        W *b = (face ? hi : lo) + m * per + j;
        if (unpack)
            *f = *b;
        else
            *b = *f;
    }
}

cudaError_t launch_halo(void *field, size_t stride, int esize, int nz, int H, long long plane, void *lo, void *hi,
                        int unpack, cudaStream_t st, int *kerr) {
    const long long total = 2LL * 5 * H * plane;
    long long blocks = (total + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (esize == 8)
        k_halo<unsigned long long><<<(int)blocks, 256, 0, st>>>(static_cast<unsigned long long *>(field), stride, nz,
                                                               H, plane, static_cast<unsigned long long *>(lo),
                                                               static_cast<unsigned long long *>(hi), unpack, kerr);
    else
        k_halo<unsigned int><<<(int)blocks, 256, 0, st>>>(static_cast<unsigned int *>(field), stride, nz, H, plane,
                                                         static_cast<unsigned int *>(lo),
                                                         static_cast<unsigned int *>(hi), unpack, kerr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Allocation-free diagnostics: the same two kernels, with the per-block
// partial sums in a fixed device array that the library itself owns.
//
// Scratch: one record of DIAG_STRIDE doubles per block of the first kernel.
// That kernel is launched with at most DIAG_MAX_BLOCKS (1216) blocks whatever
// the grid size (grid-stride loop), so 1216 records (155,648 bytes) serve
// every admissible grid.  Every record that the second kernel reads is written
// by the first kernel of the same call, so nothing has to be cleared between
// calls.  The array lives in each device's memory for as long as the library
// is loaded; every call shares it.
// ---------------------------------------------------------------------------
constexpr int NOALLOC_RECORDS = DIAG_MAX_BLOCKS;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_RECORDS * DIAG_STRIDE];

// Device address of the scratch array on the current device.  In host code
// the name g_noalloc_scratch is only a host-side stand-in, so the address is
// looked up with the device current.  The lookup allocates nothing and is
// repeated on every call rather than cached, so a context that was torn down
// and re-created (cudaDeviceReset) is served at the array's new address.
static cudaError_t noalloc_scratch(double **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<double *>(p);
    return cudaSuccess;
}

}  // namespace osb

extern "C" osb_status osb_diagnostics_noalloc(const double *Q_dev, int nx, int ny, int nz, int order,
                                              const osb_params *params, double *out_dev, void *cuda_stream) {
    using namespace osb;
    if (!Q_dev || !out_dev || !params) {
        set_last_error("osb_diagnostics_noalloc: NULL argument");
        return OSB_ERR_INVALID_ARG;
    }
    if (((uintptr_t)Q_dev & 7) || ((uintptr_t)out_dev & 7)) {
        set_last_error("osb_diagnostics_noalloc: device pointers must be 8-byte aligned");
        return OSB_ERR_BUFFER;
    }
    if (nx < 1 || ny < 1 || nz < 1 || order < 2 || order > 12 || (order & 1)) {
        set_last_error("osb_diagnostics_noalloc: sizes must be >= 1 and order even in 2..12");
        return OSB_ERR_INVALID_ARG;
    }
    if ((long long)nx * ny * nz > 0x7fffffffLL) {
        set_last_error("osb_diagnostics_noalloc: grid too large (nx*ny*nz must be below 2^31)");
        return OSB_ERR_INVALID_ARG;
    }
    if (!(params->gamma > 1) || !(params->Mach > 0) || !(params->dt > 0)) {
        set_last_error("osb_diagnostics_noalloc: need gamma > 1, Mach > 0, dt > 0");
        return OSB_ERR_INVALID_ARG;
    }
    const Dims d{nx, ny, nz, nx * ny * nz};
    if (diag_num_partials(d) > NOALLOC_RECORDS) {
        set_last_error("osb_diagnostics_noalloc: grid needs more partial records than the fixed scratch holds");
        return OSB_ERR_BUFFER;
    }
    double *scratch = nullptr;
    cudaError_t e = noalloc_scratch(&scratch);
    if (e != cudaSuccess) {
        set_last_error("osb_diagnostics_noalloc: cudaGetSymbolAddress of the scratch array failed");
        return OSB_ERR_CUDA;
    }
    Coef<double> c64;
    Coef<float> c32;
    make_coefs(order, nx, ny, nz, &c64, &c32);
    e = launch_diagnostics(d, make_phys(*params), order, c64, params->dt, Q_dev, (size_t)d.n, scratch,
                           NOALLOC_RECORDS, out_dev, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        set_last_error("osb_diagnostics_noalloc: kernel launch failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}

// ---------------------------------------------------------------------------
// FP64 arithmetic-rate probe: every thread runs eight independent chains of
// fused multiply-adds (x = x * a + b), enough independent work per warp to
// keep the FP64 pipe busy, and writes its sum so that nothing is eliminated.
// flops per launch = blocks * 256 threads * 8 chains * iters * 2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_fp64_rate(double *__restrict__ out, int iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

extern "C" osb_status osb_fp64_rate_probe(double *out_dev, int blocks, int iters, void *cuda_stream) {
    using namespace osb;
    if (!out_dev || blocks < 1 || iters < 1 || ((uintptr_t)out_dev & 7)) {
        set_last_error("osb_fp64_rate_probe: need an 8-byte aligned output, blocks >= 1, iters >= 1");
        return OSB_ERR_INVALID_ARG;
    }
    // a, b keep x bounded (x -> b / (1 - a)), so no value overflows
    k_fp64_rate<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>(out_dev, iters, 0.999999, 1e-6);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error("osb_fp64_rate_probe: launch failed");
        return OSB_ERR_CUDA;
    }
    return OSB_OK;
}
