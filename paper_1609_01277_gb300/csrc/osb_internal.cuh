// osb_internal.cuh -- internal types shared by the libosb translation units.
//
// Data layout in HBM (one grid):
//   state buffer:  U0[5] U1[5]  (FP64 RK accumulators)   qA[5] qB[5] (stage
//                  registers in the grid's precision T).  Each field starts on
//                  a 256-byte boundary (fields padded to a multiple of 256 B).
//   workspace:     aux[NAUX] fields of type T (point-wise intermediates of a
//                  stage), then the diagnostics partial sums and result.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "osb.h"
#include "dd.cuh"

namespace osb {

// Device error word of a grid (StageArgs::kerr): bit 0 a bounded in-kernel
// wait ran out, bit 1 (bounds-check build, -DOSB_BOUNDS_CHECK) an index
// computed by a stage kernel fell outside its buffer.  The bounds-check build
// tests each index where it is formed (neighbour offsets, tile and ring
// indices, global point indices, halo planes), records a failure here and
// replaces the index by 0, so the access stays inside the buffer: no trap.
constexpr int KERR_WAIT = 1, KERR_BOUNDS = 2;
#ifdef OSB_BOUNDS_CHECK
__device__ __forceinline__ bool bc_fail(int *kerr) {
    if (kerr) atomicOr(kerr, KERR_BOUNDS);
    return true;
}
#define OSB_BC_OK(cond, kerr) ((cond) || !::osb::bc_fail(kerr))
#else
#define OSB_BC_OK(cond, kerr) true
#endif

constexpr int MAXR = 6;  // orders 2..12
constexpr int BX = 32, BY = 8;  // thread block / tile of the per-point stage kernels

// Point-wise intermediate fields written by the primitive and gradient
// kernels of a stage and read by the residual kernel.
enum Aux {
    A_U = 0, A_V, A_W,        // velocity u_i = (rho u_i)/rho
    A_P, A_T,                 // pressure, temperature
    A_PXX, A_PYY, A_PZZ,      // momentum flux Phi_ii = rho u_i u_i/2 + p - g_i/(3 Re)
    A_PXY, A_PXZ, A_PYZ,      // momentum flux Phi_ij = rho u_i u_j/2 (i != j)
    A_FX, A_FY, A_FZ,         // energy flux F_j = (rho E/2 + p) u_j - u_i tau_ij
    A_DIV,                    // d_k u_k
    A_GX, A_GY, A_GZ,         // g_i = d_k u_k - d_i u_i        (viscous work form B only)
    A_TG,                     // tau_ij d_j u_i                  (viscous work form B only)
    NAUX
};

constexpr int NDIAG = 9;        // ke, enstrophy, totals[5], nonfinite, max_cfl
constexpr int DIAG_STRIDE = 16; // doubles per partial record

template <typename T>
__host__ __device__ inline size_t padded(size_t n) {
    size_t per = 256 / sizeof(T);
    return (n + per - 1) / per * per;
}

struct Dims {
    int nx, ny, nz;
    int n;    // nx*ny*nz (< 2^31)
    int sym;  // bit a set: axis a has symmetry planes at both ends (Section 2.6), else periodic
};

struct Phys {
    double Re, Mach, gamma, Pr;
    double inv_re, kappa, gm1, gM2;
};

// Stencil weights pre-divided by the grid spacing: d1[a][k] = c_k / h_a
// (k = 1..r), d2[a][k] = d_k / h_a^2 (k = 0..r).
template <typename T>
struct Coef {
    T d1[3][MAXR + 1];
    T d2[3][MAXR + 1];
};

// Folded weights of the FP64 / FP32 residual: second-derivative weights
// scaled by 1/Re (vis), 4/(3 Re) (vis43) and kappa (heat), first-derivative
// weights by 1/3 (g: viscous form B, whose g_i is stored scaled by 1/Re) and
// by 1/Re (d1ir, the gradient kernel), and the centre weights of the three
// viscous Laplacians and of the heat-flux Laplacian summed over the axes, so
// that each equation's terms accumulate with one FMA per stencil tap.
template <typename T>
struct FoldW {
    T vis[3][MAXR + 1], vis43[3][MAXR + 1], heat[3][MAXR + 1], g[3][MAXR + 1];
    T d1ir[3][MAXR + 1];  // first-derivative weights / Re: the gradient kernel forms (1/Re) d_j u_i directly
    T Re;
    T c_u, c_v, c_w, c_T;  // centre: (1/Re)(4/3 d0_x + d0_y + d0_z), ..., kappa (d0_x + d0_y + d0_z)
};

// Everything a stage launch needs.
struct StageArgs {
    Dims d;
    Phys ph;
    Coef<double> c64;
    Coef<float> c32;
    Coef<dd> cdd;           // double-float weights (OSB_DF64)
    // OSB_DF64: the double-float registers hold rho E - e_ref (e_ref =
    // 1/(gamma (gamma-1) M^2), the energy of the reference state rho = T = 1 at
    // rest), so pressure enters as p - p_ref (p_ref = (gamma-1) e_ref): the
    // stencils annihilate constants, and the small deviations keep far more
    // absolute accuracy than the full values.  0 in other precisions.
    double e_ref;
    struct {
        dd gm1, gM2, inv_re, kappa, e_ref, p_ref, c_ref;  // c_ref = e_ref/2 + p_ref
    } kdd;
    // OSB_DF64 residual: second-derivative weights scaled by 1/Re, 4/(3 Re) and
    // kappa, first-derivative weights by 1/(3 Re), so each equation's terms
    // accumulate without separate multiplications
    Coef<dd> cdd_vis, cdd_vis43, cdd_heat, cdd_g;
    FoldW<double> f64;
    FoldW<float> f32;
    int precision;          // OSB_FP64 / OSB_FP32 / OSB_DF64
    int visc_form;          // OSB_VISC_A / OSB_VISC_B
    const void *src;        // stencil source q_{k-1}
    int src_is_f64;         // 1: src holds doubles (U register), 0: type T
    int src_is_u32;         // FP32 path: src is the rounded FP32 copy of U_in (src = d2f(U_in) at every point)
    size_t src_stride;      // elements between fields of src
    void *aux;              // NAUX fields of type T
    size_t aux_stride;
    const double *U_in;     // RK accumulator read at the point
    double *U_out;          // RK accumulator written at the point (may equal U_in)
    void *q_out;            // next stage register (type T), or nullptr
    size_t u_stride, q_stride;
    double alpha_dt, beta_dt;
    void *u32_out;          // FP32 path, last stage: FP32 copy of U_out (q_stride), or nullptr
    double *R_out;          // residual-only mode: FP64 residual (5 fields, R_stride)
    size_t R_stride;
    cudaStream_t stream;
    cudaEvent_t *ev;        // optional: 4 events recorded around the 3 kernels
    int zmarch;             // FP32 path: 1 = z-marching two-kernel stage, 0 = three-kernel stage
    const float *closure;   // learned correction added to R (5 fields, stride d.n), or nullptr
    const void *ztma_flux;  // host: TMA descriptors of the z-march kernels for this stage, or nullptr
    const void *ztma_rhs;
    const void *ztma_rhs_n; // host: TMA descriptors of the narrow residual kernel (radius 3, 4), or nullptr
    int *kerr;              // device word set when a bounded in-kernel wait ran out
    // per-step diagnostics fused into the first stage (or nullptr): the
    // gradient kernel adds (1/2) rho u.u and (1/2) rho |omega|^2 over each
    // block; layout: [0] = number of block records, [2 + 2b], [3 + 2b] = the
    // two sums of block b
    double *diag_rec;
    // FP32 fused stage (one kernel per stage, orders 2 and 4): 0 = not used,
    // 1..3 = RK stage of the increment form, forward Euler = 3 without fz_has_d
    int fz_mode;
    float *fz_dinc;         // FP32 increments d (5 fields, fz_dstride)
    size_t fz_dstride;
    const float *fz_ufc;    // stage 2: FP32 copy of U at the step start (q_stride)
    int fz_has_d;           // stage 3: read d (0: forward Euler)
    const void *fz_tma;     // host: TMA descriptors of the stencil source, or nullptr
};


// Kernel kinds reported by the profiling hooks.
enum KernelKind { KK_PRIM = 0, KK_GRAD = 1, KK_RESID = 2, KK_COUNT = 3 };

struct OrderKernels {
    int order;
    cudaError_t (*stage)(const StageArgs &);     // prim + grad + residual/update
    cudaError_t (*residual)(const StageArgs &);  // prim + grad + residual only
};

// One translation unit per order provides its launcher table.
OrderKernels kernels_o2();
OrderKernels kernels_o4();
OrderKernels kernels_o6();
OrderKernels kernels_o8();
OrderKernels kernels_o10();
OrderKernels kernels_o12();
// ... and, for grids with symmetry boundaries, the mirrored-stencil variants
OrderKernels kernels_sym_o2();
OrderKernels kernels_sym_o4();
OrderKernels kernels_sym_o6();
OrderKernels kernels_sym_o8();
OrderKernels kernels_sym_o10();
OrderKernels kernels_sym_o12();

namespace zm {
// TMA descriptors of one z-march stage: haloed plane boxes (40 x (8 + 2R) x 1)
// of the ring fields and tile boxes (32 x 8 x 1) of the column-only fields.
struct ZTma {
    CUtensorMap rect[9];
    CUtensorMap col[2];
    int use;
};
// The narrow residual kernel of orders 6 and 8 (zrhs_narrow.cuh): haloed
// rectangles 40 x (4 + 2R) of its nine ring fields (conserved fields, F_x,
// F_y, g_x, g_y) and 32 x 4 tile columns of the conserved fields, F_z, g_z.
struct ZTmaN {
    CUtensorMap rect[9];
    CUtensorMap col[7];
    int use;
};
}  // namespace zm

namespace fz {
// Column tile of the fused stage: TX x TY points per CTA, one x-pair per thread.
constexpr int TX = 32, TY = 8;
// TMA descriptors of the fused stage: haloed plane boxes (40 x (TY + 4R) x 1)
// of the five fields of one stencil source.
struct FTma {
    CUtensorMap q[5];
    int use;
};
// The fused FP32 stage of radius 1 and 2 (fused_o2.cu, fused_o4.cu).
cudaError_t launch_fused_r1(const StageArgs &a);
cudaError_t launch_fused_r2(const StageArgs &a);
}  // namespace fz

// Persistent ensemble kernel (batch.cu).
constexpr int MAXB = 128;  // instances per batch

struct BatchInst {
    StageArgs st[2][3];   // [parity of (cur)][RK stage]
    int tz;               // z planes per tile
    int tiles_x, tiles_y, tiles_z;
    int zsrc[2][3];       // FP32 z-march items: stage register holding the stencil source
    zm::ZTma tma[2][2];   // FP32 z-march items: [stage register][flux, rhs]
};

struct BatchParams {
    int n;
    int tiles_total;       // items per phase sequence, all instances
    int phases;            // phases per step: 9 (three-kernel items) or 6 (FP32 z-march items)
    long long total_items;
    long long timeout_ns;  // bound on every dependency wait
    int inject_stall;      // test control: make the first wait unreachable
    const BatchInst *rec[MAXB];
    int prefix[MAXB + 1];  // tile prefix sums
    int p0[MAXB];          // parity of each instance at the first step
    unsigned long long *counter;
    unsigned *done;
    int *err;
};

cudaError_t launch_batch(const BatchParams &P, int order, int precision, int visc_form, int zmode, cudaStream_t st);

// Learned closure (closure.cu).
namespace cl {
cudaError_t closure_correction(osb_closure *c, const void *src, int src_is_f64, size_t stride, const float **C);
int closure_points(const osb_closure *c);
}  // namespace cl

// Host helpers shared by the translation units (defined in osb_api.cu).
Phys make_phys(const osb_params &prm);
void make_coefs(int order, int nx, int ny, int nz, Coef<double> *c64, Coef<float> *c32, int sym = 0);
double axis_spacing(int n, bool symmetric);
void make_coefs_dd(const Coef<double> &c64, Coef<dd> *cdd);
void set_last_error(const char *msg);

// Misc kernels (init, diagnostics).
cudaError_t launch_init_tgv(const Dims &d, const Phys &ph, double *U, size_t stride,
                            const double *noise, double amp, cudaStream_t st);
// Diagnostics of planes [zlo, zhi) of the array (zhi < 0: all); nzd planes of
// the whole box along z (0: the array's nz).
cudaError_t launch_diagnostics(const Dims &d, const Phys &ph, int order, const Coef<double> &c,
                               double dt, const double *U, size_t stride, double *partials,
                               int max_partials, double *result, cudaStream_t st, int zlo = 0, int zhi = -1,
                               int nzd = 0);
// z-slab halo: pack the H own planes next to each face of the array (nz
// planes, H ghost planes at each end) into lo/hi, or unpack lo/hi into the
// ghost planes; 5 fields of esize-byte words (4 or 8), field stride in words.
cudaError_t launch_halo(void *field, size_t stride, int esize, int nz, int H, long long plane, void *lo, void *hi,
                        int unpack, cudaStream_t st, int *kerr);
int diag_num_partials(const Dims &d);
cudaError_t launch_to_dd(const double *U, size_t u_stride, dd *q, size_t q_stride, int n, double e_ref,
                         cudaStream_t st);
cudaError_t launch_to_f32(const double *U, size_t u_stride, float *q, size_t q_stride, int n, cudaStream_t st);
// Per-step diagnostics series: sums the block records of the first stage and
// writes the two grid means into series[2 (count mod capacity)], then counts.
cudaError_t launch_series_final(const double *rec, double inv_n, double *series, int capacity, int *count,
                                cudaStream_t st);
// Upper bound on the block records of one first stage (the gradient kernel's grid).
long long series_max_records(const Dims &d);

}  // namespace osb
