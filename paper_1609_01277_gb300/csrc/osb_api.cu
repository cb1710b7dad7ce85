// osb_api.cu -- the C ABI of libosb (declared in include/osb.h): argument
// checks, buffer carving, the RK3 stage sequence and status codes.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "osb_internal.cuh"

using namespace osb;

namespace {
// NVTX range around a library call or one of its phases: visible in Nsight
// timelines when a tool is attached, a few nanoseconds otherwise.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};
const char *const kStageRange[3] = {"osb rk3 stage 1", "osb rk3 stage 2", "osb rk3 stage 3"};
}  // namespace

// Streams of the concurrent-stream ensemble mode: the instances' per-grid
// step graphs are replayed on up to kBatchStreams streams (the default number
// of hardware work queues: more streams would share them).
constexpr int kBatchStreams = 8;
struct BatchStreams {
    cudaStream_t s[kBatchStreams];
    cudaEvent_t ev[kBatchStreams + 1];  // ev[j]: stream j done; ev[kBatchStreams]: fork
};

struct osb_grid {
    osb_grid_desc desc;
    osb_params prm;
    Dims d;
    Phys ph;
    Coef<double> c64;
    Coef<float> c32;
    Coef<dd> cdd;
    OrderKernels K;
    char *state;
    char *ws;
    cudaStream_t st;
    int cur;  // which FP64 accumulator holds Q^n
    int qc;   // FP32 path: which stage register holds the FP32 copy of Q^n
    int copy_valid;
    int zmarch;  // FP32 path kernels: 2 fused stage (orders 2, 4), 1 two z-march kernels, 0 three-kernel
                 // (OSB_FP32_STAGE=fused|zmarch|split3 selects among those that apply)
    double t;
    long long step;
    double *U[2];
    void *q[2];
    size_t u_stride, q_stride;
    void *aux;
    size_t aux_stride;
    double *partials;
    int max_partials;
    double *result;
    // profiling: 4 events per stage launch, recorded on the grid's stream
    std::vector<cudaEvent_t> *prof_ev;
    int prof_used, prof_cap;
    // ensemble stepping: this grid's device record and, when it leads a
    // batch, the batch counters and the cache of captured CUDA graphs
    BatchInst *batch_rec;
    BatchInst *batch_rec_host;  // host staging copy of the record
    char *batch_ctl;
    std::map<std::string, cudaGraphExec_t> *graphs;
    cudaStream_t capture_st;  // library-owned stream the batch graphs are captured on
    // ensemble stepping on concurrent streams (lead grid only): library-owned
    // streams and their fork/join events, or nullptr
    struct BatchStreams *bstreams;
    osb_closure *closure;     // learned correction added to R in every stage, or nullptr
    // FP32 z-march stage: TMA descriptors per stage source q[b] (b = 0, 1)
    zm::ZTma *ztma;           // [2 sources][flux, rhs]
    zm::ZTmaN *ztman;         // narrow residual kernel (orders 6, 8): [2 sources], or nullptr
    fz::FTma *ftma;           // fused FP32 stage: descriptors per stage source q[b], or nullptr
    int *kerr;                // device error word of bounded in-kernel waits
    cudaGraphExec_t step_graph[2];  // one RK3 step starting with Q^n in U[0] / U[1]
    // per-step diagnostics series (osb_set_diag_series): block records of the
    // first stage (workspace), the caller's ring and its device step counter
    double *diag_rec;
    double *series;
    int series_cap;
    int *series_count;
    // z-slab of a larger periodic box (osb_set_z_slab): planes of the whole box
    // along z (0: not a slab), ghost planes at each end, next stage of
    // osb_rk3_stage
    int slab_nzd;
    int slab_h;
    int stage_pos;
};

namespace {

thread_local std::string g_err;

osb_status fail(osb_status s, const char *msg) {
    g_err = msg;
    return s;
}

osb_status cuda_fail(cudaError_t e, const char *where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();  // do not leave a non-sticky error for the next launch check
    return OSB_ERR_CUDA;
}

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

bool desc_ok(const osb_grid_desc *d) {
    if (!d) return false;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return false;
    if ((long long)d->nx * d->ny * d->nz > 0x7fffffffLL) return false;
    if (d->order < 2 || d->order > 12 || (d->order & 1)) return false;
    if (d->precision != OSB_FP64 && d->precision != OSB_FP32 && d->precision != OSB_DF64) return false;
    if (d->visc_form != OSB_VISC_A && d->visc_form != OSB_VISC_B) return false;
    return true;
}

size_t tsize(const osb_grid_desc *d) { return d->precision == OSB_FP32 ? 4 : 8; }

size_t field_bytes(size_t n, size_t es) { return round256(n * es); }

size_t npoints(const osb_grid_desc *d) { return (size_t)d->nx * d->ny * d->nz; }

size_t state_bytes(const osb_grid_desc *d) {
    const size_t n = npoints(d);
    return 2 * 5 * field_bytes(n, 8) + 2 * 5 * field_bytes(n, tsize(d));
}

size_t aux_bytes(const osb_grid_desc *d) { return NAUX * field_bytes(npoints(d), tsize(d)); }

// Per-grid ensemble block: the device record (stage arguments for both step
// parities), then the batch counters used when this grid leads a batch.
constexpr size_t BATCH_CTL_BYTES = 1024;  // counter (8 B), error word, done[MAXB]
size_t batch_bytes() { return round256(sizeof(BatchInst)) + BATCH_CTL_BYTES; }

size_t diag_bytes(const osb_grid_desc *d) {
    Dims dd{d->nx, d->ny, d->nz, (int)npoints(d)};
    return round256((size_t)(diag_num_partials(dd) + 1) * DIAG_STRIDE * sizeof(double));
}

// First-stage block records of the diagnostics series, then its step counter.
size_t series_bytes(const osb_grid_desc *d) {
    Dims dd{d->nx, d->ny, d->nz, (int)npoints(d)};
    return round256((size_t)(2 + 2 * series_max_records(dd)) * sizeof(double)) + 256;
}

size_t workspace_bytes(const osb_grid_desc *d) { return aux_bytes(d) + diag_bytes(d) + batch_bytes() + series_bytes(d); }

// Central-difference weights of order 2r (closed form): first derivative
// c_k = (-1)^{k+1} (r!)^2 / (k (r-k)! (r+k)!), second derivative d_k = 2 c_k / k,
// d_0 = -2 sum d_k (Section 2.4, arbitrary-order central differences).
void fd_weights(int order, double *c, double *dd) {
    const int r = order / 2;
    auto fact = [](int n) {
        double f = 1.0;
        for (int i = 2; i <= n; ++i) f *= i;
        return f;
    };
    const double rf2 = fact(r) * fact(r);
    double s = 0.0;
    c[0] = 0.0;
    for (int k = 1; k <= MAXR; ++k) {
        if (k > r) {
            c[k] = 0.0;
            dd[k] = 0.0;
            continue;
        }
        double ck = rf2 / ((double)k * fact(r - k) * fact(r + k));
        if (!(k & 1)) ck = -ck;
        c[k] = ck;
        dd[k] = 2.0 * ck / k;
        s += dd[k];
    }
    dd[0] = -2.0 * s;
}

OrderKernels kernels_for(int order) {
    switch (order) {
        case 2: return kernels_o2();
        case 4: return kernels_o4();
        case 6: return kernels_o6();
        case 8: return kernels_o8();
        case 10: return kernels_o10();
        case 12: return kernels_o12();
        default: return OrderKernels{0, nullptr, nullptr};
    }
}

OrderKernels kernels_sym_for(int order) {
    switch (order) {
        case 2: return kernels_sym_o2();
        case 4: return kernels_sym_o4();
        case 6: return kernels_sym_o6();
        case 8: return kernels_sym_o8();
        case 10: return kernels_sym_o10();
        case 12: return kernels_sym_o12();
        default: return OrderKernels{0, nullptr, nullptr};
    }
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        (void)cudaGetLastError();
    }
    return fn;
}

bool encode_plane_map(CUtensorMap *m, const float *base, const Dims &d, int bx, int by) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)d.nx, (cuuint64_t)d.ny, (cuuint64_t)d.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)d.nx * 4, (cuuint64_t)d.nx * d.ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA descriptors of the FP32 z-march kernels for both stage sources q[0],
// q[1].  Left unused (cp.async loads) when the x extent is not a multiple of 4
// (row strides must be 16-byte multiples), the order is above 8, or
// OSB_FP32_LOADS=cpasync.
void build_ztma(osb_grid *g) {
    g->ztma = nullptr;
    if (g->desc.precision != OSB_FP32 || g->desc.order > 8 || g->d.nx % 4) return;
    const char *env = getenv("OSB_FP32_LOADS");
    if (env && strcmp(env, "cpasync") == 0) return;
    zm::ZTma *t = new (std::nothrow) zm::ZTma[4];
    if (!t) return;
    memset(t, 0, 4 * sizeof(zm::ZTma));
    const int rh = 8 + 2 * (g->desc.order / 2);
    const float *aux = (const float *)g->aux;
    const size_t as = g->aux_stride;
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
        const float *q = (const float *)g->q[b];
        const size_t qs = g->q_stride;
        zm::ZTma &fl = t[2 * b], &rh_ = t[2 * b + 1];
        for (int f = 0; f < 4; ++f) ok = ok && encode_plane_map(&fl.rect[f], q + f * qs, g->d, 40, rh);
        ok = ok && encode_plane_map(&fl.col[0], q + 4 * qs, g->d, 32, 8);
        for (int f = 0; f < 5; ++f) ok = ok && encode_plane_map(&rh_.rect[f], q + f * qs, g->d, 40, rh);
        const int af[4] = {A_FX, A_FY, A_GX, A_GY};
        for (int f = 0; f < 4; ++f) ok = ok && encode_plane_map(&rh_.rect[5 + f], aux + af[f] * as, g->d, 40, rh);
        ok = ok && encode_plane_map(&rh_.col[0], aux + A_FZ * as, g->d, 32, 8);
        ok = ok && encode_plane_map(&rh_.col[1], aux + A_GZ * as, g->d, 32, 8);
        fl.use = rh_.use = 1;
    }
    if (!ok) {
        delete[] t;
        return;
    }
    g->ztma = t;
    // the narrow residual kernel of radius 3 and 4: rectangles 40 x (4 + 2R),
    // columns 32 x 4
    g->ztman = nullptr;
    if (g->desc.order < 6) return;
    zm::ZTmaN *tn = new (std::nothrow) zm::ZTmaN[2];
    if (!tn) return;
    memset(tn, 0, 2 * sizeof(zm::ZTmaN));
    const int rhn = 4 + 2 * (g->desc.order / 2);
    for (int b = 0; b < 2; ++b) {
        const float *q = (const float *)g->q[b];
        const size_t qs = g->q_stride;
        for (int f = 0; f < 5; ++f) ok = ok && encode_plane_map(&tn[b].rect[f], q + f * qs, g->d, 40, rhn);
        const int af[4] = {A_FX, A_FY, A_GX, A_GY};
        for (int f = 0; f < 4; ++f) ok = ok && encode_plane_map(&tn[b].rect[5 + f], aux + af[f] * as, g->d, 40, rhn);
        for (int f = 0; f < 5; ++f) ok = ok && encode_plane_map(&tn[b].col[f], q + f * qs, g->d, 32, 4);
        ok = ok && encode_plane_map(&tn[b].col[5], aux + A_FZ * as, g->d, 32, 4);
        ok = ok && encode_plane_map(&tn[b].col[6], aux + A_GZ * as, g->d, 32, 4);
        tn[b].use = 1;
    }
    if (!ok) {
        delete[] tn;
        return;
    }
    g->ztman = tn;
}

// TMA descriptors of the fused FP32 stage for both stage sources q[0], q[1]:
// haloed plane boxes of 40 x (TY + 4R) points.  Left unused (cp.async loads)
// when the x extent is not a multiple of 4 or OSB_FP32_LOADS=cpasync.
void build_ftma(osb_grid *g) {
    g->ftma = nullptr;
    if (g->desc.precision != OSB_FP32 || g->desc.order > 4 || g->d.nx % 4) return;
    const char *env = getenv("OSB_FP32_LOADS");
    if (env && strcmp(env, "cpasync") == 0) return;
    fz::FTma *t = new (std::nothrow) fz::FTma[2];
    if (!t) return;
    memset(t, 0, 2 * sizeof(fz::FTma));
    const int eh = fz::TY + 4 * (g->desc.order / 2);
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
        const float *q = (const float *)g->q[b];
        for (int f = 0; f < 5; ++f) ok = ok && encode_plane_map(&t[b].q[f], q + f * g->q_stride, g->d, 40, eh);
        t[b].use = 1;
    }
    if (!ok) {
        delete[] t;
        return;
    }
    g->ftma = t;
}

// FP32 stage kernels of a grid: the fused stage where it applies (orders 2
// and 4, viscous form A, periodic), else the two z-march kernels; the
// environment can ask for the two-kernel or the three-kernel stage.
int fp32_stage_mode(const osb_grid *g, int sym) {
    const char *env = getenv("OSB_FP32_STAGE");
    if (env && strcmp(env, "split3") == 0) return 0;
    if (sym) return 0;
    const bool fusable = g->desc.precision == OSB_FP32 && g->desc.visc_form == OSB_VISC_A && g->desc.order <= 4;
    if (env && strcmp(env, "zmarch") == 0) return 1;
    return fusable ? 2 : 1;
}

StageArgs base_args(const osb_grid *g) {
    StageArgs a;
    memset(&a, 0, sizeof(a));
    a.d = g->d;
    a.ph = g->ph;
    a.c64 = g->c64;
    a.c32 = g->c32;
    a.cdd = g->cdd;
    if (g->desc.precision == OSB_DF64) {
        const double gam = g->prm.gamma, M2 = g->prm.Mach * g->prm.Mach;
        a.e_ref = 1.0 / (gam * (gam - 1.0) * M2);
        const double p_ref = (gam - 1.0) * a.e_ref;
        a.kdd.gm1 = dd(g->ph.gm1);
        a.kdd.gM2 = dd(g->ph.gM2);
        a.kdd.inv_re = dd(g->ph.inv_re);
        a.kdd.kappa = dd(g->ph.kappa);
        a.kdd.e_ref = dd(a.e_ref);
        a.kdd.p_ref = dd(p_ref);
        a.kdd.c_ref = dd(0.5 * a.e_ref + p_ref);
        for (int ax = 0; ax < 3; ++ax)
            for (int k = 0; k <= MAXR; ++k) {
                const double d2 = g->c64.d2[ax][k], d1 = g->c64.d1[ax][k], ir = g->ph.inv_re;
                a.cdd_vis.d2[ax][k] = dd(ir * d2);
                a.cdd_vis43.d2[ax][k] = dd(ir * (4.0 / 3.0) * d2);
                a.cdd_heat.d2[ax][k] = dd(g->ph.kappa * d2);
                a.cdd_g.d1[ax][k] = dd(ir * (1.0 / 3.0) * d1);
            }
    }
    {
        const double ir = g->ph.inv_re, kap = g->ph.kappa;
        FoldW<double> &f = a.f64;
        for (int ax = 0; ax < 3; ++ax)
            for (int k = 0; k <= MAXR; ++k) {
                const double d2 = g->c64.d2[ax][k], d1 = g->c64.d1[ax][k];
                f.vis[ax][k] = ir * d2;
                f.vis43[ax][k] = ir * (4.0 / 3.0) * d2;
                f.heat[ax][k] = kap * d2;
                f.g[ax][k] = (1.0 / 3.0) * d1;
                f.d1ir[ax][k] = ir * d1;
            }
        f.Re = g->prm.Re;
        const double d0x = g->c64.d2[0][0], d0y = g->c64.d2[1][0], d0z = g->c64.d2[2][0];
        f.c_u = ir * ((4.0 / 3.0) * d0x + d0y + d0z);
        f.c_v = ir * (d0x + (4.0 / 3.0) * d0y + d0z);
        f.c_w = ir * (d0x + d0y + (4.0 / 3.0) * d0z);
        f.c_T = kap * (d0x + d0y + d0z);
        FoldW<float> &h = a.f32;
        for (int ax = 0; ax < 3; ++ax)
            for (int k = 0; k <= MAXR; ++k) {
                h.vis[ax][k] = (float)f.vis[ax][k];
                h.vis43[ax][k] = (float)f.vis43[ax][k];
                h.heat[ax][k] = (float)f.heat[ax][k];
                h.g[ax][k] = (float)f.g[ax][k];
                h.d1ir[ax][k] = (float)f.d1ir[ax][k];
            }
        h.Re = (float)f.Re;
        h.c_u = (float)f.c_u;
        h.c_v = (float)f.c_v;
        h.c_w = (float)f.c_w;
        h.c_T = (float)f.c_T;
    }
    a.precision = g->desc.precision;
    a.visc_form = g->desc.visc_form;
    a.zmarch = g->zmarch;
    a.kerr = g->kerr;
    a.aux = g->aux;
    a.aux_stride = g->aux_stride;
    a.u_stride = g->u_stride;
    a.q_stride = g->q_stride;
    a.stream = g->st;
    return a;
}

}  // namespace

namespace osb {

Phys make_phys(const osb_params &prm) {
    Phys ph;
    ph.Re = prm.Re;
    ph.Mach = prm.Mach;
    ph.gamma = prm.gamma;
    ph.Pr = prm.Pr;
    ph.inv_re = 1.0 / prm.Re;
    ph.kappa = 1.0 / ((prm.gamma - 1.0) * prm.Mach * prm.Mach * prm.Pr * prm.Re);
    ph.gm1 = prm.gamma - 1.0;
    ph.gM2 = prm.gamma * prm.Mach * prm.Mach;
    return ph;
}

// Grid spacing of an axis: periodic [0, 2 pi) with x_i = i h, or between
// symmetry planes at 0 and pi with x_i = (i + 1/2) h.
double axis_spacing(int n, bool symmetric) { return (symmetric ? M_PI : 2.0 * M_PI) / n; }

void make_coefs(int order, int nx, int ny, int nz, Coef<double> *c64, Coef<float> *c32, int sym) {
    double c[MAXR + 1], dd[MAXR + 1];
    fd_weights(order, c, dd);
    const int dims[3] = {nx, ny, nz};
    for (int a = 0; a < 3; ++a) {
        const double h = axis_spacing(dims[a], (sym >> a) & 1);
        for (int k = 0; k <= MAXR; ++k) {
            c64->d1[a][k] = c[k] / h;
            c64->d2[a][k] = dd[k] / (h * h);
            c32->d1[a][k] = (float)c64->d1[a][k];
            c32->d2[a][k] = (float)c64->d2[a][k];
        }
    }
}

// Double-float weights: head = weight rounded to FP32, tail = the remainder.
void make_coefs_dd(const Coef<double> &c64, Coef<dd> *cdd) {
    for (int a = 0; a < 3; ++a)
        for (int k = 0; k <= MAXR; ++k) {
            cdd->d1[a][k] = dd(c64.d1[a][k]);
            cdd->d2[a][k] = dd(c64.d2[a][k]);
        }
}

void set_last_error(const char *msg) { g_err = msg; }

}  // namespace osb

extern "C" {

const char *osb_status_string(osb_status s) {
    switch (s) {
        case OSB_OK: return "ok";
        case OSB_ERR_INVALID_ARG: return "invalid argument";
        case OSB_ERR_UNSUPPORTED: return "unsupported";
        case OSB_ERR_CUDA: return "CUDA error";
        case OSB_ERR_NONFINITE: return "non-finite state";
        case OSB_ERR_TIMEOUT: return "device wait timed out";
        case OSB_ERR_BUFFER: return "buffer too small or misaligned";
        case OSB_ERR_BOUNDS: return "index outside its buffer (bounds-check build)";
    }
    return "unknown status";
}

const char *osb_last_error(void) { return g_err.c_str(); }

size_t osb_state_bytes(const osb_grid_desc *d) { return desc_ok(d) ? state_bytes(d) : 0; }

size_t osb_workspace_bytes(const osb_grid_desc *d) {
    return desc_ok(d) ? workspace_bytes(d) : 0;
}

osb_status osb_grid_create(const osb_grid_desc *desc, const osb_params *prm, void *state_dev, size_t state_len,
                           void *ws_dev, size_t ws_len, void *stream, osb_grid **out) {
    if (!out) return fail(OSB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc_ok(desc)) return fail(OSB_ERR_INVALID_ARG, "invalid grid descriptor");
    if (!prm || !(prm->Re > 0) || !(prm->Mach > 0) || !(prm->Pr > 0) || !(prm->dt > 0) || !(prm->gamma > 1))
        return fail(OSB_ERR_INVALID_ARG, "invalid physical parameters");
    OrderKernels K = kernels_for(desc->order);
    if (!K.stage) return fail(OSB_ERR_UNSUPPORTED, "order not instantiated");
    if (!state_dev || !ws_dev) return fail(OSB_ERR_INVALID_ARG, "NULL device buffer");
    if (((uintptr_t)state_dev & 255) || ((uintptr_t)ws_dev & 255))
        return fail(OSB_ERR_BUFFER, "device buffers must be 256-byte aligned");
    if (state_len < state_bytes(desc)) return fail(OSB_ERR_BUFFER, "state buffer too small");
    if (ws_len < workspace_bytes(desc)) return fail(OSB_ERR_BUFFER, "workspace too small");

    osb_grid *g = new (std::nothrow) osb_grid;
    if (!g) return fail(OSB_ERR_INVALID_ARG, "host allocation failed");
    memset(g, 0, sizeof(*g));
    g->desc = *desc;
    g->prm = *prm;
    const size_t n = npoints(desc);
    g->d = Dims{desc->nx, desc->ny, desc->nz, (int)n};
    g->ph = make_phys(*prm);
    make_coefs(desc->order, desc->nx, desc->ny, desc->nz, &g->c64, &g->c32);
    make_coefs_dd(g->c64, &g->cdd);
    g->K = K;
    g->state = (char *)state_dev;
    g->ws = (char *)ws_dev;
    g->st = (cudaStream_t)stream;
    const size_t es = tsize(desc);
    const size_t f64 = field_bytes(n, 8), fT = field_bytes(n, es);
    g->u_stride = f64 / 8;
    g->q_stride = fT / es;
    g->U[0] = (double *)(g->state);
    g->U[1] = (double *)(g->state + 5 * f64);
    g->q[0] = g->state + 10 * f64;
    g->q[1] = g->state + 10 * f64 + 5 * fT;
    g->aux = g->ws;
    g->aux_stride = fT / es;
    g->partials = (double *)(g->ws + NAUX * fT);
    g->max_partials = diag_num_partials(g->d);
    g->result = g->partials + (size_t)g->max_partials * DIAG_STRIDE;
    g->batch_rec = (BatchInst *)(g->ws + aux_bytes(desc) + diag_bytes(desc));
    g->batch_ctl = (char *)g->batch_rec + round256(sizeof(BatchInst));
    g->kerr = (int *)(g->batch_ctl + BATCH_CTL_BYTES - sizeof(int));
    g->diag_rec = (double *)(g->ws + aux_bytes(desc) + diag_bytes(desc) + batch_bytes());
    g->series_count = (int *)((char *)g->diag_rec + series_bytes(desc) - 256);
    if (cudaMemsetAsync(g->kerr, 0, sizeof(int), g->st) != cudaSuccess) {
        delete g;
        return cuda_fail(cudaErrorInvalidValue, "grid create: error word reset");
    }
    build_ztma(g);
    build_ftma(g);
    g->cur = 0;
    g->zmarch = fp32_stage_mode(g, 0);
    *out = g;
    return OSB_OK;
}

static void prof_free(osb_grid *g) {
    if (!g->prof_ev) return;
    for (cudaEvent_t e : *g->prof_ev) cudaEventDestroy(e);
    delete g->prof_ev;
    g->prof_ev = nullptr;
    g->prof_used = g->prof_cap = 0;
}

osb_status osb_grid_destroy(osb_grid *g) {
    if (!g) return fail(OSB_ERR_INVALID_ARG, "grid is NULL");
    prof_free(g);
    if (g->graphs) {
        for (auto &kv : *g->graphs) cudaGraphExecDestroy(kv.second);
        delete g->graphs;
    }
    if (g->capture_st) cudaStreamDestroy(g->capture_st);
    if (g->bstreams) {
        for (int j = 0; j < kBatchStreams; ++j) {
            if (g->bstreams->s[j]) cudaStreamDestroy(g->bstreams->s[j]);
            if (g->bstreams->ev[j]) cudaEventDestroy(g->bstreams->ev[j]);
        }
        if (g->bstreams->ev[kBatchStreams]) cudaEventDestroy(g->bstreams->ev[kBatchStreams]);
        delete g->bstreams;
    }
    for (int b = 0; b < 2; ++b)
        if (g->step_graph[b]) cudaGraphExecDestroy(g->step_graph[b]);
    delete[] g->ztma;
    delete[] g->ztman;
    delete[] g->ftma;
    delete g->batch_rec_host;
    delete g;
    return OSB_OK;
}

osb_status osb_profile_start(osb_grid *g, int max_stages) {
    if (!g || max_stages < 1) return fail(OSB_ERR_INVALID_ARG, "invalid argument");
    prof_free(g);
    g->prof_ev = new (std::nothrow) std::vector<cudaEvent_t>();
    if (!g->prof_ev) return fail(OSB_ERR_INVALID_ARG, "host allocation failed");
    g->prof_ev->resize((size_t)4 * max_stages);
    for (auto &e : *g->prof_ev) {
        cudaError_t err = cudaEventCreate(&e);
        if (err != cudaSuccess) {
            e = nullptr;
            prof_free(g);
            return cuda_fail(err, "profile event create");
        }
    }
    g->prof_cap = max_stages;
    g->prof_used = 0;
    return OSB_OK;
}

osb_status osb_profile_stop(osb_grid *g, double *total_ms, long long *launches) {
    if (!g || !total_ms || !launches) return fail(OSB_ERR_INVALID_ARG, "invalid argument");
    if (!g->prof_ev) return fail(OSB_ERR_INVALID_ARG, "profiling not started");
    cudaError_t e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return cuda_fail(e, "profile sync");
    for (int k = 0; k < KK_COUNT; ++k) {
        total_ms[k] = 0.0;
        launches[k] = 0;
    }
    for (int s = 0; s < g->prof_used; ++s) {
        cudaEvent_t *ev = g->prof_ev->data() + 4 * s;
        for (int k = 0; k < KK_COUNT; ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            if (e != cudaSuccess) return cuda_fail(e, "profile elapsed");
            total_ms[k] += ms;
            launches[k] += 1;
        }
    }
    prof_free(g);
    return OSB_OK;
}

osb_status osb_init_taylor_green(osb_grid *g, const double *noise, double amp) {
    if (!g) return fail(OSB_ERR_INVALID_ARG, "grid is NULL");
    if (noise && !isfinite(amp)) return fail(OSB_ERR_INVALID_ARG, "noise amplitude not finite");
    cudaError_t e = launch_init_tgv(g->d, g->ph, g->U[g->cur], g->u_stride, noise, amp, g->st);
    if (e != cudaSuccess) return cuda_fail(e, "init_taylor_green");
    g->copy_valid = 0;
    g->t = 0.0;
    g->step = 0;
    return OSB_OK;
}

static osb_status copy_state(osb_grid *g, const double *src, double *dst, cudaMemcpyKind kind, bool sync) {
    const size_t n = g->d.n;
    for (int m = 0; m < 5; ++m) {
        const double *s;
        double *t;
        if (dst == nullptr) {  // into the grid
            s = src + m * n;
            t = g->U[g->cur] + m * g->u_stride;
        } else {
            s = g->U[g->cur] + m * g->u_stride;
            t = dst + m * n;
        }
        cudaError_t e = cudaMemcpyAsync(t, s, n * sizeof(double), kind, g->st);
        if (e != cudaSuccess) return cuda_fail(e, "state copy");
    }
    if (sync) {
        cudaError_t e = cudaStreamSynchronize(g->st);
        if (e != cudaSuccess) return cuda_fail(e, "state copy sync");
    }
    if (dst == nullptr) g->copy_valid = 0;
    return OSB_OK;
}

osb_status osb_set_state(osb_grid *g, const double *host_src) {
    if (!g || !host_src) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    osb_status s = copy_state(g, host_src, nullptr, cudaMemcpyHostToDevice, true);
    if (s == OSB_OK) {
        g->t = 0.0;
        g->step = 0;
    }
    return s;
}

osb_status osb_get_state(osb_grid *g, double *host_dst) {
    if (!g || !host_dst) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    return copy_state(g, nullptr, host_dst, cudaMemcpyDeviceToHost, true);
}

osb_status osb_set_state_device(osb_grid *g, const double *dev_src) {
    if (!g || !dev_src) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    osb_status s = copy_state(g, dev_src, nullptr, cudaMemcpyDeviceToDevice, false);
    if (s == OSB_OK) {
        g->t = 0.0;
        g->step = 0;
    }
    return s;
}

osb_status osb_get_state_device(osb_grid *g, double *dev_dst) {
    if (!g || !dev_dst) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    return copy_state(g, nullptr, dev_dst, cudaMemcpyDeviceToDevice, false);
}

static osb_status ensure_stage_copy(osb_grid *g);

osb_status osb_residual(osb_grid *g, double *R_dev) {
    if (!g || !R_dev) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    if ((uintptr_t)R_dev & 7) return fail(OSB_ERR_BUFFER, "R_dev must be 8-byte aligned");
    StageArgs a = base_args(g);
    a.src = g->U[g->cur];
    a.src_is_f64 = 1;
    a.src_stride = g->u_stride;
    if (g->desc.precision == OSB_DF64) {
        // double-float grids read their double-float copy (energy offset by e_ref)
        osb_status s0 = ensure_stage_copy(g);
        if (s0 != OSB_OK) return s0;
        a.src = g->q[g->qc];
        a.src_is_f64 = 0;
        a.src_stride = g->q_stride;
    }
    a.R_out = R_dev;
    a.R_stride = g->d.n;
    if (g->closure) {
        cudaError_t ec = cl::closure_correction(g->closure, a.src, 1, a.src_stride, &a.closure);
        if (ec != cudaSuccess) return cuda_fail(ec, "closure correction");
    }
    cudaError_t e = g->K.residual(a);
    if (e != cudaSuccess) return cuda_fail(e, "residual");
    return OSB_OK;
}

// Low-storage RK3 (Section 2.4), 2-register form with alpha = (2/3, 5/12, 3/5)
// and beta = (1/4, 3/20, 3/5).  Registers: U[cur] holds Q^n and is the stage-1
// stencil source; U[1-cur] receives U_1..U_3 in place; q[0], q[1] hold the
// stage values q_1, q_2 (no stage reads and writes the same stencil source).
static const double RK_ALPHA[3] = {2.0 / 3.0, 5.0 / 12.0, 3.0 / 5.0};
static const double RK_BETA[3] = {1.0 / 4.0, 3.0 / 20.0, 3.0 / 5.0};

// Stage k (0..2) of a step that starts with Q^n in U[cur].  FP64: stencil
// sources U[cur], q[0], q[1].  FP32: q[qc] (FP32 copy of U[cur]), q[1-qc],
// q[qc], and the last stage writes the next copy into q[1-qc]; qc == cur.
static StageArgs stage_args(const osb_grid *g, int cur, int k) {
    StageArgs a = base_args(g);
    // FP32 and double-float grids keep a copy of the accumulator in the stage
    // type as the first stage's stencil source
    const bool f32 = g->desc.precision != OSB_FP64;
    const int qc = cur;
    double *Ucur = g->U[cur], *Unext = g->U[1 - cur];
    void *src[3], *qout[3];
    if (f32) {
        src[0] = g->q[qc];
        src[1] = g->q[1 - qc];
        src[2] = g->q[qc];
        qout[0] = g->q[1 - qc];
        qout[1] = g->q[qc];
    } else {
        src[0] = Ucur;
        src[1] = g->q[0];
        src[2] = g->q[1];
        qout[0] = g->q[0];
        qout[1] = g->q[1];
    }
    qout[2] = nullptr;
    a.src = src[k];
    a.src_is_f64 = !f32;
    a.src_is_u32 = g->desc.precision == OSB_FP32 && k == 0;
    a.src_stride = (k == 0 && !f32) ? g->u_stride : g->q_stride;
    a.U_in = (k == 0) ? Ucur : Unext;
    a.U_out = Unext;
    a.q_out = qout[k];
    a.u32_out = (f32 && k == 2) ? g->q[1 - qc] : nullptr;
    a.alpha_dt = RK_ALPHA[k] * g->prm.dt;
    a.beta_dt = RK_BETA[k] * g->prm.dt;
    a.ev = nullptr;
    a.diag_rec = (k == 0 && g->series) ? g->diag_rec : nullptr;
    if (f32 && g->ztma) {
        const int b = (a.src == g->q[0]) ? 0 : 1;
        a.ztma_flux = &g->ztma[2 * b];
        a.ztma_rhs = &g->ztma[2 * b + 1];
        a.ztma_rhs_n = g->ztman ? &g->ztman[b] : nullptr;
    }
    return a;
}

// The fused FP32 stage (fused.cuh) keeps the FP64 accumulator out of stages
// 1 and 2: with Uf = q[qc] the FP32 copy of U[cur] and d the FP32 increment
// (workspace fields 0..4),
//   stage 1: src Uf;  q[1-qc] = Uf + alpha_1 dt R;  d = beta_1 dt R
//   stage 2: src q[1-qc];  q[qc] = Uf + (d + alpha_2 dt R) (in place: Uf is
//            only read at the point);  d += beta_2 dt R
//   stage 3: src q[qc];  U[1-cur] = U[cur] + (double)(d + beta_3 dt R);
//            q[1-qc] = float(U[1-cur])
// which leaves the same registers as the other FP32 stages after a step.
static bool use_fused(const osb_grid *g) { return g->zmarch == 2; }

static StageArgs stage_args_fused(const osb_grid *g, int cur, int k) {
    StageArgs a = stage_args(g, cur, k);
    const int qc = cur;
    a.fz_dinc = (float *)g->aux;
    a.fz_dstride = g->aux_stride;
    a.fz_mode = k + 1;
    a.fz_has_d = 1;
    a.fz_ufc = nullptr;
    a.U_in = g->U[cur];
    a.U_out = g->U[1 - cur];
    a.u32_out = nullptr;
    a.ztma_flux = a.ztma_rhs = a.ztma_rhs_n = nullptr;
    if (k == 0) {
        a.src = g->q[qc];
        a.q_out = g->q[1 - qc];
    } else if (k == 1) {
        a.src = g->q[1 - qc];
        a.fz_ufc = (const float *)g->q[qc];
        a.q_out = g->q[qc];
    } else {
        a.src = g->q[qc];
        a.q_out = nullptr;
        a.u32_out = g->q[1 - qc];
    }
    a.src_stride = g->q_stride;
    a.fz_tma = g->ftma ? (const void *)&g->ftma[(a.src == g->q[0]) ? 0 : 1] : nullptr;
    return a;
}

// Arguments of stage k of a per-grid RK3 step.
static StageArgs step_stage_args(const osb_grid *g, int cur, int k) {
    return use_fused(g) ? stage_args_fused(g, cur, k) : stage_args(g, cur, k);
}

static osb_status ensure_stage_copy(osb_grid *g) {
    if (g->desc.precision == OSB_FP64 || g->copy_valid) return OSB_OK;
    cudaError_t e = g->desc.precision == OSB_FP32
                        ? launch_to_f32(g->U[g->cur], g->u_stride, (float *)g->q[g->cur], g->q_stride, g->d.n, g->st)
                        : launch_to_dd(g->U[g->cur], g->u_stride, (dd *)g->q[g->cur], g->q_stride, g->d.n,
                                       base_args(g).e_ref, g->st);
    if (e != cudaSuccess) return cuda_fail(e, "stage-type copy launch");
    g->copy_valid = 1;
    return OSB_OK;
}

// After a first stage with diagnostics: append the step's two means.
static cudaError_t series_append(const osb_grid *g, cudaStream_t st) {
    if (!g->series) return cudaSuccess;
    return launch_series_final(g->diag_rec, 1.0 / (double)g->d.n, g->series, g->series_cap, g->series_count, st);
}

static osb_status rk3_one_step(osb_grid *g) {
    NvtxRange step_range("osb rk3 step");
    osb_status s0 = ensure_stage_copy(g);
    if (s0 != OSB_OK) return s0;
    for (int k = 0; k < 3; ++k) {
        NvtxRange stage_range(kStageRange[k]);
        StageArgs a = step_stage_args(g, g->cur, k);
        if (g->closure) {
            cudaError_t e = cl::closure_correction(g->closure, a.src, a.src_is_f64, a.src_stride, &a.closure);
            if (e != cudaSuccess) return cuda_fail(e, "closure correction");
        }
        if (g->prof_ev && g->prof_used < g->prof_cap) {
            a.ev = g->prof_ev->data() + 4 * g->prof_used;
            g->prof_used += 1;
        }
        cudaError_t e = g->K.stage(a);
        if (e != cudaSuccess) return cuda_fail(e, "rk3 stage launch");
        if (k == 0 && (e = series_append(g, g->st)) != cudaSuccess) return cuda_fail(e, "series launch");
    }
    g->cur = 1 - g->cur;
    g->qc = g->cur;
    g->step += 1;
    g->t = g->step * g->prm.dt;
    return OSB_OK;
}

// The launches of one RK3 step (3 stages) captured into a CUDA graph on a
// library-owned stream; replayed on the grid's stream.  Used for runs of two
// or more steps without a closure or profiling: a step is 6-9 kernel launches,
// which dominate on small grids.
static osb_status step_graph(osb_grid *g, int cur, cudaGraphExec_t *out) {
    if (g->step_graph[cur]) {
        *out = g->step_graph[cur];
        return OSB_OK;
    }
    if (!g->capture_st) {
        cudaError_t ec = cudaStreamCreateWithFlags(&g->capture_st, cudaStreamNonBlocking);
        if (ec != cudaSuccess) {
            g->capture_st = nullptr;
            return cuda_fail(ec, "step capture stream");
        }
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(g->capture_st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "step capture begin");
    cudaError_t el = cudaSuccess;
    for (int k = 0; k < 3 && el == cudaSuccess; ++k) {
        StageArgs a = step_stage_args(g, cur, k);
        a.stream = g->capture_st;
        el = g->K.stage(a);
        if (k == 0 && el == cudaSuccess) el = series_append(g, g->capture_st);
    }
    e = cudaStreamEndCapture(g->capture_st, &graph);
    if (el != cudaSuccess || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(el != cudaSuccess ? el : e, "step capture");
    }
    e = cudaGraphInstantiate(&g->step_graph[cur], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g->step_graph[cur] = nullptr;
        return cuda_fail(e, "step graph instantiate");
    }
    *out = g->step_graph[cur];
    return OSB_OK;
}

osb_status osb_rk3_step(osb_grid *g, int nsteps) {
    if (!g || nsteps < 0) return fail(OSB_ERR_INVALID_ARG, "invalid argument");
    NvtxRange range("osb_rk3_step");
    if (g->slab_nzd) return fail(OSB_ERR_UNSUPPORTED, "z-slab grids step one stage at a time (osb_rk3_stage)");
    if (g->stage_pos) return fail(OSB_ERR_INVALID_ARG, "a step begun with osb_rk3_stage is unfinished");
    const char *env = getenv("OSB_GRAPHS");
    const bool graphs = nsteps >= 2 && !g->closure && !g->prof_ev && !(env && strcmp(env, "0") == 0);
    if (graphs) {
        osb_status s0 = ensure_stage_copy(g);
        if (s0 != OSB_OK) return s0;
        for (int s = 0; s < nsteps; ++s) {
            NvtxRange step_range("osb rk3 step (graph replay)");
            cudaGraphExec_t ge = nullptr;
            osb_status st = step_graph(g, g->cur, &ge);
            if (st != OSB_OK) return st;
            cudaError_t e = cudaGraphLaunch(ge, g->st);
            if (e != cudaSuccess) return cuda_fail(e, "step graph launch");
            g->cur = 1 - g->cur;
            g->qc = g->cur;
            g->step += 1;
            g->t = g->step * g->prm.dt;
        }
        return OSB_OK;
    }
    for (int s = 0; s < nsteps; ++s) {
        osb_status st = rk3_one_step(g);
        if (st != OSB_OK) return st;
    }
    return OSB_OK;
}

// Forward Euler (Section 2.4 offers it beside the RK3 scheme): one stage per
// step, U^{n+1} = U^n + dt R(U^n), written into the other accumulator
// register; the FP32 path also writes the next step's FP32 stencil source.
osb_status osb_euler_step(osb_grid *g, int nsteps) {
    if (!g || nsteps < 0) return fail(OSB_ERR_INVALID_ARG, "invalid argument");
    NvtxRange range("osb_euler_step");
    if (g->slab_nzd) return fail(OSB_ERR_UNSUPPORTED, "z-slab grids step one stage at a time (osb_rk3_stage)");
    if (g->stage_pos) return fail(OSB_ERR_INVALID_ARG, "a step begun with osb_rk3_stage is unfinished");
    for (int s = 0; s < nsteps; ++s) {
        osb_status s0 = ensure_stage_copy(g);
        if (s0 != OSB_OK) return s0;
        StageArgs a = use_fused(g) ? stage_args_fused(g, g->cur, 2) : stage_args(g, g->cur, 0);
        a.alpha_dt = a.beta_dt = g->prm.dt;
        a.q_out = nullptr;
        if (use_fused(g)) {
            // one stage of the fused kernel's final form, without an increment
            a.src = g->q[g->qc];
            a.fz_has_d = 0;
            a.diag_rec = g->series ? g->diag_rec : nullptr;
            a.fz_tma = g->ftma ? (const void *)&g->ftma[g->qc] : nullptr;
        }
        if (g->desc.precision != OSB_FP64) a.u32_out = g->q[1 - g->qc];
        if (g->closure) {
            cudaError_t e = cl::closure_correction(g->closure, a.src, a.src_is_f64, a.src_stride, &a.closure);
            if (e != cudaSuccess) return cuda_fail(e, "closure correction");
        }
        cudaError_t e = g->K.stage(a);
        if (e != cudaSuccess) return cuda_fail(e, "euler stage launch");
        if ((e = series_append(g, g->st)) != cudaSuccess) return cuda_fail(e, "series launch");
        g->cur = 1 - g->cur;
        g->qc = g->cur;
        g->step += 1;
        g->t = g->step * g->prm.dt;
    }
    return OSB_OK;
}

osb_status osb_diagnostics(osb_grid *g, osb_diag *out) {
    if (!g || !out) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    NvtxRange range("osb_diagnostics");
    const int zlo = g->slab_nzd ? g->slab_h : 0, zhi = g->slab_nzd ? g->d.nz - g->slab_h : -1;
    cudaError_t e = launch_diagnostics(g->d, g->ph, g->desc.order, g->c64, g->prm.dt, g->U[g->cur], g->u_stride,
                                       g->partials, g->max_partials, g->result, g->st, zlo, zhi, g->slab_nzd);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics launch");
    double h[NDIAG];
    int herr = 0;
    e = cudaMemcpyAsync(h, g->result, sizeof(h), cudaMemcpyDeviceToHost, g->st);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics copy");
    e = cudaMemcpyAsync(&herr, g->kerr, sizeof(int), cudaMemcpyDeviceToHost, g->st);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics status copy");
    e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return cuda_fail(e, "diagnostics sync");
    out->t = g->t;
    out->step = g->step;
    out->ke = h[0];
    out->enstrophy = h[1];
    for (int m = 0; m < 5; ++m) out->total[m] = h[2 + m];
    out->nonfinite = (long long)h[7];
    out->max_cfl = h[8];
    if (herr & KERR_BOUNDS)
        return fail(OSB_ERR_BOUNDS, "bounds-check build: a kernel computed an index outside its buffer; the state is invalid");
    if (herr) return fail(OSB_ERR_TIMEOUT, "a bounded in-kernel wait of an earlier step ran out; the state is invalid");
    if (out->nonfinite > 0) return fail(OSB_ERR_NONFINITE, "state holds non-finite values");
    return OSB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Ensemble stepping and the tile autotuner
// ---------------------------------------------------------------------------
namespace {

struct BatchConfig {
    double wait_limit_s = 2.0;
    int test_stall = 0;
};
BatchConfig g_batch_cfg;

// Tile depth (z planes per work item) chosen by the autotuner, per grid shape.
std::mutex g_tune_mu;
std::map<std::string, int> *g_tune = nullptr;
bool g_tune_loaded = false;

std::string shape_key(const osb_grid_desc &d) {
    char b[128];
    snprintf(b, sizeof b, "%dx%dx%d/o%d/%s/v%d", d.nx, d.ny, d.nz, d.order, d.precision == OSB_FP64 ? "fp64" : (d.precision == OSB_FP32 ? "fp32" : "df64"),
             d.visc_form);
    return b;
}

// Cache file: one "key tz" pair per line at $OSB_AUTOTUNE_CACHE.
void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    if (!g_tune) g_tune = new std::map<std::string, int>();
    const char *path = getenv("OSB_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[128];
    int tz;
    while (fscanf(f, "%127s %d", key, &tz) == 2)
        if (tz >= 1 && tz <= 64) (*g_tune)[key] = tz;
    fclose(f);
}

void tune_save_locked() {
    const char *path = getenv("OSB_AUTOTUNE_CACHE");
    if (!path || !g_tune) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    for (auto &kv : *g_tune) fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    fclose(f);
}

int tile_depth(const osb_grid_desc &d) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load_locked();
    auto it = g_tune->find(shape_key(d));
    if (it != g_tune->end()) return it->second;
    return d.precision == OSB_FP32 ? 8 : 4;
}

// How an ensemble advances:
//   BATCH_PERSISTENT: one persistent kernel for all steps (work items with
//     per-instance completion counts; the only mode with device-side waits);
//   BATCH_STREAMS: each instance's per-grid step graph, instances spread over
//     concurrent library-owned streams: the per-grid kernels (register
//     budgets, weights from the constant bank, the fused FP32 stage) with the
//     small grids running side by side instead of one after another.
// OSB_BATCH_MODE = persistent | streams overrides the default (persistent for
// FP64 and FP32, streams for double-float: 64 grids of 32^3..128^3 at order 4
// measured FP64 1.94e9 / 1.91e9 point-stages/s persistent / streams, FP32
// 1.47e10 / 2.10e10, double-float 3.93e9 / 5.89e9); the wait-timeout test
// keeps the persistent kernel.
enum { BATCH_PERSISTENT = 0, BATCH_STREAMS = 1 };

static int batch_mode(int precision, bool zmode) {
    if (g_batch_cfg.test_stall) return BATCH_PERSISTENT;
    int m = precision == OSB_DF64 ? BATCH_STREAMS : BATCH_PERSISTENT;
    if (const char *e = getenv("OSB_BATCH_MODE")) {
        if (strcmp(e, "persistent") == 0) m = BATCH_PERSISTENT;
        if (strcmp(e, "streams") == 0) m = BATCH_STREAMS;
    }
    return m;
}

// BATCH_STREAMS: instances go, largest first, to the least-loaded of up to
// kBatchStreams streams; each stream replays its instances' step graphs step
// by step (an instance's steps stay in order on its stream); fork and join
// events tie the streams to the grids' stream before and after.
static osb_status batch_streams(osb_grid *const *grids, int n, int nsteps) {
    osb_grid *lead = grids[0];
    cudaStream_t st = lead->st;
    if (!lead->bstreams) {
        BatchStreams *b = new (std::nothrow) BatchStreams;
        if (!b) return fail(OSB_ERR_INVALID_ARG, "batch: host allocation failed");
        memset(b, 0, sizeof(*b));
        lead->bstreams = b;
        for (int j = 0; j < kBatchStreams; ++j) {
            cudaError_t e = cudaStreamCreateWithFlags(&b->s[j], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev[j], cudaEventDisableTiming);
            if (e != cudaSuccess) return cuda_fail(e, "batch stream creation");
        }
        cudaError_t e = cudaEventCreateWithFlags(&b->ev[kBatchStreams], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "batch event creation");
    }
    BatchStreams &B = *lead->bstreams;
    const int K = n < kBatchStreams ? n : kBatchStreams;
    std::vector<int> order(n), home(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return grids[a]->d.n > grids[b]->d.n; });
    std::vector<long long> load(K, 0);
    for (int i : order) {
        int j = 0;
        for (int q = 1; q < K; ++q)
            if (load[q] < load[j]) j = q;
        home[i] = j;
        load[j] += grids[i]->d.n;
    }
    for (int i = 0; i < n; ++i) {
        osb_status s0 = ensure_stage_copy(grids[i]);
        if (s0 != OSB_OK) return s0;
    }
    cudaError_t e = cudaEventRecord(B.ev[kBatchStreams], st);
    for (int j = 0; j < K && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(B.s[j], B.ev[kBatchStreams], 0);
    if (e != cudaSuccess) return cuda_fail(e, "batch fork");
    // the grids' stream waits for every library stream (also after a failed
    // launch, so that later work on it cannot overtake what was queued)
    auto join = [&]() {
        cudaError_t ej = cudaSuccess;
        for (int j = 0; j < K; ++j) {
            cudaError_t r = cudaEventRecord(B.ev[j], B.s[j]);
            if (r == cudaSuccess) r = cudaStreamWaitEvent(st, B.ev[j], 0);
            if (ej == cudaSuccess) ej = r;
        }
        return ej;
    };
    std::vector<int> cur(n);
    for (int i = 0; i < n; ++i) cur[i] = grids[i]->cur;
    for (int s = 0; s < nsteps; ++s)
        for (int i : order) {
            cudaGraphExec_t ge = nullptr;
            osb_status s0 = step_graph(grids[i], cur[i], &ge);
            if (s0 != OSB_OK) {
                join();
                cudaStreamSynchronize(st);
                return s0;
            }
            e = cudaGraphLaunch(ge, B.s[home[i]]);
            if (e != cudaSuccess) {
                join();
                cudaStreamSynchronize(st);
                return cuda_fail(e, "batch step graph launch; grid states are undefined");
            }
            cur[i] = 1 - cur[i];
        }
    e = join();
    if (e != cudaSuccess) return cuda_fail(e, "batch join");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    for (int i = 0; i < n; ++i) {
        osb_grid *g = grids[i];
        g->cur = cur[i];
        g->qc = g->cur;
        g->step += nsteps;
        g->t = g->step * g->prm.dt;
    }
    return OSB_OK;
}

osb_status batch_run(osb_grid *const *grids, int n, int nsteps, int force_mode = -1) {
    if (!grids || n < 1 || n > MAXB || nsteps < 0) return fail(OSB_ERR_INVALID_ARG, "batch: need 1..128 grids, nsteps >= 0");
    for (int i = 0; i < n; ++i) {
        if (!grids[i]) return fail(OSB_ERR_INVALID_ARG, "NULL grid in batch");
        if (grids[i]->closure) return fail(OSB_ERR_UNSUPPORTED, "batch: grids with a learned closure step singly");
        if (grids[i]->d.sym) return fail(OSB_ERR_UNSUPPORTED, "batch: grids with symmetry boundaries step singly");
        if (grids[i]->series) return fail(OSB_ERR_UNSUPPORTED, "batch: grids recording a diagnostics series step singly");
    }
    const osb_grid *g0 = grids[0];
    for (int i = 1; i < n; ++i) {
        const osb_grid *g = grids[i];
        if (g->st != g0->st) return fail(OSB_ERR_INVALID_ARG, "batch grids must share one stream");
        if (g->desc.order != g0->desc.order || g->desc.precision != g0->desc.precision ||
            g->desc.visc_form != g0->desc.visc_form)
            return fail(OSB_ERR_UNSUPPORTED, "batch grids must share order, precision and viscous form");
        for (int j = 0; j < i; ++j)
            if (grids[j] == g) return fail(OSB_ERR_INVALID_ARG, "a grid appears twice in the batch");
    }
    if (nsteps == 0) return OSB_OK;
    cudaStream_t st = g0->st;
    // FP32 form-A ensembles of orders <= 8 run z-march work items (row starts
    // must be 16-byte aligned: x extents multiples of 4)
    bool zmode = g0->desc.precision == OSB_FP32 && g0->desc.visc_form == OSB_VISC_A && g0->desc.order <= 8;
    for (int i = 0; i < n && zmode; ++i) zmode = grids[i]->zmarch && grids[i]->d.nx % 4 == 0;
    const int mode = force_mode >= 0 ? force_mode : batch_mode(g0->desc.precision, zmode);
    if (mode == BATCH_STREAMS) return batch_streams(grids, n, nsteps);
    BatchParams P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.phases = zmode ? 6 : 9;
    P.prefix[0] = 0;
    std::string key = std::to_string(nsteps) + "|" + std::to_string(g_batch_cfg.test_stall) + "|" +
                      std::to_string((long long)(g_batch_cfg.wait_limit_s * 1e9));
    for (int i = 0; i < n; ++i) {
        osb_grid *g = grids[i];
        osb_status s0 = ensure_stage_copy(g);
        if (s0 != OSB_OK) return s0;
        // host staging of the record (large: holds TMA descriptors), owned by the grid
        if (!g->batch_rec_host) {
            g->batch_rec_host = new (std::nothrow) BatchInst;
            if (!g->batch_rec_host) return fail(OSB_ERR_INVALID_ARG, "batch: host allocation failed");
        }
        BatchInst &rec = *g->batch_rec_host;
        memset(&rec, 0, sizeof(rec));
        for (int par = 0; par < 2; ++par)
            for (int k = 0; k < 3; ++k) {
                rec.st[par][k] = stage_args(g, par, k);
                rec.st[par][k].ztma_flux = rec.st[par][k].ztma_rhs = rec.st[par][k].ztma_rhs_n =
                    nullptr;  // host pointers: not used on the device
                rec.st[par][k].diag_rec = nullptr;
                rec.zsrc[par][k] = (rec.st[par][k].src == g->q[0]) ? 0 : 1;
            }
        rec.tz = tile_depth(g->desc);
        rec.tiles_x = (g->d.nx + BX - 1) / BX;
        rec.tiles_y = (g->d.ny + BY - 1) / BY;
        rec.tiles_z = (g->d.nz + rec.tz - 1) / rec.tz;
        if (zmode && g->ztma)
            for (int b = 0; b < 2; ++b) {
                rec.tma[b][0] = g->ztma[2 * b];
                rec.tma[b][1] = g->ztma[2 * b + 1];
            }
        // pageable source: staged before the call returns, so rec can be reused
        cudaError_t e = cudaMemcpyAsync(g->batch_rec, &rec, sizeof(rec), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "batch record upload");
        const long long tiles = (long long)rec.tiles_x * rec.tiles_y * rec.tiles_z;
        if (P.prefix[i] + tiles > 0x3fffffff) return fail(OSB_ERR_INVALID_ARG, "batch too large");
        P.prefix[i + 1] = P.prefix[i] + (int)tiles;
        P.rec[i] = g->batch_rec;
        P.p0[i] = g->cur;
        char b[64];
        snprintf(b, sizeof b, "|%p:%d:%d:%d", (void *)g, g->cur, rec.tz, (int)zmode);
        key += b;
    }
    P.tiles_total = P.prefix[n];
    P.total_items = (long long)nsteps * P.phases * P.tiles_total;
    long long max_tiles = 0;
    for (int i = 0; i < n; ++i) max_tiles = std::max(max_tiles, (long long)(P.prefix[i + 1] - P.prefix[i]));
    if ((long long)nsteps * P.phases * max_tiles > 0xffffffffLL)
        return fail(OSB_ERR_INVALID_ARG, "batch: too many steps for the 32-bit completion counters");
    P.timeout_ns = (long long)(g_batch_cfg.wait_limit_s * 1e9);
    P.inject_stall = g_batch_cfg.test_stall;
    char *ctl = g0->batch_ctl;
    P.counter = (unsigned long long *)ctl;
    P.err = (int *)(ctl + 8);
    P.done = (unsigned *)(ctl + 16);

    // one memset and one persistent launch, captured once per (grids, parity,
    // nsteps) and replayed as a CUDA graph
    osb_grid *lead = grids[0];
    if (!lead->graphs) lead->graphs = new std::map<std::string, cudaGraphExec_t>();
    cudaGraphExec_t exec = nullptr;
    // the captured launch bakes in every field of P (record addresses, tile
    // prefix sums, parities, counters): key the cache on all of it, so a grid
    // destroyed and re-created at the same host address never replays a stale
    // graph
    key.append(reinterpret_cast<const char *>(&P), sizeof(P));
    key += "|" + std::to_string(g0->desc.order) + ":" + std::to_string(g0->desc.precision) + ":" +
           std::to_string(g0->desc.visc_form) + ":" + std::to_string((int)zmode);
    auto it = lead->graphs->find(key);
    if (it != lead->graphs->end()) {
        exec = it->second;
    } else {
        // capture on a library-owned stream (the caller's may be the legacy
        // default stream, which cannot be captured); the graph is then
        // launched on the caller's stream
        if (!lead->capture_st) {
            cudaError_t ec = cudaStreamCreateWithFlags(&lead->capture_st, cudaStreamNonBlocking);
            if (ec != cudaSuccess) {
                lead->capture_st = nullptr;
                return cuda_fail(ec, "batch capture stream");
            }
        }
        cudaStream_t cs = lead->capture_st;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e, "batch capture begin");
        cudaError_t e1 = cudaMemsetAsync(ctl, 0, 16 + sizeof(unsigned) * MAXB, cs);
        cudaError_t e2 = launch_batch(P, g0->desc.order, g0->desc.precision, g0->desc.visc_form, (int)zmode, cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e), "batch capture");
        }
        e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e, "batch graph instantiate");
        if (lead->graphs->size() >= 8) {
            for (auto &kv : *lead->graphs) cudaGraphExecDestroy(kv.second);
            lead->graphs->clear();
        }
        (*lead->graphs)[key] = exec;
    }
    cudaError_t e = cudaGraphLaunch(exec, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch graph launch");
    int herr = 0;
    e = cudaMemcpyAsync(&herr, P.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "batch status copy");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "batch sync");
    for (int i = 0; i < n; ++i) {
        osb_grid *g = grids[i];
        if (nsteps & 1) g->cur = 1 - g->cur;
        g->qc = g->cur;
        g->step += nsteps;
        g->t = g->step * g->prm.dt;
    }
    if (herr) return fail(OSB_ERR_TIMEOUT, "batch: a per-instance wait exceeded its time limit; grid states are undefined");
    return OSB_OK;
}

}  // namespace

extern "C" {

osb_status osb_batch_step(osb_grid *const *grids, int n, int nsteps) {
    NvtxRange range("osb_batch_step");
    for (int i = 0; grids && i < n; ++i)
        if (grids[i] && (grids[i]->slab_nzd || grids[i]->stage_pos))
            return fail(OSB_ERR_UNSUPPORTED, "batch grids must be whole periodic boxes between steps");
    return batch_run(grids, n, nsteps);
}

osb_status osb_grid_set_closure(osb_grid *g, osb_closure *c) {
    if (!g) return fail(OSB_ERR_INVALID_ARG, "grid is NULL");
    if (c && cl::closure_points(c) != g->d.n) return fail(OSB_ERR_INVALID_ARG, "closure grid size differs from the grid's");
    if (c && g->desc.precision == OSB_DF64) return fail(OSB_ERR_UNSUPPORTED, "closures take FP64 or FP32 grids");
    if (c && g->d.sym) return fail(OSB_ERR_UNSUPPORTED, "closures take periodic grids");
    if (c && g->slab_nzd) return fail(OSB_ERR_UNSUPPORTED, "no closure on a z-slab");
    g->closure = c;
    return OSB_OK;
}

// Per-step diagnostics series (Section 3.3 kinetic energy and enstrophy of
// the state at the start of every step), fused into the first stage.
osb_status osb_set_diag_series(osb_grid *g, double *series_dev, int capacity) {
    if (!g) return fail(OSB_ERR_INVALID_ARG, "grid is NULL");
    if (series_dev && g->slab_nzd) return fail(OSB_ERR_UNSUPPORTED, "no diagnostics series on a z-slab");
    if (series_dev && (capacity < 1 || ((uintptr_t)series_dev & 7)))
        return fail(OSB_ERR_INVALID_ARG, "series: capacity >= 1 and an 8-byte aligned buffer");
    // captured step graphs hold the previous first-stage arguments
    for (int b = 0; b < 2; ++b)
        if (g->step_graph[b]) {
            cudaGraphExecDestroy(g->step_graph[b]);
            g->step_graph[b] = nullptr;
        }
    g->series = series_dev;
    g->series_cap = series_dev ? capacity : 0;
    cudaError_t e = cudaMemsetAsync(g->series_count, 0, sizeof(int), g->st);
    if (e != cudaSuccess) return cuda_fail(e, "series counter reset");
    return OSB_OK;
}

osb_status osb_diag_series_count(osb_grid *g, long long *count) {
    if (!g || !count) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, g->series_count, sizeof(int), cudaMemcpyDeviceToHost, g->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->st);
    if (e != cudaSuccess) return cuda_fail(e, "series count");
    *count = h;
    return OSB_OK;
}

// Boundary kind per axis (Section 2.6).  Symmetric axes: symmetry planes at
// 0 and pi, points at (i + 1/2) pi / n, mirrored stencil loads; periodic axes:
// [0, 2 pi), points at 2 pi i / n.
osb_status osb_set_boundaries(osb_grid *g, int bc_x, int bc_y, int bc_z) {
    if (!g) return fail(OSB_ERR_INVALID_ARG, "grid is NULL");
    if (g->slab_nzd) return fail(OSB_ERR_UNSUPPORTED, "z-slabs keep periodic boundaries");
    const int bc[3] = {bc_x, bc_y, bc_z};
    int sym = 0;
    for (int a = 0; a < 3; ++a) {
        if (bc[a] != OSB_BC_PERIODIC && bc[a] != OSB_BC_SYMMETRIC)
            return fail(OSB_ERR_INVALID_ARG, "boundary kind must be OSB_BC_PERIODIC or OSB_BC_SYMMETRIC");
        if (bc[a] == OSB_BC_SYMMETRIC) sym |= 1 << a;
    }
    if (sym && g->closure) return fail(OSB_ERR_UNSUPPORTED, "closures take periodic grids");
    OrderKernels K = sym ? kernels_sym_for(g->desc.order) : kernels_for(g->desc.order);
    if (!K.stage) return fail(OSB_ERR_UNSUPPORTED, "order not instantiated");
    // captured step graphs hold the previous kernels and weights
    for (int b = 0; b < 2; ++b)
        if (g->step_graph[b]) {
            cudaGraphExecDestroy(g->step_graph[b]);
            g->step_graph[b] = nullptr;
        }
    g->d.sym = sym;
    make_coefs(g->desc.order, g->desc.nx, g->desc.ny, g->desc.nz, &g->c64, &g->c32, sym);
    make_coefs_dd(g->c64, &g->cdd);
    g->K = K;
    // the FP32 z-march kernels wrap periodically; symmetric grids take the
    // three-kernel stage
    g->zmarch = fp32_stage_mode(g, sym);
    return OSB_OK;
}

osb_status osb_batch_configure(double wait_limit_seconds, int test_stall) {
    if (!(wait_limit_seconds > 0) || wait_limit_seconds > 3600)
        return fail(OSB_ERR_INVALID_ARG, "wait limit must be in (0, 3600] seconds");
    g_batch_cfg.wait_limit_s = wait_limit_seconds;
    g_batch_cfg.test_stall = test_stall ? 1 : 0;
    return OSB_OK;
}

osb_status osb_autotune(osb_grid *g, int trial_steps, int *best_tz) {
    if (!g || trial_steps < 1) return fail(OSB_ERR_INVALID_ARG, "invalid argument");
    const size_t n = g->d.n;
    std::vector<double> saved;
    try {
        saved.resize(5 * n);
    } catch (...) {
        return fail(OSB_ERR_INVALID_ARG, "host allocation failed");
    }
    const int cur0 = g->cur;
    const double t0 = g->t;
    const long long step0 = g->step;
    osb_status s = osb_get_state(g, saved.data());
    if (s != OSB_OK) return s;
    const std::string key = shape_key(g->desc);
    const int cand64[] = {1, 2, 4, 8, 16}, cand32[] = {4, 8, 16, 32, 0};
    const int *cand = g->desc.precision == OSB_FP32 ? cand32 : cand64;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(OSB_ERR_CUDA, "autotune: event create failed");
    int best = 4;
    float best_ms = 1e30f;
    for (int ci = 0; ci < 5; ++ci) {
        const int tz = cand[ci];
        if (tz == 0 || (tz > g->d.nz && tz != cand[0])) continue;
        {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            tune_load_locked();
            (*g_tune)[key] = tz;
        }
        osb_grid *one[1] = {g};
        s = batch_run(one, 1, 1, BATCH_PERSISTENT);  // warm-up (captures the graph); tile depths are the persistent kernel's
        if (s != OSB_OK) break;
        cudaEventRecord(e0, g->st);
        s = batch_run(one, 1, trial_steps, BATCH_PERSISTENT);
        cudaEventRecord(e1, g->st);
        if (s != OSB_OK) break;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = tz;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        (*g_tune)[key] = best;
        tune_save_locked();
    }
    // restore the state the call started from
    g->cur = cur0;
    g->qc = cur0;
    osb_status r = osb_set_state(g, saved.data());
    g->t = t0;
    g->step = step0;
    if (s != OSB_OK) return s;
    if (r != OSB_OK) return r;
    if (best_tz) *best_tz = best;
    return OSB_OK;
}

int osb_tile_depth(const osb_grid_desc *desc) {
    if (!desc_ok(desc)) return 0;
    return tile_depth(*desc);
}

osb_status osb_autotune_batch(osb_grid *const *grids, int n, int trial_steps) {
    if (!grids || n < 1 || n > MAXB || trial_steps < 1) return fail(OSB_ERR_INVALID_ARG, "invalid argument");
    for (int i = 0; i < n; ++i)
        if (!grids[i]) return fail(OSB_ERR_INVALID_ARG, "NULL grid in batch");
    NvtxRange range("osb_autotune_batch");
    // distinct shapes, largest total points first
    std::map<std::string, long long> pts;
    std::map<std::string, int> depth;
    for (int i = 0; i < n; ++i) {
        const std::string k = shape_key(grids[i]->desc);
        pts[k] += (long long)grids[i]->d.n;
        depth[k] = grids[i]->d.nz;
    }
    std::vector<std::pair<long long, std::string>> order;
    for (auto &kv : pts) order.push_back({kv.second, kv.first});
    std::sort(order.begin(), order.end(), [](const auto &a, const auto &b) { return a.first > b.first; });
    // the states to restore
    struct Saved {
        std::vector<double> q;
        int cur;
        double t;
        long long step;
    };
    std::vector<Saved> saved(n);
    for (int i = 0; i < n; ++i) {
        osb_grid *g = grids[i];
        try {
            saved[i].q.resize(5 * (size_t)g->d.n);
        } catch (...) {
            return fail(OSB_ERR_INVALID_ARG, "host allocation failed");
        }
        saved[i].cur = g->cur;
        saved[i].t = g->t;
        saved[i].step = g->step;
        osb_status s = osb_get_state(g, saved[i].q.data());
        if (s != OSB_OK) return s;
    }
    const bool f32 = grids[0]->desc.precision == OSB_FP32;
    const int cand64[] = {1, 2, 4, 8, 16}, cand32[] = {4, 8, 16, 32, 0};
    const int *cand = f32 ? cand32 : cand64;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(OSB_ERR_CUDA, "autotune: event create failed");
    osb_status s = OSB_OK;
    cudaStream_t st = grids[0]->st;
    // coordinate descent: each shape's depth in turn, the others held, timed
    // on the whole ensemble
    for (auto &ok : order) {
        const std::string &key = ok.second;
        int best = -1;
        float best_ms = 1e30f;
        for (int ci = 0; ci < 5 && s == OSB_OK; ++ci) {
            const int tz = cand[ci];
            if (tz == 0 || (tz > depth[key] && tz != cand[0])) continue;
            {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                tune_load_locked();
                (*g_tune)[key] = tz;
            }
            s = batch_run(grids, n, 1, BATCH_PERSISTENT);  // warm-up (captures the graph)
            if (s != OSB_OK) break;
            cudaEventRecord(e0, st);
            s = batch_run(grids, n, trial_steps, BATCH_PERSISTENT);
            cudaEventRecord(e1, st);
            if (s != OSB_OK) break;
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = tz;
            }
        }
        if (best > 0) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            (*g_tune)[key] = best;
        }
        if (s != OSB_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_save_locked();
    }
    osb_status r = OSB_OK;
    for (int i = 0; i < n; ++i) {
        osb_grid *g = grids[i];
        g->cur = saved[i].cur;
        g->qc = saved[i].cur;
        const osb_status ri = osb_set_state(g, saved[i].q.data());
        if (r == OSB_OK) r = ri;
        g->t = saved[i].t;
        g->step = saved[i].step;
    }
    if (s != OSB_OK) return s;
    return r;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// z-slab decomposition (one slab of planes per GPU; halo planes exchanged by
// the caller through staging buffers, e.g. with NCCL send/recv)
// ---------------------------------------------------------------------------
osb_status osb_set_z_slab(osb_grid *g, int nz_domain) {
    if (!g) return fail(OSB_ERR_INVALID_ARG, "grid is NULL");
    const int H = g->desc.order;  // 2R planes: nested first derivatives of form A reach 2R planes
    if (nz_domain < 1) return fail(OSB_ERR_INVALID_ARG, "nz_domain must be >= 1");
    if (g->desc.nz < 3 * H) return fail(OSB_ERR_INVALID_ARG, "a slab needs nz >= 3 * order planes (2 * order ghosts)");
    if (g->d.sym & 4) return fail(OSB_ERR_UNSUPPORTED, "z-slabs decompose a periodic z axis");
    if (g->series || g->closure) return fail(OSB_ERR_UNSUPPORTED, "no diagnostics series or closure on a z-slab");
    if (g->stage_pos) return fail(OSB_ERR_INVALID_ARG, "a step begun with osb_rk3_stage is unfinished");
    for (int b = 0; b < 2; ++b)
        if (g->step_graph[b]) {
            cudaGraphExecDestroy(g->step_graph[b]);
            g->step_graph[b] = nullptr;
        }
    g->slab_nzd = nz_domain;
    g->slab_h = H;
    make_coefs(g->desc.order, g->desc.nx, g->desc.ny, nz_domain, &g->c64, &g->c32, g->d.sym);
    make_coefs_dd(g->c64, &g->cdd);
    return OSB_OK;
}

size_t osb_halo_bytes(const osb_grid *g) {
    if (!g || !g->slab_nzd) return 0;
    return (size_t)5 * g->slab_h * g->desc.nx * g->desc.ny * 8;
}

// Stencil source of RK stage k (0..2) of the step in progress, or (k = 3) the
// FP64 accumulator holding Q^n; its field stride and element size.
static void halo_source(const osb_grid *g, int k, void **p, size_t *stride, int *esize) {
    if (k == 3) {
        *p = g->U[g->cur];
        *stride = g->u_stride;
        *esize = 8;
        return;
    }
    const StageArgs a = step_stage_args(g, g->cur, k);
    *p = const_cast<void *>(a.src);
    *stride = a.src_stride;
    *esize = a.src_is_f64 ? 8 : (int)tsize(&g->desc);
}

static osb_status halo_common(osb_grid *g, int source, void *lo, void *hi, int unpack) {
    if (!g || !lo || !hi) return fail(OSB_ERR_INVALID_ARG, "NULL argument");
    NvtxRange range(unpack ? "osb_halo_unpack" : "osb_halo_pack");
    if (!g->slab_nzd) return fail(OSB_ERR_INVALID_ARG, "not a z-slab (osb_set_z_slab)");
    if (source < 0 || source > 3) return fail(OSB_ERR_INVALID_ARG, "source must be 0..2 (stage) or 3 (accumulator)");
    if (source < 3 && source != g->stage_pos)
        return fail(OSB_ERR_INVALID_ARG, "the source of a stage is exchanged right before that stage");
    if (((uintptr_t)lo & 7) || ((uintptr_t)hi & 7)) return fail(OSB_ERR_BUFFER, "staging buffers must be 8-byte aligned");
    if (source == 0) {
        osb_status s0 = ensure_stage_copy(g);
        if (s0 != OSB_OK) return s0;
    }
    void *f = nullptr;
    size_t stride = 0;
    int esize = 0;
    halo_source(g, source, &f, &stride, &esize);
    const cudaError_t e = launch_halo(f, stride, esize, g->d.nz, g->slab_h, (long long)g->d.nx * g->d.ny, lo, hi,
                                      unpack, g->st, g->kerr);
    if (e != cudaSuccess) return cuda_fail(e, unpack ? "halo unpack" : "halo pack");
    return OSB_OK;
}

osb_status osb_halo_pack(osb_grid *g, int source, void *send_lo_dev, void *send_hi_dev) {
    return halo_common(g, source, send_lo_dev, send_hi_dev, 0);
}

osb_status osb_halo_unpack(osb_grid *g, int source, const void *recv_lo_dev, const void *recv_hi_dev) {
    return halo_common(g, source, const_cast<void *>(recv_lo_dev), const_cast<void *>(recv_hi_dev), 1);
}

osb_status osb_rk3_stage(osb_grid *g, int k) {
    if (!g) return fail(OSB_ERR_INVALID_ARG, "grid is NULL");
    if (k != g->stage_pos) return fail(OSB_ERR_INVALID_ARG, "stages run in order 0, 1, 2");
    NvtxRange range(kStageRange[k]);
    if (k == 0) {
        osb_status s0 = ensure_stage_copy(g);
        if (s0 != OSB_OK) return s0;
    }
    StageArgs a = step_stage_args(g, g->cur, k);
    if (g->closure) {
        cudaError_t e = cl::closure_correction(g->closure, a.src, a.src_is_f64, a.src_stride, &a.closure);
        if (e != cudaSuccess) return cuda_fail(e, "closure correction");
    }
    cudaError_t e = g->K.stage(a);
    if (e != cudaSuccess) return cuda_fail(e, "rk3 stage launch");
    if (k == 0 && (e = series_append(g, g->st)) != cudaSuccess) return cuda_fail(e, "series launch");
    if (k < 2) {
        g->stage_pos = k + 1;
        return OSB_OK;
    }
    g->stage_pos = 0;
    g->cur = 1 - g->cur;
    g->qc = g->cur;
    g->step += 1;
    g->t = g->step * g->prm.dt;
    return OSB_OK;
}
