// Host side of libbp: the C ABI declared in include/bp.h. Geometry is built
// in FP64 here (Section 2.1.1's 3x4 pinhole matrix; the explicit form is
// documented in bp.h), the launch plan is derived from the exact FP64
// footprints of the CTA tiles, and every call validates its arguments
// before launching.
#include "bp_internal.h"
#include "filter_ct.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>

namespace bp {

int plan_box_width(int need, int elem_bytes);   // k_backproject.cu

static thread_local std::string g_create_err;

bp_status fail(bp_ctx *ctx, bp_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    else g_create_err = msg;
    return st;
}

bp_status cuda_fail(bp_ctx *ctx, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(ctx, e == cudaErrorMemoryAllocation ? BP_ERR_OOM : BP_ERR_CUDA, m);
}

// Device allocations of every context still alive (a test hook reads it to
// show that a failed bp_create leaks nothing).
static std::atomic<long long> g_live_allocs{0};

// Test hook: BP_TEST_FAIL_ALLOC=n makes the n-th device allocation of each
// bp_create fail (n = 1: the first) as cudaMalloc would when out of memory.
static cudaError_t dev_alloc(bp_ctx *ctx, void **p, size_t bytes) {
    const char *f = std::getenv("BP_TEST_FAIL_ALLOC");
    const int nth = f ? std::atoi(f) : 0;
    if (nth > 0 && ++ctx->n_allocs == nth) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live_allocs;
    return e;
}

static void dev_free(void *p) {
    if (p) {
        cudaFree(p);
        --g_live_allocs;
    }
}

static void build_matrices(const bp_geometry &g, const double *angles, double *P) {
    const double cu = 0.5 * (g.nu - 1) + g.u_off_px;
    const double cv = 0.5 * (g.nv - 1) + g.v_off_px;
    const double x0 = g.ox - 0.5 * (g.nx - 1) * g.sx;
    const double y0 = g.oy - 0.5 * (g.ny - 1) * g.sy;
    const double z0 = g.oz - 0.5 * (g.nz - 1) * g.sz;
    const double mu = g.sdd / (g.sid * g.du), mv = g.sdd / (g.sid * g.dv);
    for (int s = 0; s < g.n_views; ++s) {
        const double c = std::cos(angles[s]), sn = std::sin(angles[s]);
        // world-space rows acting on (x, y, z, 1): depth w = 1 - X.e_r/sid,
        // u*w = (sdd/(sid*du)) X.e_u + cu*w, v*w = (sdd/(sid*dv)) z + cv*w
        const double rw[4] = {-c / g.sid, -sn / g.sid, 0.0, 1.0};
        const double ru[4] = {-sn * mu + cu * rw[0], c * mu + cu * rw[1], 0.0, cu};
        const double rv[4] = {cv * rw[0], cv * rw[1], mv, cv};
        const double *rows[3] = {ru, rv, rw};
        for (int r = 0; r < 3; ++r) {
            double *o = P + 12 * s + 4 * r;
            o[0] = rows[r][0] * g.sx;
            o[1] = rows[r][1] * g.sy;
            o[2] = rows[r][2] * g.sz;
            o[3] = rows[r][0] * x0 + rows[r][1] * y0 + rows[r][2] * z0 + rows[r][3];
        }
    }
}

// Depth w at the 8 corners of the volume must be positive in every view.
static bool all_in_front(const double *P, int np, int nx, int ny, int nz) {
    for (int s = 0; s < np; ++s)
        for (int c = 0; c < 8; ++c) {
            double i = (c & 1) ? nx - 1 : 0, j = (c & 2) ? ny - 1 : 0, k = (c & 4) ? nz - 1 : 0;
            const double *w = P + 12 * s + 8;
            double d = w[0] * i + w[1] * j + w[2] * k + w[3];
            if (!(d > 1e-6)) return false;
        }
    return true;
}

static int floor_div_h(int a, int b) {
    int q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Worst-case staged box over every tile and view: the corner rule of the
// device records (geom_dev.cuh make_rec) applied to exact FP64 corners with
// a wider margin.
void max_footprint(const bp_ctx *ctx, int tx, int ty, int tk, int align, int *bu, int *bv) {
    const int nx = ctx->nx, ny = ctx->ny, nz = ctx->nz, np = ctx->n_views;
    const int ntx = (nx + tx - 1) / tx, nty = (ny + ty - 1) / ty, ntz = (nz + tk - 1) / tk;
    const long long ntiles = (long long)ntx * nty * ntz;
    unsigned nthr = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<int> mu(nthr, 0), mv(nthr, 0);
    auto work = [&](unsigned t) {
        int bu_ = 0, bv_ = 0;
        for (long long tile = t; tile < ntiles; tile += nthr) {
            int i0 = (int)(tile % ntx) * tx, j0 = (int)((tile / ntx) % nty) * ty,
                k0 = (int)(tile / ((long long)ntx * nty)) * tk;
            int ex = std::min(tx, nx - i0), ey = std::min(ty, ny - j0), ez = std::min(tk, nz - k0);
            for (int s = 0; s < np; ++s) {
                const double *P = ctx->P.data() + 12 * s;
                double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
                for (int c = 0; c < 8; ++c) {
                    double i = i0 + ((c & 1) ? ex - 1 : 0), j = j0 + ((c & 2) ? ey - 1 : 0),
                           k = k0 + ((c & 4) ? ez - 1 : 0);
                    double w = P[8] * i + P[9] * j + P[10] * k + P[11];
                    double iw = 1.0 / w;
                    double u = (P[0] * i + P[1] * j + P[2] * k + P[3]) * iw;
                    double v = (P[4] * i + P[5] * j + P[6] * k + P[7]) * iw;
                    umin = std::min(umin, u); umax = std::max(umax, u);
                    vmin = std::min(vmin, v); vmax = std::max(vmax, v);
                }
                // the device divides corners in FP32 and widens them by 0.01 px;
                // 0.02 px here covers that rounding, so the plan is an upper bound
                umin = std::max(std::min(umin - 0.02, 1e8), -1e8); umax = std::max(std::min(umax + 0.02, 1e8), -1e8);
                vmin = std::max(std::min(vmin - 0.02, 1e8), -1e8); vmax = std::max(std::min(vmax + 0.02, 1e8), -1e8);
                int ub = floor_div_h((int)std::floor(umin) - 1, align) * align;
                int vb = (int)std::floor(vmin) - 1;
                bu_ = std::max(bu_, (int)std::floor(umax) + 2 - ub + 1);
                bv_ = std::max(bv_, (int)std::floor(vmax) + 2 - vb + 1);
            }
        }
        mu[t] = bu_;
        mv[t] = bv_;
    };
    std::vector<std::thread> th;
    for (unsigned t = 1; t < nthr; ++t) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();
    *bu = *std::max_element(mu.begin(), mu.end());
    *bv = *std::max_element(mv.begin(), mv.end());
}

// Shared memory of the staged back-projector: view records, 2 x 8 barrier
// slots, then one box per stage (each rounded up to 128 bytes).
static int tma_smem_bytes(int bu, int bv, int elem_bytes, int stages) {
    const int base = (256 * 48 + 2 * 8 * 8 + 127) / 128 * 128;
    return base + stages * ((bu * bv * elem_bytes + 127) / 128 * 128);
}

// Mid-plane symmetry of the matrices (Section 3.1.2): v(i, j, nz-1-k) =
// nv-1 - v(i, j, k) for every voxel and view. With u and w independent of k
// this holds iff 2 P[1][0] = (nv-1) P[2][0], 2 P[1][1] = (nv-1) P[2][1] and
// 2 P[1][3] + (nz-1) P[1][2] = (nv-1) P[2][3]; checked to 1e-10 relative.
static bool mirror_symmetric(const bp_ctx *ctx) {
    if (!ctx->zinv) return false;
    const double a = ctx->nv - 1.0, c = ctx->nz - 1.0;
    auto close = [](double x, double y) { return std::fabs(x - y) <= 1e-10 * (std::fabs(x) + std::fabs(y) + 1e-300); };
    for (int s = 0; s < ctx->n_views; ++s) {
        const double *p = &ctx->P[12 * (size_t)s];
        if (!close(2.0 * p[4], a * p[8]) || !close(2.0 * p[5], a * p[9]) || !close(2.0 * p[7] + c * p[6], a * p[11]))
            return false;
    }
    return true;
}

static void make_plan(bp_ctx *ctx) {
    Plan &pl = ctx->plan;
    pl.tx = 32;
    pl.ty = 8;
    if (ctx->stages_req < 1 || ctx->stages_req > 8) ctx->stages_req = 4;
    if (pl.tk != 64) pl.tk = 32;
    if (pl.ctas != 3) pl.ctas = 2;
    if (!ctx->zinv) {
        pl.bu = pl.bu16 = -1;
        pl.bv = 0;
        return;
    }
    int bu32, bv32, bu16, bv16;
    max_footprint(ctx, pl.tx, pl.ty, pl.tk, 4, &bu32, &bv32);
    max_footprint(ctx, pl.tx, pl.ty, pl.tk, 8, &bu16, &bv16);
    pl.bu = plan_box_width(bu32, 4);
    pl.bu16 = plan_box_width(bu16, 2);
    pl.bv = std::max(bv32, bv16);
    // shared memory budget of the TMA kernel (records + barriers + the stages):
    // the requested depth, lowered (to 2 at least) until the FP32 boxes fit
    auto fits = [&](int bu, int es, int st) { return bu > 0 && tma_smem_bytes(bu, pl.bv, es, st) <= 227 * 1024; };
    pl.stages = ctx->stages_req;
    while (pl.stages > 2 && !fits(pl.bu, 4, pl.stages)) --pl.stages;
    if (pl.bv > 256 || !fits(pl.bu, 4, pl.stages)) pl.bu = -1;
    if (pl.bv > 256 || !fits(pl.bu16, 2, pl.stages)) pl.bu16 = -1;
    // mid-plane symmetry: boxes of 16-voxel half columns, two per stage
    pl.sym_bu = pl.sym_bv = -1;
    if (ctx->sym_enable && pl.bu > 0 && mirror_symmetric(ctx)) {
        int sbu, sbv;
        max_footprint(ctx, pl.tx, pl.ty, 16, 4, &sbu, &sbv);
        sbu = plan_box_width(sbu, 4);
        if (sbu > 0 && sbv <= 256 && tma_smem_bytes(sbu, sbv, 4, 2 * pl.stages) <= 227 * 1024) {
            pl.sym_bu = sbu;
            pl.sym_bv = sbv;
        }
    }
    // forward projector: lane windows as wide as the u footprint of an 8 x 4
    // column patch (+1 column of slack for the FP32 corner rounding)
    int wbu, wbv;
    max_footprint(ctx, 8, 4, 32, 1, &wbu, &wbv);
    wbu += 1;
    wbu = fp_window_width(wbu);
    pl.fp_wbu = (pl.bu > 0 && wbu > 0 && fp_smem_bytes(wbu) <= 227 * 1024) ? wbu : -1;
}

// Ramp filter tables: real spectrum of the circularly embedded Ram-Lak
// kernel (times dp and 1/N, natural order) and the N FFT twiddles.
static bp_status make_filter_tables(bp_ctx *ctx) {
    const bp_geometry &g = ctx->g;
    int n = ct_fft_size(g.nu), lg = 0;
    ctx->fft_quad = n > 0;
    if (!ctx->fft_quad) {
        n = 1;
        while (n < 2 * g.nu - 1 || n < 16) n <<= 1;
    }
    while ((1 << lg) < n) ++lg;
    ctx->fft_n = n;
    ctx->fft_log2 = lg;
    const double dp = g.du * g.sid / g.sdd;
    std::vector<double> h(g.nu);
    for (int m = 0; m < g.nu; ++m)
        h[m] = (m == 0) ? 1.0 / (4.0 * dp * dp)
               : (m % 2 == 0) ? 0.0
               : -1.0 / (M_PI * M_PI * (double)m * (double)m * dp * dp);
    // H[k] = h[0] + 2 sum_m h[m] cos(2 pi k m / N) (even kernel -> real spectrum),
    // times dp (the convolution's quadrature weight) and 1/N (inverse FFT)
    std::vector<double> Hd(n);
    std::vector<float> Hf(n), tw(2 * (size_t)n);
    for (int k = 0; k < n; ++k) {
        double acc = h[0];
        for (int m = 1; m < g.nu; m += 2) acc += 2.0 * h[m] * std::cos(2.0 * M_PI * (double)((long long)k * m % n) / n);
        Hd[k] = acc * dp / n;
        Hf[k] = (float)Hd[k];
    }
    if (ctx->fft_quad) {
        // four-row kernel: spectrum (times sdd, the cosine weight's numerator) at
        // the digit-reversed positions of its fused step, and twiddles per pass
        std::vector<double> Hs(n);
        for (int k = 0; k < n; ++k) Hs[k] = Hd[k] * g.sdd;
        const int ntw = ct_twiddle_count(n);
        std::vector<float> cH(2 * (size_t)n), ctw(4 * (size_t)(ntw > 0 ? ntw : 1));
        ct_tables(n, Hs.data(), cH.data(), ctw.data());
        cudaError_t e = dev_alloc(ctx, &ctx->d_ctH, sizeof(float) * 2 * n);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "filter spectrum");
        e = dev_alloc(ctx, &ctx->d_cttw, sizeof(float) * ctw.size());
        if (e != cudaSuccess) return cuda_fail(ctx, e, "filter twiddles");
        e = cudaMemcpy(ctx->d_ctH, cH.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ctx->d_cttw, ctw.data(), sizeof(float) * ctw.size(), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "filter tables upload");
    }
    for (int k = 0; k < n; ++k) {
        tw[2 * k] = (float)std::cos(2.0 * M_PI * k / n);
        tw[2 * k + 1] = (float)-std::sin(2.0 * M_PI * k / n);
    }
    cudaError_t e = dev_alloc(ctx, (void **)&ctx->d_H, sizeof(float) * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "filter spectrum");
    e = dev_alloc(ctx, (void **)&ctx->d_tw, sizeof(float2) * n);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "filter twiddles");
    e = cudaMemcpy(ctx->d_H, Hf.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ctx->d_tw, tw.data(), sizeof(float2) * n, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "filter tables upload");
}

static bp_status finish_create(bp_ctx *ctx) {
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGetDevice");
    cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    const int np = ctx->n_views;
    ctx->zinv = true;
    for (int s = 0; s < np; ++s)
        if (ctx->P[12 * s + 2] != 0.0 || ctx->P[12 * s + 10] != 0.0) ctx->zinv = false;
    e = dev_alloc(ctx, (void **)&ctx->d_P, sizeof(double) * 12 * np);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "matrices");
    e = cudaMemcpy(ctx->d_P, ctx->P.data(), sizeof(double) * 12 * np, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "matrices upload");
    e = dev_alloc(ctx, (void **)&ctx->d_err, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word");
    e = cudaMemset(ctx->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error word");
    make_plan(ctx);
    if (ctx->has_geometry) {
        bp_status st = make_filter_tables(ctx);
        if (st != BP_OK) return st;
        e = dev_alloc(ctx, (void **)&ctx->d_phcoef, sizeof(float) * 20 * 256 * (size_t)np);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "phantom coefficient buffer");
    }
    return BP_OK;
}

static bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace bp

using namespace bp;

extern "C" {

bp_status bp_create(const bp_geometry *g, bp_ctx **out) {
    if (!g || !out) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: NULL argument");
    if (!(finite_pos(g->sid) && finite_pos(g->sdd) && g->sid < g->sdd))
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: need 0 < sid < sdd (finite)");
    if (g->n_views < 1 || g->nu < 2 || g->nv < 2 || g->nx < 1 || g->ny < 1 || g->nz < 1)
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: sizes must be >= 1 (detector >= 2)");
    if ((long long)g->nu * g->nv > (1ll << 31) || (long long)g->nx * g->ny * g->nz > (1ll << 40))
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: sizes too large");
    if (!(finite_pos(g->du) && finite_pos(g->dv) && finite_pos(g->sx) && finite_pos(g->sy) &&
          finite_pos(g->sz)))
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: pitches and spacings must be > 0");
    if (!(std::isfinite(g->u_off_px) && std::isfinite(g->v_off_px) && std::isfinite(g->ox) &&
          std::isfinite(g->oy) && std::isfinite(g->oz)))
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: offsets must be finite");
    bp_ctx *ctx = new (std::nothrow) bp_ctx();
    if (!ctx) return fail(nullptr, BP_ERR_OOM, "bp_create: host allocation");
    ctx->g = *g;
    ctx->angles.resize(g->n_views);
    for (int s = 0; s < g->n_views; ++s) {
        ctx->angles[s] = g->angles ? g->angles[s] : 2.0 * M_PI * s / g->n_views;
        if (!std::isfinite(ctx->angles[s])) {
            delete ctx;
            return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: non-finite angle");
        }
    }
    ctx->g.angles = nullptr;
    ctx->n_views = g->n_views;
    ctx->nu = g->nu; ctx->nv = g->nv;
    ctx->nx = g->nx; ctx->ny = g->ny; ctx->nz = g->nz;
    ctx->has_geometry = true;
    ctx->P.resize(12 * (size_t)g->n_views);
    build_matrices(ctx->g, ctx->angles.data(), ctx->P.data());
    if (!all_in_front(ctx->P.data(), ctx->n_views, ctx->nx, ctx->ny, ctx->nz)) {
        delete ctx;
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create: volume reaches behind the source");
    }
    bp_status st = finish_create(ctx);
    if (st != BP_OK) {
        g_create_err = ctx->err;
        bp_destroy(ctx);
        return st;
    }
    *out = ctx;
    return BP_OK;
}

bp_status bp_create_from_matrices(const double *P, int n_views, int nu, int nv, int nx, int ny,
                                  int nz, bp_ctx **out) {
    if (!P || !out) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create_from_matrices: NULL argument");
    if (n_views < 1 || nu < 2 || nv < 2 || nx < 1 || ny < 1 || nz < 1)
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create_from_matrices: bad sizes");
    for (long long t = 0; t < 12ll * n_views; ++t)
        if (!std::isfinite(P[t]))
            return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create_from_matrices: non-finite matrix");
    if (!all_in_front(P, n_views, nx, ny, nz))
        return fail(nullptr, BP_ERR_INVALID_ARG, "bp_create_from_matrices: depth <= 0 at a volume corner");
    bp_ctx *ctx = new (std::nothrow) bp_ctx();
    if (!ctx) return fail(nullptr, BP_ERR_OOM, "host allocation");
    ctx->n_views = n_views;
    ctx->nu = nu; ctx->nv = nv;
    ctx->nx = nx; ctx->ny = ny; ctx->nz = nz;
    ctx->P.assign(P, P + 12 * (size_t)n_views);
    bp_status st = finish_create(ctx);
    if (st != BP_OK) {
        g_create_err = ctx->err;
        bp_destroy(ctx);
        return st;
    }
    *out = ctx;
    return BP_OK;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bp_status bp_filter(bp_ctx *ctx, const float *proj, void *out, bp_dtype out_t, int batch,
                    void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_filter: NULL context");
    return bp_filter_views(ctx, proj, out, out_t, ctx->n_views, batch, stream);
}

bp_status bp_filter_views(bp_ctx *ctx, const float *proj, void *out, bp_dtype out_t, int n_views,
                          int batch, void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_filter: NULL context");
    if (n_views < 1) return fail(ctx, BP_ERR_INVALID_ARG, "bp_filter: n_views < 1");
    ctx->err.clear();
    if (!ctx->has_geometry) return fail(ctx, BP_ERR_UNSUPPORTED, "bp_filter: context has no physical geometry");
    if (!proj || !out || batch < 1) return fail(ctx, BP_ERR_INVALID_ARG, "bp_filter: NULL pointer or batch < 1");
    if (out_t != BP_F32 && out_t != BP_F16) return fail(ctx, BP_ERR_INVALID_ARG, "bp_filter: bad dtype");
    if (!aligned16(proj) || !aligned16(out)) return fail(ctx, BP_ERR_INVALID_ARG, "bp_filter: pointers must be 16-byte aligned");
    if (out_t == BP_F16 && (const void *)proj == out) return fail(ctx, BP_ERR_INVALID_ARG, "bp_filter: FP16 output may not alias the input");
    return launch_filter(ctx, proj, out, out_t, (long long)batch * n_views, (cudaStream_t)stream);
}

static bp_status check_bp_args(bp_ctx *ctx, const void *proj, bp_dtype t, int view0, int n_views,
                               long long proj_batch_stride, const float *vol, int batch, float scale) {
    if (!proj || !vol || batch < 1) return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject: NULL pointer or batch < 1");
    if (t != BP_F32 && t != BP_F16) return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject: bad dtype");
    if (view0 < 0 || n_views < 1 || view0 + n_views > ctx->n_views)
        return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject: view range outside the geometry");
    if (proj_batch_stride < 0 || (proj_batch_stride != 0 && proj_batch_stride < (long long)n_views * ctx->nu * ctx->nv))
        return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject: batch stride smaller than one batch entry");
    if (!aligned16(proj) || !aligned16(vol)) return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject: pointers must be 16-byte aligned");
    if (!std::isfinite(scale)) return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject: non-finite scale");
    return BP_OK;
}

bp_status bp_backproject_views(bp_ctx *ctx, const void *proj, bp_dtype t, int view0, int n_views,
                               long long proj_batch_stride, float *vol, int batch, float scale,
                               int accumulate, void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_backproject: NULL context");
    ctx->err.clear();
    bp_status s = check_bp_args(ctx, proj, t, view0, n_views, proj_batch_stride, vol, batch, scale);
    if (s != BP_OK) return s;
    // the whole volume: the lower half and its mirror where the symmetric kernel applies
    const bool sym = ctx->zinv && t == BP_F32 && ctx->plan.sym_bu > 0;
    return launch_backproject(ctx, proj, t, view0, n_views, proj_batch_stride, vol, batch, scale,
                              accumulate ? 1 : 0, (cudaStream_t)stream, 0, sym ? (ctx->nz + 1) / 2 : ctx->nz,
                              sym ? 1 : 0);
}

bp_status bp_backproject_slab(bp_ctx *ctx, const void *proj, bp_dtype t, int view0, int n_views,
                              long long proj_batch_stride, int z0, int nz_slab, int mirror, float *vol,
                              int batch, float scale, int accumulate, void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_backproject_slab: NULL context");
    ctx->err.clear();
    bp_status s = check_bp_args(ctx, proj, t, view0, n_views, proj_batch_stride, vol, batch, scale);
    if (s != BP_OK) return s;
    if (z0 < 0 || nz_slab < 1 || z0 + nz_slab > ctx->nz)
        return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject_slab: slice range outside the volume");
    if (mirror && z0 + nz_slab > (ctx->nz + 1) / 2)
        return fail(ctx, BP_ERR_INVALID_ARG, "bp_backproject_slab: a mirrored slab must lie in the lower half");
    return launch_backproject(ctx, proj, t, view0, n_views, proj_batch_stride, vol, batch, scale,
                              accumulate ? 1 : 0, (cudaStream_t)stream, z0, nz_slab, mirror ? 1 : 0);
}

bp_status bp_backproject(bp_ctx *ctx, const void *proj, bp_dtype t, float *vol, int batch,
                         float scale, int accumulate, void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_backproject: NULL context");
    return bp_backproject_views(ctx, proj, t, 0, ctx->n_views, 0, vol, batch, scale, accumulate, stream);
}

bp_status fp_project(bp_ctx *ctx, const float *vol, float *proj, int batch, float scale,
                     void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "fp_project: NULL context");
    ctx->err.clear();
    if (!proj || !vol || batch < 1) return fail(ctx, BP_ERR_INVALID_ARG, "fp_project: NULL pointer or batch < 1");
    if (!aligned16(proj) || !aligned16(vol)) return fail(ctx, BP_ERR_INVALID_ARG, "fp_project: pointers must be 16-byte aligned");
    if (!std::isfinite(scale)) return fail(ctx, BP_ERR_INVALID_ARG, "fp_project: non-finite scale");
    return launch_forward(ctx, vol, proj, batch, scale, (cudaStream_t)stream);
}

bp_status bp_phantom_project(bp_ctx *ctx, const double *ell, int n_ell, float *proj, void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_phantom_project: NULL context");
    ctx->err.clear();
    if (!ctx->has_geometry) return fail(ctx, BP_ERR_UNSUPPORTED, "bp_phantom_project: context has no physical geometry");
    if (!ell || !proj || n_ell < 0 || n_ell > 256) return fail(ctx, BP_ERR_INVALID_ARG, "bp_phantom_project: bad arguments (at most 256 ellipsoids)");
    for (int t = 0; t < 16 * n_ell; ++t)
        if (!std::isfinite(ell[t])) return fail(ctx, BP_ERR_INVALID_ARG, "bp_phantom_project: non-finite ellipsoid");
    for (int e = 0; e < n_ell; ++e)
        if (!(ell[16 * e + 3] > 0 && ell[16 * e + 4] > 0 && ell[16 * e + 5] > 0))
            return fail(ctx, BP_ERR_INVALID_ARG, "bp_phantom_project: semi-axes must be > 0");
    return launch_phantom(ctx, ell, n_ell, proj, (cudaStream_t)stream);
}

bp_status bp_get_matrices(const bp_ctx *ctx, double *P_out) {
    if (!ctx || !P_out) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_get_matrices: NULL argument");
    std::memcpy(P_out, ctx->P.data(), sizeof(double) * ctx->P.size());
    return BP_OK;
}

bp_status bp_get_dims(const bp_ctx *ctx, int *n_views, int *nu, int *nv, int *nx, int *ny, int *nz) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_get_dims: NULL context");
    if (n_views) *n_views = ctx->n_views;
    if (nu) *nu = ctx->nu;
    if (nv) *nv = ctx->nv;
    if (nx) *nx = ctx->nx;
    if (ny) *ny = ctx->ny;
    if (nz) *nz = ctx->nz;
    return BP_OK;
}

bp_status bp_device_status(bp_ctx *ctx, void *stream) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_device_status: NULL context");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_device_status: stream");
    unsigned w = 0;
    e = cudaMemcpy(&w, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_device_status: read");
    e = cudaMemset(ctx->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "bp_device_status: clear");
    if (w & DEV_ERR_TIMEOUT) return fail(ctx, BP_ERR_TIMEOUT, "a kernel's bounded wait ran out");
    if (w & DEV_ERR_FOOTPRINT) return fail(ctx, BP_ERR_DEVICE, "a view's footprint did not fit the staged box");
    if (w) return fail(ctx, BP_ERR_DEVICE, "kernel error word set");
    ctx->err.clear();
    return BP_OK;
}

bp_status bp_set_tuning(bp_ctx *ctx, int tk, int ctas_per_sm) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_set_tuning: NULL context");
    if (tk != 32 && tk != 64) return fail(ctx, BP_ERR_INVALID_ARG, "bp_set_tuning: tk must be 32 or 64");
    if (ctas_per_sm != 2 && ctas_per_sm != 3)
        return fail(ctx, BP_ERR_INVALID_ARG, "bp_set_tuning: ctas_per_sm must be 2 or 3");
    ctx->plan.tk = tk;
    ctx->plan.ctas = ctas_per_sm;
    make_plan(ctx);
    return BP_OK;
}

bp_status bp_set_pipeline_depth(bp_ctx *ctx, int stages) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_set_pipeline_depth: NULL context");
    if (stages < 1 || stages > 8)
        return fail(ctx, BP_ERR_INVALID_ARG, "bp_set_pipeline_depth: stages must be in [1, 8]");
    const Plan &pl = ctx->plan;
    if ((pl.bu > 0 && tma_smem_bytes(pl.bu, pl.bv, 4, stages) > 227 * 1024) ||
        (pl.bu16 > 0 && tma_smem_bytes(pl.bu16, pl.bv, 2, stages) > 227 * 1024))
        return fail(ctx, BP_ERR_INVALID_ARG, "bp_set_pipeline_depth: the staged boxes do not fit in shared memory");
    ctx->stages_req = stages;
    make_plan(ctx);
    return BP_OK;
}

bp_status bp_set_symmetry(bp_ctx *ctx, int enable) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_set_symmetry: NULL context");
    ctx->sym_enable = enable != 0;
    make_plan(ctx);
    if (enable && ctx->plan.sym_bu <= 0) {
        ctx->sym_enable = 0;
        make_plan(ctx);
        return fail(ctx, BP_ERR_UNSUPPORTED,
                    "bp_set_symmetry: the matrices are not mirror-symmetric about the central slice, "
                    "or the staged boxes do not fit");
    }
    return BP_OK;
}

bp_status bp_set_timeout(bp_ctx *ctx, double seconds) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_set_timeout: NULL context");
    if (!(seconds > 0.0 && seconds <= 60.0)) return fail(ctx, BP_ERR_INVALID_ARG, "bp_set_timeout: (0, 60] seconds");
    ctx->timeout_ns = (unsigned long long)(seconds * 1e9);
    return BP_OK;
}

bp_status bp_test_drop_view(bp_ctx *ctx, int view) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_test_drop_view: NULL context");
    ctx->test_drop_view = view;
    return BP_OK;
}

bp_status bp_get_plan(const bp_ctx *ctx, int *tk, int *bu32, int *bu16, int *bv, int *stages,
                      int *symmetric) {
    if (!ctx) return fail(nullptr, BP_ERR_INVALID_ARG, "bp_get_plan: NULL context");
    if (tk) *tk = ctx->plan.tk;
    if (bu32) *bu32 = ctx->plan.bu;
    if (bu16) *bu16 = ctx->plan.bu16;
    if (bv) *bv = ctx->plan.bv;
    if (stages) *stages = ctx->plan.stages;
    if (symmetric) *symmetric = ctx->plan.sym_bu > 0;
    return BP_OK;
}

const char *bp_last_error(const bp_ctx *ctx) {
    if (!ctx) return g_create_err.c_str();
    return ctx->err.c_str();
}

void bp_destroy(bp_ctx *ctx) {
    if (!ctx) return;
    dev_free(ctx->d_P);
    dev_free(ctx->d_err);
    dev_free(ctx->d_H);
    dev_free(ctx->d_tw);
    dev_free(ctx->d_ctH);
    dev_free(ctx->d_cttw);
    dev_free(ctx->d_phcoef);
    delete ctx;
}

int bp_test_live_allocations(void) { return (int)g_live_allocs.load(); }

}  // extern "C"
