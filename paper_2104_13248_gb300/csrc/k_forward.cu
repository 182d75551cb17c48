// Matched voxel-driven forward projector: the exact transpose of the
// back-projection of Listing 1. Every voxel value, times scale / w^2, is
// scattered to the same four detector taps with the same bilinear weights
// the back-projector reads them with. A CTA owns a 32 x 8 x 32 tile of
// voxels; each warp owns an 8 x 4 patch of its columns, one lane per voxel
// of a column, the patch's values held in registers. Records (geometry
// relative to the box origin) are the ones the back-projector uses, so the
// taps coincide.
//
// Per view, each lane accumulates its voxels' taps in a private window of
// kFpWinRows detector rows in shared memory: within a small patch the
// columns' depths differ by well under one percent, so the rows lane l's
// voxel reaches in the patch's 32 columns stay within two rows of a common
// lower bound. Private windows keep the scatter free of bank conflicts and
// of hazards between lanes (no warp barriers), where one box shared by the
// warp folds the column's ~2 x 32 rows onto 32 banks. The windows then go
// to the projection with one global reduction per window cell, so the
// overlapping windows add up there. A tap beyond its lane's window
// (columns whose rows drift further apart) is added to the projection
// directly.
#include "geom_dev.cuh"

namespace bp {

constexpr int kFpTX = 32, kFpTY = 8, kFpTK = 32;
constexpr int kFpThreads = kFpTX * kFpTY;
constexpr int kFpWinRows = 3;     // detector rows of a lane's window
constexpr int kFpRecChunk = 64;   // view records staged per pass

// Per (column, view) quantities shared by the 32 lanes that scatter the
// column's voxels (computed once per view by the thread owning the column).
struct __align__(16) FpCol {
    float v0, dv, wt, fu;   // v of the first voxel and per voxel (box-relative), 1 / W^2, u fraction
    float gu;               // 1 - fu
    int cw32, cwG, cwG1;    // window column * 32, window column * G and (column + 1) * G, G the
                            // windows a flush pass reads; wt = 0 marks a column without voxels
};

// Window layout of one warp: row dr (0..kFpWinRows-1), column c (0..wc-1)
// and lane l at word (dr * wc + c) * 32 + ((l + c * G) & 31), with G the
// number of windows the flush reads per pass (32 / used width, or 1). A
// scatter (one column, 32 lanes) touches 32 different banks, and so do the
// live lanes of a flush pass (G windows of cw consecutive columns,
// G * cw <= 32).
int fp_smem_bytes(int wc) {
    return kFpRecChunk * (int)sizeof(ViewRec) + kFpThreads * (int)sizeof(FpCol) +
           (kFpThreads / 32) * kFpWinRows * wc * 32 * (int)sizeof(float);
}

__device__ __forceinline__ void fp_tap(float *img, int nu, int nv, int row, int col, float a) {
    if (a != 0.0f && (unsigned)row < (unsigned)nv && (unsigned)col < (unsigned)nu)
        atomicAdd(img + (size_t)row * nu + col, a);
}

__device__ __forceinline__ int floor_bits(float v) { return __float_as_int(__fadd_rd(v, kMagic)); }

template <int TK>
__global__ void __launch_bounds__(kFpThreads, 3)
fp_zcol(const float *__restrict__ vol, const double *__restrict__ P, int nviews, int nu, int nv,
        int nx, int ny, int nz, int bu, int bv, int wc, float scale, float *__restrict__ proj,
        unsigned *err) {
    static_assert(TK == 32, "one lane per voxel of a 32-voxel column chunk");
    extern __shared__ __align__(16) unsigned char smem[];
    ViewRec *recs = reinterpret_cast<ViewRec *>(smem);
    FpCol *cols = reinterpret_cast<FpCol *>(smem + kFpRecChunk * sizeof(ViewRec));
    const int wwords = kFpWinRows * wc * 32;   // one warp's windows
    const int rstride = wc * 32;               // words between window rows
    float *win = reinterpret_cast<float *>(smem + kFpRecChunk * sizeof(ViewRec) + kFpThreads * sizeof(FpCol)) +
                 (threadIdx.x >> 5) * wwords;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (nx + kFpTX - 1) / kFpTX;
    const int i0 = (blockIdx.x % ntx) * kFpTX, j0 = (blockIdx.x / ntx) * kFpTY;
    const int k0 = blockIdx.y * TK;
    const int b = blockIdx.z;
    const int ex = min(kFpTX, nx - i0), ey = min(kFpTY, ny - j0), ez = min(TK, nz - k0);
    // column owned by this thread for the per-view setup (8 x 4 patch per warp)
    const int wx = warp % (kFpTX / 8), wy = warp / (kFpTX / 8);
    const int di = wx * 8 + (lane & 7), dj = wy * 4 + (lane >> 3);
    const bool col_ok = di < ex && dj < ey;
    const float fdi = (float)di, fdj = (float)dj;

    // lane l holds voxel k0 + l of each of the warp's 32 columns
    float x[32];
    {
        const size_t plane = (size_t)nx * ny;
        const bool kin = lane < ez;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const int cdi = wx * 8 + (c & 7), cdj = wy * 4 + (c >> 3);
            const bool ok = kin && cdi < ex && cdj < ey;
            x[c] = ok ? scale * vol[((size_t)b * nz + k0 + lane) * plane + (size_t)(j0 + cdj) * nx + (i0 + cdi)]
                      : 0.0f;
        }
    }
    float *pb = proj + (size_t)b * nviews * nu * nv;
    for (int t = 4 * lane; t < wwords; t += 128) *reinterpret_cast<float4 *>(win + t) = make_float4(0.f, 0.f, 0.f, 0.f);

    for (int cb = 0; cb < nviews; cb += kFpRecChunk) {
        const int cn = min(kFpRecChunk, nviews - cb);
        __syncthreads();
        for (int n = tid; n < cn; n += kFpThreads) {
            ViewRec r;
            if (!make_rec(P + 12 * (size_t)(cb + n), i0, j0, k0, ex, ey, ez, 4, bu, bv, &r))
                atomicOr(err, DEV_ERR_FOOTPRINT);
            recs[n] = r;
        }
        for (int n = 0; n < cn; ++n) {
            __syncthreads();   // records ready; previous view's column setup consumed
            const ViewRec r = recs[n];
            FpCol c;
            float uL = 0.0f, cv0 = 0.0f, cdv = 0.0f, cwt = 0.0f, cfu = 0.0f;
            int cu = 0;
            bool cok = false;
            float umin = 3e38f, umax = -3e38f, v0min = 3e38f, dvmin = 3e38f;
            if (col_ok) {
                float W = fmaf(r.Wj, fdj, fmaf(r.Wi, fdi, r.W0));
                float inv = col_rcp(W);
                uL = fmaf(r.Nuj, fdj, fmaf(r.Nui, fdi, r.Nu0)) * inv;
                cv0 = fmaf(r.Nvj, fdj, fmaf(r.Nvi, fdi, r.Nv0)) * inv;
                cdv = r.Nvk * inv;
                cwt = inv * inv;
                float tu = __fadd_rd(uL, kMagic);
                cu = __float_as_int(tu) - kMagicBits;
                cfu = uL - (tu - kMagic);
                if (uL == uL && cv0 == cv0) {
                    // every coordinate stays far inside the range of the round-to-integer trick
                    if (fabsf(cdv) < 1e4f && fabsf(cv0) < 1e6f && fabsf(uL) < 1e6f) {
                        cok = true;
                        umin = umax = uL;
                        v0min = cv0;
                        dvmin = cdv;
                    } else {
                        atomicOr(err, DEV_ERR_FOOTPRINT);
                    }
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
                umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
                v0min = fminf(v0min, __shfl_xor_sync(0xffffffffu, v0min, o));
                dvmin = fminf(dvmin, __shfl_xor_sync(0xffffffffu, dvmin, o));
            }
            const bool any = umin <= umax;
            const int uo = any ? floor_bits(umin) - kMagicBits : 0;
            const int cols_used = any ? floor_bits(umax) - kMagicBits + 2 - uo : 0;
            // A patch wider than the planned windows (not expected from the
            // plan's footprint bound) still projects every tap: all of them
            // take the direct pass below, which is correct at any width.
            const bool fits = any && cols_used <= wc;
            const int cwid = max(1, min(cols_used, 32));
            const int G = 32 / cwid;
            // A column outside the patch or without a usable geometry scatters
            // zeros at window row 0, column 0 (no branch in the scatter loop).
            c.v0 = cok ? cv0 : v0min;
            c.dv = cok ? cdv : dvmin;
            c.wt = cok ? cwt : 0.0f;
            c.fu = cok ? cfu : 0.0f;
            c.gu = 1.0f - c.fu;
            const int cwin = cok ? cu - uo : 0;
            c.cw32 = cwin * 32;
            c.cwG = cwin * G;
            c.cwG1 = c.cwG + G;
            cols[tid] = c;
            __syncwarp();
            if (!any) continue;   // uniform across the warp

            // Lane l's window starts at row floor(v0min + l * dvmin): every
            // column's row floor(v0 + l * dv) is at or above it (v0 >= v0min,
            // dv >= dvmin, l >= 0, and fmaf and the floor are monotone).
            const float fl = (float)lane;
            const int tb = floor_bits(fmaf(fl, dvmin, v0min));
            const int base = tb - kMagicBits;
            float *img = pb + (size_t)(cb + n) * nu * nv;
            unsigned dmax = fits ? 0u : ~0u;
#pragma unroll
            for (int cix = 0; fits && cix < 32; ++cix) {
                const FpCol cc = cols[warp * 32 + cix];
                const float v = fmaf(fl, cc.dv, cc.v0);
                const float tv = __fadd_rd(v, kMagic);
                const float fv = v - (tv - kMagic);
                const unsigned udr = (unsigned)(__float_as_int(tv) - tb);   // >= 0 as a signed value
                dmax = max(dmax, udr);
                const bool in = udr <= (unsigned)(kFpWinRows - 2);
                const int drc = in ? (int)udr : 0;
                const float val = in ? cc.wt * x[cix] : 0.0f;   // beyond the window: the pass below
                const float a1 = fv * val, a0 = val - a1;       // (1-fv) val, fv val
                const int w0 = drc * rstride + cc.cw32 + ((lane + cc.cwG) & 31);
                const int w1 = drc * rstride + cc.cw32 + 32 + ((lane + cc.cwG1) & 31);
                win[w0] += cc.gu * a0;
                win[w1] += cc.fu * a0;
                win[w0 + rstride] += cc.gu * a1;
                win[w1 + rstride] += cc.fu * a1;
            }
            if (__any_sync(0xffffffffu, lane < ez && dmax > (unsigned)(kFpWinRows - 2))) {
                // taps beyond a lane's window go straight to the projection
#pragma unroll
                for (int cix = 0; cix < 32; ++cix) {
                    const FpCol cc = cols[warp * 32 + cix];
                    if (cc.wt == 0.0f) continue;   // uniform across the warp
                    const float v = fmaf(fl, cc.dv, cc.v0);
                    const float tv = __fadd_rd(v, kMagic);
                    const float fv = v - (tv - kMagic);
                    const unsigned udr = (unsigned)(__float_as_int(tv) - tb);
                    const float val = cc.wt * x[cix];
                    if ((!fits || udr > (unsigned)(kFpWinRows - 2)) && val != 0.0f) {
                        const float a1 = fv * val, a0 = val - a1;
                        const int rr = r.v_box + base + (int)udr, c0 = r.u_box + uo + (cc.cw32 >> 5);
                        fp_tap(img, nu, nv, rr, c0, cc.gu * a0);
                        fp_tap(img, nu, nv, rr, c0 + 1, cc.fu * a0);
                        fp_tap(img, nu, nv, rr + 1, c0, cc.gu * a1);
                        fp_tap(img, nu, nv, rr + 1, c0 + 1, cc.fu * a1);
                    }
                }
            }
            __syncwarp();
            if (!fits) continue;   // uniform: nothing went to the windows

            // Flush: lane (g, cl) reads window it * G + g, column c0 + cl, and adds
            // its rows to the projection (windows overlap in rows; the global
            // reductions sum them).
            const int g = lane / cwid, cl = lane - g * cwid;
            // the window bases are monotone in the lane: the end lanes bound the rows
            const int bf = __shfl_sync(0xffffffffu, base, 0), bl31 = __shfl_sync(0xffffffffu, base, 31);
            const bool rows_in = r.v_box + min(bf, bl31) >= 0 && r.v_box + max(bf, bl31) + kFpWinRows - 1 < nv;
            const int nit = (32 + G - 1) / G;
            for (int c0 = 0; c0 < cols_used; c0 += cwid) {
                const int cidx = c0 + cl;
                const int gc = r.u_box + uo + cidx;
                const bool live = g < G && cidx < cols_used && gc >= 0 && gc < nu;
                const float *wcol = win + (live ? cidx : 0) * 32;
                const int cG = cidx * G;
                float *gcol = img + (live ? gc : 0);
                // all rows inside the detector (the common case): no row checks,
                // and zero cells are added too (cheaper than testing them)
                auto pass = [&](bool checked) {
                    for (int it = 0; it < nit; ++it) {
                        const int l = it * G + g;
                        const int bl = __shfl_sync(0xffffffffu, base, l & 31);
                        const bool lok = live && l < 32;
                        const int slot = (l + cG) & 31;
                        const float e0 = wcol[slot], e1 = wcol[rstride + slot], e2 = wcol[2 * rstride + slot];
                        const int row = r.v_box + bl;
                        float *d = gcol + (long long)row * nu;
                        if (!checked) {
                            if (lok) {
                                atomicAdd(d, e0);
                                atomicAdd(d + nu, e1);
                                atomicAdd(d + 2 * nu, e2);
                            }
                        } else {
                            if (lok && e0 != 0.0f && (unsigned)row < (unsigned)nv) atomicAdd(d, e0);
                            if (lok && e1 != 0.0f && (unsigned)(row + 1) < (unsigned)nv) atomicAdd(d + nu, e1);
                            if (lok && e2 != 0.0f && (unsigned)(row + 2) < (unsigned)nv) atomicAdd(d + 2 * nu, e2);
                        }
                    }
                };
                if (rows_in)
                    pass(false);
                else
                    pass(true);
            }
            __syncwarp();
            // clear the columns the scatter used, for the next view
            for (int dr = 0; dr < kFpWinRows; ++dr)
                for (int t = 4 * lane; t < cols_used * 32; t += 128)
                    *reinterpret_cast<float4 *>(win + dr * rstride + t) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

// Transpose of the per-voxel kernel for general matrices: direct global
// atomics (general matrices are the uncommon path).
__global__ void __launch_bounds__(256)
fp_voxel_gen(const float *__restrict__ vol, const double *__restrict__ P, int nviews, int nu,
             int nv, int nx, int ny, int nz, float scale, float *__restrict__ proj) {
    __shared__ ViewRecGen recs[64];
    const int tid = threadIdx.x;
    const int ntx = (nx + 7) / 8, nty = (ny + 7) / 8;
    const int t = blockIdx.x;
    const int i0 = (t % ntx) * 8, j0 = ((t / ntx) % nty) * 8, k0 = (t / (ntx * nty)) * 4;
    const int b = blockIdx.z;
    const int di = tid & 7, dj = (tid >> 3) & 7, dk = tid >> 6;
    const int i = i0 + di, j = j0 + dj, k = k0 + dk;
    const bool ok = i < nx && j < ny && k < nz;
    const float fdi = (float)di, fdj = (float)dj, fdk = (float)dk;
    const float xv = ok ? scale * vol[(((size_t)b * nz + k) * ny + j) * nx + i] : 0.0f;
    float *pb = proj + (size_t)b * nviews * nu * nv;
    for (int cb = 0; cb < nviews; cb += 64) {
        const int cn = min(64, nviews - cb);
        __syncthreads();
        for (int n = tid; n < cn; n += 256) make_rec_gen(P + 12 * (size_t)(cb + n), i0, j0, k0, &recs[n]);
        __syncthreads();
        if (!ok || xv == 0.0f) continue;
        for (int n = 0; n < cn; ++n) {
            const ViewRecGen r = recs[n];
            float W = fmaf(r.Wk, fdk, fmaf(r.Wj, fdj, fmaf(r.Wi, fdi, r.W0)));
            if (!(W > 0.0f)) continue;
            float inv = __frcp_rn(W);
            float u = fmaf(r.Nuk, fdk, fmaf(r.Nuj, fdj, fmaf(r.Nui, fdi, r.Nu0))) * inv;
            float v = fmaf(r.Nvk, fdk, fmaf(r.Nvj, fdj, fmaf(r.Nvi, fdi, r.Nv0))) * inv;
            if (!(fabsf(u) < 4e6f && fabsf(v) < 4e6f)) continue;
            float uf = floorf(u), vf = floorf(v);
            float fu = u - uf, fv = v - vf;
            int c0 = (int)uf + r.u_ref, r0 = (int)vf + r.v_ref;
            float val = inv * inv * xv;
            float a1 = fv * val, a0 = val - a1;
            float *img = pb + (size_t)(cb + n) * nu * nv;
            int rr[4] = {r0, r0, r0 + 1, r0 + 1}, cc[4] = {c0, c0 + 1, c0, c0 + 1};
            float ww[4] = {(1.0f - fu) * a0, fu * a0, (1.0f - fu) * a1, fu * a1};
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (rr[q] >= 0 && rr[q] < nv && cc[q] >= 0 && cc[q] < nu)
                    atomicAdd(img + (size_t)rr[q] * nu + cc[q], ww[q]);
        }
    }
}

bp_status launch_forward(bp_ctx *ctx, const float *vol, float *proj, int batch, float scale,
                         cudaStream_t st) {
    size_t bytes = sizeof(float) * (size_t)batch * ctx->n_views * ctx->nu * ctx->nv;
    cudaError_t e = cudaMemsetAsync(proj, 0, bytes, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fp_project: clear");
    if (!ctx->zinv || ctx->plan.bu <= 0 || ctx->plan.fp_wbu <= 0) {
        // general matrices, or patches too wide for the windows
        dim3 grid(((ctx->nx + 7) / 8) * ((ctx->ny + 7) / 8) * ((ctx->nz + 3) / 4), 1, batch);
        fp_voxel_gen<<<grid, 256, 0, st>>>(vol, ctx->d_P, ctx->n_views, ctx->nu, ctx->nv, ctx->nx,
                                           ctx->ny, ctx->nz, scale, proj);
        e = cudaGetLastError();
        return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "fp_voxel_gen launch");
    }
    // FP tiles are 32 x 8 x 32, the same shape the plan's TK=32 box covers;
    // with TK=64 plans the box is at least as large, so it still covers.
    const int bu = ctx->plan.bu, bv = ctx->plan.bv, wc = ctx->plan.fp_wbu;
    const int smem = fp_smem_bytes(wc);
    e = cudaFuncSetAttribute(fp_zcol<kFpTK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fp_zcol attribute");
    dim3 grid(((ctx->nx + kFpTX - 1) / kFpTX) * ((ctx->ny + kFpTY - 1) / kFpTY),
              (ctx->nz + kFpTK - 1) / kFpTK, batch);
    fp_zcol<kFpTK><<<grid, kFpThreads, smem, st>>>(vol, ctx->d_P, ctx->n_views, ctx->nu, ctx->nv,
                                                  ctx->nx, ctx->ny, ctx->nz, bu, bv, wc, scale, proj,
                                                  ctx->d_err);
    e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "fp_zcol launch");
}

}  // namespace bp
