// Matched voxel-driven forward projector: the exact transpose of the
// back-projection of Listing 1. Every voxel value, times scale / w^2, is
// scattered to the same four detector taps with the same bilinear weights
// the back-projector reads them with. A CTA owns a 32 x 8 x TK tile of
// voxels; each warp owns an 8 x 4 patch of its columns, one lane per voxel
// of a column, the patch's values held in registers. Per view a warp
// accumulates its patch's detector footprint in a private shared-memory box
// and then adds the box to the projection with one global reduction per
// touched pixel. Records (geometry relative to the box origin) are the ones
// the back-projector uses, so the taps coincide.
#include "geom_dev.cuh"

namespace bp {

constexpr int kFpTX = 32, kFpTY = 8, kFpTK = 32;

// Shared-memory reduction without a return value (red.shared.add.f32): the
// plain atomicAdd on a float in shared memory can come out as a
// compare-and-swap loop.
__device__ __forceinline__ void red_add_shared(float *p, float v) {
    asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(smem_addr(p)), "f"(v) : "memory");
}
constexpr int kFpThreads = kFpTX * kFpTY;

// Per (column, view) quantities shared by the 32 lanes that scatter the
// column's voxels (computed once per view by the thread owning the column).
struct __align__(16) FpCol {
    float v0, dv, wt, fu;
    int cu, ok, pad0, pad1;
};

template <int TK>
__global__ void __launch_bounds__(kFpThreads)
fp_zcol(const float *__restrict__ vol, const double *__restrict__ P, int nviews, int nu, int nv,
        int nx, int ny, int nz, int bu, int bv, int wbu, int wbv, float scale,
        float *__restrict__ proj, unsigned *err) {
    static_assert(TK == 32, "one lane per voxel of a 32-voxel column chunk");
    extern __shared__ __align__(16) unsigned char smem[];
    ViewRec *recs = reinterpret_cast<ViewRec *>(smem);
    FpCol *cols = reinterpret_cast<FpCol *>(smem + kRecChunk * sizeof(ViewRec));
    // one private box per warp, odd row pitch: the lanes of a column walk
    // down the rows at one column, which an odd pitch spreads over the banks
    const int wpitch = wbu | 1;
    const int wbox_n = wpitch * wbv;
    float *wbox = reinterpret_cast<float *>(smem + kRecChunk * sizeof(ViewRec) + kFpThreads * sizeof(FpCol)) +
                  (threadIdx.x >> 5) * wbox_n;

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

    // Scatter mapping: warp w handles the 32 columns of its patch one at a
    // time; lane l holds voxel k0 + l of each of them. The v step per voxel
    // is at least one pixel (checked per column), so within one scatter
    // instruction the lanes of a column write 32 different rows of the
    // warp's own box: plain read-add-write, no atomics.
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
    for (int t = lane; t < wbox_n; t += 32) wbox[t] = 0.0f;   // the flush keeps it clean from here on

    for (int cb = 0; cb < nviews; cb += kRecChunk) {
        const int cn = min(kRecChunk, nviews - cb);
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
            c.ok = 0;
            c.pad0 = c.pad1 = 0;
            float umin = 3e38f, umax = -3e38f, vmin = 3e38f, vmax = -3e38f;
            if (col_ok) {
                float W = fmaf(r.Wj, fdj, fmaf(r.Wi, fdi, r.W0));
                float inv = col_rcp(W);
                float uL = fmaf(r.Nuj, fdj, fmaf(r.Nui, fdi, r.Nu0)) * inv;
                c.v0 = fmaf(r.Nvj, fdj, fmaf(r.Nvi, fdi, r.Nv0)) * inv;
                c.dv = r.Nvk * inv;
                c.wt = inv * inv;
                float tu = __fadd_rd(uL, kMagic);
                c.cu = __float_as_int(tu) - kMagicBits;
                c.fu = uL - (tu - kMagic);
                float vlast = fmaf((float)(ez - 1), c.dv, c.v0);
                if (uL == uL && c.v0 == c.v0) {
                    c.ok = 1;
                    umin = umax = uL;
                    vmin = fminf(c.v0, vlast);
                    vmax = fmaxf(c.v0, vlast);
                }
            }
            // the warp's box: floor of the smallest column / row its lanes touch
            for (int o = 16; o > 0; o >>= 1) {
                umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
                umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
                vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
                vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
            }
            const bool any = umin <= umax;
            const int uo = any ? __float_as_int(__fadd_rd(umin, kMagic)) - kMagicBits : 0;
            const int vo = any ? __float_as_int(__fadd_rd(vmin, kMagic)) - kMagicBits : 0;
            const bool fits = any && (__float_as_int(__fadd_rd(umax, kMagic)) - kMagicBits) + 1 - uo <= wbu - 1 &&
                              (__float_as_int(__fadd_rd(vmax, kMagic)) - kMagicBits) + 1 - vo <= wbv - 1;
            if (any && !fits && lane == 0) atomicOr(err, DEV_ERR_FOOTPRINT);
            if (c.ok) c.cu -= uo;   // column relative to the warp box
            // At least one detector row per voxel in every column: the lanes of a
            // column then write different rows, so plain read-add-writes are safe;
            // otherwise the warp adds with shared-memory reductions for this view.
            const bool rmw = __all_sync(0xffffffffu, !c.ok || fabsf(c.dv) >= 1.0f);
            cols[tid] = c;
            __syncwarp();
            if (any && fits) {
                const float fl = (float)lane;
                // Lane l adds voxel k0 + l of each column to rows r, r + 1 and
                // columns cu, cu + 1. With the read-add-write form, the two taps
                // of one row go together (no other lane touches that row), and a
                // warp barrier separates them from the next row's taps (lane
                // l + 1's top row can be lane l's bottom row) and from the next
                // column.
                auto scatter = [&](const FpCol &cc, float xv, bool plain) {
                    float v = fmaf(fl, cc.dv, cc.v0);
                    float tv = __fadd_rd(v, kMagic);
                    float fv = v - (tv - kMagic);
                    int row = __float_as_int(tv) - kMagicBits - vo;
                    float val = cc.wt * xv;
                    float a1 = fv * val, a0 = val - a1;   // (1-fv) val, fv val
                    const bool act = lane < ez;
                    float *p = wbox + row * wpitch + cc.cu;
                    const float gu = 1.0f - cc.fu;
                    if (plain) {
                        if (act) {
                            p[0] += gu * a0;
                            p[1] += cc.fu * a0;
                        }
                        __syncwarp();
                        if (act) {
                            p[wpitch] += gu * a1;
                            p[wpitch + 1] += cc.fu * a1;
                        }
                        __syncwarp();
                    } else if (act) {
                        red_add_shared(p, gu * a0);
                        red_add_shared(p + 1, cc.fu * a0);
                        red_add_shared(p + wpitch, gu * a1);
                        red_add_shared(p + wpitch + 1, cc.fu * a1);
                    }
                };
                if (rmw) {
#pragma unroll
                    for (int cix = 0; cix < 32; ++cix) {
                        const FpCol cc = cols[warp * 32 + cix];
                        if (cc.ok) scatter(cc, x[cix], true);   // uniform across the warp
                    }
                } else {
#pragma unroll
                    for (int cix = 0; cix < 32; ++cix) {
                        const FpCol cc = cols[warp * 32 + cix];
                        if (cc.ok) scatter(cc, x[cix], false);
                    }
                    __syncwarp();
                }
                // flush the warp's box into the projection (inside the detector only)
                float *img = pb + (size_t)(cb + n) * nu * nv;
                const int rows_used = min(wbv, (__float_as_int(__fadd_rd(vmax, kMagic)) - kMagicBits) + 2 - vo);
                const int cols_used = min(wbu, (__float_as_int(__fadd_rd(umax, kMagic)) - kMagicBits) + 2 - uo);
                // Lanes take g rows of cw columns at a time (cw = the used width, at
                // most 32; G = 32 / cw rows per pass), so narrow boxes keep most lanes
                // busy. Every value read is zeroed again, so the box is clean for the
                // next view (the scatter writes only inside this region).
                const int cw = min(cols_used, 32);
                const int G = 32 / cw;
                const int g = lane / cw, cl = lane - g * cw;
                for (int c0 = 0; c0 < cols_used; c0 += cw) {
                    const int ccol = c0 + cl;
                    const int c_ = r.u_box + uo + ccol;
                    const bool cok = g < G && ccol < cols_used;
                    const bool cin = cok && c_ >= 0 && c_ < nu;
                    float *cell = wbox + g * wpitch + ccol;
                    int r_ = r.v_box + vo + g;
                    for (int rr = g; rr < rows_used; rr += G) {
                        if (cok) {
                            const float val = *cell;
                            *cell = 0.0f;
                            if (cin && val != 0.0f && r_ >= 0 && r_ < nv) atomicAdd(img + (size_t)r_ * nu + c_, val);
                        }
                        cell += G * wpitch;
                        r_ += G;
                    }
                }
            }
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
        // general matrices, or a footprint too large for the shared box
        dim3 grid(((ctx->nx + 7) / 8) * ((ctx->ny + 7) / 8) * ((ctx->nz + 3) / 4), 1, batch);
        fp_voxel_gen<<<grid, 256, 0, st>>>(vol, ctx->d_P, ctx->n_views, ctx->nu, ctx->nv, ctx->nx,
                                           ctx->ny, ctx->nz, scale, proj);
        e = cudaGetLastError();
        return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "fp_voxel_gen launch");
    }
    // FP tiles are 32 x 8 x 32, the same shape the plan's TK=32 box covers;
    // with TK=64 plans the box is at least as large, so it still covers.
    const int bu = ctx->plan.bu, bv = ctx->plan.bv;
    const int wbu = ctx->plan.fp_wbu, wbv = ctx->plan.fp_wbv;
    const int smem = kRecChunk * (int)sizeof(ViewRec) + kFpThreads * (int)sizeof(FpCol) +
                     (kFpThreads / 32) * (wbu | 1) * wbv * (int)sizeof(float);
    e = cudaFuncSetAttribute(fp_zcol<kFpTK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fp_zcol attribute");
    dim3 grid(((ctx->nx + kFpTX - 1) / kFpTX) * ((ctx->ny + kFpTY - 1) / kFpTY),
              (ctx->nz + kFpTK - 1) / kFpTK, batch);
    fp_zcol<kFpTK><<<grid, kFpThreads, smem, st>>>(vol, ctx->d_P, ctx->n_views, ctx->nu, ctx->nv,
                                                  ctx->nx, ctx->ny, ctx->nz, bu, bv, wbu, wbv, scale,
                                                  proj, ctx->d_err);
    e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "fp_zcol launch");
}

}  // namespace bp
