// Matched voxel-driven forward projector: the exact transpose of the
// back-projection of Listing 1. Every voxel value, times scale / w^2, is
// scattered to the same four detector taps with the same bilinear weights
// the back-projector reads them with. A CTA owns a 32 x 8 x TK tile of
// voxels (one thread per z-column, the tile's values held in registers);
// per view it accumulates the tile's detector footprint in a shared-memory
// box with shared atomics and then adds the box to the projection with one
// global atomic per touched pixel. Records (geometry relative to the box
// origin) are the ones the back-projector uses, so the taps coincide.
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
struct FpCol {
    float v0, dv, wt, fu;
    int cu, ok;
};

template <int TK>
__global__ void __launch_bounds__(kFpThreads)
fp_zcol(const float *__restrict__ vol, const double *__restrict__ P, int nviews, int nu, int nv,
        int nx, int ny, int nz, int bu, int bv, float scale, float *__restrict__ proj,
        unsigned *err) {
    static_assert(TK == 32, "one lane per voxel of a 32-voxel column chunk");
    extern __shared__ __align__(16) unsigned char smem[];
    ViewRec *recs = reinterpret_cast<ViewRec *>(smem);
    FpCol *cols = reinterpret_cast<FpCol *>(smem + kRecChunk * sizeof(ViewRec));
    float *box = reinterpret_cast<float *>(smem + kRecChunk * sizeof(ViewRec) + kFpThreads * sizeof(FpCol));
    // odd row pitch: the 32 lanes of a column walk down ~32-64 rows at one
    // column, which an odd pitch spreads over all 32 banks
    const int pitch = bu | 1;
    const int nbox = pitch * bv;

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

    // Scatter mapping: warp w handles the 32 columns of the same patch, one
    // at a time; lane l holds voxel k0 + l of each of them. Within one
    // scatter instruction the lanes of a column then hit 32 different
    // detector rows (the v step per voxel is >= 1 pixel here), so the
    // shared-memory adds do not contend inside the warp.
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
            __syncthreads();   // previous flush done (and records ready)
            for (int t = tid; t < nbox; t += kFpThreads) box[t] = 0.0f;
            const ViewRec r = recs[n];
            {
                FpCol c;
                c.ok = 0;
                if (col_ok) {
                    float W = fmaf(r.Wj, fdj, fmaf(r.Wi, fdi, r.W0));
                    float inv = __frcp_rn(W);
                    float uL = fmaf(r.Nuj, fdj, fmaf(r.Nui, fdi, r.Nu0)) * inv;
                    c.v0 = fmaf(r.Nvj, fdj, fmaf(r.Nvi, fdi, r.Nv0)) * inv;
                    c.dv = r.Nvk * inv;
                    c.wt = inv * inv;
                    float tu = __fadd_rd(uL, kMagic);
                    c.cu = __float_as_int(tu) - kMagicBits;
                    c.fu = uL - (tu - kMagic);
                    float vlast = fmaf((float)(ez - 1), c.dv, c.v0);
                    int rfirst = __float_as_int(__fadd_rd(c.v0, kMagic)) - kMagicBits;
                    int rlast = __float_as_int(__fadd_rd(vlast, kMagic)) - kMagicBits;
                    if (c.cu < 0 || c.cu > bu - 2 || min(rfirst, rlast) < 0 ||
                        max(rfirst, rlast) > bv - 2 || !(uL == uL))
                        atomicOr(err, DEV_ERR_FOOTPRINT);
                    else
                        c.ok = 1;
                }
                cols[tid] = c;
            }
            __syncthreads();
            const float fl = (float)lane;
#pragma unroll
            for (int c = 0; c < 32; ++c) {
                const FpCol cc = cols[warp * 32 + ((c >> 3) << 3) + (c & 7)];
                if (!cc.ok) continue;   // uniform across the warp
                float v = fmaf(fl, cc.dv, cc.v0);
                float tv = __fadd_rd(v, kMagic);
                float fv = v - (tv - kMagic);
                int row = __float_as_int(tv) - kMagicBits;
                float val = cc.wt * x[c];
                float a1 = fv * val, a0 = val - a1;   // (1-fv) val, fv val
                if (lane < ez && val != 0.0f) {
                    float *p = box + row * pitch + cc.cu;
                    const float gu = 1.0f - cc.fu;
                    red_add_shared(p, gu * a0);
                    red_add_shared(p + 1, cc.fu * a0);
                    red_add_shared(p + pitch, gu * a1);
                    red_add_shared(p + pitch + 1, cc.fu * a1);
                }
            }
            __syncthreads();
            // flush the box into the projection (pixels inside the detector only)
            float *img = pb + (size_t)(cb + n) * nu * nv;
            for (int t = tid; t < bu * bv; t += kFpThreads) {
                int rr = t / bu, cc = t - rr * bu;
                int r_ = r.v_box + rr, c_ = r.u_box + cc;
                float val = box[rr * pitch + cc];
                if (val != 0.0f && r_ >= 0 && r_ < nv && c_ >= 0 && c_ < nu)
                    atomicAdd(img + (size_t)r_ * nu + c_, val);
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
    if (!ctx->zinv || ctx->plan.bu <= 0) {
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
    const int smem = kRecChunk * (int)sizeof(ViewRec) + kFpThreads * (int)sizeof(FpCol) +
                     (bu | 1) * bv * (int)sizeof(float);
    e = cudaFuncSetAttribute(fp_zcol<kFpTK>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "fp_zcol attribute");
    dim3 grid(((ctx->nx + kFpTX - 1) / kFpTX) * ((ctx->ny + kFpTY - 1) / kFpTY),
              (ctx->nz + kFpTK - 1) / kFpTK, batch);
    fp_zcol<kFpTK><<<grid, kFpThreads, smem, st>>>(vol, ctx->d_P, ctx->n_views, ctx->nu, ctx->nv,
                                                  ctx->nx, ctx->ny, ctx->nz, bu, bv, scale, proj,
                                                  ctx->d_err);
    e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "fp_zcol launch");
}

}  // namespace bp
