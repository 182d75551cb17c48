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
//
// Window layout (one warp): row plane dr (0..2) of kPlane words, then
// column c at a pitch of 33 words, then lane l at slot (l * cw) mod 32, cw
// the odd flush width of the view. Word dr * kPlane + 33 c + ((l cw) & 31)
// is distinct for every (dr, c, l) and sits in bank (c + l cw) mod 32:
//   - a scatter (one column, 32 lanes) touches 32 banks, since cw is odd;
//   - the flush reads cell l * cw + c of a row plane with lane (l cw + c)
//     mod 32, so 32 consecutive cells are 32 banks, and consecutive lanes
//     add consecutive detector columns (coalesced reductions);
//   - a voxel's four taps are one address plus immediate offsets (+33 for
//     the next column, +kPlane for the next row).
#include "geom_dev.cuh"

namespace bp {

constexpr int kFpTX = 32, kFpTY = 8, kFpTK = 32;
constexpr int kFpThreads = kFpTX * kFpTY;
constexpr int kFpWinRows = 3;     // detector rows of a lane's window
constexpr int kFpRecChunk = 32;   // view records staged per pass
constexpr int kFpColPitch = 33;   // words between window columns

template <int WC>
struct FpWin {
    static_assert(WC % 2 == 1, "odd window widths: any used width rounds up to an odd flush width");
    static constexpr int kPlane = (WC * kFpColPitch + 31) / 32 * 32;   // a multiple of 32 words
    static constexpr int kWarpWords = kFpWinRows * kPlane;
};

// Per (column pair, view) quantities of the two columns 2p, 2p+1 of a warp's
// patch, written by the threads owning the columns and read by every lane.
struct __align__(16) FpPair {
    float2 v0, dv;   // v of the first voxel and per voxel (box-relative)
    float2 wgu, wfu; // column weights (1 - fu) / W^2 and fu / W^2 (0: a column without voxels)
};
// beside it, per pair: the window columns times 33 (int2)

// Window widths the kernel is built for (odd; the plan takes the smallest
// that holds the widest u footprint of a patch).
constexpr int kFpWidths[] = {17, 21, 25, 33, 49};

int fp_window_width(int need) {
    for (int w : kFpWidths)
        if (need <= w) return w;
    return -1;
}

static int fp_plane_words(int wc) { return (wc * kFpColPitch + 31) / 32 * 32; }

int fp_smem_bytes(int wc) {
    return kFpRecChunk * (int)sizeof(ViewRec) + (kFpThreads / 32) * 16 * (int)(sizeof(FpPair) + sizeof(int2)) +
           (kFpThreads / 32) * kFpWinRows * fp_plane_words(wc) * (int)sizeof(float);
}

__device__ __forceinline__ void fp_tap(float *img, int nu, int nv, int row, int col, float a) {
    if (a != 0.0f && (unsigned)row < (unsigned)nv && (unsigned)col < (unsigned)nu)
        atomicAdd(img + (size_t)row * nu + col, a);
}

__device__ __forceinline__ int floor_bits(float v) { return __float_as_int(__fadd_rd(v, kMagic)); }

// Order-preserving map of a float to a signed int, so warp min / max run as
// one integer reduction (redux.sync).
__device__ __forceinline__ int fkey(float f) {
    const int b = __float_as_int(f);
    return b >= 0 ? b : b ^ 0x7fffffff;
}
__device__ __forceinline__ float fkey_inv(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }
__device__ __forceinline__ float warp_fmin(float f) { return fkey_inv(__reduce_min_sync(0xffffffffu, fkey(f))); }
__device__ __forceinline__ float warp_fmax(float f) { return fkey_inv(__reduce_max_sync(0xffffffffu, fkey(f))); }

// Flush: each row plane of a warp's windows holds 32 windows x cw columns;
// lane t takes cells it * 32 + t (window l = cell / cw, column c = cell mod
// cw) and adds rows b_l, b_l + 1 and b_l + 2 of detector column ucol0 + c to
// the projection. Consecutive lanes hold consecutive columns of a window,
// so the reductions coalesce; the windows overlap in rows, and the global
// reductions sum them.
template <int kPlane>
__device__ __forceinline__ void fp_flush(const float *win, float *img, int nu, int nv, int cw, int cols_used,
                                         int base, int vbox, int ucol0, int lane) {
    // the window bases are monotone in the lane: the end lanes bound the rows
    const int bf = __shfl_sync(0xffffffffu, base, 0), bl = __shfl_sync(0xffffffffu, base, 31);
    const bool rows_in = vbox + min(bf, bl) >= 0 && vbox + max(bf, bl) + kFpWinRows - 1 < nv;
    // l = lane / cw and c = lane mod cw, and the step of 32 cells as q windows
    // plus rem columns: exact, since a quotient below 33 that is not an
    // integer lies at least 1 / cw from the next one, far beyond the rounding
    const float rcw = __frcp_rn((float)cw);
    int l = __float2int_rz(fmaf((float)lane, rcw, 0.01f));
    int c = lane - l * cw;
    const int q = __float2int_rz(fmaf(32.0f, rcw, 0.01f));
    const int rem = 32 - q * cw;
    for (int it = 0; it < cw; ++it) {
        const int rowb = __shfl_sync(0xffffffffu, base, l & 31);
        const int word = c * kFpColPitch + ((l * cw) & 31);
        const float e0 = win[word], e1 = win[word + kPlane], e2 = win[word + 2 * kPlane];
        const int gc = ucol0 + c, row = vbox + rowb;
        const bool live = c < cols_used && (unsigned)gc < (unsigned)nu;
        float *d = img + ((long long)row * nu + gc);
        if (rows_in) {
            // all rows inside the detector (the common case): no row checks,
            // and zero cells are added too (cheaper than testing them)
            if (live) {
                atomicAdd(d, e0);
                atomicAdd(d + nu, e1);
                atomicAdd(d + 2 * nu, e2);
            }
        } else if (live) {
            if (e0 != 0.0f && (unsigned)row < (unsigned)nv) atomicAdd(d, e0);
            if (e1 != 0.0f && (unsigned)(row + 1) < (unsigned)nv) atomicAdd(d + nu, e1);
            if (e2 != 0.0f && (unsigned)(row + 2) < (unsigned)nv) atomicAdd(d + 2 * nu, e2);
        }
        c += rem;
        l += q;
        if (c >= cw) {
            c -= cw;
            ++l;
        }
    }
}

// The taps of lane l's voxel in columns 2p and 2p+1 of the warp's patch:
// v, its floor and fraction for both columns as f32x2 pairs (each lane of a
// pair computed exactly as the scalar back-projector does), then the value
// times scale / W^2 split between rows floor(v) and floor(v) + 1.
// The weights are the back-projector's: (1 - fu) / W^2 and fu / W^2 on the
// two columns (from the record), 1 - fv and fv on the two rows. No packed
// subtraction (each costs integer sign flips): fv = fma(floor(v), -1, v),
// and the row shares as a1 = fv x, a0 = fma(a1, -1, x).
struct FpTaps {
    float2 fu, gu, a0, a1;   // wfu, wgu (column weights), (1 - fv) x, fv x
    int ra, rb;              // window rows floor(v) - lane base (columns 2p, 2p+1)
};

__device__ __forceinline__ FpTaps fp_taps(const FpPair &pr, float2 x, float2 fl2, int tb) {
    const float2 M2 = make_float2(kMagic, kMagic), NM2 = make_float2(-kMagic, -kMagic);
    const float2 N1 = make_float2(-1.0f, -1.0f);
    const float2 V = __ffma2_rn(fl2, pr.dv, pr.v0);
    const float2 TV = __fadd2_rd(V, M2);
    const float2 FV = __ffma2_rn(__fadd2_rn(TV, NM2), N1, V);   // v - floor(v), exact
    FpTaps t;
    t.a1 = __fmul2_rn(FV, x);
    t.a0 = __ffma2_rn(t.a1, N1, x);
    t.fu = pr.wfu;
    t.gu = pr.wgu;
    t.ra = __float_as_int(TV.x) - tb;
    t.rb = __float_as_int(TV.y) - tb;
    return t;
}

// Read-add-write of one voxel's four taps at window word w (rows drc and
// drc + 1, columns cwin and cwin + 1).
template <int kPlane>
__device__ __forceinline__ void fp_add4(float *w, float gu, float fu, float a0, float a1) {
    w[0] = fmaf(gu, a0, w[0]);
    w[kFpColPitch] = fmaf(fu, a0, w[kFpColPitch]);
    w[kPlane] = fmaf(gu, a1, w[kPlane]);
    w[kPlane + kFpColPitch] = fmaf(fu, a1, w[kPlane + kFpColPitch]);
}

// Taps straight to the projection (global reductions): every tap of the
// voxel when `all`, else only a voxel whose rows lie beyond its window.
__device__ __forceinline__ void fp_direct(float *img, int nu, int nv, int row0, int col0, float gu, float fu,
                                          float a0, float a1, int dr, bool all) {
    if (all || (unsigned)dr > (unsigned)(kFpWinRows - 2)) {
        const int rr = row0 + dr;
        fp_tap(img, nu, nv, rr, col0, gu * a0);
        fp_tap(img, nu, nv, rr, col0 + 1, fu * a0);
        fp_tap(img, nu, nv, rr + 1, col0, gu * a1);
        fp_tap(img, nu, nv, rr + 1, col0 + 1, fu * a1);
    }
}

template <int WC>
__global__ void __launch_bounds__(kFpThreads, 3)
fp_zwin(const float *__restrict__ vol, const double *__restrict__ P, int nviews, int nu, int nv,
        int nx, int ny, int nz, int bu, int bv, float scale, float *__restrict__ proj, unsigned *err) {
    constexpr int kPlane = FpWin<WC>::kPlane;
    constexpr int kWarpWords = FpWin<WC>::kWarpWords;
    extern __shared__ __align__(16) unsigned char smem[];
    ViewRec *recs = reinterpret_cast<ViewRec *>(smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    FpPair *pairs = reinterpret_cast<FpPair *>(smem + kFpRecChunk * sizeof(ViewRec)) + warp * 16;
    int2 *pcw = reinterpret_cast<int2 *>(smem + kFpRecChunk * sizeof(ViewRec) + (kFpThreads / 32) * 16 * sizeof(FpPair)) +
                warp * 16;
    float *win = reinterpret_cast<float *>(smem + kFpRecChunk * sizeof(ViewRec) +
                                           (kFpThreads / 32) * 16 * (sizeof(FpPair) + sizeof(int2))) +
                 warp * kWarpWords;

    const int ntx = (nx + kFpTX - 1) / kFpTX;
    const int i0 = (blockIdx.x % ntx) * kFpTX, j0 = (blockIdx.x / ntx) * kFpTY;
    const int k0 = blockIdx.y * kFpTK;
    const int b = blockIdx.z;
    const int ex = min(kFpTX, nx - i0), ey = min(kFpTY, ny - j0), ez = min(kFpTK, nz - k0);
    // column owned by this thread for the per-view setup (8 x 4 patch per warp)
    const int wx = warp % (kFpTX / 8), wy = warp / (kFpTX / 8);
    const int di = wx * 8 + (lane & 7), dj = wy * 4 + (lane >> 3);
    const bool col_ok = di < ex && dj < ey;
    const float fdi = (float)di, fdj = (float)dj;

    // lane l holds voxel k0 + l of columns 2p and 2p + 1 in x2[p]
    float2 x2[16];
    {
        const size_t plane = (size_t)nx * ny;
        const bool kin = lane < ez;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            const int cdi = wx * 8 + (c & 7), cdj = wy * 4 + (c >> 3);
            const bool ok = kin && cdi < ex && cdj < ey;
            const float xv = ok ? scale * vol[((size_t)b * nz + k0 + lane) * plane + (size_t)(j0 + cdj) * nx + (i0 + cdi)]
                                : 0.0f;
            if (c & 1) x2[c >> 1].y = xv;
            else x2[c >> 1].x = xv;
        }
    }
    float *pb = proj + (size_t)b * nviews * nu * nv;
    for (int t = 4 * lane; t < kWarpWords; t += 128) *reinterpret_cast<float4 *>(win + t) = make_float4(0.f, 0.f, 0.f, 0.f);
    const float fl = (float)lane;
    const float2 fl2 = make_float2(fl, fl);
    float *pf = reinterpret_cast<float *>(pairs) + (lane >> 1) * (int)(sizeof(FpPair) / 4) + (lane & 1);

    for (int cb = 0; cb < nviews; cb += kFpRecChunk) {
        const int cn = min(kFpRecChunk, nviews - cb);
        __syncthreads();   // every warp is done with the previous chunk's records
        for (int n = tid; n < cn; n += kFpThreads) {
            ViewRec r;
            if (!make_rec(P + 12 * (size_t)(cb + n), i0, j0, k0, ex, ey, ez, 4, bu, bv, &r))
                atomicOr(err, DEV_ERR_FOOTPRINT);
            recs[n] = r;
        }
        __syncthreads();
        for (int n = 0; n < cn; ++n) {
            const ViewRec r = recs[n];
            float uL = 0.0f, cv0 = 0.0f, cdv = 0.0f, cwt = 0.0f, cfu = 0.0f;
            int cu = 0;
            bool cok = false;
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
                    if (fabsf(cdv) < 1e4f && fabsf(cv0) < 1e6f && fabsf(uL) < 1e6f) cok = true;
                    else atomicOr(err, DEV_ERR_FOOTPRINT);
                }
            }
            const float umin = warp_fmin(cok ? uL : 3e38f), umax = warp_fmax(cok ? uL : -3e38f);
            if (!(umin <= umax)) continue;   // no column with voxels: uniform across the warp
            const float v0min = warp_fmin(cok ? cv0 : 3e38f), v0max = warp_fmax(cok ? cv0 : -3e38f);
            const float dvmin = warp_fmin(cok ? cdv : 3e38f), dvmax = warp_fmax(cok ? cdv : -3e38f);
            const int uo = floor_bits(umin) - kMagicBits;
            const int cols_used = floor_bits(umax) - kMagicBits + 2 - uo;
            // A column outside the patch or without a usable geometry adds zeros
            // at window row 0, column 0.
            const int cwin = cok ? cu - uo : 0;
            pf[0] = cok ? cv0 : v0min;
            pf[2] = cok ? cdv : dvmin;
            pf[4] = cok ? cwt * (1.0f - cfu) : 0.0f;
            pf[6] = cok ? cwt * cfu : 0.0f;
            reinterpret_cast<int *>(pcw)[lane] = cwin * kFpColPitch;
            __syncwarp();

            // Lane l's window starts at row floor(v0min + l * dvmin): every
            // column's row floor(v0 + l * dv) is at or above it and at or below
            // floor(v0max + l * dvmax) (v0min <= v0 <= v0max, dvmin <= dv <= dvmax,
            // l >= 0, and fmaf and the floor are monotone).
            const int tb = floor_bits(fmaf(fl, dvmin, v0min));
            const int base = tb - kMagicBits;
            float *img = pb + (size_t)(cb + n) * nu * nv;
            const int row0 = r.v_box + base, ucol0 = r.u_box + uo;
            const bool fits = cols_used <= WC;
            if (fits) {
                const int cw = cols_used | 1;   // odd flush width
                float *wl = win + ((lane * cw) & 31);
                const int th = floor_bits(fmaf(fl, dvmax, v0max));
                if (__all_sync(0xffffffffu, th - tb <= 1)) {
                    // every row of every lane is inside its window: no checks
#pragma unroll
                    for (int p = 0; p < 16; ++p) {
                        const FpPair pr = pairs[p];
                        const int2 cw2 = pcw[p];
                        const FpTaps t = fp_taps(pr, x2[p], fl2, tb);
                        fp_add4<kPlane>(wl + t.ra * kPlane + cw2.x, t.gu.x, t.fu.x, t.a0.x, t.a1.x);
                        fp_add4<kPlane>(wl + t.rb * kPlane + cw2.y, t.gu.y, t.fu.y, t.a0.y, t.a1.y);
                    }
                } else {
                    unsigned dmax = 0;
#pragma unroll
                    for (int p = 0; p < 16; ++p) {
                        const FpPair pr = pairs[p];
                        const int2 cw2 = pcw[p];
                        FpTaps t = fp_taps(pr, x2[p], fl2, tb);
                        dmax = max(dmax, max((unsigned)t.ra, (unsigned)t.rb));
                        const bool ina = (unsigned)t.ra <= (unsigned)(kFpWinRows - 2);
                        const bool inb = (unsigned)t.rb <= (unsigned)(kFpWinRows - 2);
                        // beyond the window: zeros here, the pass below adds them
                        fp_add4<kPlane>(wl + (ina ? t.ra : 0) * kPlane + cw2.x, t.gu.x, t.fu.x,
                                        ina ? t.a0.x : 0.0f, ina ? t.a1.x : 0.0f);
                        fp_add4<kPlane>(wl + (inb ? t.rb : 0) * kPlane + cw2.y, t.gu.y, t.fu.y,
                                        inb ? t.a0.y : 0.0f, inb ? t.a1.y : 0.0f);
                    }
                    if (__any_sync(0xffffffffu, lane < ez && dmax > (unsigned)(kFpWinRows - 2))) {
#pragma unroll
                        for (int p = 0; p < 16; ++p) {
                            const FpPair pr = pairs[p];
                            const int2 cw2 = pcw[p];
                            const FpTaps t = fp_taps(pr, x2[p], fl2, tb);
                            fp_direct(img, nu, nv, row0, ucol0 + cw2.x / kFpColPitch, t.gu.x, t.fu.x, t.a0.x, t.a1.x, t.ra, false);
                            fp_direct(img, nu, nv, row0, ucol0 + cw2.y / kFpColPitch, t.gu.y, t.fu.y, t.a0.y, t.a1.y, t.rb, false);
                        }
                    }
                }
                __syncwarp();
                fp_flush<kPlane>(win, img, nu, nv, cw, cols_used, base, row0 - base, ucol0, lane);
                __syncwarp();
                // clear the cells the scatter used, for the next view
                const int used = (cw * kFpColPitch + 3) & ~3;
#pragma unroll
                for (int dr = 0; dr < kFpWinRows; ++dr)
                    for (int t = 4 * lane; t < used; t += 128)
                        *reinterpret_cast<float4 *>(win + dr * kPlane + t) = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                // a patch wider than the planned windows (not expected from the
                // plan's footprint bound): every tap straight to the projection
#pragma unroll
                for (int p = 0; p < 16; ++p) {
                    const FpPair pr = pairs[p];
                    const int2 cw2 = pcw[p];
                    const FpTaps t = fp_taps(pr, x2[p], fl2, tb);
                    fp_direct(img, nu, nv, row0, ucol0 + cw2.x / kFpColPitch, t.gu.x, t.fu.x, t.a0.x, t.a1.x, t.ra, true);
                    fp_direct(img, nu, nv, row0, ucol0 + cw2.y / kFpColPitch, t.gu.y, t.fu.y, t.a0.y, t.a1.y, t.rb, true);
                }
            }
            __syncwarp();   // the pair records are rewritten for the next view
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
    dim3 grid(((ctx->nx + kFpTX - 1) / kFpTX) * ((ctx->ny + kFpTY - 1) / kFpTY),
              (ctx->nz + kFpTK - 1) / kFpTK, batch);
    auto run = [&](auto kern) -> cudaError_t {
        cudaError_t e2 = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e2 != cudaSuccess) return e2;
        kern<<<grid, kFpThreads, smem, st>>>(vol, ctx->d_P, ctx->n_views, ctx->nu, ctx->nv, ctx->nx, ctx->ny,
                                            ctx->nz, bu, bv, scale, proj, ctx->d_err);
        return cudaGetLastError();
    };
    switch (wc) {
    case 17: e = run(fp_zwin<17>); break;
    case 21: e = run(fp_zwin<21>); break;
    case 25: e = run(fp_zwin<25>); break;
    case 33: e = run(fp_zwin<33>); break;
    case 49: e = run(fp_zwin<49>); break;
    default: return fail(ctx, BP_ERR_UNSUPPORTED, "fp_project: no window width for this plan");
    }
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "fp_zwin launch");
}

}  // namespace bp
