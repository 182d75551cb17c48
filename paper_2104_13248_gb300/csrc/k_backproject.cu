// Voxel-driven cone-beam back-projection kernels (Listing 1 of Chen et al.,
// ICS '21, with the z-column hoisting of Section 3.1.2 / Algorithm 1 and the
// view-batched staging of Section 3.1.3 / Algorithm 2, redesigned for
// sm_103a):
//
//   bp_zcol_tma   one thread per z-column (i, j) owning TK voxels in
//                 registers; u, w and the u-fraction are computed once per
//                 (column, view); v is stepped linearly in k. A producer
//                 warp stages each view's detector footprint of the CTA tile
//                 into shared memory with a 4-D TMA load (zero fill outside
//                 the detector = the zero-padded sampling), STAGES views in
//                 flight on mbarriers. Software FP32 bilinear sampling,
//                 FP32 accumulation, each voxel written once.
//   bp_zcol_ldg   the same arithmetic with direct global gathers, for
//                 layouts TMA cannot describe (row pitch not a multiple of
//                 16 bytes, misaligned pointers).
//   bp_voxel_gen  one thread per voxel for general matrices (u, w depending
//                 on k).
#include "geom_dev.cuh"

#include <algorithm>
#include <cstdio>

namespace bp {

constexpr int kTX = 32;      // tile columns along x (4 warps x 8)
constexpr int kTY = 8;       // tile columns along y (2 warps x 4)
constexpr int kMaxStages = 8;   // barrier slots; the views in flight (plan.stages) are <= this
constexpr int kConsumers = kTX * kTY;
constexpr int kConsumerWarps = kConsumers / 32;
constexpr int kThreads = kConsumers + 32;   // + producer warp

__host__ __device__ constexpr int align_up(int x, int a) { return (x + a - 1) / a * a; }

template <typename T>
__host__ __device__ constexpr int stage_bytes(int bu, int bv) {
    return align_up(bu * bv * (int)sizeof(T), 128);
}

constexpr int kRecBytes = kRecChunk * (int)sizeof(ViewRec);
constexpr int kBarOffset = kRecBytes;
constexpr int kStageOffset = align_up(kRecBytes + 2 * kMaxStages * 8, 128);

// Thread -> column within the CTA tile: each warp owns an 8 x 4 patch.
__device__ __forceinline__ void consumer_column(int warp, int lane, int *di, int *dj) {
    int wx = warp % (kTX / 8), wy = warp / (kTX / 8);
    *di = wx * 8 + (lane & 7);
    *dj = wy * 4 + (lane >> 3);
}

// Packed FP32 pair arithmetic (sm_100-family f32x2 instructions): each
// operates on two independent FP32 lanes with IEEE rounding per lane, so a
// pair of voxels costs one instruction where two scalar ones were needed.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ f2 add2_rd(f2 a, f2 b) {
    f2 r;
    asm("add.rm.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Shared-memory load at a 32-bit shared address plus a compile-time byte
// offset. The tap addresses are formed in 32-bit arithmetic (one IMAD per
// tap row): pointer arithmetic on the staged box went through 64-bit
// generic addresses, several integer instructions per tap row.
template <int OFF>
__device__ __forceinline__ float lds32(unsigned a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(OFF));
    return v;
}

__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
// Per (column, view) quantities of the z-column update: the 1/W^2 weight,
// the staged-box column cu and u fraction fu, v at the tile's first slice
// and its step per slice. Returns false (and flags the device error word)
// if the taps would leave the staged box.
struct ColView {
    float wt, fu, v0, dv;
    int cu;
};

template <int BU>
__device__ __forceinline__ bool column_view(const ViewRec &r, float fdi, float fdj, int ez, int bv,
                                            unsigned *err, ColView &c) {
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
    int rfirst = __float_as_int(__fadd_rd(c.v0, kMagic)) - kMagicBits;
    int rlast = __float_as_int(__fadd_rd(vlast, kMagic)) - kMagicBits;
    if (c.cu < 0 || c.cu > BU - 2 || min(rfirst, rlast) < 0 || max(rfirst, rlast) > bv - 2 ||
        !(uL == uL) || !(c.v0 == c.v0)) {
        atomicOr(err, DEV_ERR_FOOTPRINT);
        return false;
    }
    return true;
}

// Scalar update of acc[0..TK-1] (any element type; ragged tiles): per voxel
// v, its floor (magic-number add rounding down), the fraction, four taps,
// two u-lerps, one v-lerp and the weighted accumulate.
template <typename T, int TK, int BU, bool FULL>
__device__ __forceinline__ void accumulate_scalar(const T *__restrict__ tile, const ColView &c,
                                                  int ez, float *acc) {
    const T *base = tile + c.cu;
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
        if (!FULL && kk >= ez) continue;
        float v = fmaf((float)kk, c.dv, c.v0);
        float tv = __fadd_rd(v, kMagic);
        float fv = v - (tv - kMagic);
        int row = __float_as_int(tv) - kMagicBits;
        const T *p = base + row * BU;
        float q00 = to_f32(p[0]), q01 = to_f32(p[1]);
        float q10 = to_f32(p[BU]), q11 = to_f32(p[BU + 1]);
        float s0 = fmaf(c.fu, q01 - q00, q00);
        float s1 = fmaf(c.fu, q11 - q10, q10);
        float val = fmaf(fv, s1 - s0, s0);
        acc[kk] = fmaf(c.wt, val, acc[kk]);
    }
}

// The same sampling on voxel pairs (kk, kk+1) with f32x2 instructions, the
// weights written without subtraction: (1 - fu) wt and fu wt on the two
// columns, then acc + (1 - fv) s0 + fv s1 (equal to the scalar form up to
// rounding).
// tile_s: shared address of the staged box. The row of voxel v is the bit
// pattern of v + 1.5 * 2^23 (rounded down) minus that of 1.5 * 2^23; the
// constant is folded into the base (unsigned arithmetic, exact mod 2^32).
template <int TK, int BU>
__device__ __forceinline__ void accumulate_pairs(unsigned tile_s, const ColView &c, f2 *acc2) {
    constexpr unsigned kRow = BU * 4u;
    const unsigned base = tile_s + 4u * (unsigned)c.cu - (unsigned)kMagicBits * kRow;
    // subtraction-free weights (see accumulate_sym_pairs): (1 - fu) wt and fu wt
    // on the two columns, acc + (1 - fv) s0 + fv s1 as two FMAs
    const float gu = 1.0f - c.fu;
    const f2 M2 = pk(kMagic, kMagic), GUW = pk(c.wt * gu, c.wt * gu), FUW = pk(c.wt * c.fu, c.wt * c.fu);
    const f2 NM2 = pk(-kMagic, -kMagic), N1 = pk(-1.0f, -1.0f), ONE = pk(1.0f, 1.0f);
#pragma unroll
    for (int m = 0; m < TK / 2; ++m) {
        const float va = fmaf((float)(2 * m), c.dv, c.v0);
        const float vb = fmaf((float)(2 * m + 1), c.dv, c.v0);
        const f2 V = pk(va, vb);
        const f2 TV = add2_rd(V, M2);
        const f2 FV = fma2(add2(TV, NM2), N1, V);   // v - floor(v), exact
        float ta, tb;
        upk(TV, ta, tb);
        const unsigned pa = base + __float_as_uint(ta) * kRow, pb = base + __float_as_uint(tb) * kRow;
        const f2 Q00 = pk(lds32<0>(pa), lds32<0>(pb)), Q01 = pk(lds32<4>(pa), lds32<4>(pb));
        const f2 Q10 = pk(lds32<kRow>(pa), lds32<kRow>(pb)), Q11 = pk(lds32<kRow + 4>(pa), lds32<kRow + 4>(pb));
        const f2 GV = fma2(FV, N1, ONE);
        const f2 S0 = fma2(FUW, Q01, mul2(GUW, Q00)), S1 = fma2(FUW, Q11, mul2(GUW, Q10));
        acc2[m] = fma2(FV, S1, fma2(GV, S0, acc2[m]));
    }
}

template <int TK>
__device__ __forceinline__ void store_column(float *__restrict__ vol, const float *acc, int b,
                                             int i, int j, int k0, int ez, int nx, int ny,
                                             int nz, float scale, int accumulate) {
    size_t plane = (size_t)nx * ny;
    size_t base = ((size_t)b * nz + k0) * plane + (size_t)j * nx + i;
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
        if (kk < ez) {
            float r = scale * acc[kk];
            size_t idx = base + (size_t)kk * plane;
            vol[idx] = accumulate ? vol[idx] + r : r;
        }
    }
}

// ---------------------------------------------------------------------------
// Mid-plane symmetry (Section 3.1.2, Algorithm 1). When the detector rows and
// the volume slices are centred on the same plane, v(nz-1-k) = nv-1-v(k)
// while u and w do not depend on k. A thread then owns kTH lower voxels of
// its column and their mirrors: v, its floor and fraction are computed once
// for both. The producer stages the lower box (rows vb .. vb+BV-1) and its
// vertical mirror (rows nv-vb-BV .. nv-1-vb); a lower voxel whose taps are
// box rows r, r+1 with fraction f has its mirror's taps at rows BV-1-r and
// BV-2-r of the mirrored box, weighted 1-f and f.
// ---------------------------------------------------------------------------
constexpr int kTH = 16;   // lower voxels per thread

// f32x2 pair arithmetic on voxels (k, k+1) and their mirrors, 64-bit
// accumulators, no subtraction in the weights (1825 GUPS on c3 against 1774
// for the lerps q0 + f (q1 - q0), whose packed subtractions cost integer
// sign flips).
template <int BU>
__device__ __forceinline__ void accumulate_sym_pairs(unsigned lo_s, unsigned hi_s, const ColView &c,
                                                     f2 *acc_lo, f2 *acc_hi) {
    // lo_s = shared address of the lower box + 4 c.cu; hi_s = of the mirrored
    // box + (BV-1) rows + 4 c.cu. The magic constant of the row index is
    // folded into both bases (unsigned arithmetic, exact mod 2^32).
    constexpr unsigned kRow = BU * 4u;
    const unsigned lo_m = lo_s - (unsigned)kMagicBits * kRow, hi_m = hi_s + (unsigned)kMagicBits * kRow;
    // Weights without subtractions (a packed subtraction costs two integer
    // sign flips): each u-lerp is (1 - fu) wt q0 + fu wt q1 with the view
    // weight wt folded into both, and the v-lerp is two FMAs into the
    // accumulator, acc + (1 - fv) s0 + fv s1.
    const float gu = 1.0f - c.fu;
    const f2 GUW = pk(c.wt * gu, c.wt * gu), FUW = pk(c.wt * c.fu, c.wt * c.fu);
    const f2 M2 = pk(kMagic, kMagic), NM2 = pk(-kMagic, -kMagic), N1 = pk(-1.0f, -1.0f), ONE = pk(1.0f, 1.0f);
    const f2 DV2 = pk(c.dv, c.dv), V02 = pk(c.v0, c.v0);
#pragma unroll
    for (int m = 0; m < kTH / 2; ++m) {
        const f2 V = fma2(pk((float)(2 * m), (float)(2 * m + 1)), DV2, V02);
        const f2 TV = add2_rd(V, M2);
        const f2 FV = fma2(add2(TV, NM2), N1, V);   // v - floor(v), exact
        const f2 GV = fma2(FV, N1, ONE);
        float tvx, tvy;
        upk(TV, tvx, tvy);
        const unsigned ta = __float_as_uint(tvx), tb = __float_as_uint(tvy);
        const unsigned pa = lo_m + ta * kRow, pb = lo_m + tb * kRow;
        const f2 Q00 = pk(lds32<0>(pa), lds32<0>(pb)), Q01 = pk(lds32<4>(pa), lds32<4>(pb));
        const f2 Q10 = pk(lds32<kRow>(pa), lds32<kRow>(pb)), Q11 = pk(lds32<kRow + 4>(pa), lds32<kRow + 4>(pb));
        const f2 S0 = fma2(FUW, Q01, mul2(GUW, Q00)), S1 = fma2(FUW, Q11, mul2(GUW, Q10));
        acc_lo[m] = fma2(FV, S1, fma2(GV, S0, acc_lo[m]));
        // mirror: row BV-1-r (weight 1-f) and the row above it, BV-2-r (weight f)
        const unsigned qa = hi_m - ta * kRow, qb = hi_m - tb * kRow;
        const f2 R00 = pk(lds32<0>(qa), lds32<0>(qb)), R01 = pk(lds32<4>(qa), lds32<4>(qb));
        const f2 R10 = pk(lds32<-(int)kRow>(qa), lds32<-(int)kRow>(qb));
        const f2 R11 = pk(lds32<4 - (int)kRow>(qa), lds32<4 - (int)kRow>(qb));
        const f2 T0 = fma2(FUW, R01, mul2(GUW, R00)), T1 = fma2(FUW, R11, mul2(GUW, R10));
        acc_hi[m] = fma2(FV, T1, fma2(GV, T0, acc_hi[m]));
    }
}

template <int BU>
__device__ __forceinline__ void accumulate_sym_scalar(const float *__restrict__ lo,
                                                      const float *__restrict__ hi_top, const ColView &c,
                                                      int ez, float *acc_lo, float *acc_hi) {
#pragma unroll
    for (int kk = 0; kk < kTH; ++kk) {
        if (kk >= ez) continue;
        const float v = fmaf((float)kk, c.dv, c.v0);
        const float tv = __fadd_rd(v, kMagic);
        const float fv = v - (tv - kMagic);
        const int row = __float_as_int(tv) - kMagicBits;
        const float *p = lo + row * BU;
        const float s0 = fmaf(c.fu, p[1] - p[0], p[0]);
        const float s1 = fmaf(c.fu, p[BU + 1] - p[BU], p[BU]);
        acc_lo[kk] = fmaf(c.wt, fmaf(fv, s1 - s0, s0), acc_lo[kk]);
        const float *q = hi_top - row * BU;
        const float t0 = fmaf(c.fu, q[1] - q[0], q[0]);
        const float t1 = fmaf(c.fu, q[1 - BU] - q[-BU], q[-BU]);
        acc_hi[kk] = fmaf(c.wt, fmaf(fv, t1 - t0, t0), acc_hi[kk]);
    }
}

// Lower voxels k0 .. k0+ez-1 and, for k < nz/2, their mirrors nz-1-k (the
// middle slice of an odd nz is its own mirror and is written once).
__device__ __forceinline__ void store_sym(float *__restrict__ vol, const float *lo, const float *hi, int b,
                                          int i, int j, int k0, int ez, int nx, int ny, int nz, float scale,
                                          int accumulate) {
    const size_t plane = (size_t)nx * ny;
    const size_t col = (size_t)b * nz * plane + (size_t)j * nx + i;
#pragma unroll
    for (int kk = 0; kk < kTH; ++kk) {
        if (kk < ez) {
            const int k = k0 + kk;
            const size_t a = col + (size_t)k * plane;
            const float r = scale * lo[kk];
            vol[a] = accumulate ? vol[a] + r : r;
            if (k < nz / 2) {
                const size_t m = col + (size_t)(nz - 1 - k) * plane;
                const float rm = scale * hi[kk];
                vol[m] = accumulate ? vol[m] + rm : rm;
            }
        }
    }
}

template <typename T, int TK, int BU, int MB>
__global__ void __launch_bounds__(kThreads, MB)
bp_zcol_tma(const __grid_constant__ CUtensorMap tmap, const double *__restrict__ P, int view0,
            int nviews, int nx, int ny, int nz, int bv, int align, float *__restrict__ vol,
            float scale, int accumulate, unsigned *err, unsigned long long timeout_ns,
            int drop_view, int nst, int kz0, int kz1) {
    extern __shared__ __align__(128) unsigned char smem[];
    ViewRec *recs = reinterpret_cast<ViewRec *>(smem);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem + kBarOffset);
    unsigned long long *empty = full + kMaxStages;
    unsigned char *stages = smem + kStageOffset;
    const int sbytes = stage_bytes<T>(BU, bv);
    const unsigned box_bytes = (unsigned)(BU * bv * sizeof(T));

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (nx + kTX - 1) / kTX;
    const int i0 = (blockIdx.x % ntx) * kTX, j0 = (blockIdx.x / ntx) * kTY;
    const int k0 = kz0 + blockIdx.y * TK;   // slices [kz0, kz1) of this call
    const int b = blockIdx.z;
    const int ex = min(kTX, nx - i0), ey = min(kTY, ny - j0), ez = min(TK, kz1 - k0);

    int di = 0, dj = 0;
    if (warp < kConsumerWarps) consumer_column(warp, lane, &di, &dj);
    const bool col_ok = warp < kConsumerWarps && di < ex && dj < ey;
    const float fdi = (float)di, fdj = (float)dj;

    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        fence_barrier_init();
        prefetch_tmap(&tmap);
    }
    __syncthreads();

    // accumulators: FP32 pairs (kk, kk+1) for FP32 taps, scalars otherwise
    constexpr bool kPairs = sizeof(T) == 4;
    f2 acc2[TK / 2];
    float acc[kPairs ? 1 : TK];
#pragma unroll
    for (int m = 0; m < TK / 2; ++m) acc2[m] = 0ull;
#pragma unroll
    for (int kk = 0; kk < (kPairs ? 1 : TK); ++kk) acc[kk] = 0.0f;

    __shared__ unsigned arms[kMaxStages];   // producer: armings of each full barrier
    if (tid < kMaxStages) arms[tid] = 0;
    bool alive = true;
    // pipeline position of the current view g: slot g % nst, phase (g / nst) & 1,
    // advanced per view (no division)
    int slot = 0;
    unsigned phase = 0, g = 0;
    for (int cb = 0; cb < nviews; cb += kRecChunk) {
        const int cn = min(kRecChunk, nviews - cb);
        __syncthreads();
        for (int n = tid; n < cn; n += kThreads)
            if (!make_rec(P + 12 * (size_t)(view0 + cb + n), i0, j0, k0, ex, ey, ez, align, BU,
                          bv, &recs[n]))
                atomicOr(err, DEV_ERR_FOOTPRINT);
        __syncthreads();
        if (warp == kConsumerWarps) {
            // ---- producer: one elected lane issues the TMA loads ----
            if (lane == 0 && alive) {
                for (int n = 0; n < cn; ++n, ++g) {
                    if (g >= (unsigned)nst && !mbar_wait_bounded(&empty[slot], phase ^ 1u, timeout_ns)) {
                        atomicOr(err, DEV_ERR_TIMEOUT);
                        alive = false;
                        break;
                    }
                    if (view0 + cb + n != drop_view) {   // test hook: skip this view's load
                        mbar_arrive_expect_tx(&full[slot], box_bytes);
                        tma_load_4d(stages + slot * sbytes, &tmap, recs[n].u_box, recs[n].v_box,
                                    cb + n, b, &full[slot]);
                        ++arms[slot];
                    }
                    if (++slot == nst) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
        } else {
            // ---- consumers ----
            for (int n = 0; n < cn && alive; ++n) {
                // the whole warp agrees on the outcome of the bounded wait
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[slot], phase, timeout_ns))) {
                    if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                    alive = false;
                    break;
                }
                ColView cv;
                if (col_ok && column_view<BU>(recs[n], fdi, fdj, ez, bv, err, cv)) {
                    const T *tile = reinterpret_cast<const T *>(stages + slot * sbytes);
                    if constexpr (kPairs) {
                        if (ez == TK) {
                            accumulate_pairs<TK, BU>(smem_addr(tile), cv, acc2);
                        } else {
                            float tmp[TK];
#pragma unroll
                            for (int m = 0; m < TK / 2; ++m) upk(acc2[m], tmp[2 * m], tmp[2 * m + 1]);
                            accumulate_scalar<T, TK, BU, false>(tile, cv, ez, tmp);
#pragma unroll
                            for (int m = 0; m < TK / 2; ++m) acc2[m] = pk(tmp[2 * m], tmp[2 * m + 1]);
                        }
                    } else {
                        if (ez == TK)
                            accumulate_scalar<T, TK, BU, true>(tile, cv, ez, acc);
                        else
                            accumulate_scalar<T, TK, BU, false>(tile, cv, ez, acc);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                if (++slot == nst) {
                    slot = 0;
                    phase ^= 1u;
                }
            }
        }
    }
    if (warp == kConsumerWarps && lane == 0) {
        // drain: every issued load must have landed before the CTA exits
        for (int s = 0; s < nst; ++s)
            if (arms[s] > 0 && !mbar_wait_bounded(&full[s], (arms[s] - 1) & 1, timeout_ns))
                atomicOr(err, DEV_ERR_TIMEOUT);
    }
    if (col_ok && alive) {
        if constexpr (kPairs) {
            float out[TK];
#pragma unroll
            for (int m = 0; m < TK / 2; ++m) upk(acc2[m], out[2 * m], out[2 * m + 1]);
            store_column<TK>(vol, out, b, i0 + di, j0 + dj, k0, ez, nx, ny, nz, scale, accumulate);
        } else {
            store_column<TK>(vol, acc, b, i0 + di, j0 + dj, k0, ez, nx, ny, nz, scale, accumulate);
        }
    }
}

// The staged z-column kernel with mid-plane symmetry (FP32 projections): z
// block y covers lower slices [16y, 16y+16) of the (nz+1)/2 lower slices and
// their mirrors; each stage holds the lower box and the mirrored box. The
// pipeline, bounded waits and drain are those of bp_zcol_tma.
template <int BU, int MB>
__global__ void __launch_bounds__(kThreads, MB)
bp_zsym_tma(const __grid_constant__ CUtensorMap tmap, const double *__restrict__ P, int view0,
            int nviews, int nx, int ny, int nz, int nv, int bv, int align, float *__restrict__ vol,
            float scale, int accumulate, unsigned *err, unsigned long long timeout_ns, int drop_view,
            int nst, int kz0, int kz1) {
    extern __shared__ __align__(128) unsigned char smem[];
    ViewRec *recs = reinterpret_cast<ViewRec *>(smem);
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem + kBarOffset);
    unsigned long long *empty = full + kMaxStages;
    unsigned char *stages = smem + kStageOffset;
    const unsigned box_bytes = (unsigned)(BU * bv * sizeof(float));
    const int half = stage_bytes<float>(BU, bv);   // offset of the mirrored box in a stage
    const int sbytes = 2 * half;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (nx + kTX - 1) / kTX;
    const int i0 = (blockIdx.x % ntx) * kTX, j0 = (blockIdx.x / ntx) * kTY;
    const int k0 = kz0 + blockIdx.y * kTH;   // lower slices [kz0, kz1) (kz1 <= (nz + 1) / 2) and their mirrors
    const int b = blockIdx.z;
    const int ex = min(kTX, nx - i0), ey = min(kTY, ny - j0), ez = min(kTH, kz1 - k0);

    int di = 0, dj = 0;
    if (warp < kConsumerWarps) consumer_column(warp, lane, &di, &dj);
    const bool col_ok = warp < kConsumerWarps && di < ex && dj < ey;
    const float fdi = (float)di, fdj = (float)dj;

    if (tid == 0) {
        for (int s = 0; s < nst; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kConsumerWarps);
        }
        fence_barrier_init();
        prefetch_tmap(&tmap);
    }
    __syncthreads();

    f2 acc_lo[kTH / 2], acc_hi[kTH / 2];
#pragma unroll
    for (int m = 0; m < kTH / 2; ++m) acc_lo[m] = acc_hi[m] = 0ull;

    __shared__ unsigned arms[kMaxStages];
    if (tid < kMaxStages) arms[tid] = 0;
    bool alive = true;
    int slot = 0;
    unsigned phase = 0, g = 0;
    for (int cb = 0; cb < nviews; cb += kRecChunk) {
        const int cn = min(kRecChunk, nviews - cb);
        __syncthreads();
        for (int n = tid; n < cn; n += kThreads)
            if (!make_rec(P + 12 * (size_t)(view0 + cb + n), i0, j0, k0, ex, ey, ez, align, BU, bv, &recs[n]))
                atomicOr(err, DEV_ERR_FOOTPRINT);
        __syncthreads();
        if (warp == kConsumerWarps) {
            if (lane == 0 && alive) {
                for (int n = 0; n < cn; ++n, ++g) {
                    if (g >= (unsigned)nst && !mbar_wait_bounded(&empty[slot], phase ^ 1u, timeout_ns)) {
                        atomicOr(err, DEV_ERR_TIMEOUT);
                        alive = false;
                        break;
                    }
                    if (view0 + cb + n != drop_view) {   // test hook: skip this view's loads
                        mbar_arrive_expect_tx(&full[slot], 2 * box_bytes);
                        unsigned char *st = stages + slot * sbytes;
                        tma_load_4d(st, &tmap, recs[n].u_box, recs[n].v_box, cb + n, b, &full[slot]);
                        tma_load_4d(st + half, &tmap, recs[n].u_box, nv - recs[n].v_box - bv, cb + n, b,
                                    &full[slot]);
                        ++arms[slot];
                    }
                    if (++slot == nst) {
                        slot = 0;
                        phase ^= 1u;
                    }
                }
            }
        } else {
            for (int n = 0; n < cn && alive; ++n) {
                // the whole warp agrees on the outcome of the bounded wait
                if (!__all_sync(0xffffffffu, mbar_wait_bounded(&full[slot], phase, timeout_ns))) {
                    if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                    alive = false;
                    break;
                }
                ColView cv;
                if (col_ok && column_view<BU>(recs[n], fdi, fdj, ez, bv, err, cv)) {
                    const float *lo = reinterpret_cast<const float *>(stages + slot * sbytes) + cv.cu;
                    const float *hi_top = reinterpret_cast<const float *>(stages + slot * sbytes + half) +
                                          (bv - 1) * BU + cv.cu;
                    if (ez == kTH) {
                        accumulate_sym_pairs<BU>(smem_addr(lo), smem_addr(hi_top), cv, acc_lo, acc_hi);
                    } else {
                        float tl[kTH], th[kTH];
#pragma unroll
                        for (int m = 0; m < kTH / 2; ++m) {
                            upk(acc_lo[m], tl[2 * m], tl[2 * m + 1]);
                            upk(acc_hi[m], th[2 * m], th[2 * m + 1]);
                        }
                        accumulate_sym_scalar<BU>(lo, hi_top, cv, ez, tl, th);
#pragma unroll
                        for (int m = 0; m < kTH / 2; ++m) {
                            acc_lo[m] = pk(tl[2 * m], tl[2 * m + 1]);
                            acc_hi[m] = pk(th[2 * m], th[2 * m + 1]);
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[slot]);
                if (++slot == nst) {
                    slot = 0;
                    phase ^= 1u;
                }
            }
        }
    }
    if (warp == kConsumerWarps && lane == 0) {
        for (int s = 0; s < nst; ++s)
            if (arms[s] > 0 && !mbar_wait_bounded(&full[s], (arms[s] - 1) & 1, timeout_ns))
                atomicOr(err, DEV_ERR_TIMEOUT);
    }
    if (col_ok && alive) {
        float lo[kTH], hi[kTH];
#pragma unroll
        for (int m = 0; m < kTH / 2; ++m) {
            upk(acc_lo[m], lo[2 * m], lo[2 * m + 1]);
            upk(acc_hi[m], hi[2 * m], hi[2 * m + 1]);
        }
        store_sym(vol, lo, hi, b, i0 + di, j0 + dj, k0, ez, nx, ny, nz, scale, accumulate);
    }
}

// Same arithmetic without TMA: taps are gathered from global memory with
// explicit zero padding. Records are relative to (u_box, v_box) as above.
template <typename T, int TK>
__global__ void __launch_bounds__(kConsumers)
bp_zcol_ldg(const T *__restrict__ proj, long long batch_stride, const double *__restrict__ P,
            int view0, int nviews, int nu, int nv, int nx, int ny, int nz,
            float *__restrict__ vol, float scale, int accumulate, int kz0, int kz1) {
    __shared__ ViewRec recs[128];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = (nx + kTX - 1) / kTX;
    const int i0 = (blockIdx.x % ntx) * kTX, j0 = (blockIdx.x / ntx) * kTY;
    const int k0 = kz0 + blockIdx.y * TK;   // slices [kz0, kz1) of this call
    const int b = blockIdx.z;
    const int ex = min(kTX, nx - i0), ey = min(kTY, ny - j0), ez = min(TK, kz1 - k0);
    int di, dj;
    consumer_column(warp, lane, &di, &dj);
    const bool col_ok = di < ex && dj < ey;
    const float fdi = (float)di, fdj = (float)dj;
    const T *pb = proj + (size_t)b * batch_stride;

    float acc[TK];
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) acc[kk] = 0.0f;

    for (int cb = 0; cb < nviews; cb += 128) {
        const int cn = min(128, nviews - cb);
        __syncthreads();
        for (int n = tid; n < cn; n += kConsumers) {
            ViewRec r;
            make_rec(P + 12 * (size_t)(view0 + cb + n), i0, j0, k0, ex, ey, ez, 1, 1 << 30,
                     1 << 30, &r);
            recs[n] = r;
        }
        __syncthreads();
        if (!col_ok) continue;
        for (int n = 0; n < cn; ++n) {
            const ViewRec r = recs[n];
            const T *img = pb + (size_t)(cb + n) * nu * nv;
            float W = fmaf(r.Wj, fdj, fmaf(r.Wi, fdi, r.W0));
            float inv = col_rcp(W);
            float uL = fmaf(r.Nuj, fdj, fmaf(r.Nui, fdi, r.Nu0)) * inv;
            float v0 = fmaf(r.Nvj, fdj, fmaf(r.Nvi, fdi, r.Nv0)) * inv;
            float dv = r.Nvk * inv;
            float wt = inv * inv;
            float uf = floorf(uL);
            float fu = uL - uf;
            int c0 = (int)uf + r.u_box;
            bool cin0 = c0 >= 0 && c0 < nu, cin1 = c0 + 1 >= 0 && c0 + 1 < nu;
#pragma unroll
            for (int kk = 0; kk < TK; ++kk) {
                if (kk >= ez) continue;
                float v = fmaf((float)kk, dv, v0);
                float vf = floorf(v);
                float fv = v - vf;
                int r0 = (int)vf + r.v_box;
                bool rin0 = r0 >= 0 && r0 < nv, rin1 = r0 + 1 >= 0 && r0 + 1 < nv;
                const T *row0 = img + (long long)r0 * nu + c0;
                float q00 = (rin0 && cin0) ? to_f32(row0[0]) : 0.0f;
                float q01 = (rin0 && cin1) ? to_f32(row0[1]) : 0.0f;
                float q10 = (rin1 && cin0) ? to_f32(row0[nu]) : 0.0f;
                float q11 = (rin1 && cin1) ? to_f32(row0[nu + 1]) : 0.0f;
                float s0 = fmaf(fu, q01 - q00, q00);
                float s1 = fmaf(fu, q11 - q10, q10);
                float val = fmaf(fv, s1 - s0, s0);
                acc[kk] = fmaf(wt, val, acc[kk]);
            }
        }
    }
    if (col_ok) store_column<TK>(vol, acc, b, i0 + di, j0 + dj, k0, ez, nx, ny, nz, scale, accumulate);
}

// General 3x4 matrices: one thread per voxel of an 8 x 8 x 4 tile.
template <typename T>
__global__ void __launch_bounds__(256)
bp_voxel_gen(const T *__restrict__ proj, long long batch_stride, const double *__restrict__ P,
             int view0, int nviews, int nu, int nv, int nx, int ny, int nz,
             float *__restrict__ vol, float scale, int accumulate, int kz0, int kz1) {
    __shared__ ViewRecGen recs[64];
    const int tid = threadIdx.x;
    const int ntx = (nx + 7) / 8, nty = (ny + 7) / 8;
    const int t = blockIdx.x;
    const int i0 = (t % ntx) * 8, j0 = ((t / ntx) % nty) * 8, k0 = kz0 + (t / (ntx * nty)) * 4;
    const int b = blockIdx.z;
    const int di = tid & 7, dj = (tid >> 3) & 7, dk = tid >> 6;
    const int i = i0 + di, j = j0 + dj, k = k0 + dk;
    const bool ok = i < nx && j < ny && k < kz1;
    const float fdi = (float)di, fdj = (float)dj, fdk = (float)dk;
    const T *pb = proj + (size_t)b * batch_stride;
    float acc = 0.0f;
    for (int cb = 0; cb < nviews; cb += 64) {
        const int cn = min(64, nviews - cb);
        __syncthreads();
        for (int n = tid; n < cn; n += 256) make_rec_gen(P + 12 * (size_t)(view0 + cb + n), i0, j0, k0, &recs[n]);
        __syncthreads();
        if (!ok) continue;
        for (int n = 0; n < cn; ++n) {
            const ViewRecGen r = recs[n];
            const T *img = pb + (size_t)(cb + n) * nu * nv;
            float W = fmaf(r.Wk, fdk, fmaf(r.Wj, fdj, fmaf(r.Wi, fdi, r.W0)));
            if (!(W > 0.0f)) continue;
            float inv = __frcp_rn(W);
            float u = fmaf(r.Nuk, fdk, fmaf(r.Nuj, fdj, fmaf(r.Nui, fdi, r.Nu0))) * inv;
            float v = fmaf(r.Nvk, fdk, fmaf(r.Nvj, fdj, fmaf(r.Nvi, fdi, r.Nv0))) * inv;
            if (!(fabsf(u) < 4e6f && fabsf(v) < 4e6f)) continue;
            float uf = floorf(u), vf = floorf(v);
            float fu = u - uf, fv = v - vf;
            int c0 = (int)uf + r.u_ref, r0 = (int)vf + r.v_ref;
            bool cin0 = c0 >= 0 && c0 < nu, cin1 = c0 + 1 >= 0 && c0 + 1 < nu;
            bool rin0 = r0 >= 0 && r0 < nv, rin1 = r0 + 1 >= 0 && r0 + 1 < nv;
            const T *row0 = img + (long long)r0 * nu + c0;
            float q00 = (rin0 && cin0) ? to_f32(row0[0]) : 0.0f;
            float q01 = (rin0 && cin1) ? to_f32(row0[1]) : 0.0f;
            float q10 = (rin1 && cin0) ? to_f32(row0[nu]) : 0.0f;
            float q11 = (rin1 && cin1) ? to_f32(row0[nu + 1]) : 0.0f;
            float s0 = fmaf(fu, q01 - q00, q00);
            float s1 = fmaf(fu, q11 - q10, q10);
            acc = fmaf(inv * inv, fmaf(fv, s1 - s0, s0), acc);
        }
    }
    if (ok) {
        size_t idx = (((size_t)b * nz + k) * ny + j) * nx + i;
        float r = scale * acc;
        vol[idx] = accumulate ? vol[idx] + r : r;
    }
}

// ---------------------------------------------------------------------------
// Host launcher
// ---------------------------------------------------------------------------

typedef CUresult (*PFN_encodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                    const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                    const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                    CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
    static PFN_encodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled>(p);
    }
    return fn;
}

// Box widths (elements) the TMA kernel is instantiated for. A row pitch of
// 16 mod 32 banks puts vertically adjacent taps half a bank cycle apart, so
// the 8 x 4 columns of a warp (whose taps span ~2 rows and < 16 columns)
// read without bank conflicts: FP32 widths are 16 mod 32 floats, FP16
// widths 32 mod 64 halves.
static const int kBoxWidths32[] = {48, 80, 112, 144, 176, 208, 240};
static const int kBoxWidths16[] = {32, 96, 160, 224};

int plan_box_width(int need, int elem_bytes) {
    if (elem_bytes == 2) {
        for (int w : kBoxWidths16)
            if (w >= need) return w;
    } else {
        for (int w : kBoxWidths32)
            if (w >= need) return w;
    }
    return -1;
}

template <typename T, int TK, int BU, int MB>
static cudaError_t launch_tma_t(const CUtensorMap &map, bp_ctx *ctx, int view0, int nviews,
                                int bv, int align, float *vol, int batch, float scale,
                                int accumulate, cudaStream_t st, int kz0, int kz1) {
    const int nst = ctx->plan.stages;
    const int smem = kStageOffset + nst * stage_bytes<T>(BU, bv);
    auto kern = bp_zcol_tma<T, TK, BU, MB>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(((ctx->nx + kTX - 1) / kTX) * ((ctx->ny + kTY - 1) / kTY), (kz1 - kz0 + TK - 1) / TK,
              batch);
    kern<<<grid, kThreads, smem, st>>>(map, ctx->d_P, view0, nviews, ctx->nx, ctx->ny, ctx->nz, bv,
                                       align, vol, scale, accumulate, ctx->d_err, ctx->timeout_ns,
                                       ctx->test_drop_view, nst, kz0, kz1);
    return cudaGetLastError();
}

template <typename T, int TK, int MB>
static cudaError_t launch_tma_bu(const CUtensorMap &map, bp_ctx *ctx, int bu, int view0,
                                 int nviews, int bv, int align, float *vol, int batch, float scale,
                                 int accumulate, cudaStream_t st, int kz0, int kz1) {
#define BP_TMA_CASE(W) \
    case W: return launch_tma_t<T, TK, W, MB>(map, ctx, view0, nviews, bv, align, vol, batch, scale, accumulate, st, kz0, kz1);
    if constexpr (sizeof(T) == 2) {
        switch (bu) {
            BP_TMA_CASE(32) BP_TMA_CASE(96) BP_TMA_CASE(160) BP_TMA_CASE(224)
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (bu) {
            BP_TMA_CASE(48) BP_TMA_CASE(80) BP_TMA_CASE(112) BP_TMA_CASE(144) BP_TMA_CASE(176)
            BP_TMA_CASE(208) BP_TMA_CASE(240)
            default: return cudaErrorInvalidValue;
        }
    }
#undef BP_TMA_CASE
}

template <int BU>
static cudaError_t launch_sym_t(const CUtensorMap &map, bp_ctx *ctx, int view0, int nviews, int bv,
                                float *vol, int batch, float scale, int accumulate, cudaStream_t st, int kz0,
                                int kz1) {
    const int nst = ctx->plan.stages;
    const int smem = kStageOffset + nst * 2 * stage_bytes<float>(BU, bv);
    auto kern = bp_zsym_tma<BU, 2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(((ctx->nx + kTX - 1) / kTX) * ((ctx->ny + kTY - 1) / kTY), (kz1 - kz0 + kTH - 1) / kTH, batch);
    kern<<<grid, kThreads, smem, st>>>(map, ctx->d_P, view0, nviews, ctx->nx, ctx->ny, ctx->nz, ctx->nv, bv, 4,
                                       vol, scale, accumulate, ctx->d_err, ctx->timeout_ns, ctx->test_drop_view,
                                       nst, kz0, kz1);
    return cudaGetLastError();
}

static cudaError_t launch_sym(const CUtensorMap &map, bp_ctx *ctx, int bu, int view0, int nviews, int bv,
                              float *vol, int batch, float scale, int accumulate, cudaStream_t st, int kz0,
                              int kz1) {
#define BP_SYM_CASE(W) \
    case W: return launch_sym_t<W>(map, ctx, view0, nviews, bv, vol, batch, scale, accumulate, st, kz0, kz1);
    switch (bu) {
        BP_SYM_CASE(48) BP_SYM_CASE(80) BP_SYM_CASE(112) BP_SYM_CASE(144) BP_SYM_CASE(176)
        BP_SYM_CASE(208) BP_SYM_CASE(240)
        default: return cudaErrorInvalidValue;
    }
#undef BP_SYM_CASE
}

// One launch over slices [kz0, kz1): the plain kernels, or with sym the
// mid-plane symmetric kernel over lower slices [kz0, kz1) and their mirrors.
// Returns BP_ERR_UNSUPPORTED (without launching) when sym is asked for but
// the projections cannot be staged by TMA.
static bp_status launch_range(bp_ctx *ctx, const void *proj, bp_dtype t, int view0, int nviews,
                              long long batch_stride, float *vol, int batch, float scale, int accumulate,
                              cudaStream_t st, int kz0, int kz1, bool sym) {
    const size_t es = (t == BP_F16) ? 2 : 4;
    const long long view_elems = (long long)ctx->nu * ctx->nv;
    cudaError_t e = cudaSuccess;
    if (!ctx->zinv) {
        dim3 grid(((ctx->nx + 7) / 8) * ((ctx->ny + 7) / 8) * ((kz1 - kz0 + 3) / 4), 1, batch);
        if (t == BP_F16)
            bp_voxel_gen<__half><<<grid, 256, 0, st>>>((const __half *)proj, batch_stride,
                ctx->d_P, view0, nviews, ctx->nu, ctx->nv, ctx->nx, ctx->ny, ctx->nz, vol, scale, accumulate, kz0, kz1);
        else
            bp_voxel_gen<float><<<grid, 256, 0, st>>>((const float *)proj, batch_stride, ctx->d_P,
                view0, nviews, ctx->nu, ctx->nv, ctx->nx, ctx->ny, ctx->nz, vol, scale, accumulate, kz0, kz1);
        e = cudaGetLastError();
        return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "bp_voxel_gen launch");
    }
    const Plan &pl = ctx->plan;
    const int bu = sym ? pl.sym_bu : (t == BP_F16) ? pl.bu16 : pl.bu;
    const int bv = sym ? pl.sym_bv : pl.bv;
    const int align = (t == BP_F16) ? 8 : 4;
    PFN_encodeTiled enc = get_encode();
    bool tma = enc != nullptr && bu > 0 && (((size_t)ctx->nu * es) % 16 == 0) &&
               (((uintptr_t)proj) % 16 == 0) && ((batch_stride * es) % 16 == 0) &&
               bv <= 256 && bu <= 256;
    if (tma) {
        CUtensorMap map;
        cuuint64_t dims[4] = {(cuuint64_t)ctx->nu, (cuuint64_t)ctx->nv, (cuuint64_t)nviews,
                              (cuuint64_t)batch};
        cuuint64_t strides[3] = {(cuuint64_t)(ctx->nu * es), (cuuint64_t)(view_elems * es),
                                 (cuuint64_t)(batch_stride * es)};
        cuuint32_t box[4] = {(cuuint32_t)bu, (cuuint32_t)bv, 1, 1};
        cuuint32_t estr[4] = {1, 1, 1, 1};
        CUresult r = enc(&map, t == BP_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                         4, const_cast<void *>(proj), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) tma = false;
        if (tma && sym) {
            e = launch_sym(map, ctx, bu, view0, nviews, bv, vol, batch, scale, accumulate, st, kz0, kz1);
            return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "bp_zsym_tma launch");
        }
        if (tma) {
            // variants: (voxels per thread along z, CTAs per SM the registers target)
            if (t == BP_F16) {
                if (pl.tk == 64)
                    e = launch_tma_bu<__half, 64, 1>(map, ctx, bu, view0, nviews, pl.bv, align, vol, batch, scale, accumulate, st, kz0, kz1);
                else if (pl.ctas == 3)
                    e = launch_tma_bu<__half, 32, 3>(map, ctx, bu, view0, nviews, pl.bv, align, vol, batch, scale, accumulate, st, kz0, kz1);
                else
                    e = launch_tma_bu<__half, 32, 2>(map, ctx, bu, view0, nviews, pl.bv, align, vol, batch, scale, accumulate, st, kz0, kz1);
            } else {
                if (pl.tk == 64)
                    e = launch_tma_bu<float, 64, 1>(map, ctx, bu, view0, nviews, pl.bv, align, vol, batch, scale, accumulate, st, kz0, kz1);
                else if (pl.ctas == 3)
                    e = launch_tma_bu<float, 32, 3>(map, ctx, bu, view0, nviews, pl.bv, align, vol, batch, scale, accumulate, st, kz0, kz1);
                else
                    e = launch_tma_bu<float, 32, 2>(map, ctx, bu, view0, nviews, pl.bv, align, vol, batch, scale, accumulate, st, kz0, kz1);
            }
            return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "bp_zcol_tma launch");
        }
    }
    if (sym) return BP_ERR_UNSUPPORTED;
    dim3 grid(((ctx->nx + kTX - 1) / kTX) * ((ctx->ny + kTY - 1) / kTY), (kz1 - kz0 + 31) / 32, batch);
    if (t == BP_F16)
        bp_zcol_ldg<__half, 32><<<grid, kConsumers, 0, st>>>((const __half *)proj, batch_stride,
            ctx->d_P, view0, nviews, ctx->nu, ctx->nv, ctx->nx, ctx->ny, ctx->nz, vol, scale, accumulate, kz0, kz1);
    else
        bp_zcol_ldg<float, 32><<<grid, kConsumers, 0, st>>>((const float *)proj, batch_stride,
            ctx->d_P, view0, nviews, ctx->nu, ctx->nv, ctx->nx, ctx->ny, ctx->nz, vol, scale, accumulate, kz0, kz1);
    e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "bp_zcol_ldg launch");
}

// Slices [z0, z0 + nzs) and, with mirror, the mirrored slices
// [nz - z0 - nzs, nz - z0) (the caller has checked z0 + nzs <= (nz + 1) / 2):
// one symmetric launch where the plan has the symmetric kernel and the
// projections are FP32, else plain launches over the two ranges (the middle
// slice of an odd nz only once).
bp_status launch_backproject(bp_ctx *ctx, const void *proj, bp_dtype t, int view0, int nviews,
                             long long batch_stride, float *vol, int batch, float scale,
                             int accumulate, cudaStream_t st, int z0, int nzs, int mirror) {
    const long long view_elems = (long long)ctx->nu * ctx->nv;
    if (batch_stride == 0) batch_stride = view_elems * nviews;
    const int z1 = z0 + nzs;
    if (mirror && ctx->zinv && t == BP_F32 && ctx->plan.sym_bu > 0) {
        bp_status s = launch_range(ctx, proj, t, view0, nviews, batch_stride, vol, batch, scale, accumulate, st,
                                   z0, z1, true);
        if (s != BP_ERR_UNSUPPORTED) return s;
    }
    bp_status s = launch_range(ctx, proj, t, view0, nviews, batch_stride, vol, batch, scale, accumulate, st, z0,
                               z1, false);
    if (s != BP_OK || !mirror) return s;
    const int m0 = std::max(ctx->nz - z1, z1), m1 = ctx->nz - z0;
    if (m1 <= m0) return BP_OK;
    return launch_range(ctx, proj, t, view0, nviews, batch_stride, vol, batch, scale, accumulate, st, m0, m1,
                        false);
}

}  // namespace bp
