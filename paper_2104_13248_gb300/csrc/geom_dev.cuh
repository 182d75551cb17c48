// Device helpers shared by the back-projection and forward-projection
// kernels: per-(tile, view) records in FP64, bounded mbarrier waits, TMA.
#pragma once

#include "bp_internal.h"

namespace bp {

// Largest number of views whose records one CTA keeps in shared memory at a
// time; longer view lists are processed in chunks of this size.
constexpr int kRecChunk = 256;

__device__ __forceinline__ int floor_div(int a, int b) {
    int q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

// Record of one z-invariant view for a tile with origin (i0, j0, k0) and
// extent (ex, ey, ez) voxels (already clipped to the volume). The staged
// box starts at (u_box, v_box): one column/row below the smallest corner
// projection (u_box rounded down to a multiple of `align`). Perspective maps
// the convex tile to a convex region whose extreme points are corner images,
// so the 8 corners bound the footprint. Corner coordinates are only used for
// the box, so they are divided in FP32 and widened by kFootMargin px (their
// error is below 1e-3 px); the host's plan applies a larger margin to the
// exact FP64 corners, so every box the device builds fits the planned size.
// Returns false when the taps (plus one pixel of slack per side for FP32
// rounding of the per-voxel coordinates) would leave a bu x bv box.
constexpr float kFootMargin = 0.01f;

__device__ inline bool make_rec(const double *P, int i0, int j0, int k0, int ex, int ey, int ez,
                                int align, int bu, int bv, ViewRec *r) {
    float umin = 3e38f, umax = -3e38f, vmin = 3e38f, vmax = -3e38f;
#pragma unroll 1
    for (int c = 0; c < 8; ++c) {
        double i = i0 + ((c & 1) ? ex - 1 : 0);
        double j = j0 + ((c & 2) ? ey - 1 : 0);
        double k = k0 + ((c & 4) ? ez - 1 : 0);
        float w = (float)(P[8] * i + P[9] * j + P[10] * k + P[11]);
        float u = __fdividef((float)(P[0] * i + P[1] * j + P[2] * k + P[3]), w);
        float v = __fdividef((float)(P[4] * i + P[5] * j + P[6] * k + P[7]), w);
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    // clamp to a sane integer range before conversion (far off-detector views)
    umin = fmaxf(fminf(umin - kFootMargin, 1e8f), -1e8f);
    umax = fmaxf(fminf(umax + kFootMargin, 1e8f), -1e8f);
    vmin = fmaxf(fminf(vmin - kFootMargin, 1e8f), -1e8f);
    vmax = fmaxf(fminf(vmax + kFootMargin, 1e8f), -1e8f);
    int ub = (int)floorf(umin) - 1;
    ub = floor_div(ub, align) * align;
    int vb = (int)floorf(vmin) - 1;
    bool ok = ((int)floorf(umax) + 2 - ub <= bu - 1) && ((int)floorf(vmax) + 2 - vb <= bv - 1);
    double W0 = P[8] * i0 + P[9] * j0 + P[11];
    double U0 = P[0] * i0 + P[1] * j0 + P[3];
    double V0 = P[4] * i0 + P[5] * j0 + P[6] * k0 + P[7];
    r->Nu0 = (float)(U0 - ub * W0);
    r->Nui = (float)(P[0] - ub * P[8]);
    r->Nuj = (float)(P[1] - ub * P[9]);
    r->W0 = (float)W0;
    r->Nv0 = (float)(V0 - vb * W0);
    r->Nvi = (float)(P[4] - vb * P[8]);
    r->Nvj = (float)(P[5] - vb * P[9]);
    r->Nvk = (float)P[6];
    r->Wi = (float)P[8];
    r->Wj = (float)P[9];
    r->u_box = ub;
    r->v_box = vb;
    return ok;
}

// Record for general matrices (u and w may depend on k): reference pixel is
// the rounded projection of the tile origin.
__device__ inline void make_rec_gen(const double *P, int i0, int j0, int k0, ViewRecGen *r) {
    double W0 = P[8] * i0 + P[9] * j0 + P[10] * k0 + P[11];
    double U0 = P[0] * i0 + P[1] * j0 + P[2] * k0 + P[3];
    double V0 = P[4] * i0 + P[5] * j0 + P[6] * k0 + P[7];
    float u = __fdividef((float)U0, (float)W0), v = __fdividef((float)V0, (float)W0);
    int ur = (int)floorf(fmaxf(fminf(u, 1e8f), -1e8f));
    int vr = (int)floorf(fmaxf(fminf(v, 1e8f), -1e8f));
    r->Nu0 = (float)(U0 - ur * W0);
    r->Nui = (float)(P[0] - ur * P[8]);
    r->Nuj = (float)(P[1] - ur * P[9]);
    r->Nuk = (float)(P[2] - ur * P[10]);
    r->Nv0 = (float)(V0 - vr * W0);
    r->Nvi = (float)(P[4] - vr * P[8]);
    r->Nvj = (float)(P[5] - vr * P[9]);
    r->Nvk = (float)(P[6] - vr * P[10]);
    r->W0 = (float)W0;
    r->Wi = (float)P[8];
    r->Wj = (float)P[9];
    r->Wk = (float)P[10];
    r->u_ref = ur;
    r->v_ref = vr;
    r->pad0 = r->pad1 = 0;
}

// 1/w for the per-(column, view) setup of the z-column kernels (the
// back-projectors and their transpose use the same one, so their taps and
// weights coincide): the hardware approximation, within 1 ulp, instead of the
// correctly rounded reciprocal's longer sequence. w is near 1 here.
__device__ __forceinline__ float col_rcp(float w) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(w));
    return r;
}

// floor(x) for |x| < 2^22 without a conversion instruction: adding 1.5*2^23
// with round-toward-minus-infinity leaves floor(x) in the low mantissa bits.
constexpr float kMagic = 12582912.0f;      // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;     // bit pattern of kMagic

__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__half x) { return __half2float(x); }

// ---------------------------------------------------------------------------
// mbarrier / TMA primitives (inline PTX, sm_90+ forms valid on sm_103a)
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// try_wait with a suspend-time hint: a thread whose phase is not complete
// sleeps until it completes or hint_ns passes, instead of polling (a polling
// producer warp takes issue slots from the consumer warps beside it).
#ifndef BP_WAIT_HINT_NS
#define BP_WAIT_HINT_NS 20000
#endif
__device__ __forceinline__ bool mbar_try_wait_sleep(unsigned long long *bar, unsigned parity,
                                                    unsigned hint_ns) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; gives up after timeout_ns and
// returns false (the caller records DEV_ERR_TIMEOUT and leaves its loop).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait_sleep(bar, parity, BP_WAIT_HINT_NS)) return true;
        if (global_ns() - t0 > timeout_ns) return false;
    }
}

// 4-D tiled TMA load (no multicast) into CTA shared memory, completing on bar.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1,
                                            int c2, int c3, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3),
        "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<unsigned long long>(map))
                 : "memory");
}

}  // namespace bp
