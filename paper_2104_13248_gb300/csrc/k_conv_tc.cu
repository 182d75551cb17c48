// 3x3x3 convolution forward on the 5th-generation tensor cores (tcgen05):
// implicit GEMM with M = 128 consecutive output voxels along x, N = Cout,
// K = 16 input channels of one tap, BF16 operands from shared memory and the
// FP32 accumulators in tensor memory. The paper has no learned component;
// this serves the few-view correction network.
//
// CTA tile: 4 output rows of 128 voxels stacked along z (one y), all Cout
// channels; one TMEM accumulator of Cout columns per row (lanes = voxels).
// Per 16-channel chunk of the input:
//   - the halo brick (130 x 3 x 6 voxels) arrives by two 5-D TMA loads, one
//     per 8-channel half, as two planes [voxel][8 channels] (16 bytes a voxel;
//     zero fill outside the volume is the convolution's zero padding). Eight
//     consecutive voxels of a plane are one 8 x 16-byte core matrix, so the A
//     operand of brick row (z', dy) shifted by dx is a descriptor into the
//     brick: stride 128 bytes between 8-voxel groups (SBO), the plane size
//     between the two channel halves (LBO);
//   - that A operand serves every output row rz = z' - dz (dz = 0..2) at
//     once: one MMA with N = (rows) x Cout, whose B rows are the weights of
//     taps (dz, dy, dx) for those rows, laid out [dy][dx][half][dz][cout][8]
//     by cp.async so the rows follow at a uniform 128-byte stride, and whose
//     D columns are those rows' accumulators (row rz at column (3 - rz) Cout).
//     That is 54 MMAs of N = 16-48 (Cout 16) per chunk instead of 108 of
//     N = 16, and half the A-operand reads;
//   - one thread issues them (tcgen05.mma kind::f16, M 128, K 16) and commits
//     to an mbarrier, which every thread waits for (bounded) before the next
//     chunk overwrites shared memory.
// In this per-tile kernel two CTAs share an SM, so one's loads overlap the
// other's MMAs (the brick's TMA is issued before the weight copies).
// Epilogue: each warp reads its 32 TMEM lanes (tcgen05.ld 32x32b) per row,
// adds the bias, applies ReLU and stores Cout channels per voxel.
//
// The default for layers whose weights fit is the persistent kernel further
// down (conv3d_fwd_tcp): one CTA per SM walking the tiles, resident weights,
// a producer warp streaming 32-byte-swizzled bricks into two stages, an MMA
// warp and four epilogue warps draining two TMEM accumulator sets. The
// per-tile kernel remains for layers whose weights do not fit and when
// cnn_set_tensor_path(2) forces it.
#include <cuda.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "geom_dev.cuh"
#include "../../include/unet.h"

namespace bp {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTcThreads = 128;
constexpr int kBX = 130, kBY = 3, kBZ = 6;            // halo brick
constexpr int kPlaneBytes = kBX * kBY * kBZ * 16;     // one 8-channel plane (bytes a TMA load writes)
// planes start 128-byte aligned (a TMA destination must be): 37440 -> 37504
constexpr int kPlaneStride = (kPlaneBytes + 127) / 128 * 128;
constexpr int kRows = 4;                               // output rows per CTA (4 along z)
static_assert(kPlaneStride % 128 == 0 && (2 * kPlaneStride) % 128 == 0, "TMA destinations need 128-byte alignment");

// Brick of the per-tile kernel for tiles TW voxels wide (128, or 64 with
// M = 64 MMAs): TW + 2 voxels along x.
template <int TW>
struct TileGeo {
    static constexpr int BX = TW + 2;
    static constexpr int PLANE_BYTES = BX * kBY * kBZ * 16;
    static constexpr int PLANE_STRIDE = (PLANE_BYTES + 127) / 128 * 128;
    static_assert(TW == 128 || TW == 64, "tile widths 128 and 64");
};

template <int COUT, int TW = 128>
struct TcCfg {
    static constexpr int WBYTES = 27 * 2 * COUT * 16;  // weights of one 16-channel chunk
    static constexpr int TMEM_COLS = kRows * COUT;     // 64, 128 or 256 (a power of two >= 32)
    static constexpr int SMEM = 2 * TileGeo<TW>::PLANE_STRIDE + WBYTES + 1024;   // + alignment slack
};

__device__ __forceinline__ unsigned s_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (no swizzle, K-major core matrices):
// start >> 4 in bits 0-13, leading (K) byte offset >> 4 in 16-29, stride
// (M/N) byte offset >> 4 in 32-45, descriptor version 1 in bits 46-47.
__device__ __forceinline__ unsigned long long smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
template <int N>
__device__ __forceinline__ unsigned idesc_bf16() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(128 >> 4) << 24);
}

__device__ __forceinline__ void tma_load_5d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            int c4, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(s_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4),
        "r"(s_u32(bar))
        : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s_u32(dst)), "l"(src) : "memory");
}

template <int N>
struct TmemRow;
template <>
struct TmemRow<16> {
    __device__ __forceinline__ static void load(unsigned addr, float *v) {
        unsigned r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(addr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
    }
};
template <>
struct TmemRow<32> {
    __device__ __forceinline__ static void load(unsigned addr, float *v) {
        TmemRow<16>::load(addr, v);
        TmemRow<16>::load(addr + 16, v + 16);
    }
};
template <>
struct TmemRow<64> {
    __device__ __forceinline__ static void load(unsigned addr, float *v) {
        TmemRow<32>::load(addr, v);
        TmemRow<32>::load(addr + 32, v + 32);
    }
};

// TW = 64: the tile's rows are 64 voxels (layers of width 64); each MMA has
// M = 64, whose accumulator row m sits in TMEM lane 32 (m / 16) + m % 16,
// so every epilogue warp finds its 16 rows in its first 16 lanes.
template <int COUT, bool OUT_F32, int TW>
__global__ void __launch_bounds__(kTcThreads, 2)
conv3d_fwd_tc(const __grid_constant__ CUtensorMap xmap, int xco, const bf16 *__restrict__ w,
              const float *__restrict__ bias, void *__restrict__ y, int ycs, int yco, int d, int h, int wd,
              int cin, int relu, unsigned *err, unsigned long long timeout_ns) {
    using Cfg = TcCfg<COUT, TW>;
    using G = TileGeo<TW>;
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base: planes, then weights
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *plane0 = smem;
    unsigned char *wsm = smem + 2 * G::PLANE_STRIDE;
    __shared__ __align__(8) unsigned long long tma_bar, mma_bar;
    __shared__ unsigned tmem_base;
    __shared__ int alive_s;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = wd / TW, nty = h, ntz = d / 4;
    int t = blockIdx.x;
    const int tx = t % ntx;
    t /= ntx;
    const int ty = t % nty;
    t /= nty;
    const int tz = t % ntz;
    const int nb = t / ntz;
    const int x0 = tx * TW, y0 = ty, z0 = tz * 4;

    if (tid == 0) {
        mbar_init(&tma_bar, 1);
        mbar_init(&mma_bar, 1);
        fence_barrier_init();
        alive_s = 1;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                     "r"(Cfg::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;
    const int nchunks = cin / 16;

    for (int ch = 0; ch < nchunks; ++ch) {
        // the brick's TMA first, so its latency overlaps the weight copies
        if (tid == 0) {
            mbar_arrive_expect_tx(&tma_bar, 2u * G::PLANE_BYTES);
            tma_load_5d(plane0, &xmap, xco + ch * 16, x0 - 1, y0 - 1, z0 - 1, nb, &tma_bar);
            tma_load_5d(plane0 + G::PLANE_STRIDE, &xmap, xco + ch * 16 + 8, x0 - 1, y0 - 1, z0 - 1, nb, &tma_bar);
        }
        // weights of this chunk: w[co][tap][16 ch + i] -> wsm[dy][dx][half][dz][co][8]
        for (int p = tid; p < 27 * 2 * COUT; p += kTcThreads) {
            const int half = p & 1, co = (p >> 1) % COUT, tap = (p >> 1) / COUT;
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
            cp_async16(wsm + ((((dy * 3 + dx) * 2 + half) * 3 + dz) * COUT + co) * 16,
                       w + ((size_t)co * 27 + tap) * cin + ch * 16 + half * 8);
        }
        asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core reads
        __syncthreads();
        if (tid == 0) {
            bool ok = mbar_wait_bounded(&tma_bar, ch & 1, timeout_ns);
            if (ok) {
                asm volatile("tcgen05.fence::after_thread_sync;");
                const unsigned pa = s_u32(plane0), wb = s_u32(wsm);
                // Brick row (z', dy) shifted by dx feeds output rows rz = z'-dz for
                // dz = 0..2: rows rz_hi = min(3, z') down to rz_lo = max(0, z'-2) in one
                // MMA with N = (rz_hi - rz_lo + 1) x Cout. Row rz's accumulator sits at
                // TMEM column (3 - rz) x Cout and its weights for that tap at block
                // (dy, dx, half, dz = z' - rz) of wsm, so D columns and B rows both
                // run with rz descending / dz ascending at uniform strides. The first
                // group (dy, dx) = (0, 0) issues z' = 3 (rows 1-3) and z' = 0 (row 0)
                // first, with accumulation off: every row starts exactly once.
#pragma unroll 1
                for (int g = 0; g < 9; ++g) {
                    const int dy = g / 3, dx = g % 3;
#pragma unroll 1
                    for (int q = 0; q < 6; ++q) {
                        const int zp = (g == 0) ? (q == 0 ? 3 : q == 1 ? 0 : q - 1 + (q >= 4 ? 1 : 0)) : q;
                        const int rz_hi = zp < 3 ? zp : 3, rz_lo = zp > 2 ? zp - 2 : 0;
                        const int nrows = rz_hi - rz_lo + 1;
                        const unsigned voff = (unsigned)((zp * kBY + dy) * G::BX + dx) * 16u;
                        const unsigned long long ad = smem_desc(pa + voff, G::PLANE_STRIDE, 128);
                        const unsigned boff = (unsigned)((((dy * 3 + dx) * 2) * 3 + (zp - rz_hi)) * COUT * 16);
                        const unsigned long long bd = smem_desc(wb + boff, 3 * COUT * 16, 128);
                        const unsigned id = (1u << 4) | (1u << 7) | (1u << 10) |
                                            ((unsigned)((nrows * COUT) >> 3) << 17) | ((unsigned)(TW >> 4) << 24);
                        const unsigned acc = (ch > 0 || g > 0 || q > 1) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                tmem + (unsigned)((3 - rz_hi) * COUT)),
                            "l"(ad), "l"(bd), "r"(id), "r"(acc));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    s_u32(&mma_bar)));
            } else {
                atomicOr(err, DEV_ERR_TIMEOUT);
                alive_s = 0;
                // the loads may still land: give them one more bounded wait before exiting
                mbar_wait_bounded(&tma_bar, ch & 1, timeout_ns);
            }
        }
        __syncthreads();
        if (!alive_s) break;
        // the MMAs of this chunk must have read shared memory before it is refilled
        if (!mbar_wait_bounded(&mma_bar, ch & 1, timeout_ns)) {
            if (tid == 0) atomicOr(err, DEV_ERR_TIMEOUT);
            alive_s = 0;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (!alive_s) break;
    }

    if (alive_s) {
        const size_t vox_row = (size_t)wd;
        // the voxel of this lane's accumulator row (TW = 64: lanes 16-31 hold none)
        const int xl = (TW == 128) ? warp * 32 + lane : warp * 16 + lane;
        const bool has_row = TW == 128 || lane < 16;
#pragma unroll 1
        for (int r = 0; r < kRows; ++r) {
            float v[COUT];
            TmemRow<COUT>::load(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((3 - r) * COUT), v);
            if (!has_row) continue;
            const int yy = y0, zz = z0 + r;
            const int xx = x0 + xl;
            const size_t vox = (((size_t)nb * d + zz) * h + yy) * vox_row + xx;
#pragma unroll
            for (int c = 0; c < COUT; ++c) {
                float o = v[c] + (bias ? __ldg(bias + c) : 0.0f);
                v[c] = (relu && o < 0.0f) ? 0.0f : o;
            }
            if constexpr (OUT_F32) {
                float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(y) + vox * ycs + yco);
#pragma unroll
                for (int c = 0; c < COUT / 4; ++c)
                    dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
            } else {
                uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<bf16 *>(y) + vox * ycs + yco);
#pragma unroll
                for (int c = 0; c < COUT / 8; ++c) {
                    uint4 q;
                    __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * c], v[8 * c + 1]);
                    __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * c + 2], v[8 * c + 3]);
                    __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * c + 4], v[8 * c + 5]);
                    __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * c + 6], v[8 * c + 7]);
                    q.x = *reinterpret_cast<unsigned *>(&h0);
                    q.y = *reinterpret_cast<unsigned *>(&h1);
                    q.z = *reinterpret_cast<unsigned *>(&h2);
                    q.w = *reinterpret_cast<unsigned *>(&h3);
                    dst[c] = q;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS));
}

// ---------------------------------------------------------------------------
// Persistent, warp-specialised version (the default where every chunk's
// weights fit in shared memory next to two brick stages): one CTA per SM
// walks tiles blockIdx.x, blockIdx.x + gridDim.x, ... so the CTAs in flight
// cover neighbouring tiles and share their bricks in L2.
//   - the weights of all chunks are copied once per CTA and stay resident;
//   - warp 4 (one lane) streams bricks into two stages by TMA, ahead of
//   - warp 5, which issues each (tile, chunk)'s 54 MMAs (fully unrolled, the
//     descriptors warp-uniform, one lane issuing) and commits the stage back
//     to the producer, and after a tile's last chunk commits its accumulator to
//   - warps 0-3, the epilogue, which drain one of two TMEM accumulator sets
//     (bias, ReLU, stores) while the MMAs of the next tile fill the other.
// Every wait is bounded; a role whose wait runs out records DEV_ERR_TIMEOUT
// and leaves its loop, the others' waits then run out in turn, and before the
// CTA exits the producer waits for its loads in flight and the MMA lane for
// its MMAs.
// ---------------------------------------------------------------------------
// Its bricks arrive by one TMA load per (tile, chunk) whose rows are a
// voxel's 16 channels (32 bytes), written with the 32-byte swizzle (the two
// 16-byte halves of each row swapped where address bit 7 is set); the A
// operand descriptors use the same swizzle mode, which the tensor core
// applies to absolute shared-memory addresses, so a brick row shifted by dx
// voxels is still a plain start-address offset. Half the L2 requests of two
// 16-byte-row planes, each of which fetched whole 32-byte sectors.
constexpr int kPStages = 2;
constexpr int kPThreads = 192;
// Swizzled brick of a tile TW voxels wide (TW + 2 voxels along x) and its
// stage: 74,880 / 75,776 bytes at TW = 128, 38,016 / 38,912 at TW = 64.
template <int TW>
struct PGeo {
    static constexpr int BX = TW + 2;
    static constexpr int BRICK = BX * kBY * kBZ * 32;
    static constexpr int STAGE = (BRICK + 1023) / 1024 * 1024;   // swizzle atoms stay aligned
    static_assert(STAGE % 1024 == 0, "stage bases must keep the swizzle pattern's alignment");
};
constexpr int kPSmemLimit = 232448;   // opt-in shared memory per block (227 KB)

template <int COUT, int TW = 128>
struct TcpCfg {
    static constexpr int WCHUNK = TcCfg<COUT>::WBYTES;
    static constexpr int TMEM_COLS = 2 * kRows * COUT;   // two accumulator sets: 128 or 256 columns
    __host__ __device__ static constexpr int smem(int nch) {
        return kPStages * PGeo<TW>::STAGE + nch * WCHUNK + 1024;
    }
};

// Epilogues of the persistent kernel: BF16 or FP32 activations, or the fused
// 1x1x1 output head (out[v] = res[v] + hb + sum_co hw[co] bf16(act(acc + b)),
// the same arithmetic and order as cnn_head1_forward on the BF16 activation).
enum { kEpiBf16 = 0, kEpiF32 = 1, kEpiHead = 2 };
struct HeadArgs {
    const float *hw, *hb, *res;
    float *out;
};

// TW = 64 (layers of width 64): M = 64 MMAs, whose accumulator row m sits in
// TMEM lane 32 (m / 16) + m % 16; epilogue warp w drains rows 16 w .. 16 w + 15
// from its first 16 lanes.
template <int COUT, int EPI, int TW = 128>
__global__ void __launch_bounds__(kPThreads, 1)
conv3d_fwd_tcp(const __grid_constant__ CUtensorMap xmap, int xco, const bf16 *__restrict__ w,
               const float *__restrict__ bias, void *__restrict__ y, int ycs, int yco, int d, int h, int wd,
               int cin, int relu, int ntiles, HeadArgs head, unsigned *err, unsigned long long timeout_ns) {
    using Cfg = TcpCfg<COUT, TW>;
    using G = PGeo<TW>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *stage0 = smem;
    unsigned char *wsm = smem + kPStages * G::STAGE;
    __shared__ __align__(8) unsigned long long full[kPStages], empty[kPStages], tfull[2], tempty[2], done_bar;
    __shared__ unsigned tmem_base;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = cin / 16;
    const int ntx = wd / TW, nty = h, ntz = d / 4;

    if (tid == 0) {
        for (int s = 0; s < kPStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 4);
        }
        mbar_init(&done_bar, 1);
        fence_barrier_init();
    }
    // every chunk's weights: w[co][tap][16 ch + i] -> wsm[ch][dy][dx][half][dz][co][8]
    for (int p = tid; p < nch * 27 * 2 * COUT; p += kPThreads) {
        const int half = p & 1, co = (p >> 1) % COUT, rest = (p >> 1) / COUT;
        const int tap = rest % 27, ch = rest / 27;
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        cp_async16(wsm + ch * Cfg::WCHUNK + ((((dy * 3 + dx) * 2 + half) * 3 + dz) * COUT + co) * 16,
                   w + ((size_t)co * 27 + tap) * cin + ch * 16 + half * 8);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core reads
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                     "r"(Cfg::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;

    if (warp == 4 && lane == 0) {
        // ---- producer: bricks by TMA into the two stages
        int s = 0;
        unsigned ph = 0;
        int issued[kPStages];   // parity of the load in flight on each stage, or -1
        for (int k = 0; k < kPStages; ++k) issued[k] = -1;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            int t = tile;
            const int tx = t % ntx;
            t /= ntx;
            const int ty = t % nty;
            t /= nty;
            const int tz = t % ntz;
            const int nb = t / ntz;
            for (int ch = 0; ch < nch; ++ch) {
                if (!mbar_wait_bounded(&empty[s], ph ^ 1u, timeout_ns)) {
                    atomicOr(err, DEV_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                mbar_arrive_expect_tx(&full[s], (unsigned)G::BRICK);
                tma_load_5d(stage0 + s * G::STAGE, &xmap, xco + ch * 16, tx * TW - 1, ty - 1, tz * 4 - 1, nb,
                            &full[s]);
                issued[s] = (int)ph;
                if (++s == kPStages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
        }
        // loads still in flight must land before the CTA leaves (they complete
        // on their own; the MMA lane may have consumed some of them already)
        for (int k = 0; k < kPStages; ++k)
            if (issued[k] >= 0) mbar_wait_bounded(&full[k], (unsigned)issued[k], timeout_ns);
    } else if (warp == 5) {
        // ---- MMA issue. The whole warp runs the loop so that every descriptor
        // is warp-uniform (computed on the uniform datapath, with the schedule's
        // offsets folded into constants by the full unroll); lane 0 waits,
        // issues and commits.
        const bool leader = lane == 0;
        int s = 0, a = 0;
        unsigned ph = 0, aph = 0;
        // A: 32-byte swizzle (mode 6 in bits 61-63), 8-row groups 256 bytes apart, LBO unused (1)
        const unsigned long long lbo_sbo_a = (1ull << 16) | ((unsigned long long)(256 >> 4) << 32) | (1ull << 46) |
                                             (6ull << 61);
        const unsigned long long lbo_sbo_b =
            ((unsigned long long)(((3 * COUT * 16) >> 4) & 0x3FFF) << 16) | ((unsigned long long)(128 >> 4) << 32) |
            (1ull << 46);
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            int okw = leader ? (mbar_wait_bounded(&tempty[a], aph ^ 1u, timeout_ns) ? 1 : 0) : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) {
                if (leader) atomicOr(err, DEV_ERR_TIMEOUT);
                break;
            }
            __syncwarp();
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned dbase = tmem + (unsigned)(a * kRows * COUT);
            for (int ch = 0; ch < nch; ++ch) {
                okw = leader ? (mbar_wait_bounded(&full[s], ph, timeout_ns) ? 1 : 0) : 0;
                okw = __shfl_sync(0xffffffffu, okw, 0);
                if (!okw) {
                    if (leader) atomicOr(err, DEV_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                __syncwarp();
                asm volatile("tcgen05.fence::after_thread_sync;");
                const unsigned a0 = s_u32(stage0 + s * G::STAGE) >> 4;
                const unsigned b0 = s_u32(wsm + ch * Cfg::WCHUNK) >> 4;
                const unsigned first_acc = ch > 0 ? 1u : 0u;
#pragma unroll
                for (int g = 0; g < 9; ++g) {
                    const int dy = g / 3, dx = g % 3;
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        const int zp = (g == 0) ? (q == 0 ? 3 : q == 1 ? 0 : q - 1 + (q >= 4 ? 1 : 0)) : q;
                        const int rz_hi = zp < 3 ? zp : 3, rz_lo = zp > 2 ? zp - 2 : 0;
                        const int nrows = rz_hi - rz_lo + 1;
                        const unsigned a16 = (unsigned)(2 * ((zp * kBY + dy) * G::BX + dx));
                        const unsigned b16 = (unsigned)(((((dy * 3 + dx) * 2) * 3 + (zp - rz_hi)) * COUT * 16) >> 4);
                        const unsigned id = (1u << 4) | (1u << 7) | (1u << 10) |
                                            ((unsigned)((nrows * COUT) >> 3) << 17) | ((unsigned)(TW >> 4) << 24);
                        const unsigned acc = (g == 0 && q <= 1) ? first_acc : 1u;
                        const unsigned long long ad = lbo_sbo_a | (unsigned long long)((a0 + a16) & 0x3FFF);
                        const unsigned long long bd = lbo_sbo_b | (unsigned long long)((b0 + b16) & 0x3FFF);
                        if (leader)
                            asm volatile(
                                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                    dbase + (unsigned)((3 - rz_hi) * COUT)),
                                "l"(ad), "l"(bd), "r"(id), "r"(acc));
                    }
                }
                // the stage is free once these MMAs have read it
                if (leader)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        s_u32(&empty[s])));
                __syncwarp();
                if (++s == kPStages) {
                    s = 0;
                    ph ^= 1u;
                }
            }
            if (!ok) break;
            if (leader)
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    s_u32(&tfull[a])));
            __syncwarp();
            if (++a == 2) {
                a = 0;
                aph ^= 1u;
            }
        }
        // every MMA issued must be complete before the accumulators are freed
        if (leader) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                s_u32(&done_bar)));
            if (!mbar_wait_bounded(&done_bar, 0, timeout_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---- epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (voxels x0 + 32 w + lane)
        int a = 0;
        unsigned aph = 0;
        float bv[COUT], hwv[COUT];
#pragma unroll
        for (int c = 0; c < COUT; ++c) {
            bv[c] = bias ? __ldg(bias + c) : 0.0f;
            hwv[c] = EPI == kEpiHead ? __ldg(head.hw + c) : 0.0f;
        }
        const float hb = (EPI == kEpiHead && head.hb) ? __ldg(head.hb) : 0.0f;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            int okw = 0;
            if (lane == 0) okw = mbar_wait_bounded(&tfull[a], aph, timeout_ns) ? 1 : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) {
                if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                break;
            }
            __syncwarp();
            asm volatile("tcgen05.fence::after_thread_sync;");
            int t = tile;
            const int tx = t % ntx;
            t /= ntx;
            const int ty = t % nty;
            t /= nty;
            const int tz = t % ntz;
            const int nb = t / ntz;
            const int xx = tx * TW + (TW == 128 ? warp * 32 + lane : warp * 16 + lane);
#pragma unroll 1
            for (int r = 0; r < kRows; ++r) {
                float v[COUT];
                TmemRow<COUT>::load(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(a * kRows * COUT + (3 - r) * COUT),
                                    v);
                if (TW == 64 && lane >= 16) continue;   // M = 64: rows in the first 16 lanes only
                const size_t vox = (((size_t)nb * d + tz * 4 + r) * h + ty) * (size_t)wd + xx;
#pragma unroll
                for (int c = 0; c < COUT; ++c) {
                    const float o = v[c] + bv[c];
                    v[c] = (relu && o < 0.0f) ? 0.0f : o;
                }
                if constexpr (EPI == kEpiF32) {
                    float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(y) + vox * ycs + yco);
#pragma unroll
                    for (int c = 0; c < COUT / 4; ++c)
                        dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                } else if constexpr (EPI == kEpiHead) {
                    float o = 0.0f;
#pragma unroll
                    for (int c = 0; c < COUT; ++c) o = fmaf(hwv[c], __bfloat162float(__float2bfloat16_rn(v[c])), o);
                    head.out[vox] = o + hb + (head.res ? head.res[vox] : 0.0f);
                } else {
                    uint4 *dst = reinterpret_cast<uint4 *>(reinterpret_cast<bf16 *>(y) + vox * ycs + yco);
#pragma unroll
                    for (int c = 0; c < COUT / 8; ++c) {
                        uint4 q;
                        __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * c], v[8 * c + 1]);
                        __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * c + 2], v[8 * c + 3]);
                        __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * c + 4], v[8 * c + 5]);
                        __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * c + 6], v[8 * c + 7]);
                        q.x = *reinterpret_cast<unsigned *>(&h0);
                        q.y = *reinterpret_cast<unsigned *>(&h1);
                        q.z = *reinterpret_cast<unsigned *>(&h2);
                        q.w = *reinterpret_cast<unsigned *>(&h3);
                        dst[c] = q;
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[a]);
            if (++a == 2) {
                a = 0;
                aph ^= 1u;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 5) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// The one-channel input layer (3x3x3, 1 -> 16 channels) on tcgen05, for widths
// that are multiples of 8. With one input channel the usual implicit GEMM
// (K = channels of a tap) would spend 15/16 of its products on zero channels;
// here the taps along x go into K instead. A tile is 8 outputs along x,
// 128 along y and 2 along z. Every staged input row holds the 16 values
// x0 - 4 .. x0 + 11 (K), and the weights of each (kz, ky) become a banded
// matrix B[16 xo + c][j] = w[c][kz][ky][j - xo - 3] (zero off the band), so
//   D[y][16 xo + c] += A_(z, kz, ky)[y][j] B_(kz, ky)[16 xo + c][j]
// with M = 128 rows along y, N = 128 (8 voxels x 16 channels), K = 16: nine
// MMAs per output slice, 2304 products per voxel for the 432 of the tap sum.
// K slots 0 and 1 (outside every output's taps) are staged as 1.0 and carry
// the bias (hi and lo BF16 parts) in the weights of (kz, ky) = (0, 0).
// A TMEM lane is one y row, so an epilogue thread holds all 16 channels of
// its voxels: whole-voxel stores, and the 2 x 2 x 2 pooling needs one lane
// shuffle (the y pair); the x pair and the z pair are its own columns.
//
// Persistent and warp-specialised, one CTA per SM: a tile's FP32 input
// (16 x 130 x 4 values, zero outside the volume) arrives by one TMA load two
// tiles ahead into one of two staging buffers; four producer warps round it
// to BF16 into one of two A buffers; one thread issues the MMAs into one of
// two TMEM accumulator sets
// (256 columns each), committing each output slice separately; eight
// epilogue warps drain a slice (ReLU in the BF16 conversion), stage each
// warp's 32 rows in shared memory and store them transposed (four whole
// 128-byte lines per instruction). Loads, MMAs and stores of successive
// tiles overlap; every wait is bounded.
constexpr int kSxT = 8, kSyT = 128, kSzT = 2;
constexpr int kSRows = kSyT + 2;                          // staged rows per plane (y halo)
constexpr int kSPlanes = kSzT + 2;                        // staged planes (z halo)
constexpr int kSHalf = kSPlanes * kSRows * 16;            // bytes of one 8-value K half: 8320
constexpr int kSABytes = 2 * kSHalf;                      // one staged input tile (A): 16640
constexpr int kSBBytes = 9 * 2 * 128 * 16;                // banded weights (B): 36864
constexpr int kSEpiWarps = 8, kSProdWarps = 4;
constexpr int kSThreads = (kSEpiWarps + kSProdWarps + 1) * 32;   // + the MMA warp: 416
constexpr int kSCBytes = kSEpiWarps * 32 * 128;           // epilogue staging: 32 rows x 128 bytes a warp
constexpr int kSChunks = kSPlanes * kSRows * 4;           // float4 chunks of a staged tile: 2080
constexpr int kSPer = (kSChunks + kSProdWarps * 32 - 1) / (kSProdWarps * 32);   // 17 per producer thread
constexpr int kSFBytes = kSChunks * 16;                   // one FP32 input tile as the TMA writes it: 33280
// one CTA per SM (it holds all 512 TMEM columns)
constexpr int kSSmem = 2 * kSFBytes + 2 * kSABytes + kSBBytes + kSCBytes + 128;
static_assert(kSSmem <= 227 * 1024, "stem buffers exceed the shared memory of a CTA");
static_assert(kSFBytes % 128 == 0, "TMA destinations start 128-byte aligned");
static_assert(2 * (kSSmem + 2048) > 228 * 1024, "a second CTA per SM would wait for tensor memory");
static_assert(kSHalf % 16 == 0 && kSABytes % 128 == 0, "operand buffers start 16-byte aligned");

__device__ __forceinline__ void tmem_ld32(unsigned addr, float *v) {
    unsigned r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// (lo, hi) rounded to BF16 and packed (lo in the low half); with RELU a
// negative result becomes +0 (max(x, 0) commutes with the rounding).
template <bool RELU>
__device__ __forceinline__ unsigned cvt_bf16x2(float lo, float hi) {
    unsigned r;
    if constexpr (RELU)
        asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    else
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ unsigned max_bf16x2(unsigned a, unsigned b) {
    unsigned r;
    asm("max.bf16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}

__device__ __forceinline__ unsigned bf16x2_bits(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<unsigned *>(&h);
}

struct StemTile {
    int tx, ty, tz;
    long long nb;
};
__device__ __forceinline__ StemTile stem_tile(int t, int ntx, int nty, int ntz) {
    StemTile r;
    r.tx = t % ntx;
    t /= ntx;
    r.ty = t % nty;
    t /= nty;
    r.tz = t % ntz;
    r.nb = t / ntz;
    return r;
}

template <bool POOL, bool RELU>
__global__ void __launch_bounds__(kSThreads, 1)
stem_fwd_tc(const __grid_constant__ CUtensorMap xmap, const bf16 *__restrict__ w, const float *__restrict__ b,
            bf16 *__restrict__ y, int ycs, int yco, bf16 *__restrict__ pooled, int D, int H, int W,
            int ntiles, unsigned *err, unsigned long long timeout_ns) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    unsigned char *Fs = smem;                  // two of [plane][row][16 FP32]: the input as loaded
    unsigned char *As = Fs + 2 * kSFBytes;     // two of [half][plane][row][8 BF16]: staged input
    unsigned char *Bs = As + 2 * kSABytes;     // [kz ky][half][16 xo + c][8 BF16]: banded weights
    unsigned char *Cs = Bs + kSBBytes;         // per epilogue warp [row][8 x 16 bytes], slots XOR-swizzled by row
    __shared__ __align__(8) unsigned long long f_full[2], a_full[2], a_empty[2], t_full[2][kSzT], t_empty[2],
        done_bar;
    __shared__ unsigned tmem_base;
    __shared__ float wsm[16 * 27];
    __shared__ float bsm[16];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntx = W / kSxT, nty = (H + kSyT - 1) / kSyT, ntz = (D + kSzT - 1) / kSzT;
    const int mma_warp = kSEpiWarps + kSProdWarps;

    for (int i = tid; i < 16 * 27; i += kSThreads) wsm[i] = __bfloat162float(w[i]);
    if (tid < 16) bsm[tid] = b ? b[tid] : 0.0f;
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            mbar_init(&f_full[s], 1);
            mbar_init(&a_full[s], kSProdWarps * 32);
            mbar_init(&a_empty[s], 1);
            mbar_init(&t_empty[s], kSEpiWarps);
            for (int zz = 0; zz < kSzT; ++zz) mbar_init(&t_full[s][zz], 1);
        }
        mbar_init(&done_bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    // banded weights: 16-byte row (g = 3 kz + ky, half, n = 16 xo + c) holds j = 8 half .. 8 half + 7;
    // the band uses j = 3 .. 12, and j = 0, 1 of (kz, ky) = (0, 0) hold the bias as
    // hi = bf16(b) and lo = bf16(b - hi) (within 2^-16 of b)
    for (int q = tid; q < 9 * 2 * 128; q += kSThreads) {
        const int nn = q & 127, half = (q >> 7) & 1, g = q >> 8;
        const int xo = nn >> 4, c = nn & 15;
        const float bhi = __bfloat162float(__float2bfloat16_rn(bsm[c]));
        const float blo = __bfloat162float(__float2bfloat16_rn(bsm[c] - bhi));
        unsigned v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j0 = 8 * half + 2 * e, k0 = j0 - xo - 3, k1 = k0 + 1;
            float f0 = (k0 >= 0 && k0 < 3) ? wsm[c * 27 + g * 3 + k0] : 0.0f;
            float f1 = (k1 >= 0 && k1 < 3) ? wsm[c * 27 + g * 3 + k1] : 0.0f;
            if (g == 0 && j0 == 0) {
                f0 = bhi;
                f1 = blo;
            }
            v[e] = bf16x2_bits(f0, f1);
        }
        *reinterpret_cast<uint4 *>(Bs + q * 16) = make_uint4(v[0], v[1], v[2], v[3]);
    }
    if (warp == mma_warp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_u32(&tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor core reads
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;

    if (warp >= kSEpiWarps && warp < mma_warp) {
        // ---- producers: thread p rounds float4 chunks q = p + 128 i of the loaded
        // tile (row q / 4, K values 4 (q mod 4) .. + 3) into the A buffer
        const int p = tid - kSEpiWarps * 32;
        const bool leader = p == 0;
        auto issue = [&](int tile, int fs) {
            const StemTile T = stem_tile(tile, ntx, nty, ntz);
            mbar_arrive_expect_tx(&f_full[fs], (unsigned)kSFBytes);
            tma_load_4d(Fs + fs * kSFBytes, &xmap, T.tx * kSxT - 4, T.ty * kSyT - 1, T.tz * kSzT - 1, (int)T.nb,
                        &f_full[fs]);
        };
        if (leader) {
            for (int k = 0; k < 2; ++k)
                if (blockIdx.x + k * (int)gridDim.x < ntiles) issue(blockIdx.x + k * gridDim.x, k);
        }
        int s = 0, k = 0;
        unsigned ph = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++k) {
            const int fs = k & 1;
            if (!mbar_wait_bounded(&f_full[fs], (unsigned)(k >> 1) & 1u, timeout_ns) ||
                !mbar_wait_bounded(&a_empty[s], ph ^ 1u, timeout_ns)) {
                atomicOr(err, DEV_ERR_TIMEOUT);
                ok = false;
            }
            // the producers leave together if any wait ran out (they meet on named barrier 1)
            unsigned any_out;
            asm volatile(
                "{\n .reg .pred q, r;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred r, 1, %2, q;\n"
                " selp.u32 %0, 1, 0, r;\n}"
                : "=r"(any_out)
                : "r"(ok ? 0u : 1u), "r"(kSProdWarps * 32));
            if (any_out) {
                ok = false;
                break;
            }
            const unsigned char *F = Fs + fs * kSFBytes;
            unsigned char *A = As + s * kSABytes;
#pragma unroll
            for (int i = 0; i < kSPer; ++i) {
                const int q = p + kSProdWarps * 32 * i;
                if (q < kSChunks) {
                    const float4 v = *reinterpret_cast<const float4 *>(F + q * 16);
                    const int row = q >> 2, part = q & 3;
                    const unsigned a = s_u32(A + (part >> 1) * kSHalf + row * 16 + (part & 1) * 8);
                    // K slots 0 and 1 (values x0 - 4, x0 - 3, outside every output's taps) hold 1.0
                    const unsigned lo = part == 0 ? 0x3F803F80u : bf16x2_bits(v.x, v.y);
                    asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(a), "r"(lo), "r"(bf16x2_bits(v.z, v.w))
                                 : "memory");
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&a_full[s]);
            // the loaded buffer is read by every producer: reload it two tiles ahead
            asm volatile("bar.sync 1, %0;" ::"r"(kSProdWarps * 32));
            if (leader && tile + 2 * (int)gridDim.x < ntiles) issue(tile + 2 * gridDim.x, fs);
            s ^= 1;
            ph ^= (unsigned)(s == 0);
        }
        // loads still in flight land before the CTA leaves
        if (leader) {
            for (int kk = k; kk < k + 2; ++kk)
                if (blockIdx.x + kk * (int)gridDim.x < ntiles)
                    mbar_wait_bounded(&f_full[kk & 1], (unsigned)(kk >> 1) & 1u, timeout_ns);
        }
    } else if (warp == mma_warp) {
        // ---- MMA issue (lane 0): 9 MMAs per output slice, each slice committed on its own
        if (lane == 0) {
            int s = 0, a = 0;
            unsigned ph = 0, aph = 0;
            const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(128 >> 3) << 17) |
                                   ((unsigned)(128 >> 4) << 24);
            const unsigned b_base = s_u32(Bs);
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                if (!mbar_wait_bounded(&t_empty[a], aph ^ 1u, timeout_ns) ||
                    !mbar_wait_bounded(&a_full[s], ph, timeout_ns)) {
                    atomicOr(err, DEV_ERR_TIMEOUT);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const unsigned a_base = s_u32(As + s * kSABytes);
#pragma unroll
                for (int zz = 0; zz < kSzT; ++zz) {
#pragma unroll
                    for (int g = 0; g < 9; ++g) {
                        const int kz = g / 3, ky = g % 3;
                        // A: no swizzle, K halves kSHalf apart (LBO), 8-row groups 128 bytes apart (SBO)
                        const unsigned long long ad = smem_desc(a_base + ((zz + kz) * kSRows + ky) * 16, kSHalf, 128);
                        const unsigned long long bd = smem_desc(b_base + g * 4096, 2048, 128);
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(
                                tmem + (unsigned)(a * 256 + zz * 128)),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(g > 0 ? 1u : 0u));
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                        s_u32(&t_full[a][zz])));
                }
                // the A buffer is free once these MMAs have read it
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    s_u32(&a_empty[s])));
                s ^= 1;
                ph ^= (unsigned)(s == 0);
                a ^= 1;
                aph ^= (unsigned)(a == 0);
            }
            // every MMA issued must be complete before the accumulators are freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                s_u32(&done_bar)));
            if (!mbar_wait_bounded(&done_bar, 0, timeout_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w drains TMEM lanes 32 (w mod 4) .. (rows y0 + 32 (w mod 4) + lane)
        // and voxels 4 (w / 4) .. 4 (w / 4) + 3 of the tile
        const int quarter = warp & 3, xh = warp >> 2;
        unsigned char *cw = Cs + warp * 4096;
        int a = 0;
        unsigned aph = 0;
        bool ok = true;
        for (int tile = blockIdx.x; ok && tile < ntiles; tile += gridDim.x) {
            const StemTile T = stem_tile(tile, ntx, nty, ntz);
            const int yy = T.ty * kSyT + 32 * quarter + lane;
            const int x0w = T.tx * kSxT + 4 * xh;   // first voxel of the warp's rows
            unsigned mx[2][8];                      // running maxima of the pooling windows, BF16 pairs
#pragma unroll 1
            for (int zz = 0; zz < kSzT; ++zz) {
                int okw = lane == 0 ? (mbar_wait_bounded(&t_full[a][zz], aph, timeout_ns) ? 1 : 0) : 0;
                okw = __shfl_sync(0xffffffffu, okw, 0);
                if (!okw) {
                    if (lane == 0) atomicOr(err, DEV_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                __syncwarp();
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int z = T.tz * kSzT + zz;
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {   // voxels 4 xh + 2 pp, + 1
                    float v[32];
                    tmem_ld32(tmem + ((unsigned)(32 * quarter) << 16) +
                                  (unsigned)(a * 256 + zz * 128 + (4 * xh + 2 * pp) * 16),
                              v);
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        unsigned q[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            q[k] = cvt_bf16x2<RELU>(v[16 * e + 2 * k], v[16 * e + 2 * k + 1]);
                            if constexpr (POOL) mx[pp][k] = (zz == 0 && e == 0) ? q[k] : max_bf16x2(mx[pp][k], q[k]);
                        }
                        const int xo = 2 * pp + e;
                        const int s0 = (2 * xo) ^ (lane & 7), s1 = (2 * xo + 1) ^ (lane & 7);
                        *reinterpret_cast<uint4 *>(cw + lane * 128 + s0 * 16) = make_uint4(q[0], q[1], q[2], q[3]);
                        *reinterpret_cast<uint4 *>(cw + lane * 128 + s1 * 16) = make_uint4(q[4], q[5], q[6], q[7]);
                    }
                }
                __syncwarp();
                // 8 lanes per row, 4 rows (128-byte lines) per store instruction
                const int k = lane & 7;
                bf16 *yrow = y + (((T.nb * D + z) * H + T.ty * kSyT + 32 * quarter) * (long long)W + x0w + (k >> 1)) *
                                     ycs + yco + (k & 1) * 8;
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                    const int r = 4 * it + (lane >> 3);   // row of the warp
                    const uint4 val = *reinterpret_cast<const uint4 *>(cw + r * 128 + ((k ^ (r & 7)) * 16));
                    if (T.ty * kSyT + 32 * quarter + r < H && z < D)
                        *reinterpret_cast<uint4 *>(yrow + (long long)r * W * ycs) = val;
                }
                __syncwarp();   // the staging rows are rewritten for the next slice
            }
            if (!ok) break;
            // this accumulator set is read: the MMAs of a later tile may overwrite it
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[a]);
            a ^= 1;
            aph ^= (unsigned)(a == 0);
            if constexpr (POOL) {
                // the y pair is lanes l and l ^ 1 (D, H even: a pair is whole or outside)
#pragma unroll
                for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                    for (int k = 0; k < 8; ++k)
                        mx[pp][k] = max_bf16x2(mx[pp][k], __shfl_xor_sync(0xffffffffu, mx[pp][k], 1));
                if (yy < H && (lane & 1) == 0) {
                    const int Dh = D >> 1, Hh = H >> 1, Wh = W >> 1;
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        uint4 *dst = reinterpret_cast<uint4 *>(
                            pooled + (((T.nb * Dh + T.tz) * Hh + (yy >> 1)) * (long long)Wh + (x0w >> 1) + pp) * 16);
                        dst[0] = make_uint4(mx[pp][0], mx[pp][1], mx[pp][2], mx[pp][3]);
                        dst[1] = make_uint4(mx[pp][4], mx[pp][5], mx[pp][6], mx[pp][7]);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == mma_warp) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
}

typedef CUresult (*PFN_encode5)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encode5 encode_fn() {
    static PFN_encode5 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encode5>(p);
    }
    return fn;
}

// Device error word of the tensor-core convolutions (bounded waits).
__device__ unsigned g_tc_err;

}  // namespace

static std::mutex g_tc_mu;
static unsigned *g_tc_err_addr[64] = {};
// 1 (default): tcgen05 wherever its tile applies; 0: mma.sync only
// 2: the per-tile tcgen05 kernel only (no persistent kernel)
static int g_tc_mode = 1;
static int g_num_sms[64] = {};

static cudaError_t tc_err_address(unsigned **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_tc_mu);
    if (!g_tc_err_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tc_err);
        if (e != cudaSuccess) return e;
        g_tc_err_addr[dev] = static_cast<unsigned *>(p);
    }
    *out = g_tc_err_addr[dev];
    return cudaSuccess;
}

// Streaming multiprocessors of the current device (cached per device).
static cudaError_t sm_count(int *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!g_num_sms[dev]) {
        int v = 0;
        e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_num_sms[dev] = v > 0 ? v : 1;
    }
    *out = g_num_sms[dev];
    return cudaSuccess;
}

// The tensor-core path applies when the depth is a multiple of 4, Cin a
// multiple of 16, every pointer, stride and offset 16-byte aligned, and
// either the width is a multiple of 128 with Cout 16 or 32 (tiles of 128
// voxels), or the width is a multiple of 64 but not of 128 with Cout 16, 32
// or 64 (tiles of 64 voxels, M = 64 MMAs).
bool conv_tc_applies(const void *x, int xcs, int xco, const void *w, const void *y, int ycs, int yco, int yf32,
                     int d, int h, int wd, int cin, int cout) {
    (void)yf32;
    const bool t128 = wd % 128 == 0 && (cout == 16 || cout == 32);
    const bool t64 = wd % 128 != 0 && wd % 64 == 0 && (cout == 16 || cout == 32 || cout == 64);
    return (g_tc_mode == 1 || g_tc_mode == 2) && (t128 || t64) && cin % 16 == 0 && cin > 0 && wd > 0 &&
           d % 4 == 0 && h > 0 && d > 0 && xcs % 8 == 0 && xco % 8 == 0 && ycs % 8 == 0 && yco % 8 == 0 &&
           (reinterpret_cast<uintptr_t>(x) & 15) == 0 && (reinterpret_cast<uintptr_t>(w) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(y) & 15) == 0 && encode_fn() != nullptr;
}

// Does the persistent kernel take this layer (it alone has the fused head)?
bool conv_tcp_applies(int cin, int cout) {
    if (g_tc_mode != 1 || (cout != 16 && cout != 32) || cin % 16 || cin < 16) return false;
    const int nch = cin / 16;
    return (cout == 16 ? TcpCfg<16>::smem(nch) : TcpCfg<32>::smem(nch)) <= kPSmemLimit;
}

cudaError_t conv_fwd_tc(const void *x, int xcs, int xco, const void *w, const float *b, void *y, int ycs, int yco,
                        int yf32, int n, int d, int h, int wd, int cin, int cout, int relu, cudaStream_t st,
                        const float *head_w, const float *head_b, const float *head_res, float *head_out) {
    const bool fused_head = head_out != nullptr;
    const int TW = wd % 128 == 0 ? 128 : 64;   // tile width (conv_tc_applies checked the rest)
    if (fused_head && (TW != 128 || !conv_tcp_applies(cin, cout))) return cudaErrorNotSupported;
    unsigned *err = nullptr;
    cudaError_t ea = tc_err_address(&err);
    if (ea != cudaSuccess) return ea;
    CUtensorMap map;
    const cuuint64_t es = 2;
    cuuint64_t dims[5] = {(cuuint64_t)xcs, (cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)d, (cuuint64_t)n};
    cuuint64_t strides[4] = {(cuuint64_t)xcs * es, (cuuint64_t)xcs * wd * es, (cuuint64_t)xcs * wd * h * es,
                             (cuuint64_t)xcs * wd * h * d * es};
    cuuint32_t box[5] = {8, (cuuint32_t)(TW + 2), (cuuint32_t)kBY, (cuuint32_t)kBZ, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(x), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const long long nblk = (long long)n * (d / 4) * h * (wd / TW);
    if (nblk <= 0) return cudaSuccess;
    if (nblk > 0x7fffffffLL) return cudaErrorInvalidValue;
    const unsigned long long timeout_ns = 2000000000ull;
    const int nch = cin / 16;
    // the persistent kernel keeps every chunk's weights resident; Cout 64
    // (width-64 layers) runs in one launch where all 64 channels' weights fit
    // beside the bricks (Cin 32), otherwise as two launches of 32 output
    // channels, each writing its channel slice (the bricks stay in L2 between them)
    const bool one64 = cout == 64 && TW == 64 && TcpCfg<64, 64>::smem(nch) <= kPSmemLimit;
    const int cpl = cout == 64 && !one64 ? 32 : cout;   // output channels per launch
    const int psmem = TW == 128 ? (cpl == 16 ? TcpCfg<16, 128>::smem(nch) : TcpCfg<32, 128>::smem(nch))
                                : (cpl == 16 ? TcpCfg<16, 64>::smem(nch)
                                             : cpl == 32 ? TcpCfg<32, 64>::smem(nch) : TcpCfg<64, 64>::smem(nch));
    if (g_tc_mode == 1 && psmem <= kPSmemLimit && (TW == 64 || cout != 64)) {
        // rows of 16 channels (32 bytes), 32-byte swizzle
        cuuint32_t box16[5] = {16, (cuuint32_t)(TW + 2), (cuuint32_t)kBY, (cuuint32_t)kBZ, 1};
        r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void *>(x), dims, strides, box16, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
        int sms = 0;
        cudaError_t e = sm_count(&sms);
        if (e != cudaSuccess) return e;
        const unsigned grid = (unsigned)(nblk < sms ? nblk : sms);
        const HeadArgs ha{head_w, head_b, head_res, head_out};
#define TCP_CASE(C, E, T)                                                                                       \
    {                                                                                                           \
        auto k = conv3d_fwd_tcp<C, E, T>;                                                                       \
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, psmem);                        \
        if (e != cudaSuccess) return e;                                                                         \
        for (int c0 = 0; c0 < cout; c0 += C) {                                                                  \
            k<<<grid, kPThreads, psmem, st>>>(map, xco, (const bf16 *)w + (size_t)c0 * 27 * cin, b ? b + c0 : b, \
                                              y, ycs, yco + c0, d, h, wd, cin, relu, (int)nblk, ha, err,        \
                                              timeout_ns);                                                      \
            e = cudaGetLastError();                                                                             \
            if (e != cudaSuccess) return e;                                                                     \
        }                                                                                                       \
        return cudaSuccess;                                                                                     \
    }
        if (TW == 128) {
            if (cpl == 16) {
                if (fused_head) TCP_CASE(16, kEpiHead, 128) else if (yf32) TCP_CASE(16, kEpiF32, 128) else TCP_CASE(16, kEpiBf16, 128)
            } else {
                if (fused_head) TCP_CASE(32, kEpiHead, 128) else if (yf32) TCP_CASE(32, kEpiF32, 128) else TCP_CASE(32, kEpiBf16, 128)
            }
        } else {
            if (cpl == 64) {
                if (yf32) TCP_CASE(64, kEpiF32, 64) else TCP_CASE(64, kEpiBf16, 64)
            } else if (cpl == 16) {
                if (yf32) TCP_CASE(16, kEpiF32, 64) else TCP_CASE(16, kEpiBf16, 64)
            } else {
                if (yf32) TCP_CASE(32, kEpiF32, 64) else TCP_CASE(32, kEpiBf16, 64)
            }
        }
#undef TCP_CASE
    }
#define TC_CASE(C, F, T)                                                                                        \
    {                                                                                                           \
        auto k = conv3d_fwd_tc<C, F, T>;                                                                        \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<C, T>::SMEM); \
        if (e != cudaSuccess) return e;                                                                         \
        k<<<(unsigned)nblk, kTcThreads, TcCfg<C, T>::SMEM, st>>>(map, xco, (const bf16 *)w, b, y, ycs, yco, d, h, \
                                                                 wd, cin, relu, err, timeout_ns);               \
        return cudaGetLastError();                                                                              \
    }
    if (TW == 128) {
        if (cout == 16) {
            if (yf32) TC_CASE(16, true, 128) else TC_CASE(16, false, 128)
        } else {
            if (yf32) TC_CASE(32, true, 128) else TC_CASE(32, false, 128)
        }
    } else {
        if (cout == 16) {
            if (yf32) TC_CASE(16, true, 64) else TC_CASE(16, false, 64)
        } else if (cout == 32) {
            if (yf32) TC_CASE(32, true, 64) else TC_CASE(32, false, 64)
        } else {
            if (yf32) TC_CASE(64, true, 64) else TC_CASE(64, false, 64)
        }
    }
#undef TC_CASE
}

// The tcgen05 input layer takes Cout 16 at widths that are multiples of 8,
// with 16-byte aligned tensors and channel offsets, unless
// cnn_set_tensor_path(0) selects mma.sync.
bool stem_tc_applies(const float *x, const void *y, int ycs, int yco, const void *pooled, int wd, int cout) {
    return g_tc_mode != 0 && cout == 16 && wd >= kSxT && wd % kSxT == 0 && ycs % 8 == 0 && yco % 8 == 0 &&
           (reinterpret_cast<uintptr_t>(x) & 15) == 0 && (reinterpret_cast<uintptr_t>(y) & 15) == 0 &&
           (reinterpret_cast<uintptr_t>(pooled) & 15) == 0;
}

cudaError_t stem_fwd_tc_launch(const float *x, const void *w, const float *b, void *y, int ycs, int yco,
                               void *pooled, int n, int d, int h, int wd, int relu, cudaStream_t st) {
    unsigned *err = nullptr;
    cudaError_t e = tc_err_address(&err);
    if (e != cudaSuccess) return e;
    const long long nt = (long long)n * (wd / kSxT) * ((h + kSyT - 1) / kSyT) * ((d + kSzT - 1) / kSzT);
    if (nt <= 0) return cudaSuccess;
    if (nt > 0x7fffffffLL) return cudaErrorInvalidValue;
    int sms = 0;
    e = sm_count(&sms);
    if (e != cudaSuccess) return e;
    const unsigned grid = (unsigned)(nt < sms ? nt : sms);   // one CTA per SM
    // the input as a 4-D FP32 tensor (x, y, z, batch); a box is one tile with
    // its halo, zero outside the volume
    if (!encode_fn()) return cudaErrorNotSupported;
    CUtensorMap map;
    cuuint64_t dims[4] = {(cuuint64_t)wd, (cuuint64_t)h, (cuuint64_t)d, (cuuint64_t)n};
    cuuint64_t strides[3] = {(cuuint64_t)wd * 4, (cuuint64_t)wd * h * 4, (cuuint64_t)wd * h * d * 4};
    cuuint32_t box[4] = {16, (cuuint32_t)kSRows, (cuuint32_t)kSPlanes, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float *>(x), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    auto k = pooled ? (relu ? stem_fwd_tc<true, true> : stem_fwd_tc<true, false>)
                    : (relu ? stem_fwd_tc<false, true> : stem_fwd_tc<false, false>);
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kSSmem);
    if (e != cudaSuccess) return e;
    k<<<grid, kSThreads, kSSmem, st>>>(map, (const bf16 *)w, b, (bf16 *)y, ycs, yco, (bf16 *)pooled, d, h, wd,
                                       (int)nt, err, 2000000000ull);
    return cudaGetLastError();
}

}  // namespace bp

using namespace bp;

extern "C" {

bp_status cnn_set_tensor_path(int mode) {
    if (mode < 0 || mode > 2) return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_set_tensor_path: mode must be 0, 1 or 2");
    g_tc_mode = mode;
    return BP_OK;
}

bp_status cnn_device_status(void *stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cnn_device_status: stream synchronise");
    unsigned *err = nullptr;
    e = tc_err_address(&err);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cnn_device_status: error word");
    unsigned v = 0;
    e = cudaMemcpy(&v, err, sizeof(v), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0) e = cudaMemset(err, 0, sizeof(v));
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cnn_device_status: read");
    if (v & DEV_ERR_TIMEOUT) return fail(nullptr, BP_ERR_TIMEOUT, "tensor-core convolution: a bounded wait ran out");
    if (v) return fail(nullptr, BP_ERR_DEVICE, "tensor-core convolution: device error");
    return BP_OK;
}

}  // extern "C"
