// The one-channel input layer and the additive skip connections of the
// few-view correction network. The paper has no learned component; these
// calls serve the few-view workload. Where the width is a multiple of 8 and
// Cout is 16 (the network's input layer), the layer runs on tcgen05 with the
// x taps in K (stem_fwd_tc in k_conv_tc.cu); otherwise on the tensor cores
// with mma.sync, its K dimension the 27 taps (below). The skip connections
// and the rest are element-wise passes on the CUDA cores.
//
//   stem_fwd_mma    y[v][co] = act(b[co] + sum_tap w[co][tap] bf16(x[v + tap]))
//                   for a one-channel FP32 volume: a GEMM whose K dimension
//                   is the 27 taps (not channels), so no product is spent on
//                   zero channels. A CTA stages its haloed input tile,
//                   rounded to BF16, in shared memory; each warp forms the
//                   A fragments of 16 x-consecutive voxels by direct loads
//                   at its tap offsets and runs mma.sync against weight
//                   fragments held in registers.
//   stem_wgrad      dw[co][tap] += sum_v dy[v][co] bf16(x[v + tap]) and
//                   db[co] += sum_v dy[v][co]. A CTA stages a 4 x 8 x 32
//                   voxel tile of dy and the haloed tile of x; each of its
//                   27 C + C threads owns one (tap, co) or one bias and walks
//                   the tile, then adds its sum to the global gradient.
//   upsample2_add   y[2z+a][2y+b][2x+c] = bf16(x[z][y][x] + skip[2z+a][2y+b][2x+c])
//                   (FP32 sum of the two BF16 values, rounded once), eight
//                   channels per 16-byte access.
#include "bp_internal.h"

#include <cuda_bf16.h>

#include "../../include/unet.h"

namespace bp {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kStemMaxC = 32;
constexpr int kWgZ = 4, kWgY = 8, kWgX = 32;                       // stem weight-gradient tile
constexpr int kWgHZ = kWgZ + 2, kWgHY = kWgY + 2, kWgHX = kWgX + 2;  // with halo

__device__ __forceinline__ float2 bf2f(unsigned u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}
__device__ __forceinline__ unsigned f2bf(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned *>(&h);
}
__device__ __forceinline__ float round_bf16(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// CTA tile 64 (x) x 8 (y) x 8 (z) outputs. The haloed input tile (66 x 10 x 10
// values, rounded to BF16 once and kept as BF16 bits) is staged in shared
// memory row by row (one warp per row, every load in flight before any
// store); the A fragments are byte permutes of those bits (no conversion
// per use), read at plain int indices into the tile (32-bit shared
// addressing; per-element index arithmetic in 64-bit generic addresses had
// made the layer integer-bound: 287 us at 256^3 against 181 us now). The products run on the tensor cores (mma.sync m16n8k16,
// BF16 in, FP32 accumulation) as a GEMM with M = 16 x-consecutive voxels,
// N = output channels and K = the 27 taps (zero-padded to 32): a thread's
// A-fragment entries are single shared-memory loads at the tap offsets it
// owns, the weight fragments stay in registers for the whole CTA.
constexpr int kStTX = 64, kStTY = 8, kStTZ = 8;
constexpr int kStHX = kStTX + 2, kStHY = kStTY + 2, kStHZ = kStTZ + 2;
constexpr int kStHalo = kStHX * kStHY * kStHZ;   // 2640
constexpr int kStThreads = 256;

__device__ __forceinline__ unsigned pack_bf16x2(float lo, float hi) {
    unsigned r;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma16816(float *c, const unsigned *a, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// POOL: the 2 x 2 x 2 max pooling of the (BF16) output is written as well, to
// pooled [N][D/2][H/2][W/2][C]: the tile holds whole pooling windows, a warp
// takes 2 x 2 blocks of output rows and keeps the running maximum of each
// voxel pair's rounded outputs, and the x pairs meet by a lane shuffle. The
// maxima are those of the stored values: bit for bit cnn_maxpool2_forward.
template <int C, bool POOL>
__global__ void __launch_bounds__(kStThreads)
stem_fwd_mma(const float *__restrict__ x, const bf16 *__restrict__ w, const float *__restrict__ b,
             bf16 *__restrict__ y, int ycs, int ycoff, bf16 *__restrict__ pooled, int D, int H, int W, int relu,
             int tx, int ty, int tz) {
    constexpr int NT = C / 8;   // n-tiles
    constexpr int kRowsH = kStHZ * kStHY;                          // staged rows (hz, hy)
    constexpr int kRowsPerWarp = (kRowsH + kStThreads / 32 - 1) / (kStThreads / 32);
    constexpr int kXPer = (kStHX + 31) / 32;                       // values per lane and row
    __shared__ unsigned short xs[kStHalo];   // [HZ][HY][HX], BF16 bits (rounded once when staged)
    long long r = blockIdx.x;
    const int x0 = (int)(r % tx) * kStTX;
    r /= tx;
    const int y0 = (int)(r % ty) * kStTY;
    r /= ty;
    const int z0 = (int)(r % tz) * kStTZ;
    const long long nb = r / tz;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // staging: warp w loads rows w, w + 8, ... of the haloed tile, lane l the
    // pixels l, l + 32, l + 64 of a row; every load is issued before any store
    float v[kRowsPerWarp][kXPer];
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i) {
        const int row = warp + i * (kStThreads / 32);
        const int hz = row / kStHY, hy = row - hz * kStHY;
        const int z = z0 + hz - 1, yy = y0 + hy - 1;
        const bool rok = row < kRowsH && z >= 0 && z < D && yy >= 0 && yy < H;
        const float *src = x + ((nb * D + (rok ? z : 0)) * H + (rok ? yy : 0)) * (long long)W;
#pragma unroll
        for (int j = 0; j < kXPer; ++j) {
            const int hx = lane + 32 * j, xx = x0 + hx - 1;
            v[i][j] = (rok && hx < kStHX && xx >= 0 && xx < W) ? __ldg(src + xx) : 0.0f;
        }
    }
    const int g = lane >> 2, t4 = lane & 3;
    // this thread's K slots: k = 16 s + 2 t4 + {0, 1, 8, 9}; offset of tap k in the staged tile
    int off[2][4];
    unsigned bw[2][NT][2];
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = 16 * s2 + 2 * t4 + (q & 1) + (q >> 1) * 8;
            off[s2][q] = k < 27 ? ((k / 9) * kStHY + (k / 3) % 3) * kStHX + k % 3 : -1;
        }
#pragma unroll
    for (int s2 = 0; s2 < 2; ++s2)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 16 * s2 + 2 * t4 + 8 * h, co = j * 8 + g;
                const float w0 = k < 27 ? __bfloat162float(w[co * 27 + k]) : 0.0f;
                const float w1 = k + 1 < 27 ? __bfloat162float(w[co * 27 + k + 1]) : 0.0f;
                bw[s2][j][h] = pack_bf16x2(w0, w1);
            }
    float bias[NT][2];
#pragma unroll
    for (int j = 0; j < NT; ++j) {
        bias[j][0] = b ? b[j * 8 + 2 * t4] : 0.0f;
        bias[j][1] = b ? b[j * 8 + 2 * t4 + 1] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < kRowsPerWarp; ++i) {
        const int row = warp + i * (kStThreads / 32);
#pragma unroll
        for (int j = 0; j < kXPer; ++j) {
            const int hx = lane + 32 * j;
            if (row < kRowsH && hx < kStHX) xs[row * kStHX + hx] = __bfloat16_as_ushort(__float2bfloat16_rn(v[i][j]));
        }
    }
    __syncthreads();
    // output rows (oz, oy): without pooling warp w takes rows w, w + 8, ...;
    // with pooling, the 2 x 2 row blocks w, w + 8, ... Per row four x segments
    // of 16 voxels. Shared indices are plain ints into xs (32-bit shared
    // addressing, the tap offsets compile-time within a row).
    auto row_mma = [&](int oz, int oy, int xs0, float (*acc)[4]) {
        const int rbase = (oz * kStHY + oy) * kStHX + g + xs0;   // tap (0,0,0) of voxel xs0 + g of the row
#pragma unroll
        for (int j = 0; j < NT; ++j) {
            acc[j][0] = bias[j][0];
            acc[j][1] = bias[j][1];
            acc[j][2] = bias[j][0];
            acc[j][3] = bias[j][1];
        }
#pragma unroll
        for (int s2 = 0; s2 < 2; ++s2) {
            unsigned e[2][4];   // [row g / g + 8][slot], BF16 bits
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int o = off[s2][q];
                e[0][q] = o >= 0 ? xs[rbase + o] : 0u;
                e[1][q] = o >= 0 ? xs[rbase + o + 8] : 0u;
            }
            // two BF16 values per register, the lower k in the low half
            unsigned a[4];
            a[0] = __byte_perm(e[0][0], e[0][1], 0x5410);   // row g, k = 2 t4, 2 t4 + 1
            a[1] = __byte_perm(e[1][0], e[1][1], 0x5410);   // row g + 8
            a[2] = __byte_perm(e[0][2], e[0][3], 0x5410);   // row g, k + 8
            a[3] = __byte_perm(e[1][2], e[1][3], 0x5410);   // row g + 8, k + 8
#pragma unroll
            for (int j = 0; j < NT; ++j) mma16816(acc[j], a, bw[s2][j][0], bw[s2][j][1]);
        }
    };
    // act(acc) rounded to BF16 (pairs of channels) and stored at row vrow
    auto store_row = [&](float (*acc)[4], long long vrow, int xs0, unsigned (*q)[2]) {
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                float a0 = acc[j][2 * hr], a1 = acc[j][2 * hr + 1];
                if (relu) {
                    a0 = fmaxf(a0, 0.0f);
                    a1 = fmaxf(a1, 0.0f);
                }
                q[j][hr] = f2bf(a0, a1);
            }
            const int xx = x0 + xs0 + g + 8 * hr;
            if (xx >= W) continue;
            bf16 *dst = y + (vrow + xx) * ycs + ycoff + 2 * t4;
#pragma unroll
            for (int j = 0; j < NT; ++j) *reinterpret_cast<unsigned *>(dst + j * 8) = q[j][hr];
        }
    };
    if constexpr (!POOL) {
#pragma unroll 1
        for (int orow = warp; orow < kStTZ * kStTY; orow += kStThreads / 32) {
            const int oz = orow / kStTY, oy = orow - oz * kStTY;
            const int z = z0 + oz, yy = y0 + oy;
            if (z >= D || yy >= H) continue;
            const long long vrow = ((nb * D + z) * H + yy) * (long long)W;
#pragma unroll
            for (int seg = 0; seg < 4; ++seg) {
                float acc[NT][4];
                unsigned q[NT][2];
                row_mma(oz, oy, seg * 16, acc);
                store_row(acc, vrow, seg * 16, q);
            }
        }
    } else {
        const int Dh = D >> 1, Hh = H >> 1, Wh = W >> 1;
#pragma unroll 1
        for (int blk = warp; blk < (kStTZ / 2) * (kStTY / 2); blk += kStThreads / 32) {
            const int bz = blk / (kStTY / 2), by = blk - bz * (kStTY / 2);
            const int z = z0 + 2 * bz, yy = y0 + 2 * by;
            if (z >= D || yy >= H) continue;   // D, H even: the whole block is in or out
            const long long prow = ((nb * Dh + (z >> 1)) * Hh + (yy >> 1)) * (long long)Wh;
#pragma unroll 1
            for (int seg = 0; seg < 4; ++seg) {
                float pm[NT][4];
#pragma unroll
                for (int rr = 0; rr < 4; ++rr) {
                    const int oz = 2 * bz + (rr >> 1), oy = 2 * by + (rr & 1);
                    const long long vrow = ((nb * D + z0 + oz) * H + y0 + oy) * (long long)W;
                    float acc[NT][4];
                    unsigned q[NT][2];
                    row_mma(oz, oy, seg * 16, acc);
                    store_row(acc, vrow, seg * 16, q);
#pragma unroll
                    for (int j = 0; j < NT; ++j)
#pragma unroll
                        for (int hr = 0; hr < 2; ++hr) {
                            const float2 f = bf2f(q[j][hr]);
                            pm[j][2 * hr] = rr ? fmaxf(pm[j][2 * hr], f.x) : f.x;
                            pm[j][2 * hr + 1] = rr ? fmaxf(pm[j][2 * hr + 1], f.y) : f.y;
                        }
                }
                // voxel x and x ^ 1 are lanes l and l ^ 4 (g = l / 4)
#pragma unroll
                for (int j = 0; j < NT; ++j)
#pragma unroll
                    for (int e2 = 0; e2 < 4; ++e2) pm[j][e2] = fmaxf(pm[j][e2], __shfl_xor_sync(0xffffffffu, pm[j][e2], 4));
                if ((g & 1) == 0) {
#pragma unroll
                    for (int hr = 0; hr < 2; ++hr) {
                        const int xx = x0 + seg * 16 + g + 8 * hr;
                        if (xx >= W) continue;
                        bf16 *dst = pooled + (prow + (xx >> 1)) * C + 2 * t4;
#pragma unroll
                        for (int j = 0; j < NT; ++j)
                            *reinterpret_cast<unsigned *>(dst + j * 8) = f2bf(pm[j][2 * hr], pm[j][2 * hr + 1]);
                    }
                }
            }
        }
    }
}

__global__ void stem_wgrad_kernel(const float *__restrict__ x, const bf16 *__restrict__ dy, int dcs, int dcoff,
                                  float *__restrict__ dw, float *__restrict__ db, int D, int H, int W, int C,
                                  int tx, int ty, int tz) {
    extern __shared__ __align__(16) unsigned char sm[];
    float *xs = reinterpret_cast<float *>(sm);                                  // [HZ][HY][HX]
    bf16 *gs = reinterpret_cast<bf16 *>(sm + kWgHZ * kWgHY * kWgHX * sizeof(float));   // [Z*Y*X][C]
    long long r = blockIdx.x;
    const int x0 = (int)(r % tx) * kWgX;
    r /= tx;
    const int y0 = (int)(r % ty) * kWgY;
    r /= ty;
    const int z0 = (int)(r % tz) * kWgZ;
    const long long nb = r / tz;
    for (int t = threadIdx.x; t < kWgHZ * kWgHY * kWgHX; t += blockDim.x) {
        const int hx = t % kWgHX, hy = (t / kWgHX) % kWgHY, hz = t / (kWgHX * kWgHY);
        const int z = z0 + hz - 1, yy = y0 + hy - 1, xx = x0 + hx - 1;
        xs[t] = (z >= 0 && z < D && yy >= 0 && yy < H && xx >= 0 && xx < W)
                    ? round_bf16(x[((nb * D + z) * H + yy) * (long long)W + xx]) : 0.0f;
    }
    const int c8 = C / 8;
    for (int t = threadIdx.x; t < kWgZ * kWgY * kWgX * c8; t += blockDim.x) {
        const int v = t / c8, cv = t % c8;
        const int lx = v % kWgX, ly = (v / kWgX) % kWgY, lz = v / (kWgX * kWgY);
        const int z = z0 + lz, yy = y0 + ly, xx = x0 + lx;
        uint4 q = make_uint4(0, 0, 0, 0);
        if (z < D && yy < H && xx < W)
            q = *reinterpret_cast<const uint4 *>(dy + ((nb * D + z) * H + yy) * (long long)W * dcs +
                                                 (long long)xx * dcs + dcoff + cv * 8);
        *reinterpret_cast<uint4 *>(gs + v * C + cv * 8) = q;
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t >= 28 * C) return;
    const bool is_bias = t >= 27 * C;
    const int tap = is_bias ? 0 : t / C, co = is_bias ? t - 27 * C : t % C;
    const int dz = tap / 9, dyo = (tap / 3) % 3, dx = tap % 3;
    float acc = 0.0f;
    for (int lz = 0; lz < kWgZ; ++lz)
        for (int ly = 0; ly < kWgY; ++ly) {
            const float *xr = xs + ((lz + dz) * kWgHY + ly + dyo) * kWgHX + dx;
            const bf16 *gr = gs + (lz * kWgY + ly) * kWgX * C + co;
#pragma unroll 8
            for (int lx = 0; lx < kWgX; ++lx) {
                const float g = __bfloat162float(gr[lx * C]);
                acc = is_bias ? acc + g : fmaf(g, xr[lx], acc);
            }
        }
    if (is_bias) {
        if (db) atomicAdd(&db[co], acc);
    } else {
        atomicAdd(&dw[co * 27 + tap], acc);
    }
}

__global__ void upsample2_add_v8(const uint4 *__restrict__ x, const bf16 *__restrict__ skip, int scs, int scoff,
                                 bf16 *__restrict__ y, int ycs, int ycoff, int N, int D, int H, int W, int c8) {
    const long long total = (long long)N * D * H * W * c8;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int cv = (int)(t % c8);
        long long v = t / c8;
        const int xv = (int)(v % W);
        v /= W;
        const int yv = (int)(v % H);
        v /= H;
        const int zv = (int)(v % D);
        const long long nb = v / D;
        const uint4 val = x[t];
        const float2 a0 = bf2f(val.x), a1 = bf2f(val.y), a2 = bf2f(val.z), a3 = bf2f(val.w);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long u = ((nb * (2 * D) + 2 * zv + (k >> 2)) * (2 * H) + 2 * yv + ((k >> 1) & 1)) * (2 * W) +
                                2 * xv + (k & 1);
            const uint4 s = *reinterpret_cast<const uint4 *>(skip + u * scs + scoff + cv * 8);
            const float2 s0 = bf2f(s.x), s1 = bf2f(s.y), s2 = bf2f(s.z), s3 = bf2f(s.w);
            *reinterpret_cast<uint4 *>(y + u * ycs + ycoff + cv * 8) =
                make_uint4(f2bf(a0.x + s0.x, a0.y + s0.y), f2bf(a1.x + s1.x, a1.y + s1.y),
                           f2bf(a2.x + s2.x, a2.y + s2.y), f2bf(a3.x + s3.x, a3.y + s3.y));
        }
    }
}

// 1x1x1 output head, one voxel per thread: out[v] = res[v] + b + sum_ci w[ci] x[v][ci]
// (products in channel order from 0, FP32), x BF16 with C = 8 k channels.
__global__ void head1_fwd(const bf16 *__restrict__ x, int cs, const float *__restrict__ w,
                          const float *__restrict__ bptr, const float *__restrict__ res, float *__restrict__ out,
                          long long nvox, int c8) {
    __shared__ float ws[kStemMaxC];
    for (int t = threadIdx.x; t < c8 * 8; t += blockDim.x) ws[t] = w[t];
    __syncthreads();
    const float b0 = bptr ? *bptr : 0.0f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        float acc = 0.0f;
        for (int g = 0; g < c8; ++g) {
            const uint4 q = *reinterpret_cast<const uint4 *>(x + v * cs + g * 8);
            const unsigned u[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = bf2f(u[k]);
                acc = fmaf(ws[g * 8 + 2 * k], f.x, acc);
                acc = fmaf(ws[g * 8 + 2 * k + 1], f.y, acc);
            }
        }
        out[v] = acc + b0 + (res ? res[v] : 0.0f);
    }
}

// Its gradients for an FP32 output gradient g: dx[v][ci] = bf16(w[ci] g[v]);
// dw[ci] += sum_v g[v] x[v][ci], db += sum_v g[v] (per-thread sums, a
// shared-memory reduction per CTA, one atomic per value and CTA).
__global__ void head1_bwd(const bf16 *__restrict__ x, int cs, const float *__restrict__ w,
                          const float *__restrict__ g, bf16 *__restrict__ dx, int dxcs, float *dw, float *db,
                          long long nvox, int c8) {
    __shared__ float part[kStemMaxC + 1];
    __shared__ float ws[kStemMaxC];
    const int C = c8 * 8;
    for (int t = threadIdx.x; t < C; t += blockDim.x) {
        ws[t] = w[t];
        part[t] = 0.0f;
    }
    if (threadIdx.x == 0) part[C] = 0.0f;
    __syncthreads();
    float sw[kStemMaxC];
#pragma unroll
    for (int k = 0; k < kStemMaxC; ++k) sw[k] = 0.0f;
    float sb = 0.0f;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        const float gv = g[v];
        sb += gv;
#pragma unroll
        for (int gi = 0; gi < kStemMaxC / 8; ++gi) {
            if (gi >= c8) break;
            const uint4 q = *reinterpret_cast<const uint4 *>(x + v * cs + gi * 8);
            const unsigned u[4] = {q.x, q.y, q.z, q.w};
            unsigned o[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = bf2f(u[k]);
                sw[gi * 8 + 2 * k] = fmaf(gv, f.x, sw[gi * 8 + 2 * k]);
                sw[gi * 8 + 2 * k + 1] = fmaf(gv, f.y, sw[gi * 8 + 2 * k + 1]);
                o[k] = f2bf(ws[gi * 8 + 2 * k] * gv, ws[gi * 8 + 2 * k + 1] * gv);
            }
            *reinterpret_cast<uint4 *>(dx + v * dxcs + gi * 8) = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
#pragma unroll
    for (int k = 0; k < kStemMaxC; ++k) {
        if (k >= C) break;
        float s = sw[k];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if ((threadIdx.x & 31) == 0) atomicAdd(&part[k], s);
    }
    for (int off = 16; off > 0; off >>= 1) sb += __shfl_xor_sync(0xffffffffu, sb, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(&part[C], sb);
    __syncthreads();
    for (int t = threadIdx.x; t < C; t += blockDim.x) atomicAdd(&dw[t], part[t]);
    if (threadIdx.x == 0 && db) atomicAdd(db, part[C]);
}

// Nearest upsampling of x plus the skip, rounded to BF16 per channel pair as
// upsample2_add_v8 rounds it, then the 1x1 head of head1_fwd on that value
// (same products, same channel order): bit for bit the two kernels, without
// the full-resolution sum ever reaching memory. One thread per coarse voxel
// and fine (z, y) child row: the coarse channels are loaded once for the two
// fine voxels along x, whose outputs and residuals are one float2.
__global__ void upsample2_add_head1_fwd(const bf16 *__restrict__ x, const bf16 *__restrict__ skip, int scs,
                                        int scoff, const float *__restrict__ w, const float *__restrict__ bptr,
                                        const float *__restrict__ res, float *__restrict__ out, int N, int D,
                                        int H, int W, int c8) {
    __shared__ float ws[kStemMaxC];
    for (int t = threadIdx.x; t < c8 * 8; t += blockDim.x) ws[t] = w[t];
    __syncthreads();
    const float b0 = bptr ? *bptr : 0.0f;
    const int C = c8 * 8;
    // t = ((((nb * D + z) * 2 + cz) * H + y) * 2 + cy) * W + xc: consecutive threads walk x
    const long long total = (long long)N * D * H * W * 4;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        long long r = t;
        const int xc = (int)(r % W);
        r /= W;
        const int cy = (int)(r & 1);
        r >>= 1;
        const int yc = (int)(r % H);
        r /= H;
        const int cz = (int)(r & 1);
        r >>= 1;
        const int zc = (int)(r % D);
        const long long nb = r / D;
        const long long cv = ((nb * D + zc) * H + yc) * W + xc;
        const long long v0 = ((nb * 2 * D + 2 * zc + cz) * (2 * H) + 2 * yc + cy) * (2LL * W) + 2 * xc;
        float acc0 = 0.0f, acc1 = 0.0f;
        for (int g = 0; g < c8; ++g) {
            const uint4 q = *reinterpret_cast<const uint4 *>(x + cv * C + g * 8);
            const uint4 s0 = *reinterpret_cast<const uint4 *>(skip + v0 * scs + scoff + g * 8);
            const uint4 s1 = *reinterpret_cast<const uint4 *>(skip + (v0 + 1) * scs + scoff + g * 8);
            const unsigned qa[4] = {q.x, q.y, q.z, q.w};
            const unsigned sa[4] = {s0.x, s0.y, s0.z, s0.w}, sb[4] = {s1.x, s1.y, s1.z, s1.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 a = bf2f(qa[k]), u = bf2f(sa[k]), o = bf2f(sb[k]);
                const float2 f0 = bf2f(f2bf(a.x + u.x, a.y + u.y)), f1 = bf2f(f2bf(a.x + o.x, a.y + o.y));
                acc0 = fmaf(ws[g * 8 + 2 * k], f0.x, acc0);
                acc0 = fmaf(ws[g * 8 + 2 * k + 1], f0.y, acc0);
                acc1 = fmaf(ws[g * 8 + 2 * k], f1.x, acc1);
                acc1 = fmaf(ws[g * 8 + 2 * k + 1], f1.y, acc1);
            }
        }
        float2 rr = make_float2(0.0f, 0.0f);
        if (res) rr = *reinterpret_cast<const float2 *>(res + v0);
        *reinterpret_cast<float2 *>(out + v0) = make_float2(acc0 + b0 + rr.x, acc1 + b0 + rr.y);
    }
}

unsigned blocks_for(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bp_status launched(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(nullptr, e, what);
}

}  // namespace
}  // namespace bp

using namespace bp;

namespace bp {
bool stem_tc_applies(const float *x, const void *y, int ycs, int yco, const void *pooled, int wd, int cout);
cudaError_t stem_fwd_tc_launch(const float *x, const void *w, const float *b, void *y, int ycs, int yco,
                               void *pooled, int n, int d, int h, int wd, int relu, cudaStream_t st);
}  // namespace bp

static bp_status launch_stem(const float *x, const void *w, const float *b, void *y, int y_cstride, int y_coff,
                             void *pooled, int n, int d, int h, int wd, int cout, int relu, void *stream) {
    // tcgen05 with the x taps in K (k_conv_tc.cu) where its tile fits
    if (stem_tc_applies(x, y, y_cstride, y_coff, pooled, wd, cout)) {
        cudaError_t e = stem_fwd_tc_launch(x, w, b, y, y_cstride, y_coff, pooled, n, d, h, wd, relu,
                                           (cudaStream_t)stream);
        return e == cudaSuccess ? BP_OK : cuda_fail(nullptr, e, "stem_fwd_tc");
    }
    const int tx = (wd + kStTX - 1) / kStTX, ty = (h + kStTY - 1) / kStTY, tz = (d + kStTZ - 1) / kStTZ;
    const long long nt = (long long)n * tx * ty * tz;
    if (nt > 0x7fffffffLL) return fail(nullptr, BP_ERR_INVALID_ARG, "stem: volume too large");
    cudaStream_t st = (cudaStream_t)stream;
    bf16 *p = (bf16 *)pooled;
#define STEM_CASE(C)                                                                                              \
    case C:                                                                                                       \
        if (p)                                                                                                    \
            stem_fwd_mma<C, true><<<(unsigned)nt, kStThreads, 0, st>>>(x, (const bf16 *)w, b, (bf16 *)y,           \
                                                                       y_cstride, y_coff, p, d, h, wd, relu, tx, ty, tz); \
        else                                                                                                      \
            stem_fwd_mma<C, false><<<(unsigned)nt, kStThreads, 0, st>>>(x, (const bf16 *)w, b, (bf16 *)y,          \
                                                                        y_cstride, y_coff, p, d, h, wd, relu, tx, ty, tz); \
        break;
    switch (cout) {
        STEM_CASE(8)
        STEM_CASE(16)
        STEM_CASE(24)
        default: STEM_CASE(32)
    }
#undef STEM_CASE
    return launched("stem_fwd_mma");
}

extern "C" {

bp_status cnn_stem_forward(const float *x, const void *w, const float *b, void *y, int y_cstride, int y_coff,
                           int n, int d, int h, int wd, int cout, int relu, void *stream) {
    if (!x || !w || !y || n < 1 || d < 1 || h < 1 || wd < 4 || wd % 4 || cout < 8 || cout % 8 ||
        cout > kStemMaxC || y_cstride % 8 || y_coff % 8 || y_coff < 0 || y_coff + cout > y_cstride || !al16(y))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_stem_forward: bad arguments");
    return launch_stem(x, w, b, y, y_cstride, y_coff, nullptr, n, d, h, wd, cout, relu, stream);
}

bp_status cnn_stem_pool_forward(const float *x, const void *w, const float *b, void *y, int y_cstride, int y_coff,
                                void *pooled, int n, int d, int h, int wd, int cout, int relu, void *stream) {
    if (!x || !w || !y || !pooled || n < 1 || d < 2 || h < 2 || wd < 4 || wd % 4 || d % 2 || h % 2 || cout < 8 ||
        cout % 8 || cout > kStemMaxC || y_cstride % 8 || y_coff % 8 || y_coff < 0 || y_coff + cout > y_cstride ||
        !al16(y) || !al16(pooled))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_stem_pool_forward: bad arguments");
    return launch_stem(x, w, b, y, y_cstride, y_coff, pooled, n, d, h, wd, cout, relu, stream);
}

bp_status cnn_stem_wgrad(const float *x, const void *dy, int dy_cstride, int dy_coff, float *dw, float *db, int n,
                         int d, int h, int wd, int cout, void *stream) {
    if (!x || !dy || !dw || n < 1 || d < 1 || h < 1 || wd < 1 || cout < 8 || cout % 8 || cout > kStemMaxC ||
        dy_cstride % 8 || dy_coff % 8 || dy_coff < 0 || dy_coff + cout > dy_cstride || !al16(dy))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_stem_wgrad: bad arguments");
    const int tx = (wd + kWgX - 1) / kWgX, ty = (h + kWgY - 1) / kWgY, tz = (d + kWgZ - 1) / kWgZ;
    const long long nt = (long long)n * tx * ty * tz;
    if (nt > 0x7fffffffLL) return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_stem_wgrad: volume too large");
    const size_t smem = kWgHZ * kWgHY * kWgHX * sizeof(float) + (size_t)kWgZ * kWgY * kWgX * cout * sizeof(bf16);
    if (smem > 48 * 1024) {   // cout 32: 73 KB, above the default limit
        cudaError_t e = cudaFuncSetAttribute(stem_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cnn_stem_wgrad: shared memory limit");
    }
    const int threads = (28 * cout + 31) / 32 * 32;
    stem_wgrad_kernel<<<(unsigned)nt, threads, smem, (cudaStream_t)stream>>>(
        x, (const bf16 *)dy, dy_cstride, dy_coff, dw, db, d, h, wd, cout, tx, ty, tz);
    return launched("stem_wgrad_kernel");
}

bp_status cnn_head1_forward(const void *x, int x_cstride, const float *w, const float *b, const float *res,
                            float *out, long long nvox, int cin, void *stream) {
    if (!x || !w || !out || nvox < 1 || cin < 8 || cin % 8 || cin > kStemMaxC || x_cstride % 8 ||
        cin > x_cstride || !al16(x))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_head1_forward: bad arguments");
    head1_fwd<<<blocks_for(nvox), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, x_cstride, w, b, res, out, nvox,
                                                                 cin / 8);
    return launched("head1_fwd");
}

bp_status cnn_head1_backward(const void *x, int x_cstride, const float *w, const float *g, void *dx,
                             int dx_cstride, float *dw, float *db, long long nvox, int cin, void *stream) {
    if (!x || !w || !g || !dx || !dw || nvox < 1 || cin < 8 || cin % 8 || cin > kStemMaxC || x_cstride % 8 ||
        dx_cstride % 8 || cin > x_cstride || cin > dx_cstride || !al16(x) || !al16(dx))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_head1_backward: bad arguments");
    long long nb = (nvox + 255) / 256;
    if (nb > 4096) nb = 4096;   // per-thread sums over a grid-stride loop
    head1_bwd<<<(unsigned)nb, 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, x_cstride, w, g, (bf16 *)dx,
                                                              dx_cstride, dw, db, nvox, cin / 8);
    return launched("head1_bwd");
}

bp_status cnn_upsample2_add_forward(const void *x, const void *skip, int s_cstride, int s_coff, void *y,
                                    int y_cstride, int y_coff, int n, int d, int h, int wd, int c, void *stream) {
    if (!x || !skip || !y || n < 1 || d < 1 || h < 1 || wd < 1 || c < 8 || c % 8 || s_cstride % 8 || s_coff % 8 ||
        y_cstride % 8 || y_coff % 8 || s_coff < 0 || y_coff < 0 || s_coff + c > s_cstride ||
        y_coff + c > y_cstride || !al16(x) || !al16(skip) || !al16(y))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_upsample2_add_forward: bad arguments");
    const long long tot8 = (long long)n * d * h * wd * (c / 8);
    upsample2_add_v8<<<blocks_for(tot8), 256, 0, (cudaStream_t)stream>>>(
        (const uint4 *)x, (const bf16 *)skip, s_cstride, s_coff, (bf16 *)y, y_cstride, y_coff, n, d, h, wd, c / 8);
    return launched("upsample2_add_v8");
}

bp_status cnn_upsample2_add_head1_forward(const void *x, const void *skip, int s_cstride, int s_coff,
                                          const float *w, const float *b, const float *res, float *out, int n,
                                          int d, int h, int wd, int c, void *stream) {
    if (!x || !skip || !w || !out || n < 1 || d < 1 || h < 1 || wd < 1 || c < 8 || c % 8 || c > kStemMaxC ||
        s_cstride % 8 || s_coff % 8 || s_coff < 0 || s_coff + c > s_cstride || !al16(x) || !al16(skip))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_upsample2_add_head1_forward: bad arguments");
    if (((uintptr_t)out & 7u) || ((uintptr_t)res & 7u))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_upsample2_add_head1_forward: res and out must be 8-byte aligned");
    const long long nthreads = 4LL * n * d * h * wd;
    upsample2_add_head1_fwd<<<blocks_for(nthreads), 256, 0, (cudaStream_t)stream>>>(
        (const bf16 *)x, (const bf16 *)skip, s_cstride, s_coff, w, b, res, out, n, d, h, wd, c / 8);
    return launched("upsample2_add_head1_fwd");
}

}  // extern "C"
