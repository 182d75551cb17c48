// 3x3x3 convolutions of the few-view correction network as implicit GEMMs on
// the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation),
// plus the element-wise kernels a U-Net needs (pooling, upsampling, ReLU
// backward, loss, Adam). The paper has no learned component; the calls
// serve the few-view workload.
//
// Forward / input-gradient tile: 16 (x) x 4 (y) x 2 (z) output voxels per
// CTA of 4 warps; each warp owns two 16-voxel rows (two m16 tiles) and all
// output channels. Per 16-channel input chunk the CTA stages the halo brick
// (18 x 6 x 4 voxels) in shared memory once and, per z-plane of taps, the
// weights of 9 taps; the 27 taps then read shifted rows of the brick with
// ldmatrix. Rows are padded to 48 bytes so the 8 rows of an ldmatrix land
// in 8 distinct bank groups. The input gradient is the forward kernel run on
// the output gradient with flipped, transposed weights.
//
// Weight gradient: the GEMM over voxels dy^T (Cout x V) x x_shift (V x 16)
// per tap, split over CTAs that each walk several tiles and keep the
// partial sums of one z-plane of taps (9 taps) in registers; ldmatrix.trans
// turns the channels-last tiles into the operand layouts.
#include "bp_internal.h"

#include <cuda_bf16.h>

#include <mutex>

#include "../../include/unet.h"

namespace bp {

typedef __nv_bfloat16 bf16;

constexpr int kTX = 16, kTY = 4, kTZ = 2;                  // output tile
constexpr int kHX = kTX + 2, kHY = kTY + 2, kHZ = kTZ + 2;  // halo brick
constexpr int kHV = kHX * kHY * kHZ;                        // 432 voxels
constexpr int kRowPad = 24;                                 // bf16 per staged row (16 + 8 pad)
constexpr int kConvThreads = 128;

__device__ __forceinline__ unsigned s_addr(const void *p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                        unsigned &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned &r0, unsigned &r1, unsigned &r2,
                                          unsigned &r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float *c, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Tile geometry shared by the kernels: tile index -> (n, z0, y0, x0).
struct TileGrid {
    int tx, ty, tz;   // tiles per dimension
    __device__ __forceinline__ void decode(long long t, int d, int &n, int &z0, int &y0, int &x0) const {
        x0 = (int)(t % tx) * kTX;
        long long r = t / tx;
        y0 = (int)(r % ty) * kTY;
        r /= ty;
        z0 = (int)(r % tz) * kTZ;
        n = (int)(r / tz);
    }
};

// Stage the 16-channel chunk [c0, c0+16) of the halo brick around a tile
// (zero outside the volume) into As[kHV][kRowPad].
__device__ __forceinline__ void stage_halo(bf16 *As, const bf16 *__restrict__ x, int cs, int coff,
                                           int c0, int n, int z0, int y0, int x0, int D, int H,
                                           int W) {
    for (int t = threadIdx.x; t < kHV * 2; t += blockDim.x) {
        const int hv = t >> 1, half = t & 1;
        const int hx = hv % kHX, hy = (hv / kHX) % kHY, hz = hv / (kHX * kHY);
        const int z = z0 + hz - 1, y = y0 + hy - 1, xx = x0 + hx - 1;
        uint4 val = make_uint4(0, 0, 0, 0);
        if (z >= 0 && z < D && y >= 0 && y < H && xx >= 0 && xx < W) {
            const size_t vox = (((size_t)n * D + z) * H + y) * W + xx;
            val = *reinterpret_cast<const uint4 *>(x + vox * cs + coff + c0 + half * 8);
        }
        *reinterpret_cast<uint4 *>(As + hv * kRowPad + half * 8) = val;
    }
}

// ---------------------------------------------------------------------------
// Forward (and input-gradient) implicit GEMM
// ---------------------------------------------------------------------------
template <int COUT, bool OUT_F32>
__global__ void __launch_bounds__(kConvThreads)
conv3d_fwd_kernel(const bf16 *__restrict__ x, int xcs, int xco, const bf16 *__restrict__ w,
                  const float *__restrict__ bias, void *__restrict__ y, int ycs, int yco, int D,
                  int H, int W, int cin, int relu, TileGrid grid) {
    __shared__ __align__(128) bf16 As[kHV * kRowPad];
    __shared__ __align__(128) bf16 Bs[9 * COUT * kRowPad];
    constexpr int NT = COUT / 8;

    int n, z0, y0, x0;
    grid.decode(blockIdx.x, D, n, z0, y0, x0);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.0f;

    // ldmatrix lane roles
    const int a_row = lane & 15, a_koff = (lane >> 4) * 8;
    const int b_n = (lane >> 4) * 8 + (lane & 7), b_koff = ((lane >> 3) & 1) * 8;

    for (int c0 = 0; c0 < cin; c0 += 16) {
        __syncthreads();
        stage_halo(As, x, xcs, xco, c0, n, z0, y0, x0, D, H, W);
        for (int dz = 0; dz < 3; ++dz) {
            __syncthreads();
            // weights of taps dz*9 .. dz*9+8, channels c0..c0+15
            for (int t = threadIdx.x; t < 9 * COUT * 2; t += kConvThreads) {
                const int half = t & 1, row = t >> 1;        // row = tap9 * COUT + co
                const int t9 = row / COUT, co = row % COUT;
                const uint4 val = *reinterpret_cast<const uint4 *>(
                    w + ((size_t)co * 27 + dz * 9 + t9) * cin + c0 + half * 8);
                *reinterpret_cast<uint4 *>(Bs + row * kRowPad + half * 8) = val;
            }
            __syncthreads();
#pragma unroll 1
            for (int t9 = 0; t9 < 9; ++t9) {
                const int dy = t9 / 3, dx = t9 % 3;
                unsigned a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const int mrow = warp * 2 + mt;            // 0..7 -> (zz, yy)
                    const int zz = mrow / kTY, yy = mrow % kTY;
                    const int hv = ((zz + dz) * kHY + (yy + dy)) * kHX + (a_row + dx);
                    ldsm_x4(s_addr(As + hv * kRowPad + a_koff), a[mt][0], a[mt][1], a[mt][2], a[mt][3]);
                }
#pragma unroll
                for (int np = 0; np < NT / 2; ++np) {
                    unsigned b0, b1, b2, b3;
                    ldsm_x4(s_addr(Bs + (t9 * COUT + np * 16 + b_n) * kRowPad + b_koff), b0, b1, b2, b3);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
                        mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
                    }
                }
            }
        }
    }

    // epilogue: bias, ReLU, store (c0,c1: row g; c2,c3: row g+8; cols 2q, 2q+1)
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
        const int mrow = warp * 2 + mt;
        const int z = z0 + mrow / kTY, yv = y0 + mrow % kTY;
        if (z >= D || yv >= H) continue;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int xv = x0 + g + half * 8;
            if (xv >= W) continue;
            const size_t vox = (((size_t)n * D + z) * H + yv) * W + xv;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int co = nt * 8 + 2 * q;
                float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
                if (bias) {
                    v0 += bias[co];
                    v1 += bias[co + 1];
                }
                if (relu) {
                    v0 = fmaxf(v0, 0.0f);
                    v1 = fmaxf(v1, 0.0f);
                }
                if (OUT_F32) {
                    *reinterpret_cast<float2 *>(reinterpret_cast<float *>(y) + vox * ycs + yco + co) =
                        make_float2(v0, v1);
                } else {
                    *reinterpret_cast<__nv_bfloat162 *>(reinterpret_cast<bf16 *>(y) + vox * ycs + yco + co) =
                        __floats2bfloat162_rn(v0, v1);
                }
            }
        }
    }
}

// wt[ci][tap][co] = w[co][26 - tap][ci]: the weights of the input-gradient
// convolution (taps mirrored, input and output channels swapped)
__global__ void flip_transpose_kernel(const bf16 *__restrict__ w, bf16 *__restrict__ wt, int cin,
                                      int cout) {
    const long long n = 27LL * cin * cout;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(t % cout);
        const int tap = (int)((t / cout) % 27);
        const int ci = (int)(t / (27LL * cout));
        wt[t] = w[((size_t)co * 27 + (26 - tap)) * cin + ci];
    }
}

// ---------------------------------------------------------------------------
// Weight gradient
// ---------------------------------------------------------------------------
constexpr int kWgTiles = 16;   // tiles per CTA

template <int COUT>
__global__ void __launch_bounds__(kConvThreads)
conv3d_wgrad_kernel(const bf16 *__restrict__ x, int xcs, int xco, const bf16 *__restrict__ dy,
                    int dycs, int dyco, float *__restrict__ dw, int D, int H, int W, int cin,
                    long long ntiles, TileGrid grid) {
    constexpr int DYP = COUT + 8;                 // staged dy row: COUT + 8 bf16
    constexpr int MT = COUT / 16;                 // m16 tiles (output channels)
    constexpr int WPM = 4 / MT;                   // warps sharing one m tile (split over k)
    __shared__ __align__(128) bf16 As[kHV * kRowPad];
    __shared__ __align__(128) bf16 Ds[kTX * kTY * kTZ * DYP];

    const int c0 = blockIdx.y * 16;
    const int dz = blockIdx.z;                    // this CTA's z-plane of taps
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = warp % MT, ks = warp / MT;     // m tile, k-split slot

    float acc[9][2][4];
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[t][nt][e] = 0.0f;

    const int a_v = (lane >> 4) * 8 + (lane & 7), a_coff = ((lane >> 3) & 1) * 8;
    const int b_v = ((lane >> 3) & 1) * 8 + (lane & 7), b_coff = (lane >> 4) * 8;

    const long long t_begin = (long long)blockIdx.x * kWgTiles;
    const long long t_end = min(ntiles, t_begin + kWgTiles);
    for (long long tile = t_begin; tile < t_end; ++tile) {
        int n, z0, y0, x0;
        grid.decode(tile, D, n, z0, y0, x0);
        __syncthreads();
        stage_halo(As, x, xcs, xco, c0, n, z0, y0, x0, D, H, W);
        // dy tile (zero outside the volume)
        for (int t = threadIdx.x; t < kTX * kTY * kTZ * (COUT / 8); t += kConvThreads) {
            const int v = t / (COUT / 8), part = t % (COUT / 8);
            const int xx = v % kTX, yy = (v / kTX) % kTY, zz = v / (kTX * kTY);
            const int z = z0 + zz, yv = y0 + yy, xv = x0 + xx;
            uint4 val = make_uint4(0, 0, 0, 0);
            if (z < D && yv < H && xv < W) {
                const size_t vox = (((size_t)n * D + z) * H + yv) * W + xv;
                val = *reinterpret_cast<const uint4 *>(dy + vox * dycs + dyco + part * 8);
            }
            *reinterpret_cast<uint4 *>(Ds + v * DYP + part * 8) = val;
        }
        __syncthreads();
        // k steps: 8 rows of 16 voxels; this warp takes rows ks, ks+WPM, ...
#pragma unroll 1
        for (int kr = ks; kr < kTY * kTZ; kr += WPM) {
            const int zz = kr / kTY, yy = kr % kTY;
            unsigned a0, a1, a2, a3;
            ldsm_x4_t(s_addr(Ds + (kr * kTX + a_v) * DYP + mt * 16 + a_coff), a0, a1, a2, a3);
#pragma unroll
            for (int t9 = 0; t9 < 9; ++t9) {
                const int ddy = t9 / 3, ddx = t9 % 3;
                const int hv = ((zz + dz) * kHY + (yy + ddy)) * kHX + (b_v + ddx);
                unsigned b0, b1, b2, b3;
                ldsm_x4_t(s_addr(As + hv * kRowPad + b_coff), b0, b1, b2, b3);
                mma_bf16(acc[t9][0], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[t9][1], a0, a1, a2, a3, b2, b3);
            }
        }
    }
    // c0,c1: (co = g, ci = 2q, 2q+1); c2,c3: (co = g+8, ...)
    const int g = lane >> 2, q = lane & 3;
#pragma unroll
    for (int t9 = 0; t9 < 9; ++t9) {
        const int tap = dz * 9 + t9;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int ci = c0 + nt * 8 + 2 * q;
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const int co = mt * 16 + g + half * 8;
                float *p = dw + ((size_t)co * 27 + tap) * cin + ci;
                atomicAdd(p, acc[t9][nt][2 * half]);
                atomicAdd(p + 1, acc[t9][nt][2 * half + 1]);
            }
        }
    }
}

// db[co] += sum_v dy[v][co]
__global__ void bias_grad_kernel(const bf16 *__restrict__ dy, int cs, int coff, float *db,
                                 long long nvox, int c) {
    extern __shared__ float part[];
    for (int t = threadIdx.x; t < c; t += blockDim.x) part[t] = 0.0f;
    __syncthreads();
    const int lanes_per_vox = c;   // one thread per (voxel, channel)
    const long long total = nvox * c;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / lanes_per_vox;
        const int ch = (int)(t % lanes_per_vox);
        atomicAdd(&part[ch], __bfloat162float(dy[v * cs + coff + ch]));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < c; t += blockDim.x) atomicAdd(&db[t], part[t]);
}

// ---------------------------------------------------------------------------
// Output head (cin -> 1 channel) on the CUDA cores
// ---------------------------------------------------------------------------
__global__ void head_fwd_kernel(const bf16 *__restrict__ x, int cs, const float *__restrict__ w,
                                const float *__restrict__ bptr, const float *__restrict__ res,
                                float *__restrict__ out, int N, int D, int H, int W, int cin) {
    extern __shared__ float ws[];   // [27][cin]
    for (int t = threadIdx.x; t < 27 * cin; t += blockDim.x) ws[t] = w[t];
    __syncthreads();
    const float b0 = bptr ? *bptr : 0.0f;
    const long long nvox = (long long)N * D * H * W;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        const int xv = (int)(v % W), yv = (int)((v / W) % H), z = (int)((v / ((long long)W * H)) % D);
        const long long nb = v / ((long long)W * H * D);
        float acc = b0;
        for (int tap = 0; tap < 27; ++tap) {
            const int zz = z + tap / 9 - 1, yy = yv + (tap / 3) % 3 - 1, xx = xv + tap % 3 - 1;
            if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            const bf16 *p = x + (((nb * D + zz) * H + yy) * W + xx) * cs;
            for (int ci = 0; ci < cin; ++ci) acc = fmaf(ws[tap * cin + ci], __bfloat162float(p[ci]), acc);
        }
        out[v] = acc + (res ? res[v] : 0.0f);
    }
}

// dx[v][ci] = sum_tap w[tap][ci] g[v - off(tap)]
__global__ void head_dgrad_kernel(const float *__restrict__ g, const float *__restrict__ w,
                                  bf16 *__restrict__ dx, int cs, int N, int D, int H, int W, int cin) {
    extern __shared__ float ws[];
    for (int t = threadIdx.x; t < 27 * cin; t += blockDim.x) ws[t] = w[t];
    __syncthreads();
    const long long nvox = (long long)N * D * H * W;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        const int xv = (int)(v % W), yv = (int)((v / W) % H), z = (int)((v / ((long long)W * H)) % D);
        const long long nb = v / ((long long)W * H * D);
        float gt[27];
#pragma unroll
        for (int tap = 0; tap < 27; ++tap) {
            const int zz = z - (tap / 9 - 1), yy = yv - ((tap / 3) % 3 - 1), xx = xv - (tap % 3 - 1);
            gt[tap] = (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W)
                          ? 0.0f : g[((nb * D + zz) * H + yy) * W + xx];
        }
        for (int ci = 0; ci < cin; ++ci) {
            float acc = 0.0f;
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) acc = fmaf(ws[tap * cin + ci], gt[tap], acc);
            dx[v * cs + ci] = __float2bfloat16_rn(acc);
        }
    }
}

// dw[tap][ci] += sum_v g[v] x[v + off(tap)][ci]; db += sum_v g[v]
__global__ void head_wgrad_kernel(const float *__restrict__ g, const bf16 *__restrict__ x, int cs,
                                  float *dw, float *db, int N, int D, int H, int W, int cin) {
    extern __shared__ float part[];   // [27*cin + 1]
    for (int t = threadIdx.x; t < 27 * cin + 1; t += blockDim.x) part[t] = 0.0f;
    __syncthreads();
    const long long nvox = (long long)N * D * H * W;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        const float gv = g[v];
        if (gv == 0.0f) continue;
        const int xv = (int)(v % W), yv = (int)((v / W) % H), z = (int)((v / ((long long)W * H)) % D);
        const long long nb = v / ((long long)W * H * D);
        atomicAdd(&part[27 * cin], gv);
        for (int tap = 0; tap < 27; ++tap) {
            const int zz = z + tap / 9 - 1, yy = yv + (tap / 3) % 3 - 1, xx = xv + tap % 3 - 1;
            if (zz < 0 || zz >= D || yy < 0 || yy >= H || xx < 0 || xx >= W) continue;
            const bf16 *p = x + (((nb * D + zz) * H + yy) * W + xx) * cs;
            for (int ci = 0; ci < cin; ++ci) atomicAdd(&part[tap * cin + ci], gv * __bfloat162float(p[ci]));
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 27 * cin; t += blockDim.x) atomicAdd(&dw[t], part[t]);
    if (threadIdx.x == 0) atomicAdd(db, part[27 * cin]);
}

// ---------------------------------------------------------------------------
// Element-wise kernels
// ---------------------------------------------------------------------------
__global__ void maxpool2_fwd_kernel(const bf16 *__restrict__ x, int cs, int coff, bf16 *__restrict__ y,
                                    int N, int D, int H, int W, int c) {
    const int Do = D / 2, Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Do * Ho * Wo * c;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(t % c);
        long long v = t / c;
        const int xo = (int)(v % Wo), yo = (int)((v / Wo) % Ho), zo = (int)((v / ((long long)Wo * Ho)) % Do);
        const long long nb = v / ((long long)Wo * Ho * Do);
        float m = -3.0e38f;
        for (int k = 0; k < 8; ++k) {
            const int z = 2 * zo + (k >> 2), yy = 2 * yo + ((k >> 1) & 1), xx = 2 * xo + (k & 1);
            m = fmaxf(m, __bfloat162float(x[(((nb * D + z) * H + yy) * W + xx) * cs + coff + ch]));
        }
        y[v * c + ch] = __float2bfloat16_rn(m);
    }
}

__global__ void maxpool2_bwd_kernel(const bf16 *__restrict__ x, int cs, int coff,
                                    const bf16 *__restrict__ dy, bf16 *__restrict__ dx, int dcs,
                                    int dcoff, int N, int D, int H, int W, int c) {
    const int Do = D / 2, Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Do * Ho * Wo * c;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(t % c);
        long long v = t / c;
        const int xo = (int)(v % Wo), yo = (int)((v / Wo) % Ho), zo = (int)((v / ((long long)Wo * Ho)) % Do);
        const long long nb = v / ((long long)Wo * Ho * Do);
        float m = -3.0e38f;
        int arg = 0;
        for (int k = 0; k < 8; ++k) {
            const int z = 2 * zo + (k >> 2), yy = 2 * yo + ((k >> 1) & 1), xx = 2 * xo + (k & 1);
            const float val = __bfloat162float(x[(((nb * D + z) * H + yy) * W + xx) * cs + coff + ch]);
            if (val > m) {
                m = val;
                arg = k;
            }
        }
        const int z = 2 * zo + (arg >> 2), yy = 2 * yo + ((arg >> 1) & 1), xx = 2 * xo + (arg & 1);
        bf16 *p = dx + (((nb * D + z) * H + yy) * W + xx) * dcs + dcoff + ch;
        *p = __float2bfloat16_rn(__bfloat162float(*p) + __bfloat162float(dy[v * c + ch]));
    }
}

// ---- 8-channel (16-byte) versions of the element-wise kernels: one index
// decomposition per 8 channels instead of per element; used when every
// channel stride and offset is a multiple of 8 and the pointers are 16-byte
// aligned (which channels-last tensors of this library always are).
__device__ __forceinline__ float2 bf2f(unsigned u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}
__device__ __forceinline__ unsigned f2bf(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<unsigned *>(&h);
}

__global__ void upsample2_fwd_v8(const uint4 *__restrict__ x, bf16 *__restrict__ y, int ycs, int ycoff,
                                 int N, int D, int H, int W, int c8) {
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
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long u = ((nb * (2 * D) + 2 * zv + (k >> 2)) * (2 * H) + 2 * yv + ((k >> 1) & 1)) * (2 * W) +
                                2 * xv + (k & 1);
            *reinterpret_cast<uint4 *>(y + u * ycs + ycoff + cv * 8) = val;
        }
    }
}

__global__ void upsample2_bwd_v8(const bf16 *__restrict__ dy, int dycs, int dycoff, uint4 *__restrict__ dx,
                                 int N, int D, int H, int W, int c8) {
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
        float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const long long u = ((nb * (2 * D) + 2 * zv + (k >> 2)) * (2 * H) + 2 * yv + ((k >> 1) & 1)) * (2 * W) +
                                2 * xv + (k & 1);
            const uint4 q = *reinterpret_cast<const uint4 *>(dy + u * dycs + dycoff + cv * 8);
            const float2 a = bf2f(q.x), b = bf2f(q.y), c = bf2f(q.z), d = bf2f(q.w);
            s[0] += a.x; s[1] += a.y; s[2] += b.x; s[3] += b.y;
            s[4] += c.x; s[5] += c.y; s[6] += d.x; s[7] += d.y;
        }
        dx[t] = make_uint4(f2bf(s[0], s[1]), f2bf(s[2], s[3]), f2bf(s[4], s[5]), f2bf(s[6], s[7]));
    }
}

__global__ void relu_bwd_v8(bf16 *__restrict__ g, int gcs, int gcoff, const bf16 *__restrict__ y, int ycs,
                            int ycoff, long long nvox, int c8) {
    const long long total = nvox * c8;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / c8;
        const int cv = (int)(t % c8);
        uint4 *gp = reinterpret_cast<uint4 *>(g + v * gcs + gcoff + cv * 8);
        const uint4 yq = *reinterpret_cast<const uint4 *>(y + v * ycs + ycoff + cv * 8);
        uint4 gq = *gp;
        unsigned *gw = reinterpret_cast<unsigned *>(&gq);
        const unsigned *yw = reinterpret_cast<const unsigned *>(&yq);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float2 yy = bf2f(yw[i]);
            // keep each half where y > 0, else +0
            unsigned keep = (yy.x > 0.0f ? 0x0000FFFFu : 0u) | (yy.y > 0.0f ? 0xFFFF0000u : 0u);
            gw[i] &= keep;
        }
        *gp = gq;
    }
}

__global__ void pack_input_v8(const float *__restrict__ x, uint4 *__restrict__ y, int c8, long long nvox) {
    const long long total = nvox * c8;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / c8;
        const int cv = (int)(t % c8);
        y[t] = cv == 0 ? make_uint4(f2bf(x[v], 0.0f), 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
    }
}

// Output head, four consecutive voxels along x per thread: per (dz, dy) the
// six input voxels x-1 .. x+4 are loaded once, 8 channels at a time (16-byte
// loads), and serve the three dx taps of all four outputs; the weights are
// read from shared memory as broadcasts.
__global__ void head_fwd_v4(const bf16 *__restrict__ x, int cs, const float *__restrict__ w,
                            const float *__restrict__ bptr, const float *__restrict__ res,
                            float *__restrict__ out, int N, int D, int H, int W, int cin) {
    extern __shared__ float ws[];   // [27][cin]
    for (int t = threadIdx.x; t < 27 * cin; t += blockDim.x) ws[t] = w[t];
    __syncthreads();
    const float b0 = bptr ? *bptr : 0.0f;
    const int W4 = W / 4;
    const long long total = (long long)N * D * H * W4;
    const int c8n = cin / 8;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        long long v = t;
        const int x0 = (int)(v % W4) * 4;
        v /= W4;
        const int yv = (int)(v % H);
        v /= H;
        const int z = (int)(v % D);
        const long long nb = v / D;
        float acc[4] = {b0, b0, b0, b0};
        for (int dz = 0; dz < 3; ++dz) {
            const int zz = z + dz - 1;
            if (zz < 0 || zz >= D) continue;
            for (int dy = 0; dy < 3; ++dy) {
                const int yy = yv + dy - 1;
                if (yy < 0 || yy >= H) continue;
                const bf16 *row = x + ((nb * D + zz) * H + yy) * (long long)W * cs;
                const float *wt = ws + (dz * 3 + dy) * 3 * cin;
                for (int g8 = 0; g8 < c8n; ++g8) {
                    float in[6][8];
#pragma unroll
                    for (int p = 0; p < 6; ++p) {
                        const int xx = x0 + p - 1;
                        if (xx >= 0 && xx < W) {
                            const uint4 q = *reinterpret_cast<const uint4 *>(row + (long long)xx * cs + g8 * 8);
                            const float2 a = bf2f(q.x), b = bf2f(q.y), c = bf2f(q.z), d = bf2f(q.w);
                            in[p][0] = a.x; in[p][1] = a.y; in[p][2] = b.x; in[p][3] = b.y;
                            in[p][4] = c.x; in[p][5] = c.y; in[p][6] = d.x; in[p][7] = d.y;
                        } else {
#pragma unroll
                            for (int j = 0; j < 8; ++j) in[p][j] = 0.0f;
                        }
                    }
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float wv = wt[dx * cin + g8 * 8 + j];
#pragma unroll
                            for (int o = 0; o < 4; ++o) acc[o] = fmaf(wv, in[o + dx][j], acc[o]);
                        }
                    }
                }
            }
        }
        const long long vo = ((nb * D + z) * H + yv) * (long long)W + x0;
#pragma unroll
        for (int o = 0; o < 4; ++o) out[vo + o] = acc[o] + (res ? res[vo + o] : 0.0f);
    }
}

// FP32 pairs: fma.rn.f32x2 (sm_100 family) computes two independent IEEE
// FMAs per instruction.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 upk2(f2x r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ f2x fma2x(f2x a, f2x b, f2x c) {
    f2x r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// A BF16 pair word (channel 2c in the low half) as its FP32 pair: BF16 is the
// upper half of the FP32 encoding, so one shift and one mask.
__device__ __forceinline__ f2x bfw2f2(unsigned u) {
    return pk2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}

// Output head (16 channels -> 1) on a shared-memory tile: 64 (x) x 8 (y) x 2
// (z) outputs per CTA of 256 threads, each owning four x-consecutive
// outputs. The haloed input (66 x 10 x 4 voxels, 16 BF16 channels = two
// 16-byte halves a voxel) is staged once. Within each 128-byte group of four
// voxels the eight halves are permuted by the group index, so the eight
// threads of a quarter-warp, which read the same offset of eight consecutive
// groups, hit eight different bank groups. Products run on channel pairs with
// fma.rn.f32x2; the pair sums are added once at the end.
constexpr int kHdTX = 64, kHdTY = 8, kHdTZ = 2, kHdCin = 16;
constexpr int kHdHX = kHdTX + 2, kHdHY = kHdTY + 2, kHdHZ = kHdTZ + 2;
constexpr int kHdRowChunks = (kHdHX + 3) / 4 * 8;   // 16-byte slots per staged row (17 groups)
constexpr int kHdSmem = kHdHZ * kHdHY * kHdRowChunks * 16;   // 87,040 bytes
constexpr int kHdThreads = 256;

__device__ __forceinline__ int head_slot(int row, int i, int h) {
    const int g = i >> 2;
    return row * kHdRowChunks + g * 8 + (((i & 3) * 2 + h) ^ (g & 7));
}

__global__ void __launch_bounds__(kHdThreads)
head_fwd_tile(const bf16 *__restrict__ x, int cs, const float *__restrict__ w, const float *__restrict__ bptr,
              const float *__restrict__ res, float *__restrict__ out, int D, int H, int W, int tx, int ty, int tz) {
    extern __shared__ __align__(128) uint4 hs[];
    __shared__ __align__(16) float ws[27 * kHdCin];
    long long r = blockIdx.x;
    const int x0 = (int)(r % tx) * kHdTX;
    r /= tx;
    const int y0 = (int)(r % ty) * kHdTY;
    r /= ty;
    const int z0 = (int)(r % tz) * kHdTZ;
    const long long nb = r / tz;
    for (int t = threadIdx.x; t < 27 * kHdCin; t += kHdThreads) ws[t] = w[t];
    // every copy of the CTA in flight at once (cp.async, zero fill outside the volume)
    for (int c = threadIdx.x; c < kHdHZ * kHdHY * kHdHX * 2; c += kHdThreads) {
        const int row = c / (kHdHX * 2), rem = c - row * (kHdHX * 2);
        const int i = rem >> 1, h = rem & 1;
        const int z = z0 + row / kHdHY - 1, yy = y0 + row % kHdHY - 1, xx = x0 + i - 1;
        const bool in = z >= 0 && z < D && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const bf16 *src = in ? x + (((nb * D + z) * H + yy) * (long long)W + xx) * cs + h * 8 : x;
        const unsigned dst = static_cast<unsigned>(__cvta_generic_to_shared(hs + head_slot(row, i, h)));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(in ? 16 : 0)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int t = threadIdx.x;
    const int ox = (t & 15) * 4, oy = (t >> 4) & 7, oz = t >> 7;
    const f2x *w2 = reinterpret_cast<const f2x *>(ws);   // [27][8] channel pairs
    f2x acc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int dz = 0; dz < 3; ++dz) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
            const int row = (oz + dz) * kHdHY + oy + dy;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                f2x X[6][4];
#pragma unroll
                for (int p = 0; p < 6; ++p) {
                    const uint4 q = hs[head_slot(row, ox + p, h)];
                    X[p][0] = bfw2f2(q.x);
                    X[p][1] = bfw2f2(q.y);
                    X[p][2] = bfw2f2(q.z);
                    X[p][3] = bfw2f2(q.w);
                }
#pragma unroll
                for (int dx = 0; dx < 3; ++dx) {
                    const int tap = (dz * 3 + dy) * 3 + dx;
                    f2x Wp[4];
#pragma unroll
                    for (int c2 = 0; c2 < 4; ++c2) Wp[c2] = w2[tap * 8 + h * 4 + c2];
#pragma unroll
                    for (int o = 0; o < 4; ++o)
#pragma unroll
                        for (int c2 = 0; c2 < 4; ++c2) acc[o] = fma2x(Wp[c2], X[o + dx][c2], acc[o]);
                }
            }
        }
    }
    const int z = z0 + oz, yy = y0 + oy;
    if (z >= D || yy >= H) return;
    const float b0 = bptr ? *bptr : 0.0f;
    const long long vo = ((nb * D + z) * H + yy) * (long long)W;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        const int xx = x0 + ox + o;
        if (xx < W) {
            const float2 a = upk2(acc[o]);
            out[vo + xx] = (a.x + a.y) + b0 + (res ? res[vo + xx] : 0.0f);
        }
    }
}

// 2x2x2 max pooling, eight channels (16 bytes) per thread; y dense.
__global__ void maxpool2_fwd_v8(const bf16 *__restrict__ x, int cs, int coff, uint4 *__restrict__ y, int N,
                                int D, int H, int W, int c8) {
    const int Do = D / 2, Ho = H / 2, Wo = W / 2;
    const long long total = (long long)N * Do * Ho * Wo * c8;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int cv = (int)(t % c8);
        long long v = t / c8;
        const int xo = (int)(v % Wo);
        v /= Wo;
        const int yo = (int)(v % Ho);
        v /= Ho;
        const int zo = (int)(v % Do);
        const long long nb = v / Do;
        float m[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) m[j] = -3.0e38f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int z = 2 * zo + (k >> 2), yy = 2 * yo + ((k >> 1) & 1), xx = 2 * xo + (k & 1);
            const uint4 q =
                *reinterpret_cast<const uint4 *>(x + (((nb * D + z) * H + yy) * (long long)W + xx) * cs + coff + cv * 8);
            const float2 a = bf2f(q.x), b = bf2f(q.y), c = bf2f(q.z), d = bf2f(q.w);
            m[0] = fmaxf(m[0], a.x); m[1] = fmaxf(m[1], a.y); m[2] = fmaxf(m[2], b.x); m[3] = fmaxf(m[3], b.y);
            m[4] = fmaxf(m[4], c.x); m[5] = fmaxf(m[5], c.y); m[6] = fmaxf(m[6], d.x); m[7] = fmaxf(m[7], d.y);
        }
        y[t] = make_uint4(f2bf(m[0], m[1]), f2bf(m[2], m[3]), f2bf(m[4], m[5]), f2bf(m[6], m[7]));
    }
}

__global__ void upsample2_fwd_kernel(const bf16 *__restrict__ x, bf16 *__restrict__ y, int ycs,
                                     int ycoff, int N, int D, int H, int W, int c) {
    const int Du = 2 * D, Hu = 2 * H, Wu = 2 * W;
    const long long total = (long long)N * Du * Hu * Wu * c;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(t % c);
        long long v = t / c;
        const int xu = (int)(v % Wu), yu = (int)((v / Wu) % Hu), zu = (int)((v / ((long long)Wu * Hu)) % Du);
        const long long nb = v / ((long long)Wu * Hu * Du);
        y[v * ycs + ycoff + ch] = x[(((nb * D + zu / 2) * H + yu / 2) * W + xu / 2) * c + ch];
    }
}

__global__ void upsample2_bwd_kernel(const bf16 *__restrict__ dy, int dycs, int dycoff,
                                     bf16 *__restrict__ dx, int N, int D, int H, int W, int c) {
    const long long total = (long long)N * D * H * W * c;
    const int Hu = 2 * H, Wu = 2 * W, Du = 2 * D;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(t % c);
        long long v = t / c;
        const int xv = (int)(v % W), yv = (int)((v / W) % H), z = (int)((v / ((long long)W * H)) % D);
        const long long nb = v / ((long long)W * H * D);
        float s = 0.0f;
        for (int k = 0; k < 8; ++k) {
            const int zu = 2 * z + (k >> 2), yu = 2 * yv + ((k >> 1) & 1), xu = 2 * xv + (k & 1);
            s += __bfloat162float(dy[(((nb * Du + zu) * Hu + yu) * Wu + xu) * dycs + dycoff + ch]);
        }
        dx[v * c + ch] = __float2bfloat16_rn(s);
    }
}

__global__ void relu_bwd_kernel(bf16 *__restrict__ g, int gcs, int gcoff, const bf16 *__restrict__ y,
                                int ycs, int ycoff, long long nvox, int c) {
    const long long total = nvox * c;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const long long v = t / c;
        const int ch = (int)(t % c);
        if (!(__bfloat162float(y[v * ycs + ycoff + ch]) > 0.0f))
            g[v * gcs + gcoff + ch] = __float2bfloat16_rn(0.0f);
    }
}

__global__ void pack_input_kernel(const float *__restrict__ x, bf16 *__restrict__ y, int cs,
                                  long long nvox) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox;
         v += (long long)gridDim.x * blockDim.x) {
        y[v * cs] = __float2bfloat16_rn(x[v]);
        for (int c = 1; c < cs; ++c) y[v * cs + c] = __float2bfloat16_rn(0.0f);
    }
}

__global__ void mse_kernel(const float *__restrict__ p, const float *__restrict__ t, float *__restrict__ g,
                           float *loss, long long n) {
    __shared__ float red[32];
    float s = 0.0f;
    const float inv = 2.0f / (float)n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float d = p[i] - t[i];
        g[i] = inv * d;
        s = fmaf(d, d, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(loss, s);
    }
}

__global__ void adam_kernel(float *__restrict__ p, float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, bf16 *__restrict__ p16, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (p16) p16[i] = __float2bfloat16_rn(pi);
        g[i] = 0.0f;
    }
}

// ---------------------------------------------------------------------------
// Host wrappers
// ---------------------------------------------------------------------------
static unsigned ew_blocks(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535LL * 16 ? 65535LL * 16 : b));
}

static bp_status launch_ok(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(nullptr, e, what);
}

static bool al16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static TileGrid make_grid(int n, int d, int h, int wd, long long *ntiles) {
    TileGrid g;
    g.tx = (wd + kTX - 1) / kTX;
    g.ty = (h + kTY - 1) / kTY;
    g.tz = (d + kTZ - 1) / kTZ;
    *ntiles = (long long)n * g.tx * g.ty * g.tz;
    return g;
}

bool conv_tc_applies(const void *x, int xcs, int xco, const void *w, const void *y, int ycs, int yco, int yf32,
                     int d, int h, int wd, int cin, int cout);
cudaError_t conv_fwd_tc(const void *x, int xcs, int xco, const void *w, const float *b, void *y, int ycs, int yco,
                        int yf32, int n, int d, int h, int wd, int cin, int cout, int relu, cudaStream_t st,
                        const float *head_w = nullptr, const float *head_b = nullptr,
                        const float *head_res = nullptr, float *head_out = nullptr);
bool conv_tcp_applies(int cin, int cout);

static bp_status conv_fwd(const bf16 *x, int xcs, int xco, const bf16 *w, const float *b, void *y,
                          int ycs, int yco, int yf32, int n, int d, int h, int wd, int cin, int cout,
                          int relu, cudaStream_t st) {
    // tcgen05 implicit GEMM (k_conv_tc.cu) where its tile fits the layer
    if (conv_tc_applies(x, xcs, xco, w, y, ycs, yco, yf32, d, h, wd, cin, cout)) {
        cudaError_t e = conv_fwd_tc(x, xcs, xco, w, b, y, ycs, yco, yf32, n, d, h, wd, cin, cout, relu, st);
        return e == cudaSuccess ? BP_OK : cuda_fail(nullptr, e, "conv3d_fwd_tc");
    }
    long long nt;
    TileGrid g = make_grid(n, d, h, wd, &nt);
    if (nt > 0x7fffffffLL) return fail(nullptr, BP_ERR_INVALID_ARG, "conv3d: volume too large");
#define CONV_CASE(C)                                                                                 \
    case C:                                                                                          \
        if (yf32)                                                                                    \
            conv3d_fwd_kernel<C, true><<<(unsigned)nt, kConvThreads, 0, st>>>(x, xcs, xco, w, b, y, ycs, yco, d, h, wd, cin, relu, g); \
        else                                                                                         \
            conv3d_fwd_kernel<C, false><<<(unsigned)nt, kConvThreads, 0, st>>>(x, xcs, xco, w, b, y, ycs, yco, d, h, wd, cin, relu, g); \
        break;
    switch (cout) {
        CONV_CASE(16) CONV_CASE(32) CONV_CASE(64)
        default: return fail(nullptr, BP_ERR_UNSUPPORTED, "conv3d: cout must be 16, 32 or 64");
    }
#undef CONV_CASE
    return launch_ok("conv3d_fwd_kernel");
}

static bool conv_args_ok(int cs, int coff, int c) { return cs % 8 == 0 && coff % 8 == 0 && coff + c <= cs; }

// Scratch of cnn_conv3d_dgrad_noalloc: the flipped, transposed weights live
// in this fixed device array instead of a caller buffer. 27 * 128 * 128 BF16
// values (864 KiB), reserved on every GPU that loads the library until the
// process exits. Host code must not pass the name itself to a kernel (on the
// host it only stands for the symbol); the device address comes from
// cudaGetSymbolAddress, looked up once per device and cached.
constexpr long long kNoAllocScratchElems = 27LL * 128 * 128;
static __device__ __align__(256) bf16 g_dgrad_scratch[kNoAllocScratchElems];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static void *g_scratch_addr[kMaxDevices] = {};

static bp_status dgrad_scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cnn_conv3d_dgrad_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices)
        return fail(nullptr, BP_ERR_UNSUPPORTED, "cnn_conv3d_dgrad_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_dgrad_scratch);
        if (e != cudaSuccess || !p)
            return cuda_fail(nullptr, e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                             "cnn_conv3d_dgrad_noalloc: cudaGetSymbolAddress");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BP_OK;
}

}  // namespace bp

using namespace bp;

extern "C" {

bp_status cnn_conv3d_forward(const void *x, int x_cstride, int x_coff, const void *w, const float *b,
                             void *y, int y_cstride, int y_coff, int y_fp32, int n, int d, int h,
                             int wd, int cin, int cout, int relu, void *stream) {
    if (!x || !w || !y || n < 1 || d < 1 || h < 1 || wd < 1 || cin < 16 || cin % 16 ||
        !conv_args_ok(x_cstride, x_coff, cin) || !conv_args_ok(y_cstride, y_coff, cout) ||
        !al16(x) || !al16(w) || !al16(y))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_conv3d_forward: bad arguments");
    return conv_fwd((const bf16 *)x, x_cstride, x_coff, (const bf16 *)w, b, y, y_cstride, y_coff,
                    y_fp32, n, d, h, wd, cin, cout, relu, (cudaStream_t)stream);
}

bp_status cnn_conv3d_forward_head(const void *x, int x_cstride, int x_coff, const void *w, const float *b,
                                  const float *head_w, const float *head_b, const float *res, float *out, int n,
                                  int d, int h, int wd, int cin, int cout, int relu, void *stream) {
    if (!x || !w || !head_w || !out || n < 1 || d < 1 || h < 1 || wd < 1 || cin < 16 || cin % 16 ||
        !conv_args_ok(x_cstride, x_coff, cin) || !al16(x) || !al16(w))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_conv3d_forward_head: bad arguments");
    if (wd % 128 != 0 || !conv_tcp_applies(cin, cout) ||
        !conv_tc_applies(x, x_cstride, x_coff, w, out, cout, 0, 0, d, h, wd, cin, cout))
        return fail(nullptr, BP_ERR_UNSUPPORTED, "cnn_conv3d_forward_head: layer outside the persistent tcgen05 kernel");
    cudaError_t e = conv_fwd_tc(x, x_cstride, x_coff, w, b, nullptr, cout, 0, 0, n, d, h, wd, cin, cout, relu,
                                (cudaStream_t)stream, head_w, head_b, res, out);
    return e == cudaSuccess ? BP_OK : cuda_fail(nullptr, e, "conv3d_fwd_tcp (fused head)");
}

bp_status cnn_conv3d_dgrad(const void *dy, int dy_cstride, int dy_coff, const void *w, void *wt,
                           void *dx, int dx_cstride, int dx_coff, int n, int d, int h, int wd,
                           int cin, int cout, void *stream) {
    if (!dy || !w || !wt || !dx || cin < 16 || cin % 16 || cout % 16 ||
        !conv_args_ok(dy_cstride, dy_coff, cout) || !conv_args_ok(dx_cstride, dx_coff, cin) ||
        !al16(dy) || !al16(w) || !al16(wt) || !al16(dx))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_conv3d_dgrad: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    flip_transpose_kernel<<<ew_blocks(27LL * cin * cout), 256, 0, st>>>((const bf16 *)w, (bf16 *)wt, cin, cout);
    bp_status s = launch_ok("flip_transpose_kernel");
    if (s != BP_OK) return s;
    // dx = conv(dy, wt) with cin' = cout, cout' = cin, no bias, no activation;
    // the input-gradient channels go in blocks of 64, 32 or 16 (the tile
    // widths the tensor-core kernel is built for)
    for (int ci0 = 0; ci0 < cin;) {
        const int left = cin - ci0;
        const int blk = left >= 64 ? 64 : (left >= 32 ? 32 : 16);
        s = conv_fwd((const bf16 *)dy, dy_cstride, dy_coff, (const bf16 *)wt + (size_t)ci0 * 27 * cout,
                     nullptr, dx, dx_cstride, dx_coff + ci0, 0, n, d, h, wd, cout, blk, 0, st);
        if (s != BP_OK) return s;
        ci0 += blk;
    }
    return BP_OK;
}

// Same result as cnn_conv3d_dgrad without the caller's weight buffer: for
// callers that cannot allocate device memory (see unet.h). Allocates
// nothing; the scratch is the library's static array above.
bp_status cnn_conv3d_dgrad_noalloc(const void *dy, int dy_cstride, int dy_coff, const void *w,
                                   void *dx, int dx_cstride, int dx_coff, int n, int d, int h,
                                   int wd, int cin, int cout, void *stream) {
    if (!dy || !w || !dx || cin < 16 || cin % 16 || cout % 16 ||
        !conv_args_ok(dy_cstride, dy_coff, cout) || !conv_args_ok(dx_cstride, dx_coff, cin) ||
        !al16(dy) || !al16(w) || !al16(dx))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_conv3d_dgrad_noalloc: bad arguments");
    if (27LL * cin * cout > kNoAllocScratchElems)
        return fail(nullptr, BP_ERR_INVALID_ARG,
                    "cnn_conv3d_dgrad_noalloc: cin * cout exceeds the static scratch limit of 16384 "
                    "(27 * cin * cout BF16 values must fit 442368); use cnn_conv3d_dgrad");
    void *wt = nullptr;
    bp_status s = dgrad_scratch_address(&wt);
    if (s != BP_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    // every element of the scratch that the convolution reads is written
    // here first, so nothing left by an earlier call is ever used
    flip_transpose_kernel<<<ew_blocks(27LL * cin * cout), 256, 0, st>>>((const bf16 *)w, (bf16 *)wt, cin, cout);
    s = launch_ok("flip_transpose_kernel");
    if (s != BP_OK) return s;
    for (int ci0 = 0; ci0 < cin;) {
        const int left = cin - ci0;
        const int blk = left >= 64 ? 64 : (left >= 32 ? 32 : 16);
        s = conv_fwd((const bf16 *)dy, dy_cstride, dy_coff, (const bf16 *)wt + (size_t)ci0 * 27 * cout,
                     nullptr, dx, dx_cstride, dx_coff + ci0, 0, n, d, h, wd, cout, blk, 0, st);
        if (s != BP_OK) return s;
        ci0 += blk;
    }
    return BP_OK;
}

bp_status cnn_conv3d_wgrad(const void *x, int x_cstride, int x_coff, const void *dy, int dy_cstride,
                           int dy_coff, float *dw, float *db, int n, int d, int h, int wd, int cin,
                           int cout, void *stream) {
    if (!x || !dy || !dw || cin < 16 || cin % 16 || !conv_args_ok(x_cstride, x_coff, cin) ||
        !conv_args_ok(dy_cstride, dy_coff, cout) || !al16(x) || !al16(dy))
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_conv3d_wgrad: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    long long nt;
    TileGrid g = make_grid(n, d, h, wd, &nt);
    dim3 grid((unsigned)((nt + kWgTiles - 1) / kWgTiles), cin / 16, 3);
    switch (cout) {
        case 16: conv3d_wgrad_kernel<16><<<grid, kConvThreads, 0, st>>>((const bf16 *)x, x_cstride, x_coff, (const bf16 *)dy, dy_cstride, dy_coff, dw, d, h, wd, cin, nt, g); break;
        case 32: conv3d_wgrad_kernel<32><<<grid, kConvThreads, 0, st>>>((const bf16 *)x, x_cstride, x_coff, (const bf16 *)dy, dy_cstride, dy_coff, dw, d, h, wd, cin, nt, g); break;
        case 64: conv3d_wgrad_kernel<64><<<grid, kConvThreads, 0, st>>>((const bf16 *)x, x_cstride, x_coff, (const bf16 *)dy, dy_cstride, dy_coff, dw, d, h, wd, cin, nt, g); break;
        default: return fail(nullptr, BP_ERR_UNSUPPORTED, "cnn_conv3d_wgrad: cout must be 16, 32 or 64");
    }
    bp_status s = launch_ok("conv3d_wgrad_kernel");
    if (s != BP_OK || !db) return s;
    const long long nvox = (long long)n * d * h * wd;
    bias_grad_kernel<<<ew_blocks(nvox * cout / 64), 256, cout * sizeof(float), st>>>(
        (const bf16 *)dy, dy_cstride, dy_coff, db, nvox, cout);
    return launch_ok("bias_grad_kernel");
}

bp_status cnn_head_forward(const void *x, int x_cstride, const float *w, const float *b, const float *res,
                           float *out, int n, int d, int h, int wd, int cin, void *stream) {
    if (!x || !w || !out || cin < 1 || cin > x_cstride || n < 1)
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_head_forward: bad arguments");
    const long long nvox = (long long)n * d * h * wd;
    if (cin == kHdCin && x_cstride % 8 == 0 && al16(x)) {
        const int tx = (wd + kHdTX - 1) / kHdTX, ty = (h + kHdTY - 1) / kHdTY, tz = (d + kHdTZ - 1) / kHdTZ;
        const long long nt = (long long)n * tx * ty * tz;
        if (nt > 0x7fffffffLL) return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_head_forward: volume too large");
        cudaError_t e = cudaFuncSetAttribute(head_fwd_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, kHdSmem);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cnn_head_forward: shared memory limit");
        head_fwd_tile<<<(unsigned)nt, kHdThreads, kHdSmem, (cudaStream_t)stream>>>(
            (const bf16 *)x, x_cstride, w, b, res, out, d, h, wd, tx, ty, tz);
        return launch_ok("head_fwd_tile");
    }
    if (cin % 8 == 0 && x_cstride % 8 == 0 && wd % 4 == 0 && al16(x)) {
        head_fwd_v4<<<ew_blocks(nvox / 4), 256, 27 * cin * sizeof(float), (cudaStream_t)stream>>>(
            (const bf16 *)x, x_cstride, w, b, res, out, n, d, h, wd, cin);
        return launch_ok("head_fwd_v4");
    }
    head_fwd_kernel<<<ew_blocks(nvox), 256, 27 * cin * sizeof(float), (cudaStream_t)stream>>>(
        (const bf16 *)x, x_cstride, w, b, res, out, n, d, h, wd, cin);
    return launch_ok("head_fwd_kernel");
}

bp_status cnn_head_backward(const void *x, int x_cstride, const float *w, const float *g, void *dx,
                            int dx_cstride, float *dw, float *db, int n, int d, int h, int wd,
                            int cin, void *stream) {
    if (!x || !w || !g || !dx || !dw || !db || cin < 1 || cin > x_cstride || cin > dx_cstride)
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_head_backward: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const long long nvox = (long long)n * d * h * wd;
    head_dgrad_kernel<<<ew_blocks(nvox), 256, 27 * cin * sizeof(float), st>>>(g, w, (bf16 *)dx, dx_cstride, n, d, h, wd, cin);
    bp_status s = launch_ok("head_dgrad_kernel");
    if (s != BP_OK) return s;
    head_wgrad_kernel<<<ew_blocks(nvox / 8), 256, (27 * cin + 1) * sizeof(float), st>>>(g, (const bf16 *)x, x_cstride, dw, db, n, d, h, wd, cin);
    return launch_ok("head_wgrad_kernel");
}

bp_status cnn_maxpool2_forward(const void *x, int x_cstride, int x_coff, void *y, int n, int d, int h,
                               int wd, int c, void *stream) {
    if (!x || !y || d % 2 || h % 2 || wd % 2 || x_coff + c > x_cstride)
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_maxpool2_forward: bad arguments");
    if (c % 8 == 0 && x_cstride % 8 == 0 && x_coff % 8 == 0 && al16(x) && al16(y)) {
        const long long tot8 = (long long)n * (d / 2) * (h / 2) * (wd / 2) * (c / 8);
        maxpool2_fwd_v8<<<ew_blocks(tot8), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, x_cstride, x_coff, (uint4 *)y, n, d, h, wd, c / 8);
        return launch_ok("maxpool2_fwd_v8");
    }
    const long long tot = (long long)n * (d / 2) * (h / 2) * (wd / 2) * c;
    maxpool2_fwd_kernel<<<ew_blocks(tot), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, x_cstride, x_coff, (bf16 *)y, n, d, h, wd, c);
    return launch_ok("maxpool2_fwd_kernel");
}

bp_status cnn_maxpool2_backward(const void *x, int x_cstride, int x_coff, const void *dy, void *dx,
                                int dx_cstride, int dx_coff, int n, int d, int h, int wd, int c,
                                void *stream) {
    if (!x || !dy || !dx || d % 2 || h % 2 || wd % 2)
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_maxpool2_backward: bad arguments");
    const long long tot = (long long)n * (d / 2) * (h / 2) * (wd / 2) * c;
    maxpool2_bwd_kernel<<<ew_blocks(tot), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, x_cstride, x_coff, (const bf16 *)dy, (bf16 *)dx, dx_cstride, dx_coff, n, d, h, wd, c);
    return launch_ok("maxpool2_bwd_kernel");
}

bp_status cnn_upsample2_forward(const void *x, void *y, int y_cstride, int y_coff, int n, int d, int h,
                                int wd, int c, void *stream) {
    if (!x || !y || y_coff + c > y_cstride)
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_upsample2_forward: bad arguments");
    if (c % 8 == 0 && y_cstride % 8 == 0 && y_coff % 8 == 0 && al16(x) && al16(y)) {
        const long long tot8 = (long long)n * d * h * wd * (c / 8);
        upsample2_fwd_v8<<<ew_blocks(tot8), 256, 0, (cudaStream_t)stream>>>((const uint4 *)x, (bf16 *)y, y_cstride, y_coff, n, d, h, wd, c / 8);
        return launch_ok("upsample2_fwd_v8");
    }
    const long long tot = (long long)n * 8 * d * h * wd * c;
    upsample2_fwd_kernel<<<ew_blocks(tot), 256, 0, (cudaStream_t)stream>>>((const bf16 *)x, (bf16 *)y, y_cstride, y_coff, n, d, h, wd, c);
    return launch_ok("upsample2_fwd_kernel");
}

bp_status cnn_upsample2_backward(const void *dy, int dy_cstride, int dy_coff, void *dx, int n, int d,
                                 int h, int wd, int c, void *stream) {
    if (!dy || !dx || dy_coff + c > dy_cstride)
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_upsample2_backward: bad arguments");
    if (c % 8 == 0 && dy_cstride % 8 == 0 && dy_coff % 8 == 0 && al16(dy) && al16(dx)) {
        const long long tot8 = (long long)n * d * h * wd * (c / 8);
        upsample2_bwd_v8<<<ew_blocks(tot8), 256, 0, (cudaStream_t)stream>>>((const bf16 *)dy, dy_cstride, dy_coff, (uint4 *)dx, n, d, h, wd, c / 8);
        return launch_ok("upsample2_bwd_v8");
    }
    const long long tot = (long long)n * d * h * wd * c;
    upsample2_bwd_kernel<<<ew_blocks(tot), 256, 0, (cudaStream_t)stream>>>((const bf16 *)dy, dy_cstride, dy_coff, (bf16 *)dx, n, d, h, wd, c);
    return launch_ok("upsample2_bwd_kernel");
}

bp_status cnn_relu_backward(void *g, int g_cstride, int g_coff, const void *y, int y_cstride, int y_coff,
                            long long nvox, int c, void *stream) {
    if (!g || !y || g_coff + c > g_cstride || y_coff + c > y_cstride)
        return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_relu_backward: bad arguments");
    if (c % 8 == 0 && g_cstride % 8 == 0 && g_coff % 8 == 0 && y_cstride % 8 == 0 && y_coff % 8 == 0 && al16(g) &&
        al16(y)) {
        relu_bwd_v8<<<ew_blocks(nvox * (c / 8)), 256, 0, (cudaStream_t)stream>>>((bf16 *)g, g_cstride, g_coff, (const bf16 *)y, y_cstride, y_coff, nvox, c / 8);
        return launch_ok("relu_bwd_v8");
    }
    relu_bwd_kernel<<<ew_blocks(nvox * c), 256, 0, (cudaStream_t)stream>>>((bf16 *)g, g_cstride, g_coff, (const bf16 *)y, y_cstride, y_coff, nvox, c);
    return launch_ok("relu_bwd_kernel");
}

bp_status cnn_pack_input(const float *x, void *y, int cstride, long long nvox, void *stream) {
    if (!x || !y || cstride < 1) return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_pack_input: bad arguments");
    if (cstride % 8 == 0 && al16(y)) {
        pack_input_v8<<<ew_blocks(nvox * (cstride / 8)), 256, 0, (cudaStream_t)stream>>>(x, (uint4 *)y, cstride / 8, nvox);
        return launch_ok("pack_input_v8");
    }
    pack_input_kernel<<<ew_blocks(nvox), 256, 0, (cudaStream_t)stream>>>(x, (bf16 *)y, cstride, nvox);
    return launch_ok("pack_input_kernel");
}

bp_status cnn_mse(const float *p, const float *t, float *g, float *loss, long long n, void *stream) {
    if (!p || !t || !g || !loss || n < 1) return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_mse: bad arguments");
    mse_kernel<<<ew_blocks(n) > 4096 ? 4096 : ew_blocks(n), 256, 0, (cudaStream_t)stream>>>(p, t, g, loss, n);
    return launch_ok("mse_kernel");
}

bp_status cnn_adam(float *p, float *g, float *m, float *v, void *p16, long long n, float lr, float b1,
                   float b2, float eps, int t, void *stream) {
    if (!p || !g || !m || !v || n < 1 || t < 1) return fail(nullptr, BP_ERR_INVALID_ARG, "cnn_adam: bad arguments");
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    adam_kernel<<<ew_blocks(n), 256, 0, (cudaStream_t)stream>>>(p, g, m, v, (bf16 *)p16, n, lr, b1, b2, eps, c1, c2);
    return launch_ok("adam_kernel");
}

}  // extern "C"
