// FDK pre-filter (the paper assumes filtered projections, Section 2.1.2):
// cosine weight, then the linear convolution of every detector row with the
// discrete Ram-Lak kernel, done as a zero-padded FFT convolution in shared
// memory. Rows of up to 5120 pixels go to the four-row kernel of
// filter_ct.cuh; this file holds the dispatch, the host tables of that
// kernel and, for longer rows (N = 16384), a two-row kernel with one float2
// per point. Two real rows travel as the real and imaginary parts of one
// complex FFT: the kernel's spectrum is real and even, so the product keeps
// the two rows apart.
//
// The two-row kernel's FFT is a Stockham autosort transform with radix-16
// passes (a last pass of radix 2/4/8 when log2 N is not a multiple of 4):
// every thread holds R points of one butterfly group in registers, applies
// the inter-pass twiddles from a table, runs an R-point DFT in registers and
// writes the results to their sorted positions, so each pass reads and
// writes shared memory once and the output comes out in natural order. The
// first forward pass reads the projections from global memory (with the
// cosine weight); the last forward pass multiplies by the spectrum of the
// kernel (which carries dp and the 1/N of the inverse); the last inverse
// pass writes the first nu samples of each row to global memory.
#include <cmath>
#include <cstdint>

#include "bp_internal.h"
#include "filter_ct.cuh"

namespace bp {

constexpr int kFilterThreads = 256;

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// x * exp(DIR * i * pi / 2): forward (DIR = -1) multiplies by -i
template <int DIR>
__device__ __forceinline__ float2 rot4(float2 x) {
    return DIR < 0 ? make_float2(x.y, -x.x) : make_float2(-x.y, x.x);
}

// cos and sin of 2*pi*m/16, m = 0..15
__device__ __constant__ float kC16[16] = {
    1.0f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f, 0.0f,
    -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f, -1.0f,
    -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f, 0.0f,
    0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
__device__ __constant__ float kS16[16] = {
    0.0f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f, 1.0f,
    0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f, 0.0f,
    -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f, -1.0f,
    -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f};

// exp(DIR * 2 pi i * m / 16) with m a compile-time constant after unrolling
template <int DIR>
__device__ __forceinline__ float2 w16(int m) {
    m &= 15;
    return make_float2(kC16[m], DIR < 0 ? -kS16[m] : kS16[m]);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
    float2 a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = rot4<DIR>(csub(x1, x3));
    x0 = cadd(a, c);
    x2 = csub(a, c);
    x1 = cadd(b, d);
    x3 = csub(b, d);
}

template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<2, DIR> {
    __device__ __forceinline__ static void run(float2 *v) {
        float2 a = v[0];
        v[0] = cadd(a, v[1]);
        v[1] = csub(a, v[1]);
    }
};

template <int DIR>
struct Dft<4, DIR> {
    __device__ __forceinline__ static void run(float2 *v) { dft4<DIR>(v[0], v[1], v[2], v[3]); }
};

template <int DIR>
struct Dft<8, DIR> {
    // X[k1 + 4 k2] = E[k1] + (-1)^k2 W8^k1 O[k1], E/O = DFT4 of even/odd inputs
    __device__ __forceinline__ static void run(float2 *v) {
        float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4<DIR>(e0, e1, e2, e3);
        dft4<DIR>(o0, o1, o2, o3);
        o1 = cmul(o1, w16<DIR>(2));
        o2 = rot4<DIR>(o2);
        o3 = cmul(o3, w16<DIR>(6));
        v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
        v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
        v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
        v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
    }
};

template <int DIR>
struct Dft<16, DIR> {
    // n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W16^(n2 k1), DFT4 over n2
    __device__ __forceinline__ static void run(float2 *v) {
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4<DIR>(v[n2], v[n2 + 4], v[n2 + 8], v[n2 + 12]);
        // after the first layer, v[n2 + 4 k1] holds A[n2][k1]
#pragma unroll
        for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
            for (int k1 = 1; k1 < 4; ++k1) v[n2 + 4 * k1] = cmul(v[n2 + 4 * k1], w16<DIR>(n2 * k1));
        float2 t[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            float2 a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
            dft4<DIR>(a0, a1, a2, a3);
            t[k1] = a0; t[k1 + 4] = a1; t[k1 + 8] = a2; t[k1 + 12] = a3;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = t[i];
    }
};

template <typename TO>
__device__ __forceinline__ void store_out(TO *p, float v);
template <>
__device__ __forceinline__ void store_out<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_out<__half>(__half *p, float v) { *p = __float2half_rn(v); }

struct FilterArgs {
    const float *in;
    void *out;
    long long nrows;
    int nu, nv, pairs;
    const float *H;     // [N] natural order
    const float2 *tw;   // [N] exp(-2 pi i m / N)
    float sdd, du, dv, cu, cv;
};

// Shared-memory position of complex sample m: one pad slot every 16 samples,
// so the stride-16 writes of the first Stockham pass hit distinct banks.
__device__ __forceinline__ int pad16(int m) { return m + (m >> 4); }

// Row pairs per CTA for transform size N: 4096 complex points per CTA.
template <int N>
struct PairsPerCta {
    static constexpr int value = N >= 4096 ? 1 : 4096 / N;
};

// One Stockham pass of radix R over all row pairs of the CTA. Each thread
// loads every group it owns before the barrier and stores after it, so the
// pass can work in place.
//   MODE 0: smem -> smem;  MODE 1: global (cosine-weighted) -> smem;
//   MODE 2: smem -> smem with the spectrum multiply;  MODE 3: smem -> global
template <typename TO, int N, int R, int NS, int DIR, int MODE>
__device__ __forceinline__ void stockham_pass(float2 *buf, const FilterArgs &a, long long row0) {
    constexpr int G = N / R;
    constexpr int NG = PairsPerCta<N>::value * G;
    constexpr int GPT = (NG + kFilterThreads - 1) / kFilterThreads;
    float2 v[GPT][R];
#pragma unroll
    for (int q = 0; q < GPT; ++q) {
        const int g = q * kFilterThreads + threadIdx.x;
        if (g >= NG) continue;
        const int p = g / G, j = g % G;
        const int k = j % NS;
        if (MODE == 1) {
            const long long ra = row0 + 2 * p, rb = ra + 1;
            const float sdd2 = a.sdd * a.sdd;
            float vma = ((float)(ra % a.nv) - a.cv) * a.dv;
            float vmb = ((float)(rb % a.nv) - a.cv) * a.dv;
            vma *= vma;
            vmb *= vmb;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = j + r * G;
                float xa = 0.0f, xb = 0.0f;
                // N >= 2 nu - 1 gives nu <= N/2 = (R/2) G, so r >= R/2 reads only padding
                if (r < R / 2 && m < a.nu) {
                    float um = ((float)m - a.cu) * a.du;
                    um *= um;
                    if (ra < a.nrows) xa = a.in[ra * a.nu + m] * (a.sdd * rsqrtf(sdd2 + um + vma));
                    if (rb < a.nrows) xb = a.in[rb * a.nu + m] * (a.sdd * rsqrtf(sdd2 + um + vmb));
                }
                v[q][r] = make_float2(xa, xb);
            }
        } else {
            // (j + r G) >> 4 = (j >> 4) + r G/16 for G a multiple of 16: one
            // padded base address and compile-time offsets
            const float2 *src = buf + pad16(p * N + j);
#pragma unroll
            for (int r = 0; r < R; ++r)
                v[q][r] = (G % 16 == 0) ? src[r * (G + G / 16)] : buf[pad16(p * N + j + r * G)];
        }
        if (NS > 1) {
            // twiddles w^r: powers of two from the table, the others as one
            // product of two table entries (error of a few ulp at most)
            float2 w[R];
            w[0] = make_float2(1.0f, 0.0f);
#pragma unroll
            for (int r = 1; r < R; ++r) {
                if (r == 1 || r == 4 || r == 8 || (r == 2 && R <= 4)) {
                    w[r] = __ldg(&a.tw[(k * r) * (N / (NS * R))]);
                    if (DIR > 0) w[r].y = -w[r].y;
                } else if (r == 2) {
                    w[r] = cmul(w[1], w[1]);
                } else {
                    const int hb = (r >= 8) ? 8 : (r >= 4 ? 4 : 2);
                    w[r] = cmul(w[hb], w[r - hb]);
                }
            }
#pragma unroll
            for (int r = 1; r < R; ++r) v[q][r] = cmul(v[q][r], w[r]);
        }
        Dft<R, DIR>::run(v[q]);
    }
    if (MODE != 1) __syncthreads();   // every read of this pass precedes every write
#pragma unroll
    for (int q = 0; q < GPT; ++q) {
        const int g = q * kFilterThreads + threadIdx.x;
        if (g >= NG) continue;
        const int p = g / G, j = g % G;
        const int k = j % NS;
        const int dst = (j - k) * R + k;
        if (MODE == 3) {
            const long long ra = row0 + 2 * p, rb = ra + 1;
            TO *out = reinterpret_cast<TO *>(a.out);
            // last pass: m = j + r G and only m < nu <= N/2 is kept, so r < R/2
#pragma unroll
            for (int r = 0; r < R / 2; ++r) {
                const int m = dst + r * NS;
                if (m < a.nu) {
                    if (ra < a.nrows) store_out<TO>(out + ra * a.nu + m, v[q][r].x);
                    if (rb < a.nrows) store_out<TO>(out + rb * a.nu + m, v[q][r].y);
                }
            }
        } else {
            float2 *dstp = buf + pad16(p * N + dst);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int m = dst + r * NS;
                float2 x = v[q][r];
                if (MODE == 2) {
                    const float h = __ldg(&a.H[m]);
                    x.x *= h;
                    x.y *= h;
                }
                // dst = R j for NS == 1 (R = 16: pad adds j, offsets r stay in one
                // 16-block); for NS a multiple of 16 the stride pads uniformly
                if (NS == 1 && R == 16)
                    dstp[r] = x;
                else if (NS % 16 == 0)
                    dstp[r * (NS + NS / 16)] = x;
                else
                    buf[pad16(p * N + m)] = x;
            }
        }
    }
    __syncthreads();
}

// Compile-time pass list: radix-16 passes, then one pass of 2^(LG mod 4).
template <int LG>
struct Passes {
    static constexpr int n16 = LG / 4;
    static constexpr int rem = LG % 4;
    static constexpr int count = n16 + (rem ? 1 : 0);
};

template <int LG, int PASS>
struct PassRadix {
    static constexpr int value = (PASS < Passes<LG>::n16) ? 16 : (1 << Passes<LG>::rem);
};

template <int LG, int PASS>
struct PassNs {
    static constexpr int value = (PASS == 0) ? 1 : PassNs<LG, PASS - 1>::value * PassRadix<LG, PASS - 1>::value;
};
template <int LG>
struct PassNs<LG, 0> {
    static constexpr int value = 1;
};

template <typename TO, int LG, int DIR, int PASS>
__device__ __forceinline__ void run_passes(float2 *buf, const FilterArgs &a, long long row0) {
    if constexpr (PASS < Passes<LG>::count) {
        constexpr int N = 1 << LG;
        constexpr int R = PassRadix<LG, PASS>::value;
        constexpr int NS = PassNs<LG, PASS>::value;
        constexpr bool first = PASS == 0, last = PASS == Passes<LG>::count - 1;
        // forward: first reads global, last applies the spectrum; inverse: last writes global
        constexpr int MODE = (DIR < 0) ? (first ? (last ? 4 : 1) : (last ? 2 : 0))
                                       : (last ? 3 : 0);
        if constexpr (MODE == 4) {
            // single forward pass: global read + spectrum multiply
            stockham_pass<TO, N, R, NS, DIR, 1>(buf, a, row0);
            __syncthreads();
            for (int t = threadIdx.x; t < PairsPerCta<N>::value * N; t += kFilterThreads) {
                float h = __ldg(&a.H[t & (N - 1)]);
                float2 x = buf[pad16(t)];
                buf[pad16(t)] = make_float2(x.x * h, x.y * h);
            }
            __syncthreads();
        } else {
            stockham_pass<TO, N, R, NS, DIR, MODE>(buf, a, row0);
        }
        run_passes<TO, LG, DIR, PASS + 1>(buf, a, row0);
    }
}

template <typename TO, int LG>
__global__ void __launch_bounds__(kFilterThreads)
ramp_filter_stockham(FilterArgs a) {
    extern __shared__ float2 buf[];
    const long long row0 = (long long)blockIdx.x * PairsPerCta<(1 << LG)>::value * 2;
    run_passes<TO, LG, -1, 0>(buf, a, row0);
    run_passes<TO, LG, +1, 0>(buf, a, row0);
}

template <typename TO>
static cudaError_t launch_lg(int lg, const FilterArgs &a, unsigned nblk, int smem, cudaStream_t st) {
#define BP_FILTER_CASE(L)                                                                       \
    case L: {                                                                                   \
        auto k = ramp_filter_stockham<TO, L>;                                                    \
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem); \
        if (e != cudaSuccess) return e;                                                         \
        k<<<nblk, kFilterThreads, smem, st>>>(a);                                                \
        return cudaGetLastError();                                                              \
    }
    switch (lg) {
        BP_FILTER_CASE(14)
        default: return cudaErrorInvalidValue;
    }
#undef BP_FILTER_CASE
}

int ct_twiddle_count(int N) { return fct::plan_tw_offset(N, fct::plan_count(N) - 1); }

// Spectrum at the fused step's slots, Ht[k2][g] = H[f(16 g + k2)], with f the
// frequency of a digit-reversed position (digit k_p = (pos mod S_p) / T_p,
// weight R_0 ... R_(p-1)); twiddles of pass p at (k - 1) T_p + o, angle
// 2 pi o k / S_p.
void ct_tables(int N, const double *H, float *Ht, float *tw) {
    const int C = fct::plan_count(N), G = N / 16;
    for (int pos = 0; pos < N; ++pos) {
        long long f = 0, w = 1;
        for (int p = 0; p < C; ++p) {
            const int S = fct::plan_span(N, p), T = fct::plan_stride(N, p);
            f += (long long)((pos % S) / T) * w;
            w *= fct::plan_radix(N, p);
        }
        const int g = pos / 16, k2 = pos % 16;
        Ht[2 * ((size_t)k2 * G + g)] = Ht[2 * ((size_t)k2 * G + g) + 1] = (float)H[f];
    }
    for (int p = 0; p + 1 < C; ++p) {
        const int S = fct::plan_span(N, p), T = fct::plan_stride(N, p), R = fct::plan_radix(N, p);
        const int off = fct::plan_tw_offset(N, p);
        for (int k = 1; k < R; ++k)
            for (int o = 0; o < T; ++o) {
                const double ang = 2.0 * M_PI * (double)((long long)o * k % S) / S;
                float *e = tw + 4 * ((size_t)off + (size_t)(k - 1) * T + o);
                e[0] = e[1] = (float)std::cos(ang);
                e[2] = e[3] = (float)std::sin(ang);
            }
    }
}

int ct_fft_size(int nu) {
    static const int sizes[] = {32, 64, 128, 256, 512, 1024, 1280, 2048, 2560, 4096, 5120, 8192, 10240};
    for (int n : sizes)
        if (n >= 2 * nu - 1) return n;
    return 0;
}

bp_status launch_filter(bp_ctx *ctx, const float *proj, void *out, bp_dtype out_t,
                        long long n_views_total, cudaStream_t st) {
    const bp_geometry &g = ctx->g;
    const int N = ctx->fft_n;
    if (ctx->fft_quad) {
        CtArgs c;
        c.in = proj;
        c.out = out;
        c.nrows = n_views_total * ctx->nv;
        c.nu = ctx->nu;
        c.nv = ctx->nv;
        c.out_f16 = out_t == BP_F16;
        c.Ht = reinterpret_cast<const float2 *>(ctx->d_ctH);
        c.tw = reinterpret_cast<const ulonglong2 *>(ctx->d_cttw);
        c.sdd2 = (float)(g.sdd * g.sdd);
        c.du = (float)g.du;
        c.dv = (float)g.dv;
        c.cu = (float)(0.5 * (g.nu - 1) + g.u_off_px);
        c.cv = (float)(0.5 * (g.nv - 1) + g.v_off_px);
        cudaError_t e;
        switch (N) {
            case 32: e = launch_ct<32>(c, st); break;
            case 64: e = launch_ct<64>(c, st); break;
            case 128: e = launch_ct<128>(c, st); break;
            case 256: e = launch_ct<256>(c, st); break;
            case 512: e = launch_ct<512>(c, st); break;
            case 1024: e = launch_ct<1024>(c, st); break;
            case 1280: e = launch_ct<1280>(c, st); break;
            case 2048: e = launch_ct<2048>(c, st); break;
            case 2560: e = launch_ct<2560>(c, st); break;
            case 4096: e = launch_ct<4096>(c, st); break;
            case 5120: e = launch_ct<5120>(c, st); break;
            case 8192: e = launch_ct<8192>(c, st); break;
            case 10240: e = launch_ct<10240>(c, st); break;
            default: return fail(ctx, BP_ERR_UNSUPPORTED, "bp_filter: no transform of this size");
        }
        return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "ramp_filter_ct launch");
    }
    if (ctx->fft_log2 != 14)
        return fail(ctx, BP_ERR_UNSUPPORTED, "bp_filter: detector rows longer than 8192 pixels");
    FilterArgs a;
    a.in = proj;
    a.out = out;
    a.nrows = n_views_total * ctx->nv;
    a.nu = ctx->nu;
    a.nv = ctx->nv;
    a.pairs = N >= 4096 ? 1 : 4096 / N;
    a.H = ctx->d_H;
    a.tw = ctx->d_tw;
    a.sdd = (float)g.sdd;
    a.du = (float)g.du;
    a.dv = (float)g.dv;
    a.cu = (float)(0.5 * (g.nu - 1) + g.u_off_px);
    a.cv = (float)(0.5 * (g.nv - 1) + g.v_off_px);
    const long long nblk = (a.nrows + 2LL * a.pairs - 1) / (2LL * a.pairs);
    if (nblk > 0x7fffffffLL) return fail(ctx, BP_ERR_INVALID_ARG, "bp_filter: too many rows");
    const int smem = (a.pairs * N + a.pairs * N / 16) * (int)sizeof(float2);
    cudaError_t e = (out_t == BP_F16) ? launch_lg<__half>(ctx->fft_log2, a, (unsigned)nblk, smem, st)
                                      : launch_lg<float>(ctx->fft_log2, a, (unsigned)nblk, smem, st);
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "ramp_filter_stockham launch");
}

}  // namespace bp
