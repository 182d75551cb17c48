// FDK pre-filter (the paper assumes filtered projections, Section 2.1.2):
// cosine weight, then the linear convolution of every detector row with the
// discrete Ram-Lak kernel, done as a zero-padded FFT convolution in shared
// memory. Two real rows travel as the real and imaginary parts of one
// complex FFT: the kernel's spectrum is real and even, so the product keeps
// the two rows apart. Forward transform: radix-2 decimation in frequency
// (natural in, bit-reversed out); the spectrum table is stored bit-reversed;
// inverse: radix-2 decimation in time (bit-reversed in, natural out). The
// 1/N of the inverse and the isocenter pitch dp are folded into the table.
#include "bp_internal.h"

namespace bp {

constexpr int kFilterThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

__device__ __forceinline__ void store_out(float *p, float v) { *p = v; }
__device__ __forceinline__ void store_out(__half *p, float v) { *p = __float2half_rn(v); }

// One CTA filters `pairs` row pairs; buf holds pairs * N complex values.
template <typename TO>
__global__ void __launch_bounds__(kFilterThreads)
ramp_filter_fft(const float *__restrict__ in, TO *__restrict__ out, long long nrows, int nu,
                int nv, int lg, int pairs, const float *__restrict__ Hbr,
                const float2 *__restrict__ tw, float sdd, float du, float dv, float cu, float cv) {
    extern __shared__ float2 buf[];
    const int N = 1 << lg;
    const int half_n = N >> 1;
    const long long row0 = (long long)blockIdx.x * pairs * 2;
    const float sdd2 = sdd * sdd;

    // load with cosine weight; zero padding beyond nu
    for (int t = threadIdx.x; t < pairs * N; t += kFilterThreads) {
        int p = t / N, m = t - p * N;
        long long ra = row0 + 2 * p, rb = ra + 1;
        float a = 0.0f, b = 0.0f;
        if (m < nu) {
            float um = ((float)m - cu) * du;
            float um2 = um * um;
            if (ra < nrows) {
                float vm = ((float)(ra % nv) - cv) * dv;
                a = in[ra * nu + m] * (sdd * rsqrtf(sdd2 + um2 + vm * vm));
            }
            if (rb < nrows) {
                float vm = ((float)(rb % nv) - cv) * dv;
                b = in[rb * nu + m] * (sdd * rsqrtf(sdd2 + um2 + vm * vm));
            }
        }
        buf[t] = make_float2(a, b);
    }
    __syncthreads();

    // forward: decimation in frequency
    for (int h = half_n, ts = 1; h >= 1; h >>= 1, ts <<= 1) {
        for (int t = threadIdx.x; t < pairs * half_n; t += kFilterThreads) {
            int p = t / half_n, j = t - p * half_n;
            int off = j & (h - 1);
            int i0 = p * N + ((j - off) << 1) + off, i1 = i0 + h;
            float2 a = buf[i0], b = buf[i1];
            buf[i0] = make_float2(a.x + b.x, a.y + b.y);
            buf[i1] = cmul(make_float2(a.x - b.x, a.y - b.y), tw[off * ts]);
        }
        __syncthreads();
    }
    // multiply by the real spectrum (bit-reversed order)
    for (int t = threadIdx.x; t < pairs * N; t += kFilterThreads) {
        float hv = Hbr[t & (N - 1)];
        float2 x = buf[t];
        buf[t] = make_float2(x.x * hv, x.y * hv);
    }
    __syncthreads();
    // inverse: decimation in time with conjugate twiddles
    for (int h = 1, ts = half_n; h <= half_n; h <<= 1, ts >>= 1) {
        for (int t = threadIdx.x; t < pairs * half_n; t += kFilterThreads) {
            int p = t / half_n, j = t - p * half_n;
            int off = j & (h - 1);
            int i0 = p * N + ((j - off) << 1) + off, i1 = i0 + h;
            float2 w = tw[off * ts];
            float2 a = buf[i0], b = cmul(buf[i1], make_float2(w.x, -w.y));
            buf[i0] = make_float2(a.x + b.x, a.y + b.y);
            buf[i1] = make_float2(a.x - b.x, a.y - b.y);
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < pairs * nu; t += kFilterThreads) {
        int p = t / nu, m = t - p * nu;
        long long ra = row0 + 2 * p, rb = ra + 1;
        float2 x = buf[p * N + m];
        if (ra < nrows) store_out(out + ra * nu + m, x.x);
        if (rb < nrows) store_out(out + rb * nu + m, x.y);
    }
}

bp_status launch_filter(bp_ctx *ctx, const float *proj, void *out, bp_dtype out_t,
                        long long n_views_total, cudaStream_t st) {
    const bp_geometry &g = ctx->g;
    const int N = ctx->fft_n;
    const long long nrows = n_views_total * ctx->nv;
    const int pairs = N >= 4096 ? 1 : 4096 / N;
    const long long nblk = (nrows + 2LL * pairs - 1) / (2LL * pairs);
    const int smem = pairs * N * (int)sizeof(float2);
    const float cu = (float)(0.5 * (g.nu - 1) + g.u_off_px);
    const float cv = (float)(0.5 * (g.nv - 1) + g.v_off_px);
    if (nblk > 0x7fffffffLL) return fail(ctx, BP_ERR_INVALID_ARG, "bp_filter: too many rows");
    cudaError_t e;
    if (out_t == BP_F16) {
        e = cudaFuncSetAttribute(ramp_filter_fft<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            ramp_filter_fft<__half><<<(unsigned)nblk, kFilterThreads, smem, st>>>(
                proj, (__half *)out, nrows, ctx->nu, ctx->nv, ctx->fft_log2, pairs, ctx->d_H,
                ctx->d_tw, (float)g.sdd, (float)g.du, (float)g.dv, cu, cv);
    } else {
        e = cudaFuncSetAttribute(ramp_filter_fft<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            ramp_filter_fft<float><<<(unsigned)nblk, kFilterThreads, smem, st>>>(
                proj, (float *)out, nrows, ctx->nu, ctx->nv, ctx->fft_log2, pairs, ctx->d_H,
                ctx->d_tw, (float)g.sdd, (float)g.du, (float)g.dv, cu, cv);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "ramp_filter_fft launch");
}

}  // namespace bp
