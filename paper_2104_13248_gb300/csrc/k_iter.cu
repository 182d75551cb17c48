// Element-wise steps of MLEM / ordered-subset EM and block SART (include/
// iter.h): the ratio or normalised residual on the detector side and the
// multiplicative or additive update on the volume side. Each is one pass
// over HBM, grid-stride, with 16-byte vector accesses when every array is
// 16-byte aligned. The comparisons and the order of the FP32 operations are
// the ones iter.h states, so a threshold decision matches the FP64 oracle's
// except for values within rounding of eps.
#include <cstdint>

#include "bp_internal.h"
#include "../../include/iter.h"

namespace bp {

namespace {

constexpr int kItThreads = 256;

struct Fill {
    float v;
    __device__ float operator()(float) const { return v; }
};

__device__ __forceinline__ float ratio1(float p, float y, float eps) { return y > eps ? p / y : 0.0f; }
__device__ __forceinline__ float resid1(float p, float y, float w, float eps) {
    return w > eps ? (p - y) / w : 0.0f;
}
__device__ __forceinline__ float mlem1(float x, float b, float s, float eps) { return s > eps ? (x * b) / s : x; }
__device__ __forceinline__ float sart1(float x, float b, float s, float lam, int nonneg, float eps) {
    float r = s > eps ? x + (lam * b) / s : x;
    return (nonneg && r < 0.0f) ? 0.0f : r;
}

__global__ void __launch_bounds__(kItThreads) fill_kernel(float *x, long long n, float v, int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        float4 *x4 = reinterpret_cast<float4 *>(x);
        for (; i < n / 4; i += stride) x4[i] = make_float4(v, v, v, v);
        for (long long t = (n / 4) * 4 + (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride)
            x[t] = v;
    } else {
        for (; i < n; i += stride) x[i] = v;
    }
}

__global__ void __launch_bounds__(kItThreads) ratio_kernel(const float *__restrict__ p, const float *__restrict__ y,
                                                           float *r, long long n, float eps, int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tail = 0;
    if (vec) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p), *y4 = reinterpret_cast<const float4 *>(y);
        float4 *r4 = reinterpret_cast<float4 *>(r);
        for (long long i = t0; i < n / 4; i += stride) {
            const float4 a = p4[i], b = y4[i];
            r4[i] = make_float4(ratio1(a.x, b.x, eps), ratio1(a.y, b.y, eps), ratio1(a.z, b.z, eps),
                                ratio1(a.w, b.w, eps));
        }
        tail = (n / 4) * 4;
    }
    for (long long i = tail + t0; i < n; i += stride) r[i] = ratio1(p[i], y[i], eps);
}

__global__ void __launch_bounds__(kItThreads) resid_kernel(const float *__restrict__ p, const float *__restrict__ y,
                                                           const float *__restrict__ w, float *r, long long n,
                                                           float eps, int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tail = 0;
    if (vec) {
        const float4 *p4 = reinterpret_cast<const float4 *>(p), *y4 = reinterpret_cast<const float4 *>(y);
        const float4 *w4 = reinterpret_cast<const float4 *>(w);
        float4 *r4 = reinterpret_cast<float4 *>(r);
        for (long long i = t0; i < n / 4; i += stride) {
            const float4 a = p4[i], b = y4[i], c = w4[i];
            r4[i] = make_float4(resid1(a.x, b.x, c.x, eps), resid1(a.y, b.y, c.y, eps),
                                resid1(a.z, b.z, c.z, eps), resid1(a.w, b.w, c.w, eps));
        }
        tail = (n / 4) * 4;
    }
    for (long long i = tail + t0; i < n; i += stride) r[i] = resid1(p[i], y[i], w[i], eps);
}

__global__ void __launch_bounds__(kItThreads) mlem_kernel(float *x, const float *__restrict__ b,
                                                          const float *__restrict__ s, long long n, float eps,
                                                          int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tail = 0;
    if (vec) {
        float4 *x4 = reinterpret_cast<float4 *>(x);
        const float4 *b4 = reinterpret_cast<const float4 *>(b), *s4 = reinterpret_cast<const float4 *>(s);
        for (long long i = t0; i < n / 4; i += stride) {
            const float4 a = x4[i], c = b4[i], d = s4[i];
            x4[i] = make_float4(mlem1(a.x, c.x, d.x, eps), mlem1(a.y, c.y, d.y, eps), mlem1(a.z, c.z, d.z, eps),
                                mlem1(a.w, c.w, d.w, eps));
        }
        tail = (n / 4) * 4;
    }
    for (long long i = tail + t0; i < n; i += stride) x[i] = mlem1(x[i], b[i], s[i], eps);
}

__global__ void __launch_bounds__(kItThreads) sart_kernel(float *x, const float *__restrict__ b,
                                                          const float *__restrict__ s, long long n, float lam,
                                                          int nonneg, float eps, int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tail = 0;
    if (vec) {
        float4 *x4 = reinterpret_cast<float4 *>(x);
        const float4 *b4 = reinterpret_cast<const float4 *>(b), *s4 = reinterpret_cast<const float4 *>(s);
        for (long long i = t0; i < n / 4; i += stride) {
            const float4 a = x4[i], c = b4[i], d = s4[i];
            x4[i] = make_float4(sart1(a.x, c.x, d.x, lam, nonneg, eps), sart1(a.y, c.y, d.y, lam, nonneg, eps),
                                sart1(a.z, c.z, d.z, lam, nonneg, eps), sart1(a.w, c.w, d.w, lam, nonneg, eps));
        }
        tail = (n / 4) * 4;
    }
    for (long long i = tail + t0; i < n; i += stride) x[i] = sart1(x[i], b[i], s[i], lam, nonneg, eps);
}

// Least squares: r = y - p and the block's share of 0.5 sum r^2 in FP64,
// added to *loss once per block (the order of the blocks' additions varies,
// so the loss may differ from run to run in its last bits; r does not).
__global__ void __launch_bounds__(kItThreads) ls_resid_kernel(const float *__restrict__ y, const float *__restrict__ p,
                                                              float *r, long long n, double *loss, int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double acc = 0.0;
    long long tail = 0;
    if (vec) {
        const float4 *y4 = reinterpret_cast<const float4 *>(y), *p4 = reinterpret_cast<const float4 *>(p);
        float4 *r4 = reinterpret_cast<float4 *>(r);
        for (long long i = t0; i < n / 4; i += stride) {
            const float4 a = y4[i], b = p4[i];
            const float4 d = make_float4(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z),
                                         __fsub_rn(a.w, b.w));
            r4[i] = d;
            acc += (double)d.x * d.x + (double)d.y * d.y + (double)d.z * d.z + (double)d.w * d.w;
        }
        tail = (n / 4) * 4;
    }
    for (long long i = tail + t0; i < n; i += stride) {
        const float d = __fsub_rn(y[i], p[i]);
        r[i] = d;
        acc += (double)d * d;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double part[kItThreads / 32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kItThreads / 32; ++w) s += part[w];
        atomicAdd(loss, 0.5 * s);
    }
}

// out = r * (float)(*s): the loss gradient times a device-side scale.
__global__ void __launch_bounds__(kItThreads) scale_kernel(const float *__restrict__ r, const double *__restrict__ s,
                                                           float *out, long long n, int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const float c = (float)*s;
    long long tail = 0;
    if (vec) {
        const float4 *r4 = reinterpret_cast<const float4 *>(r);
        float4 *o4 = reinterpret_cast<float4 *>(out);
        for (long long i = t0; i < n / 4; i += stride) {
            const float4 a = r4[i];
            o4[i] = make_float4(__fmul_rn(a.x, c), __fmul_rn(a.y, c), __fmul_rn(a.z, c), __fmul_rn(a.w, c));
        }
        tail = (n / 4) * 4;
    }
    for (long long i = tail + t0; i < n; i += stride) out[i] = __fmul_rn(r[i], c);
}

// Gradient step x = x - (step * g), two roundings (no fused multiply-add).
__global__ void __launch_bounds__(kItThreads) gd_kernel(float *x, const float *__restrict__ g, long long n, float step,
                                                        int vec) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tail = 0;
    if (vec) {
        float4 *x4 = reinterpret_cast<float4 *>(x);
        const float4 *g4 = reinterpret_cast<const float4 *>(g);
        for (long long i = t0; i < n / 4; i += stride) {
            const float4 a = x4[i], b = g4[i];
            x4[i] = make_float4(__fsub_rn(a.x, __fmul_rn(step, b.x)), __fsub_rn(a.y, __fmul_rn(step, b.y)),
                                __fsub_rn(a.z, __fmul_rn(step, b.z)), __fsub_rn(a.w, __fmul_rn(step, b.w)));
        }
        tail = (n / 4) * 4;
    }
    for (long long i = tail + t0; i < n; i += stride) x[i] = __fsub_rn(x[i], __fmul_rn(step, g[i]));
}

// Enough CTAs to fill the GPU (the loops stride over the rest).
unsigned it_blocks(long long n) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 148;
    }
    const long long want = (n + kItThreads - 1) / kItThreads;
    const long long cap = 8LL * sms;
    return (unsigned)(want < 1 ? 1 : (want > cap ? cap : want));
}

bool a16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bp_status it_done(const char *what) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(nullptr, e, what);
}

}  // namespace

}  // namespace bp

using namespace bp;

extern "C" {

bp_status it_fill(float *x, long long n, float value, void *stream) {
    if (n < 0 || (n > 0 && !x)) return fail(nullptr, BP_ERR_INVALID_ARG, "it_fill: bad arguments");
    if (n == 0) return BP_OK;
    fill_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(x, n, value, a16(x));
    return it_done("it_fill launch");
}

bp_status it_ratio(const float *p, const float *y, float *r, long long n, float eps, void *stream) {
    if (n < 0 || (n > 0 && (!p || !y || !r))) return fail(nullptr, BP_ERR_INVALID_ARG, "it_ratio: bad arguments");
    if (n == 0) return BP_OK;
    ratio_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(p, y, r, n, eps,
                                                                          a16(p) && a16(y) && a16(r));
    return it_done("it_ratio launch");
}

bp_status it_residual(const float *p, const float *y, const float *w, float *r, long long n, float eps,
                      void *stream) {
    if (n < 0 || (n > 0 && (!p || !y || !w || !r)))
        return fail(nullptr, BP_ERR_INVALID_ARG, "it_residual: bad arguments");
    if (n == 0) return BP_OK;
    resid_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(p, y, w, r, n, eps,
                                                                          a16(p) && a16(y) && a16(w) && a16(r));
    return it_done("it_residual launch");
}

bp_status it_mlem_update(float *x, const float *b, const float *s, long long n, float eps, void *stream) {
    if (n < 0 || (n > 0 && (!x || !b || !s)))
        return fail(nullptr, BP_ERR_INVALID_ARG, "it_mlem_update: bad arguments");
    if (n == 0) return BP_OK;
    mlem_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(x, b, s, n, eps,
                                                                         a16(x) && a16(b) && a16(s));
    return it_done("it_mlem_update launch");
}

bp_status it_sart_update(float *x, const float *b, const float *s, long long n, float lambda, int nonneg,
                         float eps, void *stream) {
    if (n < 0 || (n > 0 && (!x || !b || !s)))
        return fail(nullptr, BP_ERR_INVALID_ARG, "it_sart_update: bad arguments");
    if (n == 0) return BP_OK;
    sart_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(x, b, s, n, lambda, nonneg, eps,
                                                                         a16(x) && a16(b) && a16(s));
    return it_done("it_sart_update launch");
}

bp_status it_ls_residual(const float *y, const float *p, float *r, long long n, double *loss, void *stream) {
    if (n < 0 || !loss || (n > 0 && (!y || !p || !r)))
        return fail(nullptr, BP_ERR_INVALID_ARG, "it_ls_residual: bad arguments");
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(double), (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "it_ls_residual: clear");
    if (n == 0) return BP_OK;
    ls_resid_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(y, p, r, n, loss,
                                                                             a16(y) && a16(p) && a16(r));
    return it_done("it_ls_residual launch");
}

bp_status it_scale(const float *r, const double *s, float *out, long long n, void *stream) {
    if (n < 0 || !s || (n > 0 && (!r || !out))) return fail(nullptr, BP_ERR_INVALID_ARG, "it_scale: bad arguments");
    if (n == 0) return BP_OK;
    scale_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(r, s, out, n, a16(r) && a16(out));
    return it_done("it_scale launch");
}

bp_status it_gd_step(float *x, const float *g, long long n, float step, void *stream) {
    if (n < 0 || (n > 0 && (!x || !g))) return fail(nullptr, BP_ERR_INVALID_ARG, "it_gd_step: bad arguments");
    if (n == 0) return BP_OK;
    gd_kernel<<<it_blocks(n), kItThreads, 0, (cudaStream_t)stream>>>(x, g, n, step, a16(x) && a16(g));
    return it_done("it_gd_step launch");
}

}  // extern "C"
