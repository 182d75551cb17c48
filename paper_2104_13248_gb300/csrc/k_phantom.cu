// Input data: analytic line integrals of an ellipsoid phantom on the
// detector (not part of the reconstruction method). For every (view,
// ellipsoid) the host derives, in FP64, the ray direction in the
// ellipsoid's unit-sphere frame as an affine function of the pixel's
// detector coordinates (U, V), d' = D0 + U D1 + V D2, and the cross product
// of the source position with it, X = X0 + U X1 + V X2 (same frame). The
// squared distance of the ray from the sphere centre is |X|^2/|d'|^2, and
// the chord is 2 sqrt((1 - |X|^2/|d'|^2)/|d'|^2) times the source-pixel
// distance. The cross-product form avoids the cancellation of the usual
// quadratic discriminant, so the per-pixel work runs in FP32.
#include "bp_internal.h"

#include <cmath>
#include <vector>

namespace bp {

constexpr int kPhCoef = 20;

__global__ void __launch_bounds__(256)
phantom_kernel(const float *__restrict__ coef, int n_ell, int nu, int nv, float du, float dv,
               float cu, float cv, float sdd, float *__restrict__ proj) {
    extern __shared__ float cs[];
    const int s = blockIdx.y;
    const float *cv_ = coef + (size_t)s * n_ell * kPhCoef;
    for (int t = threadIdx.x; t < n_ell * kPhCoef; t += blockDim.x) cs[t] = cv_[t];
    __syncthreads();
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix >= (long long)nu * nv) return;
    const int r = (int)(pix / nu), c = (int)(pix % nu);
    const float U = ((float)c - cu) * du, V = ((float)r - cv) * dv;
    const float L = sqrtf(sdd * sdd + U * U + V * V);
    float sum = 0.0f;
    for (int e = 0; e < n_ell; ++e) {
        const float *q = cs + e * kPhCoef;
        float dx = fmaf(V, q[6], fmaf(U, q[3], q[0]));
        float dy = fmaf(V, q[7], fmaf(U, q[4], q[1]));
        float dz = fmaf(V, q[8], fmaf(U, q[5], q[2]));
        float A = dx * dx + dy * dy + dz * dz;
        float xx = fmaf(V, q[15], fmaf(U, q[12], q[9]));
        float xy = fmaf(V, q[16], fmaf(U, q[13], q[10]));
        float xz = fmaf(V, q[17], fmaf(U, q[14], q[11]));
        float m2 = (xx * xx + xy * xy + xz * xz) / A;
        if (m2 < 1.0f) sum += q[18] * 2.0f * sqrtf((1.0f - m2) / A) * L;
    }
    proj[(size_t)s * nu * nv + pix] = sum;
}

static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

bp_status launch_phantom(bp_ctx *ctx, const double *ell, int n_ell, float *proj, cudaStream_t st) {
    const bp_geometry &g = ctx->g;
    const int np = ctx->n_views;
    if (n_ell == 0) {
        cudaError_t e = cudaMemsetAsync(proj, 0, sizeof(float) * (size_t)np * ctx->nu * ctx->nv, st);
        return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "phantom clear");
    }
    std::vector<float> coef((size_t)np * n_ell * kPhCoef, 0.0f);
    for (int s = 0; s < np; ++s) {
        const double c = std::cos(ctx->angles[s]), sn = std::sin(ctx->angles[s]);
        const double er[3] = {c, sn, 0.0}, eu[3] = {-sn, c, 0.0}, ev[3] = {0.0, 0.0, 1.0};
        for (int e = 0; e < n_ell; ++e) {
            const double *E = ell + 16 * e;
            const double *R = E + 6;   // body -> world, row-major
            double rt[3][3], pS[3];
            const double *axes[3] = {er, eu, ev};
            const double S[3] = {g.sid * c - E[0], g.sid * sn - E[1], -E[2]};
            for (int a = 0; a < 3; ++a) {
                for (int m = 0; m < 3; ++m)
                    rt[m][a] = (R[0 * 3 + a] * axes[m][0] + R[1 * 3 + a] * axes[m][1] +
                                R[2 * 3 + a] * axes[m][2]) / E[3 + a];
                pS[a] = (R[0 * 3 + a] * S[0] + R[1 * 3 + a] * S[1] + R[2 * 3 + a] * S[2]) / E[3 + a];
            }
            double D0[3] = {-g.sdd * rt[0][0], -g.sdd * rt[0][1], -g.sdd * rt[0][2]};
            double X0[3], X1[3], X2[3];
            cross3(pS, D0, X0);
            cross3(pS, rt[1], X1);
            cross3(pS, rt[2], X2);
            float *q = coef.data() + ((size_t)s * n_ell + e) * kPhCoef;
            for (int a = 0; a < 3; ++a) {
                q[a] = (float)D0[a];
                q[3 + a] = (float)rt[1][a];
                q[6 + a] = (float)rt[2][a];
                q[9 + a] = (float)X0[a];
                q[12 + a] = (float)X1[a];
                q[15 + a] = (float)X2[a];
            }
            q[18] = (float)E[15];
        }
    }
    cudaError_t e = cudaMemcpyAsync(ctx->d_phcoef, coef.data(), sizeof(float) * coef.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "phantom coefficients upload");
    // the host vector dies at return: make sure the (pageable) copy has consumed it
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "phantom coefficients upload");
    dim3 grid((unsigned)(((long long)ctx->nu * ctx->nv + 255) / 256), np);
    phantom_kernel<<<grid, 256, n_ell * kPhCoef * sizeof(float), st>>>(
        ctx->d_phcoef, n_ell, ctx->nu, ctx->nv, (float)g.du, (float)g.dv,
        (float)(0.5 * (g.nu - 1) + g.u_off_px), (float)(0.5 * (g.nv - 1) + g.v_off_px),
        (float)g.sdd, proj);
    e = cudaGetLastError();
    return e == cudaSuccess ? BP_OK : cuda_fail(ctx, e, "phantom_kernel launch");
}

}  // namespace bp
