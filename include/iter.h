/*
 * iter.h - C ABI of the element-wise steps of iterative reconstruction on
 * the projector pair of bp.h: MLEM / ordered-subset EM (Shepp and Vardi;
 * Hudson and Larkin) and block SART (Andersen and Kak). The paper names
 * these methods as the reason back-projection is called repeatedly
 * (Section 1); it prints no formula for them, and these calls follow the
 * published update rules:
 *
 *   MLEM, per view subset t:  y = A_t x;  r = p / y  (0 where y <= eps);
 *                             x <- x (A_t^T r) / (A_t^T 1)  (unchanged where A_t^T 1 <= eps)
 *   SART, per view subset t:  y = A_t x;  r = (p - y) / (A_t 1)  (0 where A_t 1 <= eps);
 *                             x <- x + lambda (A_t^T r) / (A_t^T 1)  (unchanged where A_t^T 1 <= eps),
 *                             then max(x, 0) when nonneg
 *
 * A is fp_project and A^T bp_backproject, both with scale 1. These calls do
 * the element-wise parts; the caller chains them with the projectors.
 *
 * Conventions: all arrays are FP32 device arrays of n elements owned by the
 * caller (n >= 0, 4-byte aligned; 16-byte aligned arrays take vector
 * loads). Outputs may alias inputs of the same index (in place). Calls are
 * asynchronous on `stream` (NULL = legacy default stream), never allocate,
 * and return bp_status (bp.h) with the message in bp_last_error(NULL).
 * Divisions are IEEE FP32 (round to nearest) in the order written above:
 * (x * b) / s for MLEM and x + (lambda * b) / s for SART.
 */
#ifndef ITER_H
#define ITER_H

#include "bp.h"

#ifdef __cplusplus
extern "C" {
#endif

/* x[i] = value. */
bp_status it_fill(float *x, long long n, float value, void *stream);

/* r[i] = p[i] / y[i] where y[i] > eps, else 0 (MLEM's ratio of measured to
 * estimated projections). */
bp_status it_ratio(const float *p, const float *y, float *r, long long n, float eps, void *stream);

/* r[i] = (p[i] - y[i]) / w[i] where w[i] > eps, else 0 (SART's residual
 * normalised by the ray sums w = A 1). */
bp_status it_residual(const float *p, const float *y, const float *w, float *r, long long n,
                      float eps, void *stream);

/* x[i] = (x[i] * b[i]) / s[i] where s[i] > eps, else unchanged (MLEM update;
 * b = A^T r, s = A^T 1). */
bp_status it_mlem_update(float *x, const float *b, const float *s, long long n, float eps,
                         void *stream);

/* x[i] += (lambda * b[i]) / s[i] where s[i] > eps; then x[i] = max(x[i], 0)
 * when nonneg != 0 (SART update; b = A^T r, s = A^T 1). */
bp_status it_sart_update(float *x, const float *b, const float *s, long long n, float lambda,
                         int nonneg, float eps, void *stream);

/* Least squares on the projector pair (the differentiable reconstruction:
 * gradient descent on L(x) = 0.5 ||A x - p||^2, A = fp_project):
 *   it_ls_residual  r[i] = y[i] - p[i] (FP32) and *loss = 0.5 sum r[i]^2,
 *                   summed in FP64 (loss is a device double, overwritten;
 *                   the blocks' partial sums are added in a varying order,
 *                   so the loss's last bits may differ between runs, r's
 *                   never do). y = A x, p the measured projections.
 *   it_scale        out[i] = r[i] * (float)(*s), s a device double (the
 *                   gradient of the loss for an upstream gradient s).
 *   it_gd_step      x[i] = x[i] - (step * g[i]), two FP32 roundings. */
bp_status it_ls_residual(const float *y, const float *p, float *r, long long n, double *loss, void *stream);
bp_status it_scale(const float *r, const double *s, float *out, long long n, void *stream);
bp_status it_gd_step(float *x, const float *g, long long n, float step, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* ITER_H */
