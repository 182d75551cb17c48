// Interface of the four-row FFT ramp filter (filter_ct.cuh holds the kernel;
// k_filter_c*.cu instantiate it for each transform size).
#pragma once

#include <cuda_runtime.h>

namespace bp {

struct CtArgs {
    const float *in;             // [nrows][nu] raw projections
    void *out;                   // [nrows][nu] FP32 or FP16 filtered projections
    long long nrows;
    int nu, nv, out_f16;
    const float2 *Ht;            // [16][N/16] (H, H): spectrum at the fused step's positions (ct_tables)
    const ulonglong2 *tw;        // twiddles (cos, cos, sin, sin) of every pass but the last (ct_tables)
    float sdd2, du, dv, cu, cv;  // sdd^2; pixel pitches; detector centre in pixels
};

// Transform size for rows of nu pixels: the smallest supported N >= 2 nu - 1
// (powers of two from 32 to 8192 and 1280, 2560, 5120, 10240); 0 when nu is
// too long for this kernel.
int ct_fft_size(int nu);

// Host tables of transform size N for the kernel: Ht (2 floats per entry,
// 16 * (N / 16) entries) and tw (4 floats per entry, ct_twiddle_count(N)
// entries). H[k] (k in natural order) is the kernel spectrum, already
// scaled by everything the convolution multiplies it with.
int ct_twiddle_count(int N);
void ct_tables(int N, const double *H, float *Ht, float *tw);

// Launch over all rows (four rows per transform pair); defined for the sizes
// ct_fft_size returns.
template <int N>
cudaError_t launch_ct(const CtArgs &a, cudaStream_t st);

}  // namespace bp
