// Interface of the four-row FFT ramp filter (filter_quad.cuh holds the
// kernel; k_filter_q*.cu instantiate it for each transform size).
#pragma once

#include <cuda_runtime.h>

namespace bp {

struct QArgs {
    const float *in;          // [nrows][nu] raw projections
    void *out;                // [nrows][nu] FP32 or FP16 filtered projections
    long long nrows;
    int nu, nv, out_f16;
    int in_vec;               // in 16-byte aligned and nu % 4 == 0 (16-byte row copies)
    const float2 *H2;         // [N] (H[k], H[k]): kernel spectrum x dp / N
    const ulonglong2 *tw4;    // [N] (cos, cos, sin, sin) of 2 pi e / N
    float sdd, du, dv, cu, cv;
};

// Transform size for rows of nu pixels: the smallest supported N >= 2 nu - 1
// (powers of two from 32 to 8192 and 1280, 2560, 5120, 10240); 0 when nu is
// too long for this kernel.
int quad_fft_size(int nu);

// Launch over all rows (four rows per transform pair); defined for the sizes
// quad_fft_size returns.
template <int N>
cudaError_t launch_quad(const QArgs &a, cudaStream_t st);

}  // namespace bp
