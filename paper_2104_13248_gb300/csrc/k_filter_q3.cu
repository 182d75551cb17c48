// Instantiations of the four-row FFT ramp filter (filter_quad.cuh), split
// across translation units so they compile in parallel.
#include "filter_quad.cuh"

namespace bp {
template cudaError_t launch_quad<1280>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<5120>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<8192>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<10240>(const QArgs &, cudaStream_t);
}  // namespace bp
