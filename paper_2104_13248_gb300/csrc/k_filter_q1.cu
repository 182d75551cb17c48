// Instantiations of the four-row FFT ramp filter (filter_quad.cuh), split
// across translation units so they compile in parallel.
#include "filter_quad.cuh"

namespace bp {
template cudaError_t launch_quad<2560>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<1024>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<256>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<32>(const QArgs &, cudaStream_t);
}  // namespace bp
