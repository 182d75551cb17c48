// Instantiations of the four-row FFT ramp filter (filter_quad.cuh), split
// across translation units so they compile in parallel.
#include "filter_quad.cuh"

namespace bp {
template cudaError_t launch_quad<4096>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<2048>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<512>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<64>(const QArgs &, cudaStream_t);
template cudaError_t launch_quad<128>(const QArgs &, cudaStream_t);
}  // namespace bp
