// Instantiations of the four-row FFT ramp filter (filter_ct.cuh), split
// across translation units so they compile in parallel.
#include "filter_ct.cuh"

namespace bp {
template cudaError_t launch_ct<4096>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<2048>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<512>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<64>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<128>(const CtArgs &, cudaStream_t);
}  // namespace bp
