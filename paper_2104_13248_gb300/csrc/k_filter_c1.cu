// Instantiations of the four-row FFT ramp filter (filter_ct.cuh), split
// across translation units so they compile in parallel.
#include "filter_ct.cuh"

namespace bp {
template cudaError_t launch_ct<2560>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<1024>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<256>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<32>(const CtArgs &, cudaStream_t);
}  // namespace bp
