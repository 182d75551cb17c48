// Instantiations of the four-row FFT ramp filter (filter_ct.cuh), split
// across translation units so they compile in parallel.
#include "filter_ct.cuh"

namespace bp {
template cudaError_t launch_ct<1280>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<5120>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<8192>(const CtArgs &, cudaStream_t);
template cudaError_t launch_ct<10240>(const CtArgs &, cudaStream_t);
}  // namespace bp
