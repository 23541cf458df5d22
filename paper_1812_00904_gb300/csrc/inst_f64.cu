// Instantiations of the streaming kernel for double values and double vectors (one translation unit
// per value type, so that the instantiations compile in parallel).
#include "stream_kernel.cuh"

namespace gbk {

cudaError_t launch_stream_f64(int mode, int kb, const LaunchArgs &a) { return launch_mode<double, double>(mode, kb, a); }

}  // namespace gbk
