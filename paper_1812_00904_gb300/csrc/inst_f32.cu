// Instantiations of the streaming kernel for float values and float vectors (one translation unit
// per value type, so that the instantiations compile in parallel).
#include "stream_kernel.cuh"

namespace gbk {

cudaError_t launch_stream_f32(int mode, int kb, const LaunchArgs &a) { return launch_mode<float, float>(mode, kb, a); }

}  // namespace gbk
