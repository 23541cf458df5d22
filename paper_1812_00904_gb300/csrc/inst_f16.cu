// Instantiations of the streaming kernel for __half values and float vectors (one translation unit
// per value type, so that the instantiations compile in parallel).
#include "stream_kernel.cuh"

namespace gbk {

cudaError_t launch_stream_f16(int mode, int kb, const LaunchArgs &a) { return launch_mode<__half, float>(mode, kb, a); }

}  // namespace gbk
