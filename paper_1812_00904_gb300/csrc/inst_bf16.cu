// Instantiations of the streaming kernel for __nv_bfloat16 values and float vectors (one translation unit
// per value type, so that the instantiations compile in parallel).
#include "stream_kernel.cuh"

namespace gbk {

cudaError_t launch_stream_bf16(int mode, int kb, const LaunchArgs &a) { return launch_mode<__nv_bfloat16, float>(mode, kb, a); }

}  // namespace gbk
