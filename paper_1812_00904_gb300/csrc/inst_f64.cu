// Instantiations of the streaming kernel for double values and double vectors.
#include "stream_kernel.cuh"

namespace gbk {

cudaError_t launch_stream_f64(int mode, int kb, const LaunchArgs &a) {
    using VT = double;
    using XT = double;
    if (mode == MODE_DVALUES) {
        return a.smemv ? launch_one<VT, XT, MODE_DVALUES, 1, true>(a) : launch_one<VT, XT, MODE_DVALUES, 1, false>(a);
    }
    if (!a.smemv) {
        if (mode == MODE_SCATTER) return kb == 1 ? launch_one<VT, XT, MODE_SCATTER, 1, false>(a) : cudaErrorInvalidValue;
        // several vectors: interleaved in global memory (vin[0])
        if (kb <= 1) return launch_one<VT, XT, MODE_SEGDOT, 1, false>(a);
        if (kb <= 2) return launch_one<VT, XT, MODE_SEGDOT, 2, false>(a);
        if (kb <= 4) return launch_one<VT, XT, MODE_SEGDOT, 4, false>(a);
        return launch_one<VT, XT, MODE_SEGDOT, 8, false>(a);
    }
    if (mode == MODE_SCATTER) {
        if (kb <= 1) return launch_one<VT, XT, MODE_SCATTER, 1, true>(a);
        if (kb <= 2) return launch_one<VT, XT, MODE_SCATTER, 2, true>(a);
        if (kb <= 4) return launch_one<VT, XT, MODE_SCATTER, 4, true>(a);
        return launch_one<VT, XT, MODE_SCATTER, 8, true>(a);
    }
    if (kb <= 1) return launch_one<VT, XT, MODE_SEGDOT, 1, true>(a);
    if (kb <= 2) return launch_one<VT, XT, MODE_SEGDOT, 2, true>(a);
    if (kb <= 4) return launch_one<VT, XT, MODE_SEGDOT, 4, true>(a);
    return launch_one<VT, XT, MODE_SEGDOT, 8, true>(a);
}

}  // namespace gbk
