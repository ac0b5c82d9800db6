// Block stream instantiated with the FP64 arithmetic policy (see stream_impl.cuh).
#include "stream_impl.cuh"

namespace htlr {

void launch_stream_fp64(const StreamArgs &a) { launch_stream_policy<PolicyFP64>(a); }

}  // namespace htlr
