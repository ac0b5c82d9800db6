// Block stream instantiated with the FP32 arithmetic policy (see stream_impl.cuh).
#include "stream_impl.cuh"

namespace htlr {

void launch_stream_fp32(const StreamArgs &a) { launch_stream_policy<PolicyFP32>(a); }

}  // namespace htlr
