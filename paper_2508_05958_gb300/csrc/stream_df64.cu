// Block stream instantiated with the DF64 arithmetic policy (see stream_impl.cuh).
#include "stream_impl.cuh"

namespace htlr {

void launch_stream_df64(const StreamArgs &a) { launch_stream_policy<PolicyDF64>(a); }

}  // namespace htlr
