// Generated near field instantiated in FP64 arithmetic (see near_gen_impl.cuh).
#include "near_gen_impl.cuh"

namespace htlr {

void launch_near_generated_f64(const NearGenArgs &a, cudaStream_t s) { launch_gen_prec<double>(a, s); }

}  // namespace htlr
