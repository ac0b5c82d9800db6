// Generated near field: the inadmissible leaves of Algorithm 2 applied without storing
// their dense blocks (eq. (4.1) evaluated on the fly).  The kernels are in
// near_gen_impl.cuh, compiled once per precision (near_gen_f32.cu, near_gen_f64.cu).
#include "htlr_internal.h"

namespace htlr {

void launch_near_generated_f32(const NearGenArgs &a, cudaStream_t s);
void launch_near_generated_f64(const NearGenArgs &a, cudaStream_t s);

void launch_near_generated(int prec, const NearGenArgs &a, cudaStream_t s)
{
    if (prec == kPrecFP32) launch_near_generated_f32(a, s);
    else launch_near_generated_f64(a, s);
}

}  // namespace htlr
