// Block cluster tree walk (Def. 2.4) on the GPU, one level at a time.
//
// The cluster tree is the 2^d uniform partition of [0,1]^d (§2.2, Def. 3.3).  A pair
// (tau, sigma) of level l is visited when its parents form an inadmissible non-leaf pair
// of level l-1; it becomes an admissible leaf (far) if the admissibility test passes,
// otherwise it is handed to level l+1 (or is an inadmissible leaf at the last level).
//
// Admissibility is decided on integers (reading of Def. 2.2/2.3 on the geometric cells
// of one level, side s): with the box offset o = sigma - tau and the per-dimension gap
// g_k = max(|o_k| - 1, 0) (in units of s), diam^2 = d s^2 and dist^2 = |g|^2 s^2, so the
// strong test is d <= eta^2 |g|^2 (ties admissible, relative slack 1e-12 on eta^2); the
// weak test (zero-measure overlap of the cells) is o != 0.
#include "htlr_internal.h"

namespace htlr {

__device__ __forceinline__ bool admissible_int(int d, const int *o, double eta)
{
    if (eta <= 0.0) {
        for (int k = 0; k < d; ++k)
            if (o[k] != 0) return true;
        return false;
    }
    int g2 = 0;
    for (int k = 0; k < d; ++k) {
        int a = o[k] < 0 ? -o[k] : o[k];
        int g = a > 1 ? a - 1 : 0;
        g2 += g * g;
    }
    return (double)d <= eta * eta * (double)g2 * (1.0 + 1e-12);
}

// pass 0: count far / near children per target box; pass 1: write them at the offsets.
__global__ void walk_kernel(int pass, int d, int level, double eta, const int *prev_rowptr,
                            const int *prev_col, int *far_cnt, int *near_cnt,
                            const int *far_off, const int *near_off, int *far_col,
                            int *near_col)
{
    const int nb1 = 1 << level;
    const int nbox = 1 << (d * level);
    int tau = blockIdx.x * blockDim.x + threadIdx.x;
    if (tau >= nbox) return;
    int t[3], par = 0;
    for (int k = 0; k < d; ++k) {
        t[k] = (tau >> (level * k)) & (nb1 - 1);
        par |= (t[k] >> 1) << ((level - 1) * k);
    }
    int nf = 0, nn = 0;
    int fo = pass ? far_off[tau] : 0, no = pass ? near_off[tau] : 0;
    const int pb1 = nb1 >> 1;
    for (int e = prev_rowptr[par]; e < prev_rowptr[par + 1]; ++e) {
        int sp = prev_col[e];
        int spk[3];
        for (int k = 0; k < d; ++k) spk[k] = (sp >> ((level - 1) * k)) & (pb1 - 1);
        for (int c = 0; c < (1 << d); ++c) {
            int o[3], sig = 0;
            for (int k = 0; k < d; ++k) {
                int sk = 2 * spk[k] + ((c >> k) & 1);
                o[k] = sk - t[k];
                sig |= sk << (level * k);
            }
            if (admissible_int(d, o, eta)) {
                if (pass) far_col[fo + nf] = sig;
                ++nf;
            } else {
                if (pass) near_col[no + nn] = sig;
                ++nn;
            }
        }
    }
    if (!pass) {
        far_cnt[tau] = nf;
        near_cnt[tau] = nn;
    }
}

void launch_walk(int pass, int d, int level, double eta, const int *d_prev_rowptr,
                 const int *d_prev_col, int *d_far_cnt, int *d_near_cnt, const int *d_far_off,
                 const int *d_near_off, int *d_far_col, int *d_near_col, cudaStream_t s)
{
    int nbox = 1 << (d * level);
    int threads = 128;
    int blocks = (nbox + threads - 1) / threads;
    walk_kernel<<<blocks, threads, 0, s>>>(pass, d, level, eta, d_prev_rowptr, d_prev_col,
                                           d_far_cnt, d_near_cnt, d_far_off, d_near_off,
                                           d_far_col, d_near_col);
}

}  // namespace htlr
