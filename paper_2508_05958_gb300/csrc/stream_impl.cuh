// The block stream of HMultVec (the hot loop): H_tau += G_{tau sigma} W_sigma for every
// admissible block and f_tau += A_{tau sigma} u_sigma for every inadmissible leaf
// (eq. (4.3) and the dense case of Algorithm 2).
//
// One warp per task.  A task is a run of consecutive entries of one block row; for every
// entry the warp stages x_sigma (W_sigma, or u_sigma gathered from natural order for the
// dense blocks) in shared memory, then streams the block column by column: lane l owns
// rows l, l + 32, ... (RPL of them), so every column load is one coalesced 256-byte
// access (128 bytes for FP32 blocks), with four columns in flight.  The task's partial
// result goes to `part` in FP64; rows are reduced in task order afterwards.
//
// The arithmetic is a policy, one translation unit each:
//   PolicyFP64  blocks and products in FP64 (1 FMA per streamed double).
//   PolicyDF64  blocks pre-split into float pairs (hi, lo) with hi + lo equal to the
//               FP64 value to 2^-48 relative; each product is formed with the exact FMA
//               error term plus the two cross terms and summed with TwoSum (Knuth), all
//               in the FP32 pipe, which GB300 runs 58x faster than its FP64 pipe.  The
//               partial result is converted to FP64 once per task.
//   PolicyFP32  blocks, products and accumulation in FP32 (mixed-precision far field).
#pragma once

#include "htlr_internal.h"

namespace htlr {

struct PolicyFP64 {
    using BlockT = double;
    using XT = double;
    struct Acc {
        double v;
    };
    static __device__ __forceinline__ void zero(Acc &a) { a.v = 0.0; }
    static __device__ __forceinline__ XT stage(double x) { return x; }
    template <bool CS>
    static __device__ __forceinline__ BlockT load(const BlockT *p)
    {
        if (CS) return __ldcs(p);
        return __ldg(p);
    }
    static __device__ __forceinline__ void mac(Acc &a, BlockT g, XT x) { a.v = fma(g, x, a.v); }
    static __device__ __forceinline__ double out(const Acc &a) { return a.v; }
};

struct PolicyDF64 {
    using BlockT = float2;  // (hi, lo)
    using XT = float2;
    struct Acc {
        float hi, lo;
    };
    static __device__ __forceinline__ void zero(Acc &a) { a.hi = a.lo = 0.f; }
    static __device__ __forceinline__ XT stage(double x)
    {
        float h = __double2float_rn(x);
        return make_float2(h, __double2float_rn(x - (double)h));
    }
    template <bool CS>
    static __device__ __forceinline__ BlockT load(const BlockT *p)
    {
        if (CS) return __ldcs(p);
        return __ldg(p);
    }
    // acc += g * x.  The _rn intrinsics keep the compiler from contracting the
    // additions with the product (which would break the error-free transformations).
    static __device__ __forceinline__ void mac(Acc &a, BlockT g, XT x)
    {
        float p = __fmul_rn(g.x, x.x);
        float e = __fmaf_rn(g.x, x.x, -p);          // g.hi x.hi - p, exactly
        e = __fmaf_rn(g.x, x.y, e);                 // + g.hi x.lo
        e = __fmaf_rn(g.y, x.x, e);                 // + g.lo x.hi
        float t = __fadd_rn(a.hi, p);               // TwoSum(a.hi, p)
        float z = __fsub_rn(t, a.hi);
        float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(t, z)), __fsub_rn(p, z));
        a.hi = t;
        a.lo = __fadd_rn(a.lo, __fadd_rn(err, e));
    }
    static __device__ __forceinline__ double out(const Acc &a) { return (double)a.hi + (double)a.lo; }
};

struct PolicyFP32 {
    using BlockT = float;
    using XT = float;
    struct Acc {
        float v;
    };
    static __device__ __forceinline__ void zero(Acc &a) { a.v = 0.f; }
    static __device__ __forceinline__ XT stage(double x) { return __double2float_rn(x); }
    template <bool CS>
    static __device__ __forceinline__ BlockT load(const BlockT *p)
    {
        if (CS) return __ldcs(p);
        return __ldg(p);
    }
    static __device__ __forceinline__ void mac(Acc &a, BlockT g, XT x) { a.v = __fmaf_rn(g, x, a.v); }
    static __device__ __forceinline__ double out(const Acc &a) { return (double)a.v; }
};

template <class P, int RPL, int NR, bool CS>
__device__ __forceinline__ void stream_task(const Task &T, const KindDesc &K, int lane,
                                            typename P::XT *xs, int d, int n, int leaf,
                                            int nl_level, const double *__restrict__ u,
                                            long long ldu, double *__restrict__ part)
{
    using BlockT = typename P::BlockT;
    typename P::Acc acc[RPL][NR];
#pragma unroll
    for (int k = 0; k < RPL; ++k)
#pragma unroll
        for (int r = 0; r < NR; ++r) P::zero(acc[k][r]);
    const int cols = K.cols, ld = K.ld;
    for (int e = T.e0; e < T.e1; ++e) {
        const int sg = K.col[e];
        const long long bi = K.blk[e];
        // stage x_sigma as xs[j * NR + r]
        if (K.is_near) {
            int s3[3] = {0, 0, 0};
            const int nl1 = 1 << nl_level;
            for (int k = 0; k < d; ++k) s3[k] = (sg >> (nl_level * k)) & (nl1 - 1);
            for (int j = lane; j < cols; j += 32) {
                int jj = j;
                long long nat = 0, str = 1;
                for (int k = 0; k < d; ++k) {
                    nat += (long long)(s3[k] * leaf + jj % leaf) * str;
                    jj /= leaf;
                    str *= n;
                }
#pragma unroll
                for (int r = 0; r < NR; ++r) xs[j * NR + r] = P::stage(u[nat + ldu * r]);
            }
        } else {
            const double *xb = K.x + (long long)sg * K.x_box_stride;
            for (int j = lane; j < cols; j += 32)
#pragma unroll
                for (int r = 0; r < NR; ++r) xs[j * NR + r] = P::stage(xb[(long long)r * cols + j]);
        }
        __syncwarp();
        const BlockT *__restrict__ G =
            static_cast<const BlockT *>(K.blocks) + bi * K.blk_stride + lane;
        int s = 0;
        for (; s + 4 <= cols; s += 4) {
            BlockT g[4][RPL];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int k = 0; k < RPL; ++k)
                    g[q][k] = P::template load<CS>(G + (long long)(s + q) * ld + 32 * k);
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const typename P::XT xv = xs[(s + q) * NR + r];
#pragma unroll
                    for (int k = 0; k < RPL; ++k) P::mac(acc[k][r], g[q][k], xv);
                }
        }
        for (; s < cols; ++s) {
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const typename P::XT xv = xs[s * NR + r];
#pragma unroll
                for (int k = 0; k < RPL; ++k)
                    P::mac(acc[k][r], P::template load<CS>(G + (long long)s * ld + 32 * k), xv);
            }
        }
        __syncwarp();
    }
    double *out = part + T.part;
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
        for (int k = 0; k < RPL; ++k) out[(long long)r * ld + lane + 32 * k] = P::out(acc[k][r]);
}

template <class P, int NR, bool CS>
__global__ void __launch_bounds__(256) stream_kernel(const Task *__restrict__ tasks, int t0, int t1,
                                                     const KindDesc *__restrict__ kinds, int d,
                                                     int n, int leaf, int nl_level,
                                                     const double *__restrict__ u, long long ldu,
                                                     int max_cols, double *__restrict__ part,
                                                     int *err)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    using XT = typename P::XT;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    XT *xs = reinterpret_cast<XT *>(sm_raw) + (long long)wib * max_cols * NR;
    const int wpb = blockDim.x >> 5;
    for (int t = t0 + blockIdx.x * wpb + wib; t < t1; t += gridDim.x * wpb) {
        const Task T = tasks[t];
        const KindDesc K = kinds[T.kind];
        switch (K.rpl) {
#define HTLR_RPL_CASE(R)                                                                        \
    case R: stream_task<P, R, NR, CS>(T, K, lane, xs, d, n, leaf, nl_level, u, ldu, part); break;
            HTLR_RPL_CASE(1) HTLR_RPL_CASE(2) HTLR_RPL_CASE(3) HTLR_RPL_CASE(4)
            HTLR_RPL_CASE(5) HTLR_RPL_CASE(6) HTLR_RPL_CASE(7) HTLR_RPL_CASE(8)
            HTLR_RPL_CASE(9) HTLR_RPL_CASE(10) HTLR_RPL_CASE(11) HTLR_RPL_CASE(12)
            HTLR_RPL_CASE(13) HTLR_RPL_CASE(14) HTLR_RPL_CASE(15) HTLR_RPL_CASE(16)
#undef HTLR_RPL_CASE
        default:
            if (lane == 0) atomicExch(err, (int)kDevBadTask);
        }
    }
}

template <class P, int NR, bool CS>
static void launch_stream_policy_t(const StreamArgs &a, int blocks, int threads, size_t smem)
{
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(stream_kernel<P, NR, CS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    stream_kernel<P, NR, CS><<<blocks, threads, smem, a.stream>>>(
        a.tasks, a.t0, a.t1, a.kinds, a.d, a.n, a.leaf, a.nl_level, a.u, a.ldu, a.max_cols,
        a.part, a.err);
}

template <class P>
static void launch_stream_policy(const StreamArgs &a)
{
    const int ntasks = a.t1 - a.t0;
    if (ntasks <= 0) return;
    const int threads = a.threads == 128 ? 128 : 256, wpb = threads / 32;
    int blocks = (ntasks + wpb - 1) / wpb;
    const int cap = 152 * (a.ctas_per_sm > 0 ? a.ctas_per_sm : 8);
    if (blocks > cap) blocks = cap;
    size_t smem = sizeof(typename P::XT) * (size_t)wpb * a.max_cols * a.nrhs;
#define HTLR_NR_CASE(R)                                                          \
    case R:                                                                      \
        if (a.streaming)                                                         \
            launch_stream_policy_t<P, R, true>(a, blocks, threads, smem);       \
        else                                                                     \
            launch_stream_policy_t<P, R, false>(a, blocks, threads, smem);      \
        break;
    switch (a.nrhs) {
        HTLR_NR_CASE(1) HTLR_NR_CASE(2) HTLR_NR_CASE(3) HTLR_NR_CASE(4)
    default: break;
    }
#undef HTLR_NR_CASE
}

}  // namespace htlr
