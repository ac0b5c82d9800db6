// HMultVec (Algorithm 2) on the GPU, level-batched.
//
// Algorithm 2 applies each admissible block (tau, sigma) as W = U_sigma x_l V_l^T,
// H = G W, F = H x_l U_l (eq. (4.3)), and each inadmissible leaf as a dense gemv.  The
// factors of a box depend on that box alone (on a uniform grid they are even the same
// for every box of a level), so the source-side contraction W_sigma is shared by every
// block with source sigma and the target-side expansion is linear in H_tau; the same
// sums are taken as
//   up      W_sigma = u_sigma x_1 V_1^T ... x_d V_d^T    once per (level, box)
//   stream  H_tau = sum_sigma G_{tau sigma} W_sigma     every admissible block
//           f_tau = sum_sigma A_{tau sigma} u_sigma     every inadmissible leaf
//   out     f_tau += sum_levels H_anc x_1 U_1 ... x_d U_d  restricted to the leaf's rows
// The stream step reads every core and dense block once; it is the hot loop.
#include <algorithm>

#include "htlr_internal.h"

namespace htlr {

// Arithmetic of the up and out contractions.  ArithFP64: plain FP64 FMAs (the FP64 mode).
// ArithDF64: float pairs (hi, lo) with hi + lo equal to the FP64 value to 2^-48, products
// formed with the exact FMA error term and the two cross terms, sums by TwoSum, all on the
// FP32 pipe; used with the df64, FP32 and BF16X6 far fields, whose own arithmetic is no
// more accurate.  Both hold 8 bytes per value, so the shared-memory layouts agree.
struct ArithFP64 {
    using T = double;
    static __device__ __forceinline__ T from(double x) { return x; }
    static __device__ __forceinline__ double to(T a) { return a; }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T mac(T a, T b, T acc) { return fma(a, b, acc); }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
};

struct ArithDF64 {
    using T = float2;  // (hi, lo)
    // FP64 -> (hi, lo) by integer operations (no FP64 instructions): hi keeps the sign,
    // the exponent and the leading 24 bits of the significand, lo the next 24 of the
    // remaining 29 (relative error below 2^-48).  |x| below 2^-100 gives zero, which is
    // far under the operands of the product.
    static __device__ __forceinline__ T from(double x)
    {
        const unsigned long long b = (unsigned long long)__double_as_longlong(x);
        const uint32_t e = (uint32_t)(b >> 52) & 0x7FFu;
        const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
        if (e < 1023u - 100u) return make_float2(0.f, 0.f);
        const float hi = __uint_as_float(sgn | ((e - 896u) << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
        // remainder r 2^(e - 1075), r < 2^29: as a float, normalised by its leading bit
        const uint32_t r = (uint32_t)(b & 0x1FFFFFFFu);
        if (r == 0u) return make_float2(hi, 0.f);
        const int lz = __clz(r);                  // r < 2^29: lz >= 3
        const int top = 31 - lz;                  // index of the leading bit of r
        // significand: the 23 bits below the leading one (truncated)
        const uint32_t man = top >= 23 ? (r >> (top - 23)) & 0x7FFFFFu : (r << (23 - top)) & 0x7FFFFFu;
        const int ex = (int)e - 1075 + top + 127; // biased exponent of r 2^(e - 1075)
        const float lo = ex > 0 ? __uint_as_float(sgn | ((uint32_t)ex << 23) | man) : 0.f;
        return make_float2(hi, lo);
    }
    static __device__ __forceinline__ double to(T a) { return (double)a.x + (double)a.y; }
    static __device__ __forceinline__ T zero() { return make_float2(0.f, 0.f); }
    // acc + a b, renormalised (|lo| <= ulp(hi) / 2).  The _rn intrinsics keep the compiler
    // from contracting the error-free transformations.
    static __device__ __forceinline__ T mac(T a, T b, T acc)
    {
        const float p = __fmul_rn(a.x, b.x);
        float e = __fmaf_rn(a.x, b.x, -p);          // a.hi b.hi - p, exactly
        e = __fmaf_rn(a.x, b.y, e);
        e = __fmaf_rn(a.y, b.x, e);
        const float t = __fadd_rn(acc.x, p);        // TwoSum(acc.hi, p)
        const float z = __fsub_rn(t, acc.x);
        const float err = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(t, z)), __fsub_rn(p, z));
        const float lo = __fadd_rn(acc.y, __fadd_rn(err, e));
        const float hi = __fadd_rn(t, lo);          // renormalise
        return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, t)));
    }
    static __device__ __forceinline__ T add(T a, T b)
    {
        const float t = __fadd_rn(a.x, b.x);
        const float z = __fsub_rn(t, a.x);
        const float err = __fadd_rn(__fsub_rn(a.x, __fsub_rn(t, z)), __fsub_rn(b.x, z));
        const float lo = __fadd_rn(__fadd_rn(a.y, b.y), err);
        const float hi = __fadd_rn(t, lo);
        return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, t)));
    }
};

struct BoxDims {
    int first[3], cnt[3];
    const double *U[3], *V[3];
};

__device__ __forceinline__ BoxDims box_dims(const LevelGeom &g, int d, int box)
{
    BoxDims b;
    const int m = (1 << g.level) - 1;
    for (int k = 0; k < 3; ++k) {
        if (k < d) {
            int bk = (box >> (g.level * k)) & m;
            b.first[k] = g.first[k][bk];
            b.cnt[k] = g.cnt[k][bk];
            b.U[k] = g.Upool + g.uoff[k][bk];
            b.V[k] = g.Vpool + g.voff[k][bk];
        } else {
            b.first[k] = 0;
            b.cnt[k] = 1;
            b.U[k] = b.V[k] = nullptr;
        }
    }
    return b;
}

// ---------------------------------------------------------------------------------
// up: one CTA per (box, rhs).  Mode products in the order 1, 2, (3), slab by slab of
// the last dimension so that shared memory stays bounded for large boxes.
// ---------------------------------------------------------------------------------
template <class AR>
__global__ void __launch_bounds__(128) up_kernel(int d, int n, LevelGeom g,
                                                 const double *__restrict__ u, long long ldu,
                                                 int nrc, double *__restrict__ W, int slab,
                                                 int urows, int vsm)
{
    using T = typename AR::T;
    extern __shared__ __align__(16) unsigned char up_sm[];
    T *sm = reinterpret_cast<T *>(up_sm);
    const int box = blockIdx.x, r = blockIdx.y;
    const int pe = g.pe, mc = g.maxcnt;
    const BoxDims b = box_dims(g, d, box);
    const double *ur = u + ldu * r;
    const int n3 = (d == 3) ? mc : 1;
    T *Vs = sm;                           // d factors, mc x pe each (leading dim cnt_k)
    T *Y1 = Vs + (vsm ? 3 * mc * pe : 0); // pe x c2 x slab
    T *Y2 = Y1 + pe * mc * slab;          // pe x pe x c3
    T *Us = Y2 + pe * pe * n3;            // rows of u_sigma (c1 values each), converted once
    // the factors in shared memory when they fit (vsm), else read (and converted) in place
    if (vsm) {
        for (int k = 0; k < d; ++k)
            for (int i = threadIdx.x; i < b.cnt[k] * pe; i += blockDim.x)
                Vs[k * mc * pe + i] = AR::from(b.V[k][i]);
        __syncthreads();
    }
    const int c1 = b.cnt[0], c2 = b.cnt[1], c3 = (d == 3) ? b.cnt[2] : 1;
    auto vf = [&](int k, int i) -> T { return vsm ? Vs[k * mc * pe + i] : AR::from(b.V[k][i]); };
    const long long base = (long long)b.first[0] + (long long)n * b.first[1] +
                           (d == 3 ? (long long)n * n * b.first[2] : 0);
    for (int i3g = 0; i3g < c3; i3g += slab) {
        const int ns = min(slab, c3 - i3g);
        // mode 1: Y1[mu1 + pe (i2 + c2 j3)] = sum_i1 V1[i1, mu1] u[i1, i2, i3], over the
        // rows (i2, j3) of the slab in chunks of `urows` rows staged in shared memory
        const int nrow = c2 * ns;
        for (int r0 = 0; r0 < nrow; r0 += urows) {
            const int nr = min(urows, nrow - r0);
            for (int idx = threadIdx.x; idx < c1 * nr; idx += blockDim.x) {
                const int i1 = idx % c1, row = r0 + idx / c1;
                const int i2 = row % c2, j3 = row / c2;
                Us[idx] = AR::from(ur[base + i1 + (long long)n * i2 + (long long)n * n * (i3g + j3)]);
            }
            __syncthreads();
            for (int idx = threadIdx.x; idx < pe * nr; idx += blockDim.x) {
                const int mu1 = idx % pe, row = idx / pe;
                const T *ru = Us + c1 * row;
                T acc = AR::zero();
                for (int i1 = 0; i1 < c1; ++i1) acc = AR::mac(vf(0, i1 + c1 * mu1), ru[i1], acc);
                Y1[mu1 + pe * (r0 + row)] = acc;
            }
            __syncthreads();
        }
        // mode 2: Y2[mu1 + pe (mu2 + pe i3)] = sum_i2 V2[i2, mu2] Y1[mu1 + pe (i2 + c2 j3)]
        for (int idx = threadIdx.x; idx < pe * pe * ns; idx += blockDim.x) {
            int mu1 = idx % pe, rest = idx / pe;
            int mu2 = rest % pe, j3 = rest / pe;
            T acc = AR::zero();
            for (int i2 = 0; i2 < c2; ++i2)
                acc = AR::mac(vf(1, i2 + c2 * mu2), Y1[mu1 + pe * (i2 + c2 * j3)], acc);
            Y2[mu1 + pe * (mu2 + pe * (i3g + j3))] = acc;
        }
        __syncthreads();
    }
    const int pd = g.pd;
    double *Wout = W + ((long long)box * nrc + r) * pd;
    if (d == 2) {
        for (int idx = threadIdx.x; idx < pd; idx += blockDim.x) Wout[idx] = AR::to(Y2[idx]);
        return;
    }
    // mode 3: W[mu1 + pe (mu2 + pe mu3)] = sum_i3 V3[i3, mu3] Y2[mu1 + pe (mu2 + pe i3)]
    for (int idx = threadIdx.x; idx < pd; idx += blockDim.x) {
        int m12 = idx % (pe * pe), mu3 = idx / (pe * pe);
        T acc = AR::zero();
        for (int i3 = 0; i3 < c3; ++i3) acc = AR::mac(vf(2, i3 + c3 * mu3), Y2[m12 + pe * pe * i3], acc);
        Wout[idx] = AR::to(acc);
    }
}

void launch_up(int d, int n, const LevelGeom &g, const double *u, int nrhs_here, long long ldu,
               int nrc, double *d_W, cudaStream_t s, bool df64)
{
    const int nbox = 1 << (d * g.level);
    const int mc = g.maxcnt, pe = g.pe;
    const int n3 = (d == 3) ? mc : 1;
    // slab of the last dimension so that the mode-1 buffer stays within 1024 values, and
    // rows of u staged at most 1024 values at a time (no more rows than a slab holds,
    // c2 x slab <= mc x slab): large boxes then take about 28 KB of shared memory and run
    // 8 CTAs per SM instead of 4 (their mode products wait on shared-memory latency)
    int slab = n3;
    while (slab > 1 && (long long)pe * mc * slab > 1024) slab = (slab + 1) / 2;
    const int urows = std::max(1, std::min(1024 / mc, mc * slab));
    const int vsm = 3 * mc * pe <= 8192 ? 1 : 0;   // factors staged when within 64 KB
    size_t smem = sizeof(double) * ((vsm ? (size_t)3 * mc * pe : 0) + (size_t)pe * mc * slab +
                                    (size_t)pe * pe * n3 + (size_t)mc * urows);
    dim3 grid(nbox, nrhs_here);
    if (df64) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(up_kernel<ArithDF64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        up_kernel<ArithDF64><<<grid, 128, smem, s>>>(d, n, g, u, ldu, nrc, d_W, slab, urows, vsm);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(up_kernel<ArithFP64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        up_kernel<ArithFP64><<<grid, 128, smem, s>>>(d, n, g, u, ldu, nrc, d_W, slab, urows, vsm);
    }
}

// The block stream (the hot loop) lives in stream_impl.cuh, instantiated per
// precision in stream_fp64.cu, stream_df64.cu and stream_fp32.cu.
void launch_stream(int prec, const StreamArgs &a)
{
    switch (prec) {
    case kPrecDF64: launch_stream_df64(a); break;
    case kPrecFP32: launch_stream_fp32(a); break;
    default: launch_stream_fp64(a); break;
    }
}

int leaf_level(int n, int leaf)
{
    int l = 0;
    while ((leaf << l) < n) ++l;
    return l;
}

// ---------------------------------------------------------------------------------
// reduce: H_tau[r][t] = sum over the row's tasks (in task order) of their partials.
// ---------------------------------------------------------------------------------
__global__ void reduce_far_kernel(int nbox, int pd, int ld, int nrc, int nrhs_here,
                                  const int *__restrict__ row_task, const Task *__restrict__ tasks,
                                  const double *__restrict__ part, double *__restrict__ H)
{
    long long total = (long long)nbox * nrhs_here * pd;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int t = (int)(idx % pd);
        long long rest = idx / pd;
        int r = (int)(rest % nrhs_here);
        int box = (int)(rest / nrhs_here);
        double acc = 0.0;
        for (int k = row_task[box]; k < row_task[box + 1]; ++k)
            acc += part[tasks[k].part + (long long)r * ld + t];
        H[((long long)box * nrc + r) * pd + t] = acc;
    }
}

void launch_reduce_far(int nbox, int pd, int ld, int nrc, int nrhs_here, const int *d_row_task,
                       const Task *d_tasks, const double *d_part, double *d_H, cudaStream_t s)
{
    long long total = (long long)nbox * nrhs_here * pd;
    int threads = 256;
    long long blocks = (total + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    reduce_far_kernel<<<(int)blocks, threads, 0, s>>>(nbox, pd, ld, nrc, nrhs_here, d_row_task,
                                                      d_tasks, d_part, d_H);
}

// ---------------------------------------------------------------------------------
// out: one CTA per (leaf, rhs).  f_tau = base + sum over the far levels of
// H_anc x_1 U_1 x_2 U_2 (x_3 U_3), each U restricted to the rows of the leaf inside its
// ancestor; written once, in natural order.  The base is the sum of the leaf's
// dense-block partials in task order [+ a u], or the generated near field already in f.
// ---------------------------------------------------------------------------------
// PER: row slots per thread (leaves of up to PER * 256 points), a template argument so
// that the slots stay in registers and only as many as the largest leaf needs are held.
template <class AR, int PER>
__global__ void __launch_bounds__(256) out_kernel(OutArgs A)
{
    constexpr int kOutPer = PER;
    using T = typename AR::T;
    extern __shared__ __align__(16) unsigned char out_sm[];
    T *sm = reinterpret_cast<T *>(out_sm);
    const int tau = blockIdx.x, r = blockIdx.y, d = A.d, n = A.n, L = A.L;
    const BoxDims lb = box_dims(A.leafg, d, tau);
    int t3[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) t3[k] = (tau >> (L * k)) & ((1 << L) - 1);
    const int rows = lb.cnt[0] * lb.cnt[1] * lb.cnt[2];
    const int per = (rows + blockDim.x - 1) / blockDim.x;
    double base[kOutPer];        // near field (+ a u + diagonal), FP64
    T far[kOutPer];              // far field of all levels, in the arithmetic AR
    long long nat[kOutPer];
#pragma unroll
    for (int m = 0; m < kOutPer; ++m) {
        base[m] = 0.0;
        far[m] = AR::zero();
        nat[m] = -1;
        const int i = threadIdx.x + blockDim.x * m;
        if (m < per && i < rows) {
            const int j1 = i % lb.cnt[0], j23 = i / lb.cnt[0];
            const int j2 = j23 % lb.cnt[1], j3 = j23 / lb.cnt[1];
            const long long na = (long long)(lb.first[0] + j1) + (long long)n * (lb.first[1] + j2) +
                                 (d == 3 ? (long long)n * n * (lb.first[2] + j3) : 0);
            nat[m] = na;
            double sb = 0.0;
            if (A.near_in_f) {
                sb = A.f[na + A.ldf * r];
            } else {
                for (int k = A.near_row_task[tau]; k < A.near_row_task[tau + 1]; ++k)
                    sb += A.part[A.tasks[k].part + (long long)r * A.near_ld + i];
                if (A.a_add) sb += A.a_add[na] * A.u[na + A.ldu * r];
                if (A.diag_add) sb += A.diag_add[na] * A.u[na + A.ldu * r];
            }
            base[m] = sb;
        }
    }
    const int c1 = lb.cnt[0], c2 = lb.cnt[1], c3 = lb.cnt[2];
    for (int q = 0; q < A.ndown; ++q) {
        const DownLevel &D = A.down[q];
        const int pe = D.g.pe, lev = D.g.level;
        int anc = 0;
        for (int k = 0; k < d; ++k) anc |= (t3[k] >> (L - lev)) << (lev * k);
        const BoxDims ab = box_dims(D.g, d, anc);
        int o[3];
        for (int k = 0; k < 3; ++k) o[k] = lb.first[k] - ab.first[k];
        const double *Hb = D.H + ((long long)anc * A.nrc + r) * D.g.pd;
        T *Hs = sm;                               // pd
        T *Z3 = Hs + D.g.pd;                      // pe^2 * c3
        T *Z2 = Z3 + pe * pe * c3;                // pe * c2 * c3
        T *Us = Z2 + pe * c2 * c3;                // the ancestor's factors on the leaf's rows
        T *U1 = Us, *U2 = Us + c1 * pe, *U3 = U2 + c2 * pe;
        for (int i = threadIdx.x; i < D.g.pd; i += blockDim.x) Hs[i] = AR::from(Hb[i]);
        for (int i = threadIdx.x; i < c1 * pe; i += blockDim.x)
            U1[i] = AR::from(ab.U[0][o[0] + i % c1 + ab.cnt[0] * (i / c1)]);
        for (int i = threadIdx.x; i < c2 * pe; i += blockDim.x)
            U2[i] = AR::from(ab.U[1][o[1] + i % c2 + ab.cnt[1] * (i / c2)]);
        if (d == 3)
            for (int i = threadIdx.x; i < c3 * pe; i += blockDim.x)
                U3[i] = AR::from(ab.U[2][o[2] + i % c3 + ab.cnt[2] * (i / c3)]);
        __syncthreads();
        const T *Zsrc = Hs;
        if (d == 3) {
            // Z3[mu1 + pe (mu2 + pe j3)] = sum_mu3 U3[j3, mu3] H[mu1 + pe (mu2 + pe mu3)]
            for (int idx = threadIdx.x; idx < pe * pe * c3; idx += blockDim.x) {
                int m12 = idx % (pe * pe), j3 = idx / (pe * pe);
                T acc = AR::zero();
                for (int m3 = 0; m3 < pe; ++m3)
                    acc = AR::mac(U3[j3 + c3 * m3], Hs[m12 + pe * pe * m3], acc);
                Z3[idx] = acc;
            }
            __syncthreads();
            Zsrc = Z3;
        }
        // Z2[mu1 + pe (j2 + c2 j3)] = sum_mu2 U2[j2, mu2] Zsrc[mu1 + pe (mu2 + pe j3)]
        for (int idx = threadIdx.x; idx < pe * c2 * c3; idx += blockDim.x) {
            int mu1 = idx % pe, rest = idx / pe;
            int j2 = rest % c2, j3 = rest / c2;
            T acc = AR::zero();
            for (int m2 = 0; m2 < pe; ++m2)
                acc = AR::mac(U2[j2 + c2 * m2], Zsrc[mu1 + pe * (m2 + pe * j3)], acc);
            Z2[idx] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < kOutPer; ++m) {
            const int i = threadIdx.x + blockDim.x * m;
            if (m < per && i < rows) {
                int j1 = i % c1, j23 = i / c1;
                T acc = far[m];
                for (int m1 = 0; m1 < pe; ++m1) acc = AR::mac(U1[j1 + c1 * m1], Z2[m1 + pe * j23], acc);
                far[m] = acc;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < kOutPer; ++m)
        if (nat[m] >= 0) A.f[nat[m] + A.ldf * r] = base[m] + AR::to(far[m]);
}

template <class AR, int PER>
static void launch_out_per(const OutArgs &a, size_t smem, dim3 grid, int threads, cudaStream_t s)
{
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(out_kernel<AR, PER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    out_kernel<AR, PER><<<grid, threads, smem, s>>>(a);
}

template <class AR>
static void launch_out_ar(const OutArgs &a, int per, size_t smem, dim3 grid, int threads,
                          cudaStream_t s)
{
    if (per <= 1) launch_out_per<AR, 1>(a, smem, grid, threads, s);
    else if (per <= 2) launch_out_per<AR, 2>(a, smem, grid, threads, s);
    else if (per <= 4) launch_out_per<AR, 4>(a, smem, grid, threads, s);
    else launch_out_per<AR, 8>(a, smem, grid, threads, s);
}

void launch_out(const OutArgs &a, int max_rows, cudaStream_t s, bool df64)
{
    size_t smem = 0;
    const int mcl = a.leafg.maxcnt > 1 ? a.leafg.maxcnt : 1;  // largest leaf extent
    for (int q = 0; q < a.ndown; ++q) {
        const int pe = a.down[q].g.pe;
        size_t need = (size_t)a.down[q].g.pd + (size_t)pe * pe * (a.d == 3 ? mcl : 1) +
                      (size_t)pe * mcl * (a.d == 3 ? mcl : 1) + (size_t)3 * mcl * pe;
        if (need > smem) smem = need;
    }
    smem *= sizeof(double);
    if (smem == 0) smem = sizeof(double);
    int threads = max_rows < 256 ? ((max_rows + 31) / 32) * 32 : 256;
    const int per = (max_rows + threads - 1) / threads;   // row slots per thread, <= 8
    dim3 grid(1 << (a.d * a.L), a.nrhs);
    if (df64) launch_out_ar<ArithDF64>(a, per, smem, grid, threads, s);
    else launch_out_ar<ArithFP64>(a, per, smem, grid, threads, s);
}

}  // namespace htlr
