// Generated near field: the inadmissible leaves of Algorithm 2 applied without storing
// their dense blocks (eq. (4.1) evaluated on the fly).  Compiled once per precision
// (near_gen_f32.cu, near_gen_f64.cu); near_gen.cu dispatches.
//   f_i = sum_{sigma near tau} sum_{j in sigma, j != i} k(x_i, y_j) w_j u_j
//         + (K_ii w_i + a_i) u_i,                                  i in tau,
// with w_j the cell measure of point j (h^d on a uniform grid).  Used where the dense
// blocks cannot be held (tensor grids, whose blocks differ pair by pair, or very large
// uniform grids).  One CTA per target leaf; the source points of each near leaf are
// staged in shared memory (coordinates relative to the target leaf's corner, w_j u_j)
// and every thread sweeps them for its own target rows.  FP64 or FP32 arithmetic; the
// relative coordinates keep FP32 distances accurate for neighbouring points.
#pragma once

#include "htlr_internal.h"

namespace htlr {

template <typename T>
__device__ __forceinline__ T kernel_value(const KernelDesc &k, int d, T r2, const T *dx);

template <>
__device__ __forceinline__ double kernel_value<double>(const KernelDesc &k, int d, double r2,
                                                       const double *dx)
{
    switch (k.type) {
    case HTLR_K_LOG: return k.scale * 0.5 * log(r2);
    case HTLR_K_INV_R: return k.scale / sqrt(r2);
    case HTLR_K_EXP_R: return k.scale * exp(-sqrt(r2));
    case HTLR_K_GAUSS: return k.scale * exp(-r2 / (2.0 * k.param * k.param));
    case HTLR_K_POLY: {
        int deg = (int)k.param;
        double v = k.scale;
        for (int l = 0; l < d; ++l) {
            double b = dx[l] + 2.0 + 0.5 * l, pw = 1.0;
            for (int e = 0; e < deg; ++e) pw *= b;
            v *= pw;
        }
        return v;
    }
    default: return k.scale;
    }
}

template <>
__device__ __forceinline__ float kernel_value<float>(const KernelDesc &k, int d, float r2,
                                                     const float *dx)
{
    const float sc = (float)k.scale;
    switch (k.type) {
    case HTLR_K_LOG: return sc * 0.5f * logf(r2);
    case HTLR_K_INV_R: return sc / sqrtf(r2);
    case HTLR_K_EXP_R: return sc * expf(-sqrtf(r2));
    case HTLR_K_GAUSS: return sc * expf(-r2 / (float)(2.0 * k.param * k.param));
    case HTLR_K_POLY: {
        int deg = (int)k.param;
        float v = sc;
        for (int l = 0; l < d; ++l) {
            float b = dx[l] + 2.0f + 0.5f * l, pw = 1.0f;
            for (int e = 0; e < deg; ++e) pw *= b;
            v *= pw;
        }
        return v;
    }
    default: return sc;
    }
}

// One CTA per target leaf; thread t owns the target rows t, t + T, ..., t + (PER-1) T
// (T threads).  The source points of one near leaf at a time are staged in shared memory
// as (y relative to the target leaf's corner, w_j u_j for every RHS, contiguous), and
// every thread sweeps them with its PER rows held in registers, so one staged point
// feeds PER kernel evaluations and PER x NR multiply-adds.  The kernel type is resolved
// once per launch (a template argument of the sweep), not per pair.  All small per-
// dimension arrays are indexed with compile-time indices so they stay in registers.
struct KParams {
    double scale, param, inv2s2;  // inv2s2 = 1 / (2 sigma^2) for the Gaussian
    int deg;
};

// 2^x by the SFU's base-2 exponential (relative error near 2^-22; x <= 0 here, results
// in (0, 1], never subnormal for the distances of neighbouring leaves).
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/sqrt(x) by the SFU (relative error near 2^-23).  x is a squared distance between
// distinct points here, never subnormal; x = 0 (a point with itself) gives +inf, and the
// sweep replaces that pair's value.
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Scale applied to the FP32 coordinates when they are staged, so that the exponential
// kernels need no multiply per pair: exp(-r) = 2^(-r log2 e) with coordinates scaled by
// log2 e, and exp(-r^2 / (2 sigma^2)) = 2^(-r^2) with coordinates scaled by
// sqrt(log2 e / (2 sigma^2)).  FP64 arithmetic and the other kernels use the plain
// coordinates.
template <typename T>
__host__ __device__ inline double coord_scale(int ktype, double sigma)
{
    const double log2e = 1.4426950408889634;
    if (sizeof(T) != 4) return 1.0;
    if (ktype == HTLR_K_EXP_R) return log2e;
    if (ktype == HTLR_K_GAUSS) return sqrt(log2e / (2.0 * sigma * sigma));
    return 1.0;
}

// Kernel values without the kernel's scale factor, which the sweep folds into w_j u_j.
// FP32 coordinates arrive scaled by coord_scale<float>.
template <typename T, int KT>
__device__ __forceinline__ T kv_eval(const KParams &k, int d, T r2, T dx0, T dx1, T dx2)
{
    if constexpr (KT == HTLR_K_LOG) {
        return (T)0.5 * log(r2);
    } else if constexpr (KT == HTLR_K_INV_R) {
        if constexpr (sizeof(T) == 4) return rsqrt_approx(r2);
        else return 1.0 / sqrt(r2);
    } else if constexpr (KT == HTLR_K_EXP_R) {
        if constexpr (sizeof(T) == 4) return ex2_approx(-(r2 * rsqrt_approx(r2)));
        else return exp(-sqrt(r2));
    } else if constexpr (KT == HTLR_K_GAUSS) {
        if constexpr (sizeof(T) == 4) return ex2_approx(-r2);
        else return exp(-r2 * k.inv2s2);
    } else if constexpr (KT == HTLR_K_POLY) {
        const T dxs[3] = {dx0, dx1, dx2};
        T v = (T)1;
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            if (l < d) {
                const T b = dxs[l] + (T)2 + (T)0.5 * (T)l;
                T pw = (T)1;
                for (int e = 0; e < k.deg; ++e) pw *= b;
                v *= pw;
            }
        }
        return v;
    } else {
        return (T)1;
    }
}

// FP32 row totals: slot m of this thread, RHS r, at tot[r * nslot + threadIdx.x +
// blockDim.x * m]; the first source leaf stores, the others add.
__device__ __forceinline__ void fold_total(float *__restrict__ tot, int nslot, int m, int r,
                                           bool first, float v)
{
    float &t = tot[r * nslot + (int)threadIdx.x + (int)blockDim.x * m];
    t = first ? v : t + v;
}

// Sweeps the staged source leaf for the first PA (<= PER) row slots of the thread: the
// others hold no row of the leaf for any lane of the warp.  FP64 accumulates into acc;
// FP32 sums the leaf in registers and folds the sums into the row totals (fold_total),
// so a row's sum over all its near leaves is two short FP32 sums, not one long one.
template <typename T, int NR, int PER, int PA, int KT, bool SELF>
__device__ __forceinline__ void sweep(const KParams &k, int d, int cols,
                                      const T *__restrict__ sy, const T *__restrict__ swu,
                                      const T (&xr)[PER][3], const int (&irow)[PER],
                                      T (&acc)[PER][NR], float *__restrict__ tot, int nslot,
                                      bool first)
{
    if constexpr (sizeof(T) == 4 && NR % 2 == 0) {
        // FP32: the multiply-adds of two right-hand sides in one packed FMA (f32x2)
        float2 a2[PER][NR / 2];
#pragma unroll
        for (int m = 0; m < PA; ++m)
#pragma unroll
            for (int r = 0; r < NR / 2; ++r) a2[m][r] = make_float2(0.f, 0.f);
        const float2 *swu2 = reinterpret_cast<const float2 *>(swu);
        for (int j = 0; j < cols; ++j) {
            const T y0 = sy[4 * j], y1 = sy[4 * j + 1], y2 = sy[4 * j + 2];
            float2 wu[NR / 2];
#pragma unroll
            for (int r = 0; r < NR / 2; ++r) wu[r] = swu2[j * (NR / 2) + r];
#pragma unroll
            for (int m = 0; m < PA; ++m) {
                const T dx0 = xr[m][0] - y0, dx1 = xr[m][1] - y1, dx2 = xr[m][2] - y2;
                const T r2 = dx0 * dx0 + dx1 * dx1 + dx2 * dx2;
                T kv = kv_eval<T, KT>(k, d, r2, dx0, dx1, dx2);
                if constexpr (SELF) kv = j == irow[m] ? (T)0 : kv;   // diagonal: added apart
                const float2 kv2 = make_float2(kv, kv);
#pragma unroll
                for (int r = 0; r < NR / 2; ++r) a2[m][r] = __ffma2_rn(kv2, wu[r], a2[m][r]);
            }
        }
#pragma unroll
        for (int m = 0; m < PA; ++m)
#pragma unroll
            for (int r = 0; r < NR / 2; ++r) {
                fold_total(tot, nslot, m, 2 * r, first, a2[m][r].x);
                fold_total(tot, nslot, m, 2 * r + 1, first, a2[m][r].y);
            }
    } else if constexpr (sizeof(T) == 4) {
        float l[PER][NR];
#pragma unroll
        for (int m = 0; m < PA; ++m)
#pragma unroll
            for (int r = 0; r < NR; ++r) l[m][r] = 0.f;
        for (int j = 0; j < cols; ++j) {
            const T y0 = sy[4 * j], y1 = sy[4 * j + 1], y2 = sy[4 * j + 2];
            T wu[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) wu[r] = swu[j * NR + r];
#pragma unroll
            for (int m = 0; m < PA; ++m) {
                const T dx0 = xr[m][0] - y0, dx1 = xr[m][1] - y1, dx2 = xr[m][2] - y2;
                const T r2 = dx0 * dx0 + dx1 * dx1 + dx2 * dx2;
                T kv = kv_eval<T, KT>(k, d, r2, dx0, dx1, dx2);
                if constexpr (SELF) kv = j == irow[m] ? (T)0 : kv;   // the diagonal is added apart
#pragma unroll
                for (int r = 0; r < NR; ++r) l[m][r] = __fmaf_rn(kv, wu[r], l[m][r]);
            }
        }
#pragma unroll
        for (int m = 0; m < PA; ++m)
#pragma unroll
            for (int r = 0; r < NR; ++r) fold_total(tot, nslot, m, r, first, l[m][r]);
    } else {
        for (int j = 0; j < cols; ++j) {
            const T y0 = sy[4 * j], y1 = sy[4 * j + 1], y2 = sy[4 * j + 2];
            T wu[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) wu[r] = swu[j * NR + r];
#pragma unroll
            for (int m = 0; m < PA; ++m) {
                const T dx0 = xr[m][0] - y0, dx1 = xr[m][1] - y1, dx2 = xr[m][2] - y2;
                const T r2 = dx0 * dx0 + dx1 * dx1 + dx2 * dx2;
                T kv = kv_eval<T, KT>(k, d, r2, dx0, dx1, dx2);
                if constexpr (SELF) kv = j == irow[m] ? (T)0 : kv;   // the diagonal is added apart
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[m][r] += kv * wu[r];
            }
        }
    }
}

// Dispatch on the warp's count of active row slots pa (warp-uniform): sweep the first pa.
template <typename T, int NR, int PER, int PA, int KT, bool SELF>
__device__ __forceinline__ void sweep_active(int pa, const KParams &k, int d, int cols,
                                             const T *__restrict__ sy, const T *__restrict__ swu,
                                             const T (&xr)[PER][3], const int (&irow)[PER],
                                             T (&acc)[PER][NR], float *__restrict__ tot,
                                             int nslot, bool first)
{
    if constexpr (PA >= 1) {
        if (pa == PA)
            sweep<T, NR, PER, PA, KT, SELF>(k, d, cols, sy, swu, xr, irow, acc, tot, nslot, first);
        else
            sweep_active<T, NR, PER, PA - 1, KT, SELF>(pa, k, d, cols, sy, swu, xr, irow, acc,
                                                       tot, nslot, first);
    }
}

// box of leaf index g: first grid line and point count per dimension (unused dims: 0, 1)
__device__ __forceinline__ void leaf_box(const LevelGeom &lg, int d, int L, int g, int (&f)[3],
                                         int (&c)[3])
{
    const int m1 = (1 << L) - 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        f[k] = 0;
        c[k] = 1;
        if (k < d) {
            const int bk = (g >> (L * k)) & m1;
            f[k] = lg.first[k][bk];
            c[k] = lg.cnt[k][bk];
        }
    }
}

template <typename T, int NR, int PER>
__global__ void __launch_bounds__(256) near_gen_kernel(NearGenArgs A, int r0, int nr)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int tau = blockIdx.x, d = A.d, n = A.n, L = A.L;
    int tf[3], tc[3];
    leaf_box(A.leafg, d, L, tau, tf, tc);
    double lo[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) lo[k] = k < d ? ldexp((double)((tau >> (L * k)) & ((1 << L) - 1)), -L) : 0.0;
    const int rows = tc[0] * tc[1] * tc[2];
    KParams kp;
    kp.scale = A.k.scale;
    kp.param = A.k.param;
    kp.inv2s2 = A.k.type == HTLR_K_GAUSS ? 1.0 / (2.0 * A.k.param * A.k.param) : 0.0;
    kp.deg = (int)A.k.param;
    const double cs = coord_scale<T>(A.k.type, A.k.param);
    // shared: source points (4 per point: y_1..y_3, pad), w u (max_rows x NR)
    T *sy = reinterpret_cast<T *>(sm_raw);
    T *swu = sy + 4 * A.max_rows;
    float *stot = reinterpret_cast<float *>(swu + (size_t)A.max_rows * NR);   // FP32 only
    const int nslot = PER * (int)blockDim.x;
    T xr[PER][3];
    int irow[PER];
    long long nat[PER];
    T acc[PER][NR];
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int i = threadIdx.x + blockDim.x * m;
        irow[m] = i;
        nat[m] = -1;
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[m][r] = (T)0;
        // rows past the leaf evaluate a far-away dummy point (finite, never written)
        xr[m][0] = xr[m][1] = xr[m][2] = (T)4;
        if (i < rows) {
            const int j1 = i % tc[0], j23 = i / tc[0], j2 = j23 % tc[1], j3 = j23 / tc[1];
            const int gi[3] = {tf[0] + j1, tf[1] + j2, tf[2] + j3};
            long long na = 0, str = 1;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                xr[m][k] = (T)0;
                if (k < d) {
                    xr[m][k] = (T)((A.coords[(long long)k * n + gi[k]] - lo[k]) * cs);
                    na += (long long)gi[k] * str;
                    str *= n;
                }
            }
            nat[m] = na;
        }
    }
    // Row slot m of warp w holds rows 32 (w + W m) ... + 31 (W warps): slots past the
    // leaf's last row are skipped for the whole warp, so a leaf smaller than the CTA's
    // PER x T row slots costs only its own rows (rounded up to 32).
    const int wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5, groups = (rows + 31) >> 5;
    int pa = 0;
#pragma unroll
    for (int m = 0; m < PER; ++m)
        if (wid + nwarp * m < groups) pa = m + 1;
    for (int e = A.rowptr[tau]; e < A.rowptr[tau + 1]; ++e) {
        const int sg = A.col[e];
        int sf[3], sc[3];
        leaf_box(A.leafg, d, L, sg, sf, sc);
        const int cols = sc[0] * sc[1] * sc[2];
        __syncthreads();
        for (int j = threadIdx.x; j < cols; j += blockDim.x) {
            const int j1 = j % sc[0], j23 = j / sc[0], j2 = j23 % sc[1], j3 = j23 / sc[1];
            const int gj[3] = {sf[0] + j1, sf[1] + j2, sf[2] + j3};
            long long na = 0, str = 1;
            double w = 1.0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                T y = (T)0;
                if (k < d) {
                    y = (T)((A.coords[(long long)k * n + gj[k]] - lo[k]) * cs);
                    w *= A.width[(long long)k * n + gj[k]];
                    na += (long long)gj[k] * str;
                    str *= n;
                }
                sy[4 * j + k] = y;
            }
            sy[4 * j + 3] = (T)0;
#pragma unroll
            for (int r = 0; r < NR; ++r)
                swu[j * NR + r] = r < nr ? (T)(A.k.scale * w * A.u[na + A.ldu * (r0 + r)]) : (T)0;
        }
        __syncthreads();
        const bool self = (sg == tau), first = (e == A.rowptr[tau]);
#define HTLR_SWEEP(KT)                                                                      \
    (self ? sweep_active<T, NR, PER, PER, KT, true>(pa, kp, d, cols, sy, swu, xr, irow, acc, \
                                                    stot, nslot, first)                     \
          : sweep_active<T, NR, PER, PER, KT, false>(pa, kp, d, cols, sy, swu, xr, irow, acc, \
                                                     stot, nslot, first))
        switch (A.k.type) {
        case HTLR_K_LOG: HTLR_SWEEP(HTLR_K_LOG); break;
        case HTLR_K_INV_R: HTLR_SWEEP(HTLR_K_INV_R); break;
        case HTLR_K_EXP_R: HTLR_SWEEP(HTLR_K_EXP_R); break;
        case HTLR_K_GAUSS: HTLR_SWEEP(HTLR_K_GAUSS); break;
        case HTLR_K_POLY: HTLR_SWEEP(HTLR_K_POLY); break;
        default: HTLR_SWEEP(HTLR_K_CONST); break;
        }
#undef HTLR_SWEEP
    }
    if constexpr (sizeof(T) == 4) {   // FP32: the row totals (each thread reads its own)
        if (A.rowptr[tau + 1] > A.rowptr[tau]) {
#pragma unroll
            for (int m = 0; m < PER; ++m)
                if (m < pa) {
#pragma unroll
                    for (int r = 0; r < NR; ++r)
                        acc[m][r] = stot[r * nslot + threadIdx.x + blockDim.x * m];
                }
        }
    }
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        if (nat[m] < 0) continue;
        const double dg = A.diag[nat[m]] + (A.a ? A.a[nat[m]] : 0.0);
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (r < nr) {
                const double uv = A.u[nat[m] + A.ldu * (r0 + r)];
                A.f[nat[m] + A.ldf * (r0 + r)] = (double)acc[m][r] + dg * uv;
            }
        }
    }
}

template <typename T, int NR, int PER>
static void launch_gen_t(const NearGenArgs &a, int r0, int nr, int threads, cudaStream_t s)
{
    size_t smem = sizeof(T) * (size_t)a.max_rows * (4 + NR);
    if (sizeof(T) == 4) smem += sizeof(float) * (size_t)PER * threads * NR;   // row totals
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(near_gen_kernel<T, NR, PER>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    near_gen_kernel<T, NR, PER><<<1 << (a.d * a.L), threads, smem, s>>>(a, r0, nr);
}

template <typename T, int NR>
static void launch_gen_nr(const NearGenArgs &a, int r0, int nr, cudaStream_t s)
{
    // the fewest rows per thread that cover the largest leaf with at most 256 threads
    int per = 2;
    while (per < 4 && (a.max_rows + per - 1) / per > 256) ++per;
    int threads = ((a.max_rows + per - 1) / per + 31) / 32 * 32;
    if (threads < 32) threads = 32;
    if (per == 2) launch_gen_t<T, NR, 2>(a, r0, nr, threads, s);
    else if (per == 3) launch_gen_t<T, NR, 3>(a, r0, nr, threads, s);
    else launch_gen_t<T, NR, 4>(a, r0, nr, threads, s);
}

template <typename T>
inline void launch_gen_prec(const NearGenArgs &a, cudaStream_t s)
{
    for (int r0 = 0; r0 < a.nrhs; r0 += 16) {
        int nr = a.nrhs - r0 < 16 ? a.nrhs - r0 : 16;
        if (nr <= 1) launch_gen_nr<T, 1>(a, r0, nr, s);
        else if (nr <= 4) launch_gen_nr<T, 4>(a, r0, nr, s);
        else launch_gen_nr<T, 16>(a, r0, nr, s);
    }
}

}  // namespace htlr
