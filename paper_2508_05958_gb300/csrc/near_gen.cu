// Generated near field: the inadmissible leaves of Algorithm 2 applied without storing
// their dense blocks (eq. (4.1) evaluated on the fly):
//   f_i = sum_{sigma near tau} sum_{j in sigma, j != i} k(x_i, y_j) w_j u_j
//         + (K_ii w_i + a_i) u_i,                                  i in tau,
// with w_j the cell measure of point j (h^d on a uniform grid).  Used where the dense
// blocks cannot be held (tensor grids, whose blocks differ pair by pair, or very large
// uniform grids).  One CTA per target leaf; the source points of each near leaf are
// staged in shared memory (coordinates relative to the target leaf's corner, w_j u_j)
// and every thread sweeps them for its own target rows.  FP64 or FP32 arithmetic; the
// relative coordinates keep FP32 distances accurate for neighbouring points.
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

constexpr int kGenPer = 4;  // target rows per thread: leaves of up to 1024 points

template <typename T, int NR>
__global__ void __launch_bounds__(256) near_gen_kernel(NearGenArgs A, int r0, int nr)
{
    extern __shared__ __align__(16) unsigned char sm_raw[];
    const int tau = blockIdx.x, d = A.d, n = A.n, L = A.L;
    const int m1 = (1 << L) - 1;
    int tf[3] = {0, 0, 0}, tc[3] = {1, 1, 1};
    double lo[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < d; ++k) {
        int tk = (tau >> (L * k)) & m1;
        tf[k] = A.leafg.first[k][tk];
        tc[k] = A.leafg.cnt[k][tk];
        lo[k] = ldexp((double)tk, -L);
    }
    const int rows = tc[0] * tc[1] * tc[2];
    // shared: source coordinates (d x max_rows, T), w u (NR x max_rows, T)
    T *sy = reinterpret_cast<T *>(sm_raw);
    T *swu = sy + 3 * A.max_rows;
    // own target rows
    T xr[kGenPer][3];
    long long nat[kGenPer];
    T acc[kGenPer][NR];
    for (int m = 0; m < kGenPer; ++m) {
        const int i = threadIdx.x + blockDim.x * m;
        nat[m] = -1;
        for (int r = 0; r < NR; ++r) acc[m][r] = (T)0;
        for (int k = 0; k < 3; ++k) xr[m][k] = (T)0;
        if (i < rows) {
            int j1 = i % tc[0], j23 = i / tc[0], j2 = j23 % tc[1], j3 = j23 / tc[1];
            int gi[3] = {tf[0] + j1, tf[1] + j2, tf[2] + j3};
            long long na = 0, str = 1;
            for (int k = 0; k < d; ++k) {
                xr[m][k] = (T)(A.coords[(long long)k * n + gi[k]] - lo[k]);
                na += (long long)gi[k] * str;
                str *= n;
            }
            nat[m] = na;
        }
    }
    for (int e = A.rowptr[tau]; e < A.rowptr[tau + 1]; ++e) {
        const int sg = A.col[e];
        int sf[3] = {0, 0, 0}, sc[3] = {1, 1, 1};
        for (int k = 0; k < d; ++k) {
            int sk = (sg >> (L * k)) & m1;
            sf[k] = A.leafg.first[k][sk];
            sc[k] = A.leafg.cnt[k][sk];
        }
        const int cols = sc[0] * sc[1] * sc[2];
        __syncthreads();
        for (int j = threadIdx.x; j < cols; j += blockDim.x) {
            int j1 = j % sc[0], j23 = j / sc[0], j2 = j23 % sc[1], j3 = j23 / sc[1];
            int gj[3] = {sf[0] + j1, sf[1] + j2, sf[2] + j3};
            long long na = 0, str = 1;
            double w = 1.0;
            for (int k = 0; k < d; ++k) {
                sy[k * A.max_rows + j] = (T)(A.coords[(long long)k * n + gj[k]] - lo[k]);
                w *= A.width[(long long)k * n + gj[k]];
                na += (long long)gj[k] * str;
                str *= n;
            }
            for (int r = 0; r < nr; ++r)
                swu[r * A.max_rows + j] = (T)(w * A.u[na + A.ldu * (r0 + r)]);
        }
        __syncthreads();
        const bool self = (sg == tau);
        for (int m = 0; m < kGenPer; ++m) {
            const int i = threadIdx.x + blockDim.x * m;
            if (i >= rows) continue;
            for (int j = 0; j < cols; ++j) {
                if (self && j == i) continue;
                T dx[3];
                T r2 = (T)0;
                for (int k = 0; k < d; ++k) {
                    dx[k] = xr[m][k] - sy[k * A.max_rows + j];
                    r2 += dx[k] * dx[k];
                }
                const T kv = kernel_value<T>(A.k, d, r2, dx);
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if (r < nr) acc[m][r] += kv * swu[r * A.max_rows + j];
            }
        }
    }
    for (int m = 0; m < kGenPer; ++m) {
        if (nat[m] < 0) continue;
        const double dg = A.diag[nat[m]] + (A.a ? A.a[nat[m]] : 0.0);
        for (int r = 0; r < nr; ++r) {
            const double uv = A.u[nat[m] + A.ldu * (r0 + r)];
            A.f[nat[m] + A.ldf * (r0 + r)] = (double)acc[m][r] + dg * uv;
        }
    }
}

template <typename T, int NR>
static void launch_gen_t(const NearGenArgs &a, int r0, int nr, cudaStream_t s)
{
    size_t smem = sizeof(T) * (size_t)a.max_rows * (3 + NR);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(near_gen_kernel<T, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    near_gen_kernel<T, NR><<<1 << (a.d * a.L), 256, smem, s>>>(a, r0, nr);
}

template <typename T>
static void launch_gen_prec(const NearGenArgs &a, cudaStream_t s)
{
    for (int r0 = 0; r0 < a.nrhs; r0 += 16) {
        int nr = a.nrhs - r0 < 16 ? a.nrhs - r0 : 16;
        if (nr <= 1) launch_gen_t<T, 1>(a, r0, nr, s);
        else if (nr <= 2) launch_gen_t<T, 2>(a, r0, nr, s);
        else if (nr <= 4) launch_gen_t<T, 4>(a, r0, nr, s);
        else if (nr <= 8) launch_gen_t<T, 8>(a, r0, nr, s);
        else launch_gen_t<T, 16>(a, r0, nr, s);
    }
}

void launch_near_generated(int prec, const NearGenArgs &a, cudaStream_t s)
{
    if (prec == kPrecFP32) launch_gen_prec<float>(a, s);
    else launch_gen_prec<double>(a, s);
}

}  // namespace htlr
