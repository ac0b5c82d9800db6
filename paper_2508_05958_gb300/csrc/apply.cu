// HMultVec (Algorithm 2) on the GPU, level-batched.
//
// Algorithm 2 applies each admissible block (tau, sigma) as W = U_sigma x_l V_l^T,
// H = G W, F = H x_l U_l (eq. (4.3)), and each inadmissible leaf as a dense gemv.  On a
// uniform grid the factors of a level are the same for every box, so the source-side
// contraction W_sigma depends on sigma alone and the target-side expansion is linear in
// H_tau: the same sums are taken as
//   up      W_sigma = u_sigma x_1 F^T ... x_d F^T        once per (level, box)
//   stream  H_tau = sum_sigma G_{tau sigma} W_sigma     every admissible block
//           f_tau = sum_sigma A_{tau sigma} u_sigma     every inadmissible leaf
//   out     f_tau += sum_levels H_anc x_1 F ... x_d F   restricted to the leaf's rows
// The stream step reads every core and dense block once; it is the hot loop.
#include "htlr_internal.h"

namespace htlr {

// ---------------------------------------------------------------------------------
// up: one CTA per (box, rhs).  Mode products in the order 1, 2, (3), slab by slab of
// the last dimension so that shared memory stays bounded for large boxes.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(128) up_kernel(int d, int n, int level, int nb, int pe,
                                                 const double *__restrict__ F,
                                                 const double *__restrict__ u, long long ldu,
                                                 int nrc, double *__restrict__ W, int slab)
{
    extern __shared__ double sm[];
    const int box = blockIdx.x, r = blockIdx.y;
    const int nb1 = 1 << level;
    int b[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) b[k] = (box >> (level * k)) & (nb1 - 1);
    const double *ur = u + ldu * r;
    double *Fs = sm;                      // nb x pe
    double *Y1 = Fs + nb * pe;            // pe x nb x slab  (mode-1 result of a slab)
    double *Y2 = Y1 + pe * nb * slab;     // pe x pe x nb    (d = 3) or pe x pe (d = 2)
    for (int i = threadIdx.x; i < nb * pe; i += blockDim.x) Fs[i] = F[i];
    __syncthreads();
    const int n3 = (d == 3) ? nb : 1;
    const long long base = (long long)b[0] * nb + (long long)n * b[1] * nb +
                           (d == 3 ? (long long)n * n * b[2] * nb : 0);
    for (int i3g = 0; i3g < n3; i3g += slab) {
        int ns = min(slab, n3 - i3g);
        // mode 1 on the slab: Y1[mu1 + pe (i2 + nb j3)] = sum_i1 F[i1, mu1] u[i1, i2, i3]
        for (int idx = threadIdx.x; idx < pe * nb * ns; idx += blockDim.x) {
            int mu1 = idx % pe, rest = idx / pe;
            int i2 = rest % nb, j3 = rest / nb;
            const double *row = ur + base + (long long)n * i2 + (long long)n * n * (i3g + j3);
            double acc = 0.0;
            for (int i1 = 0; i1 < nb; ++i1) acc = fma(Fs[i1 + nb * mu1], row[i1], acc);
            Y1[idx] = acc;
        }
        __syncthreads();
        // mode 2: Y2[mu1 + pe (mu2 + pe i3)] = sum_i2 F[i2, mu2] Y1[mu1 + pe (i2 + nb j3)]
        for (int idx = threadIdx.x; idx < pe * pe * ns; idx += blockDim.x) {
            int mu1 = idx % pe, rest = idx / pe;
            int mu2 = rest % pe, j3 = rest / pe;
            double acc = 0.0;
            for (int i2 = 0; i2 < nb; ++i2)
                acc = fma(Fs[i2 + nb * mu2], Y1[mu1 + pe * (i2 + nb * j3)], acc);
            Y2[mu1 + pe * (mu2 + pe * (i3g + j3))] = acc;
        }
        __syncthreads();
    }
    const int pd = (d == 3) ? pe * pe * pe : pe * pe;
    double *Wout = W + ((long long)box * nrc + r) * pd;
    if (d == 2) {
        for (int idx = threadIdx.x; idx < pd; idx += blockDim.x) Wout[idx] = Y2[idx];
        return;
    }
    // mode 3: W[mu1 + pe (mu2 + pe mu3)] = sum_i3 F[i3, mu3] Y2[mu1 + pe (mu2 + pe i3)]
    for (int idx = threadIdx.x; idx < pd; idx += blockDim.x) {
        int m12 = idx % (pe * pe), mu3 = idx / (pe * pe);
        double acc = 0.0;
        for (int i3 = 0; i3 < nb; ++i3) acc = fma(Fs[i3 + nb * mu3], Y2[m12 + pe * pe * i3], acc);
        Wout[idx] = acc;
    }
}

void launch_up(int d, int n, int level, int nb, int pe, const double *d_F, const double *u,
               int nrhs_here, long long ldu, int nrc, double *d_W, cudaStream_t s)
{
    int nbox = 1 << (d * level);
    int n3 = (d == 3) ? nb : 1;
    // slab so that the mode-1 buffer stays within ~64 KB
    int slab = n3;
    while (slab > 1 && (long long)pe * nb * slab > 8192) slab = (slab + 1) / 2;
    size_t smem = sizeof(double) * ((size_t)nb * pe + (size_t)pe * nb * slab +
                                    (size_t)pe * pe * n3);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(up_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(nbox, nrhs_here);
    up_kernel<<<grid, 128, smem, s>>>(d, n, level, nb, pe, d_F, u, ldu, nrc, d_W, slab);
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
// out: one CTA per (leaf, rhs).  f_tau = (sum of the leaf's inadmissible-block partials)
// [+ a u] + sum over the far levels of H_anc x_1 F x_2 F (x_3 F), F restricted to the
// rows of the leaf inside its ancestor; written once, in natural order.
// ---------------------------------------------------------------------------------
struct DownArgs {
    int ndown;
    DownLevel lv[HTLR_MAX_LEVELS];
};

__global__ void __launch_bounds__(256) out_kernel(int d, int n, int leaf, int L, int nrc,
                                                  const int *__restrict__ near_row_task,
                                                  const Task *__restrict__ tasks,
                                                  const double *__restrict__ part, int near_ld,
                                                  const double *__restrict__ a_add,
                                                  const double *__restrict__ u, long long ldu,
                                                  DownArgs down, double *__restrict__ f,
                                                  long long ldf)
{
    extern __shared__ double sm[];
    const int tau = blockIdx.x, r = blockIdx.y;
    const int nl1 = 1 << L;
    int t3[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) t3[k] = (tau >> (L * k)) & (nl1 - 1);
    int rows = 1;
    for (int k = 0; k < d; ++k) rows *= leaf;
    // per-thread accumulators for rows i = threadIdx.x + blockDim.x * m
    const int per = (rows + blockDim.x - 1) / blockDim.x;  // <= 8 (leaf^d <= 2048)
    double acc[8];
    long long nat[8];
    for (int m = 0; m < per && m < 8; ++m) {
        int i = threadIdx.x + blockDim.x * m;
        acc[m] = 0.0;
        nat[m] = -1;
        if (i < rows) {
            int ii = i;
            long long na = 0, str = 1;
            for (int k = 0; k < d; ++k) {
                na += (long long)(t3[k] * leaf + ii % leaf) * str;
                ii /= leaf;
                str *= n;
            }
            nat[m] = na;
            double s = 0.0;
            for (int k = near_row_task[tau]; k < near_row_task[tau + 1]; ++k)
                s += part[tasks[k].part + (long long)r * near_ld + i];
            if (a_add) s += a_add[na] * u[na + ldu * r];
            acc[m] = s;
        }
    }
    // far levels, in increasing level order
    for (int q = 0; q < down.ndown; ++q) {
        const DownLevel D = down.lv[q];
        const int pe = D.pe, nb = D.nb, lev = D.level;
        int anc = 0, o[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) {
            int ak = t3[k] >> (L - lev);
            anc |= ak << (lev * k);
            o[k] = (t3[k] - (ak << (L - lev))) * leaf;
        }
        const double *Hb = D.H + ((long long)anc * nrc + r) * D.pd;
        double *Hs = sm;                          // pd
        double *Z3 = Hs + D.pd;                   // pe^2 * leaf   (d = 3)
        double *Z2 = Z3 + pe * pe * leaf;         // pe * leaf^(d-1)
        for (int i = threadIdx.x; i < D.pd; i += blockDim.x) Hs[i] = Hb[i];
        __syncthreads();
        const double *Zsrc = Hs;
        if (d == 3) {
            // Z3[mu1 + pe (mu2 + pe j3)] = sum_mu3 F[o3 + j3, mu3] H[mu1 + pe (mu2 + pe mu3)]
            for (int idx = threadIdx.x; idx < pe * pe * leaf; idx += blockDim.x) {
                int m12 = idx % (pe * pe), j3 = idx / (pe * pe);
                double s = 0.0;
                for (int m3 = 0; m3 < pe; ++m3)
                    s = fma(D.F[o[2] + j3 + nb * m3], Hs[m12 + pe * pe * m3], s);
                Z3[idx] = s;
            }
            __syncthreads();
            Zsrc = Z3;
        }
        // Z2[mu1 + pe (j2 + leaf j3)] = sum_mu2 F[o2 + j2, mu2] Zsrc[mu1 + pe (mu2 + pe j3)]
        const int n3 = (d == 3) ? leaf : 1;
        for (int idx = threadIdx.x; idx < pe * leaf * n3; idx += blockDim.x) {
            int mu1 = idx % pe, rest = idx / pe;
            int j2 = rest % leaf, j3 = rest / leaf;
            double s = 0.0;
            for (int m2 = 0; m2 < pe; ++m2)
                s = fma(D.F[o[1] + j2 + nb * m2], Zsrc[mu1 + pe * (m2 + pe * j3)], s);
            Z2[idx] = s;
        }
        __syncthreads();
        for (int m = 0; m < per && m < 8; ++m) {
            int i = threadIdx.x + blockDim.x * m;
            if (i < rows) {
                int j1 = i % leaf, j23 = i / leaf;
                double s = 0.0;
                for (int m1 = 0; m1 < pe; ++m1)
                    s = fma(D.F[o[0] + j1 + nb * m1], Z2[m1 + pe * j23], s);
                acc[m] += s;
            }
        }
        __syncthreads();
    }
    for (int m = 0; m < per && m < 8; ++m)
        if (nat[m] >= 0) f[nat[m] + ldf * r] = acc[m];
}

void launch_out(int d, int n, int leaf, int L, int nrc, int nrhs_here, const int *d_near_row_task,
                const Task *d_tasks, const double *d_part, int near_ld, const double *d_a_add,
                const double *u, long long ldu, const DownLevel *down, int ndown, double *f,
                long long ldf, cudaStream_t s)
{
    DownArgs args;
    args.ndown = ndown;
    size_t smem = 0;
    for (int q = 0; q < ndown && q < HTLR_MAX_LEVELS; ++q) {
        args.lv[q] = down[q];
        int pe = down[q].pe;
        size_t need = (size_t)down[q].pd + (size_t)pe * pe * leaf +
                      (size_t)pe * leaf * (d == 3 ? leaf : 1);
        if (need > smem) smem = need;
    }
    smem *= sizeof(double);
    if (smem == 0) smem = sizeof(double);
    int rows = 1;
    for (int k = 0; k < d; ++k) rows *= leaf;
    int threads = rows < 256 ? ((rows + 31) / 32) * 32 : 256;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(out_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(1 << (d * L), nrhs_here);
    out_kernel<<<grid, threads, smem, s>>>(d, n, leaf, L, nrc, d_near_row_task, d_tasks, d_part,
                                           near_ld, d_a_add, u, ldu, args, f, ldf);
}

}  // namespace htlr
