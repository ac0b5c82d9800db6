// Construct (Algorithm 1) on the GPU: interpolation factors and their QR, the Nystrom
// diagonal, core tensors of admissible blocks and dense inadmissible blocks.
#include "htlr_internal.h"

namespace htlr {

// k(x, y) of the displacement r = x - y (every supported kernel depends on x - y only).
__device__ __forceinline__ double kernel_of(const KernelDesc &k, int d, const double *r)
{
    double r2 = 0.0;
    for (int l = 0; l < d; ++l) r2 = fma(r[l], r[l], r2);
    switch (k.type) {
    case HTLR_K_LOG: return k.scale * 0.5 * log(r2);
    case HTLR_K_INV_R: return k.scale / sqrt(r2);
    case HTLR_K_EXP_R: return k.scale * exp(-sqrt(r2));
    case HTLR_K_GAUSS: return k.scale * exp(-r2 / (2.0 * k.param * k.param));
    case HTLR_K_POLY: {
        int deg = (int)k.param;
        double v = k.scale;
        for (int l = 0; l < d; ++l) {
            double b = r[l] + 2.0 + 0.5 * l, pw = 1.0;
            for (int e = 0; e < deg; ++e) pw *= b;
            v *= pw;
        }
        return v;
    }
    case HTLR_K_CONST: return k.scale;
    }
    return 0.0;
}

// ---------------------------------------------------------------------------------
// Factor of one level (eq. (3.5)) and its economy QR (Algorithm 1).
// U(i, mu) = L_mu(x_i) for the box-relative points x_i = (i + 1/2) h, i < nb, on the
// Chebyshev points of [0, side], evaluated with the barycentric formula of the first
// kind Chebyshev points (weights (-1)^j sin((2j+1) pi / (2p))).  Then Householder QR
// U = F R with F (nb x pe) orthonormal, R (pe x p) upper triangular.
// ---------------------------------------------------------------------------------
__global__ void factor_kernel(int nb, int p, int pe, double side, double h, int orth,
                              double *F, double *R, double *work)
{
    const double pi = 3.141592653589793238462643;
    // U into work (nb x p, column-major)
    for (int idx = threadIdx.x; idx < nb * p; idx += blockDim.x) {
        int i = idx % nb, mu = idx / nb;
        double x = (i + 0.5) * h;
        double num = 0.0, den = 0.0;
        int hit = -1;
        for (int j = 0; j < p; ++j) {
            double xj = 0.5 * side * cos((2 * j + 1) * pi / (2.0 * p)) + 0.5 * side;
            double wj = ((j & 1) ? -1.0 : 1.0) * sin((2 * j + 1) * pi / (2.0 * p));
            double dx = x - xj;
            if (dx == 0.0) hit = j;
            double t = wj / dx;
            den += t;
            if (j == mu) num = t;
        }
        double v = (hit >= 0) ? (hit == mu ? 1.0 : 0.0) : num / den;
        work[i + (size_t)nb * mu] = v;
    }
    __syncthreads();
    if (!orth) {
        for (int idx = threadIdx.x; idx < nb * p; idx += blockDim.x) F[idx] = work[idx];
        for (int idx = threadIdx.x; idx < p * p; idx += blockDim.x)
            R[idx] = (idx % p == idx / p) ? 1.0 : 0.0;
        return;
    }
    if (threadIdx.x != 0) return;
    // Householder QR in place on work; reflector j kept in work[j+1.., j] with v_j = 1
    // implied, its scalar in tauv[j].
    double tauv[kMaxP];
    for (int j = 0; j < pe; ++j) {
        double *a = work + (size_t)nb * j;
        double sig = 0.0;
        for (int i = j + 1; i < nb; ++i) sig += a[i] * a[i];
        double alpha = a[j];
        if (sig == 0.0) {
            tauv[j] = 0.0;  // already upper triangular in this column
            continue;
        }
        double nrm = sqrt(alpha * alpha + sig);
        double beta = alpha <= 0.0 ? nrm : -nrm;  // new diagonal entry
        double v0 = alpha - beta;
        tauv[j] = (beta - alpha) / beta;
        for (int i = j + 1; i < nb; ++i) a[i] /= v0;
        a[j] = beta;
        // apply H_j = I - tau v v^T to the remaining columns
        for (int c = j + 1; c < p; ++c) {
            double *b = work + (size_t)nb * c;
            double s = b[j];
            for (int i = j + 1; i < nb; ++i) s += a[i] * b[i];
            s *= tauv[j];
            b[j] -= s;
            for (int i = j + 1; i < nb; ++i) b[i] -= s * a[i];
        }
    }
    for (int c = 0; c < p; ++c)
        for (int r = 0; r < pe; ++r) R[r + pe * c] = (r <= c) ? work[r + (size_t)nb * c] : 0.0;
    // F = H_0 ... H_{pe-1} [I; 0]
    for (int c = 0; c < pe; ++c)
        for (int i = 0; i < nb; ++i) F[i + (size_t)nb * c] = (i == c) ? 1.0 : 0.0;
    for (int j = pe - 1; j >= 0; --j) {
        if (tauv[j] == 0.0) continue;
        const double *a = work + (size_t)nb * j;
        for (int c = 0; c < pe; ++c) {
            double *f = F + (size_t)nb * c;
            double s = f[j];
            for (int i = j + 1; i < nb; ++i) s += a[i] * f[i];
            s *= tauv[j];
            f[j] -= s;
            for (int i = j + 1; i < nb; ++i) f[i] -= s * a[i];
        }
    }
}

void launch_factor(int nb, int p, int pe, double side, double h, int orth, double *d_F,
                   double *d_R, cudaStream_t s)
{
    // the work array sits behind F's storage region (allocated by the caller as
    // nb * p doubles after F)
    double *work = d_F + (size_t)nb * p;
    factor_kernel<<<1, 128, 0, s>>>(nb, p, pe, side, h, orth, d_F, d_R, work);
}

// ---------------------------------------------------------------------------------
// Nystrom diagonal (eq. (1.4)): int over the cell centred at x of k(x, y) dy, with the
// cell split at x into 2^d boxes of side h/2 and a q^d Gauss-Legendre rule on each.
// ---------------------------------------------------------------------------------
__global__ void diag_kernel(KernelDesc k, int d, double h, int q, const double *gx,
                            const double *gw, double *out)
{
    __shared__ double red[256];
    long long qd = 1;
    for (int l = 0; l < d; ++l) qd *= q;
    long long total = qd << d;
    double acc = 0.0;
    const double half = 0.25 * h;  // half-width of a sub-box of side h/2
    for (long long m = threadIdx.x; m < total; m += blockDim.x) {
        int c = (int)(m / qd);
        long long r = m % qd;
        double disp[3], w = 1.0;
        for (int l = 0; l < d; ++l) {
            int kq = (int)(r % q);
            r /= q;
            double sgn = ((c >> l) & 1) ? 1.0 : -1.0;
            double y = sgn * (half + half * gx[kq]);   // y - x on the sub-box
            disp[l] = -y;                               // x - y
            w *= half * gw[kq];
        }
        acc += w * kernel_of(k, d, disp);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

void launch_diag(const KernelDesc &k, int d, double h, int q, const double *d_gx,
                 const double *d_gw, double *d_out, cudaStream_t s)
{
    diag_kernel<<<1, 256, 0, s>>>(k, d, h, q, d_gx, d_gw, d_out);
}

// ---------------------------------------------------------------------------------
// Core tensors (eq. (3.5) + the core update of Algorithm 1):
//   G = (w K) x_1 R ... x_d R x_{d+1} R ... x_{2d} R,  K(t, s) = k(xi_t, eta_s),
// where xi_t, eta_s are the tensor Chebyshev points of the target and source cells of
// one level (offset o = tau - sigma in boxes).  One CTA per core, grid-stride; each CTA
// owns two scratch tensors of p^{2d} doubles.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) cores_kernel(KernelDesc k, int d, int p, int pe, int ld,
                                                    int apply_r, double side, double wgt,
                                                    const double *R,
                                                    long long ncores, const int *off,
                                                    double *cores, double *scratch,
                                                    long long scratch_per_cta)
{
    const double pi = 3.141592653589793238462643;
    __shared__ double cn[kMaxP];
    __shared__ double Rs[kMaxP * kMaxP];
    if (threadIdx.x < p)
        cn[threadIdx.x] = 0.5 * side * cos((2 * threadIdx.x + 1) * pi / (2.0 * p)) + 0.5 * side;
    for (int i = threadIdx.x; i < pe * p; i += blockDim.x) Rs[i] = R[i];
    __syncthreads();
    long long pdf = 1, pde = 1;
    for (int l = 0; l < d; ++l) {
        pdf *= p;
        pde *= pe;
    }
    double *A = scratch + scratch_per_cta * blockIdx.x;
    double *B = A + pdf * pdf;
    for (long long c = blockIdx.x; c < ncores; c += gridDim.x) {
        int o[3] = {off[3 * c], off[3 * c + 1], off[3 * c + 2]};
        // kernel values at the node pairs, t fastest
        for (long long idx = threadIdx.x; idx < pdf * pdf; idx += blockDim.x) {
            long long t = idx % pdf, s = idx / pdf;
            double disp[3];
            for (int l = 0; l < d; ++l) {
                int tl = (int)(t % p), sl = (int)(s % p);
                t /= p;
                s /= p;
                disp[l] = o[l] * side + (cn[tl] - cn[sl]);
            }
            A[idx] = wgt * kernel_of(k, d, disp);
        }
        __syncthreads();
        double *src = A, *dst = B;
        int dims[6];
        for (int m = 0; m < 2 * d; ++m) dims[m] = p;
        if (apply_r) {
            for (int m = 0; m < 2 * d; ++m) {
                long long inner = 1, outer = 1;
                for (int j = 0; j < m; ++j) inner *= dims[j];
                for (int j = m + 1; j < 2 * d; ++j) outer *= dims[j];
                long long nout = inner * pe * outer;
                int dm = dims[m];
                for (long long idx = threadIdx.x; idx < nout; idx += blockDim.x) {
                    long long in_ = idx % inner, rest = idx / inner;
                    int mu = (int)(rest % pe);
                    long long ou = rest / pe;
                    const double *x = src + in_ + inner * dm * ou;
                    double acc = 0.0;
                    for (int kk = 0; kk < dm; ++kk) acc = fma(Rs[mu + pe * kk], x[inner * kk], acc);
                    dst[idx] = acc;
                }
                dims[m] = pe;
                __syncthreads();
                double *t = src;
                src = dst;
                dst = t;
            }
        }
        // src holds pe^{2d} values, t fastest: write [s][t] with padding rows zeroed
        double *out = cores + (long long)c * ld * pde;
        for (long long idx = threadIdx.x; idx < (long long)ld * pde; idx += blockDim.x) {
            long long t = idx % ld, s = idx / ld;
            out[idx] = (t < pde) ? src[t + pde * s] : 0.0;
        }
        __syncthreads();
    }
}

void launch_cores(const KernelDesc &k, int d, int p, int pe, int ld, int apply_r, double side,
                  double wgt, const double *d_R, int64_t ncores, const int *d_off, double *d_cores,
                  double *d_scratch, int nscratch_ctas, cudaStream_t s)
{
    if (ncores <= 0) return;
    long long pdf = 1;
    for (int l = 0; l < d; ++l) pdf *= p;
    int grid = (int)(ncores < nscratch_ctas ? ncores : nscratch_ctas);
    cores_kernel<<<grid, 256, 0, s>>>(k, d, p, pe, ld, apply_r, side, wgt, d_R, ncores, d_off,
                                      d_cores, d_scratch, 2 * pdf * pdf);
}

// ---------------------------------------------------------------------------------
// Precision conversions of finished blocks.
// df64: x = hi + lo with hi = fl32(x), lo = fl32(x - hi); the pair overwrites x in place.
// ---------------------------------------------------------------------------------
__global__ void split_df64_kernel(double *buf, size_t count)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x) {
        double x = buf[i];
        float h = __double2float_rn(x);
        float l = __double2float_rn(x - (double)h);
        reinterpret_cast<float2 *>(buf)[i] = make_float2(h, l);
    }
}

__global__ void to_fp32_kernel(const double *src, float *dst, size_t count)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < count;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = __double2float_rn(src[i]);
}

void launch_split_df64(double *d_buf, size_t count, cudaStream_t s)
{
    if (count) split_df64_kernel<<<152 * 8, 256, 0, s>>>(d_buf, count);
}

void launch_to_fp32(const double *d_src, float *d_dst, size_t count, cudaStream_t s)
{
    if (count) to_fp32_kernel<<<152 * 8, 256, 0, s>>>(d_src, d_dst, count);
}

// ---------------------------------------------------------------------------------
// Dense inadmissible leaves (eq. (4.1)): A_ij = a(x_i) delta_ij + K_ij h^d, with the
// diagonal K_ii h^d from the quadrature above.  Leaf-local lexicographic indices,
// column-major [j][i] with leading dimension ld.
// ---------------------------------------------------------------------------------
__global__ void near_kernel(KernelDesc k, int d, int n, int leaf, int ld, double h, double wgt,
                            double diag, const double *a, long long nblk, const int *off,
                            const int *tau, double *blocks)
{
    int rows = 1;
    for (int l = 0; l < d; ++l) rows *= leaf;
    long long per = (long long)ld * rows;
    long long total = per * nblk;
    int nl1 = n / leaf;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long b = idx / per;
        int rem = (int)(idx % per);
        int i = rem % ld, j = rem / ld;
        double v = 0.0;
        if (i < rows) {
            int ii = i, jj = j;
            double disp[3];
            bool same = true;
            for (int l = 0; l < d; ++l) {
                int il = ii % leaf, jl = jj % leaf;
                ii /= leaf;
                jj /= leaf;
                int ol = off[3 * b + l];
                int dl = ol * leaf + il - jl;
                if (dl != 0) same = false;
                disp[l] = dl * h;
            }
            if (same) {
                v = diag;
                if (a) {
                    int t = tau[b];
                    long long nat = 0, str = 1;
                    int i2 = i;
                    for (int l = 0; l < d; ++l) {
                        int tl = t % nl1;
                        t /= nl1;
                        nat += (long long)(tl * leaf + i2 % leaf) * str;
                        i2 /= leaf;
                        str *= n;
                    }
                    v += a[nat];
                }
            } else {
                v = wgt * kernel_of(k, d, disp);
            }
        }
        blocks[idx] = v;
    }
}

void launch_near(const KernelDesc &k, int d, int n, int leaf, int ld, double h, double wgt,
                 double diag, const double *d_a, int64_t nblk, const int *d_off, const int *d_tau,
                 double *d_blocks, cudaStream_t s)
{
    if (nblk <= 0) return;
    near_kernel<<<152 * 8, 256, 0, s>>>(k, d, n, leaf, ld, h, wgt, diag, d_a, nblk, d_off, d_tau,
                                        d_blocks);
}

// ---------------------------------------------------------------------------------
// Remove the diagonal entries of the listed dense blocks (they are added separately, in
// FP64, when the blocks are used in a lower precision).
// ---------------------------------------------------------------------------------
__global__ void zero_diag_kernel(double *blocks, int ld, int rows, const int *ids, int nids)
{
    const long long total = (long long)nids * rows;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int b = ids[idx / rows], i = (int)(idx % rows);
        blocks[(long long)b * ld * rows + (long long)i * ld + i] = 0.0;
    }
}

void launch_zero_diag(double *blocks, int ld, int rows, const int *d_ids, int nids, cudaStream_t s)
{
    if (nids > 0) zero_diag_kernel<<<152 * 4, 256, 0, s>>>(blocks, ld, rows, d_ids, nids);
}

// ---------------------------------------------------------------------------------
// Tensor grids (§3.3 weights, Def. 3.3 tensor boxes): factors of every 1-D box of a
// level.  U(i, mu) = L_mu(x_i) and V(i, mu) = L_mu(x_i) w_i on the Chebyshev points of
// the box's geometric cell [k 2^-l, (k+1) 2^-l], barycentric form; w_i is the 1-D cell
// width, so that the core needs no quadrature weight.  Grid (dimension, 1-D box).
// ---------------------------------------------------------------------------------
__global__ void factor_tensor_kernel(int n, int level, int p, const double *coords,
                                     const double *width, const int *geo, double *Upool,
                                     double *Vpool)
{
    const double pi = 3.141592653589793238462643;
    const int l = blockIdx.y, k = blockIdx.x, nb1 = 1 << level;
    const int *g = geo + (size_t)l * 4 * nb1;  // first, cnt, uoff, voff
    const int first = g[k], cnt = g[nb1 + k], uo = g[2 * nb1 + k], vo = g[3 * nb1 + k];
    const double side = ldexp(1.0, -level), lo = k * side;
    for (int idx = threadIdx.x; idx < cnt * p; idx += blockDim.x) {
        const int i = idx % cnt, mu = idx / cnt;
        const double x = coords[(size_t)l * n + first + i];
        double num = 0.0, den = 0.0;
        int hit = -1;
        for (int j = 0; j < p; ++j) {
            double xj = lo + 0.5 * side * cos((2 * j + 1) * pi / (2.0 * p)) + 0.5 * side;
            double wj = ((j & 1) ? -1.0 : 1.0) * sin((2 * j + 1) * pi / (2.0 * p));
            double dx = x - xj;
            if (dx == 0.0) hit = j;
            double t = wj / dx;
            den += t;
            if (j == mu) num = t;
        }
        const double v = (hit >= 0) ? (hit == mu ? 1.0 : 0.0) : num / den;
        Upool[uo + idx] = v;
        Vpool[vo + idx] = v * width[(size_t)l * n + first + i];
    }
}

void launch_factor_tensor(int d, int n, int level, int p, const double *coords,
                          const double *width, const int *geo, double *Upool, double *Vpool,
                          cudaStream_t s)
{
    dim3 grid(1 << level, d);
    factor_tensor_kernel<<<grid, 128, 0, s>>>(n, level, p, coords, width, geo, Upool, Vpool);
}

// ---------------------------------------------------------------------------------
// Tensor grids: K_ii w_i = int over the cell of point i of k(x_i, y) dy (eq. (1.4) with
// the cell measure of §3.3), the cell split at x_i into 2^d boxes (of unequal sides when
// x_i is off-centre), a q^d Gauss-Legendre rule on each.  One warp per point; lanes
// split the nodes and a fixed shuffle tree reduces them.
// ---------------------------------------------------------------------------------
__global__ void diag_points_kernel(KernelDesc k, int d, int n, const double *coords,
                                   const double *edges, int q, const double *gx,
                                   const double *gw, double *diag)
{
    const long long N = (long long)n * n * (d == 3 ? n : 1);
    const int lane = threadIdx.x & 31;
    long long qd = 1;
    for (int l = 0; l < d; ++l) qd *= q;
    const long long total = qd << d;
    for (long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; i < N;
         i += ((long long)gridDim.x * blockDim.x) >> 5) {
        double x[3], a[3], b[3];
        long long r = i;
        for (int l = 0; l < d; ++l) {
            int il = (int)(r % n);
            r /= n;
            x[l] = coords[(size_t)l * n + il];
            a[l] = edges[(size_t)l * (n + 1) + il];
            b[l] = edges[(size_t)l * (n + 1) + il + 1];
        }
        double acc = 0.0;
        for (long long m = lane; m < total; m += 32) {
            int c = (int)(m / qd);
            long long rq = m % qd;
            double disp[3], w = 1.0;
            for (int l = 0; l < d; ++l) {
                int kq = (int)(rq % q);
                rq /= q;
                double lo = ((c >> l) & 1) ? x[l] : a[l];
                double hi = ((c >> l) & 1) ? b[l] : x[l];
                double half = 0.5 * (hi - lo);
                double y = 0.5 * (lo + hi) + half * gx[kq];
                disp[l] = x[l] - y;
                w *= half * gw[kq];
            }
            acc += w * kernel_of(k, d, disp);
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) diag[i] = acc;
    }
}

void launch_diag_points(const KernelDesc &k, int d, int n, const double *coords,
                        const double *edges, int q, const double *gx, const double *gw,
                        double *diag, cudaStream_t s)
{
    diag_points_kernel<<<152 * 16, 256, 0, s>>>(k, d, n, coords, edges, q, gx, gw, diag);
}

}  // namespace htlr
