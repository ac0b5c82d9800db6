// Restarted GMRES for the second-kind system a(x) u + K u = f (eq. (1.1) inverted, the
// "backward evaluation" of §1), with HMultVec as the operator.
//
// nrhs systems are solved together: every Arnoldi step is one multi-RHS matvec.  The
// Arnoldi process runs in FP64 with classical Gram-Schmidt applied twice (CGS2); its
// inner products use fixed-order block reductions, so results are bitwise repeatable.
// The small Hessenberg least-squares problems are solved on the host with Givens
// rotations.  With a second (e.g. mixed-precision) operator, the solve is wrapped in
// iterative refinement: r = f - A u with the accurate operator, A_inner e = r solved to
// a looser tolerance, u += e, until ||f - A u|| <= tol ||f||.
#include <cmath>
#include <cstdio>
#include <vector>

#include "htlr_internal.h"

namespace htlr {

int matvec_enqueue(const htlr_handle *H, const double *u, double *f, int nrhs);

namespace {

constexpr int kDotBlocks = 152 * 2;  // row chunks of the two-pass reductions

// part[(blk * nrhs + r) * k + j] = sum over the rows of chunk blk of V_j[r] . w[r]
// (V_j of RHS r at V + (j * nrhs + r) * N).  grid (kDotBlocks, nrhs), 256 threads.
__global__ void dots_partial(long long N, int nrhs, int k, const double *__restrict__ V,
                             const double *__restrict__ w, double *__restrict__ part)
{
    __shared__ double red[256];
    const int r = blockIdx.y, blk = blockIdx.x, nb = gridDim.x;
    const long long chunk = (N + nb - 1) / nb;
    const long long i0 = blk * chunk, i1 = i0 + chunk < N ? i0 + chunk : N;
    const double *wr = w + (long long)r * N;
    for (int j = 0; j < k; ++j) {
        const double *vj = V + ((long long)j * nrhs + r) * N;
        double s = 0.0;
        for (long long i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(vj[i], wr[i], s);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = blockDim.x / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[((long long)blk * nrhs + r) * k + j] = red[0];
        __syncthreads();
    }
}

// out[r * k + j] = sum over blk (in order) of part[(blk * nrhs + r) * k + j]
__global__ void dots_final(int nb, int nrhs, int k, const double *__restrict__ part,
                           double *__restrict__ out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nrhs * k) return;
    const int r = idx / k, j = idx % k;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[((long long)b * nrhs + r) * k + j];
    out[idx] = s;
}

// w[r] -= sum_j V_j[r] c[r * k + j]   (c on the device)
__global__ void sub_combination(long long N, int nrhs, int k, const double *__restrict__ V,
                                const double *__restrict__ c, double *__restrict__ w)
{
    const long long total = N * nrhs;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / N);
        const long long i = idx % N;
        double s = w[idx];
        for (int j = 0; j < k; ++j) s -= V[((long long)j * nrhs + r) * N + i] * c[r * k + j];
        w[idx] = s;
    }
}

// out[r] = x[r] * scale[r]  (scale on the device; a zero scale gives zero)
__global__ void scale_vec(long long N, int nrhs, const double *__restrict__ x,
                          const double *__restrict__ scale, double *__restrict__ out)
{
    const long long total = N * nrhs;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x)
        out[idx] = x[idx] * scale[idx / N];
}

// out = a - b
__global__ void sub_vec(long long total, const double *__restrict__ a, const double *__restrict__ b,
                        double *__restrict__ out)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x)
        out[idx] = a[idx] - b[idx];
}

// u[r] += sum_j V_j[r] y[r * k + j]
__global__ void add_combination(long long N, int nrhs, int k, const double *__restrict__ V,
                                const double *__restrict__ y, double *__restrict__ u)
{
    const long long total = N * nrhs;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(idx / N);
        const long long i = idx % N;
        double s = u[idx];
        for (int j = 0; j < k; ++j) s = fma(V[((long long)j * nrhs + r) * N + i], y[r * k + j], s);
        u[idx] = s;
    }
}

struct Work {
    long long N = 0;
    int nrhs = 0, m = 0;
    double *V = nullptr;     // (m + 1) x nrhs x N
    double *w = nullptr;     // nrhs x N
    double *r = nullptr;     // nrhs x N
    double *e = nullptr;     // nrhs x N (refinement correction)
    double *part = nullptr;  // kDotBlocks x nrhs x (m + 1)
    double *c = nullptr;     // nrhs x (m + 1)
    double *c2 = nullptr;    // nrhs x (m + 1): second Gram-Schmidt pass
    double *nn = nullptr;    // nrhs: squared norms
    ~Work()
    {
        for (double *p : {V, w, r, e, part, c, c2, nn})
            if (p) cudaFree(p);
    }
};

const int kThreads = 256, kGrid = 152 * 8;

// out[r * k + j] = V_j[r] . w[r] for j < k (device), then copied to host hv.
int dots(const Work &W, cudaStream_t s, const double *V, const double *w, int k, double *d_out,
         std::vector<double> *hv)
{
    dim3 g(kDotBlocks, W.nrhs);
    dots_partial<<<g, kThreads, 0, s>>>(W.N, W.nrhs, k, V, w, W.part);
    dots_final<<<(W.nrhs * k + 255) / 256, 256, 0, s>>>(kDotBlocks, W.nrhs, k, W.part, d_out);
    if (hv) {
        hv->resize((size_t)W.nrhs * k);
        cudaError_t e = cudaMemcpyAsync(hv->data(), d_out, sizeof(double) * hv->size(),
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "gmres dots copy");
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "gmres dots");
    }
    return HTLR_OK;
}

// GMRES(m) on A x = b (all on the device, x is the initial guess and the result), to
// ||b - A x|| <= tol ||b|| per RHS (estimated by the Arnoldi recurrence, checked with the
// true residual at every restart).  Returns the relative residuals in rel_out.
int gmres_solve(const htlr_handle *A, Work &W, const double *b, double *x, double tol,
                int max_iters, int *iters_out, int *matvecs_out, std::vector<double> &rel_out)
{
    cudaStream_t s = A->stream;
    const long long N = W.N;
    const int nrhs = W.nrhs, m = W.m;
    std::vector<double> bnorm, beta, tmp;
    int rc = dots(W, s, b, b, 1, W.c, &bnorm);  // ||b||^2 (V_0 slot reused as b)
    if (rc) return rc;
    for (double &v : bnorm) v = std::sqrt(v);
    int iters = 0, matvecs = 0;
    std::vector<double> Hh((size_t)nrhs * (m + 1) * m), cs((size_t)nrhs * m), sn((size_t)nrhs * m),
        g((size_t)nrhs * (m + 1)), y((size_t)nrhs * m);
    std::vector<double> scale(nrhs), hcol;
    rel_out.assign(nrhs, 0.0);
    while (true) {
        // r = b - A x
        if ((rc = matvec_enqueue(A, x, W.w, nrhs))) return rc;
        ++matvecs;
        sub_vec<<<kGrid, kThreads, 0, s>>>(N * nrhs, b, W.w, W.r);
        if ((rc = dots(W, s, W.r, W.r, 1, W.c, &beta))) return rc;
        bool all_done = true;
        for (int r = 0; r < nrhs; ++r) {
            beta[r] = std::sqrt(beta[r]);
            rel_out[r] = bnorm[r] > 0 ? beta[r] / bnorm[r] : 0.0;
            if (rel_out[r] > tol) all_done = false;
        }
        if (all_done || iters >= max_iters) break;
        // V_0 = r / beta
        for (int r = 0; r < nrhs; ++r) scale[r] = beta[r] > 0 ? 1.0 / beta[r] : 0.0;
        cudaMemcpyAsync(W.c, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s);
        scale_vec<<<kGrid, kThreads, 0, s>>>(N, nrhs, W.r, W.c, W.V);
        std::fill(g.begin(), g.end(), 0.0);
        for (int r = 0; r < nrhs; ++r) g[(size_t)r * (m + 1)] = beta[r];
        std::vector<int> kdim(nrhs, 0), frozen(nrhs, 0);
        for (int r = 0; r < nrhs; ++r) frozen[r] = rel_out[r] <= tol;
        int k = 0;
        for (; k < m && iters < max_iters; ++k, ++iters) {
            double *Vk = W.V + (long long)k * nrhs * N;
            if ((rc = matvec_enqueue(A, Vk, W.w, nrhs))) return rc;
            ++matvecs;
            // CGS2: h = V^T w, w -= V h, twice; then ||w||^2.  The coefficients stay on the
            // device between the passes; the host reads them once per step
            if ((rc = dots(W, s, W.V, W.w, k + 1, W.c, nullptr))) return rc;
            sub_combination<<<kGrid, kThreads, 0, s>>>(N, nrhs, k + 1, W.V, W.c, W.w);
            if ((rc = dots(W, s, W.V, W.w, k + 1, W.c2, nullptr))) return rc;
            sub_combination<<<kGrid, kThreads, 0, s>>>(N, nrhs, k + 1, W.V, W.c2, W.w);
            if ((rc = dots(W, s, W.w, W.w, 1, W.nn, nullptr))) return rc;
            std::vector<double> h1((size_t)nrhs * (k + 1)), h2(h1.size()), nn((size_t)nrhs);
            cudaMemcpyAsync(h1.data(), W.c, sizeof(double) * h1.size(), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(h2.data(), W.c2, sizeof(double) * h2.size(), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(nn.data(), W.nn, sizeof(double) * nn.size(), cudaMemcpyDeviceToHost, s);
            {
                cudaError_t e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) return cuda_fail(e, "gmres step");
            }
            bool all_conv = true;
            for (int r = 0; r < nrhs; ++r) {
                double *hc = &Hh[((size_t)r * m + k) * (m + 1)];
                for (int j = 0; j <= k; ++j) hc[j] = h1[(size_t)r * (k + 1) + j] + h2[(size_t)r * (k + 1) + j];
                hc[k + 1] = std::sqrt(nn[r]);
                scale[r] = (hc[k + 1] > 0 && !frozen[r]) ? 1.0 / hc[k + 1] : 0.0;
                if (frozen[r]) continue;
                // previous rotations, then a new one zeroing hc[k+1]
                for (int j = 0; j < k; ++j) {
                    double c0 = cs[(size_t)r * m + j], s0 = sn[(size_t)r * m + j];
                    double t = c0 * hc[j] + s0 * hc[j + 1];
                    hc[j + 1] = -s0 * hc[j] + c0 * hc[j + 1];
                    hc[j] = t;
                }
                double a0 = hc[k], b0 = hc[k + 1], rr = std::hypot(a0, b0);
                double c0 = rr > 0 ? a0 / rr : 1.0, s0 = rr > 0 ? b0 / rr : 0.0;
                cs[(size_t)r * m + k] = c0;
                sn[(size_t)r * m + k] = s0;
                hc[k] = rr;
                hc[k + 1] = 0.0;
                double *gr = &g[(size_t)r * (m + 1)];
                gr[k + 1] = -s0 * gr[k];
                gr[k] = c0 * gr[k];
                kdim[r] = k + 1;
                const double est = bnorm[r] > 0 ? std::fabs(gr[k + 1]) / bnorm[r] : 0.0;
                if (est <= tol || rr == 0.0) frozen[r] = 1;
                if (!frozen[r]) all_conv = false;
            }
            // V_{k+1} = w / h_{k+1,k}
            cudaMemcpyAsync(W.c, scale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, s);
            scale_vec<<<kGrid, kThreads, 0, s>>>(N, nrhs, W.w, W.c, W.V + (long long)(k + 1) * nrhs * N);
            if (all_conv) {
                ++k;
                ++iters;
                break;
            }
        }
        // y = R^{-1} g per RHS, x += V y
        const int kk = k;
        std::fill(y.begin(), y.end(), 0.0);
        std::vector<double> yk((size_t)nrhs * (kk > 0 ? kk : 1), 0.0);
        for (int r = 0; r < nrhs; ++r) {
            const int kr = kdim[r];
            for (int i = kr - 1; i >= 0; --i) {
                double v = g[(size_t)r * (m + 1) + i];
                for (int j = i + 1; j < kr; ++j) v -= Hh[((size_t)r * m + j) * (m + 1) + i] * yk[(size_t)r * kk + j];
                const double d = Hh[((size_t)r * m + i) * (m + 1) + i];
                yk[(size_t)r * kk + i] = d != 0.0 ? v / d : 0.0;
            }
        }
        if (kk > 0) {
            cudaMemcpyAsync(W.c, yk.data(), sizeof(double) * yk.size(), cudaMemcpyHostToDevice, s);
            add_combination<<<kGrid, kThreads, 0, s>>>(N, nrhs, kk, W.V, W.c, x);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "gmres kernels");
    }
    *iters_out += iters;
    *matvecs_out += matvecs;
    return HTLR_OK;
}

}  // namespace

bool handle_is_live(const htlr_handle *H);

}  // namespace htlr

using namespace htlr;

extern "C" int htlr_gmres(const htlr_handle *H, const htlr_handle *H_inner, const double *f,
                          double *u, int nrhs, const htlr_gmres_options *o,
                          htlr_gmres_result *res)
{
    if (!handle_is_live(H) || (H_inner && !handle_is_live(H_inner))) {
        set_error("htlr_gmres: not a live HTLR handle");
        return HTLR_EINVAL;
    }
    if (!f || !u || nrhs < 1) {
        set_error("htlr_gmres: f and u must be device pointers and nrhs >= 1");
        return HTLR_EINVAL;
    }
    if (H_inner && (H_inner->d != H->d || H_inner->n != H->n)) {
        set_error("htlr_gmres: the inner operator must have the same grid size");
        return HTLR_EINVAL;
    }
    htlr_gmres_options def = {30, 3000, 1e-10, 1e-6, 20};
    const htlr_gmres_options &O = o ? *o : def;
    if (O.restart < 1 || O.restart > 200 || O.max_iters < 1 || !(O.tol > 0) ||
        (H_inner && !(O.inner_tol > 0))) {
        set_error("htlr_gmres: invalid options");
        return HTLR_EINVAL;
    }
    Work W;
    long long N = 1;
    for (int k = 0; k < H->d; ++k) N *= H->n;
    W.N = N;
    W.nrhs = nrhs;
    W.m = O.restart;
    const size_t vec = (size_t)N * nrhs;
    cudaError_t e;
    if ((e = device_malloc((void **)&W.V, sizeof(double) * vec * (W.m + 1))) != cudaSuccess ||
        (e = device_malloc((void **)&W.w, sizeof(double) * vec)) != cudaSuccess ||
        (e = device_malloc((void **)&W.r, sizeof(double) * vec)) != cudaSuccess ||
        (e = device_malloc((void **)&W.part, sizeof(double) * kDotBlocks * nrhs * (W.m + 1))) != cudaSuccess ||
        (e = device_malloc((void **)&W.c, sizeof(double) * nrhs * (W.m + 1))) != cudaSuccess ||
        (e = device_malloc((void **)&W.c2, sizeof(double) * nrhs * (W.m + 1))) != cudaSuccess ||
        (e = device_malloc((void **)&W.nn, sizeof(double) * nrhs)) != cudaSuccess)
        return cuda_fail(e, "htlr_gmres workspace");
    int iters = 0, matvecs = 0, refinements = 0, rc;
    std::vector<double> rel;
    if (!H_inner) {
        rc = gmres_solve(H, W, f, u, O.tol, O.max_iters, &iters, &matvecs, rel);
        if (rc) return rc;
    } else {
        // iterative refinement: residual with H (accurate), corrections with H_inner
        if ((e = device_malloc((void **)&W.e, sizeof(double) * vec)) != cudaSuccess)
            return cuda_fail(e, "htlr_gmres workspace");
        double *rr = nullptr;
        if ((e = device_malloc((void **)&rr, sizeof(double) * vec)) != cudaSuccess)
            return cuda_fail(e, "htlr_gmres workspace");
        std::vector<double> fn, rn;
        rc = dots(W, H->stream, f, f, 1, W.c, &fn);
        for (int it = 0; rc == HTLR_OK; ++it) {
            if ((rc = matvec_enqueue(H, u, W.w, nrhs))) break;
            ++matvecs;
            sub_vec<<<kGrid, kThreads, 0, H->stream>>>((long long)vec, f, W.w, rr);
            if ((rc = dots(W, H->stream, rr, rr, 1, W.c, &rn))) break;
            rel.assign(nrhs, 0.0);
            bool done = true;
            for (int r = 0; r < nrhs; ++r) {
                rel[r] = fn[r] > 0 ? std::sqrt(rn[r] / fn[r]) : 0.0;
                if (rel[r] > O.tol) done = false;
            }
            if (done || it >= O.max_refine || iters >= O.max_iters) break;
            cudaMemsetAsync(W.e, 0, sizeof(double) * vec, H->stream);
            if ((e = cudaStreamSynchronize(H->stream)) != cudaSuccess) {
                rc = cuda_fail(e, "htlr_gmres");
                break;
            }
            std::vector<double> rel_in;
            if ((rc = gmres_solve(H_inner, W, rr, W.e, O.inner_tol, O.max_iters - iters, &iters,
                                  &matvecs, rel_in)))
                break;
            if ((e = cudaStreamSynchronize(H_inner->stream)) != cudaSuccess) {
                rc = cuda_fail(e, "htlr_gmres");
                break;
            }
            // u += e
            std::vector<double> one((size_t)nrhs, 1.0);
            cudaMemcpyAsync(W.c, one.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice,
                            H->stream);
            add_combination<<<kGrid, kThreads, 0, H->stream>>>(N, nrhs, 1, W.e, W.c, u);
            ++refinements;
        }
        cudaFree(rr);
        if (rc) return rc;
    }
    e = cudaStreamSynchronize(H->stream);
    if (e != cudaSuccess) return cuda_fail(e, "htlr_gmres");
    if (H_inner && (e = cudaStreamSynchronize(H_inner->stream)) != cudaSuccess)
        return cuda_fail(e, "htlr_gmres");
    // a device check that failed in any matvec of the solve (a bounded wait that ran out)
    // invalidates the result
    if ((rc = check_device_error(H, "htlr_gmres"))) return rc;
    if (H_inner && (rc = check_device_error(H_inner, "htlr_gmres (inner operator)"))) return rc;
    if (res) {
        res->iterations = iters;
        res->matvecs = matvecs;
        res->refinements = refinements;
        double mx = 0.0;
        for (double v : rel) mx = v > mx ? v : mx;
        res->rel_residual = mx;
        res->converged = mx <= O.tol;
    }
    return HTLR_OK;
}
