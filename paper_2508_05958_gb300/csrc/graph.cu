// Matvec plans: the launch sequence of one HMultVec (Algorithm 2) for fixed device
// operands, captured once into a CUDA graph and replayed with a single graph launch.
// A matvec is 10-40 kernel launches (per level: upward contraction, stream, reduction;
// the output kernel); for small operators their launch latency is most of the time.
#include <new>

#include "htlr_internal.h"

namespace htlr {
int matvec_enqueue_on(const htlr_handle *H, const double *u, double *f, int nrhs,
                      cudaStream_t s);
bool handle_is_live(const htlr_handle *H);
}  // namespace htlr

struct htlr_plan {
    const htlr_handle *H = nullptr;
    const double *u = nullptr;
    double *f = nullptr;
    int nrhs = 0;
    int generation = -1;
    int launches = 0;
    cudaGraphExec_t exec = nullptr;
};

using namespace htlr;

namespace {

int fail(int code, const char *msg)
{
    set_error(msg);
    return code;
}

void drop(htlr_plan *P)
{
    if (P->exec) cudaGraphExecDestroy(P->exec);
    P->exec = nullptr;
}

// Capture the matvec on a private stream (the legacy default stream cannot be captured).
int capture(htlr_plan *P)
{
    drop(P);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "htlr_plan: stream");
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = HTLR_OK;
    if (e == cudaSuccess) {
        rc = matvec_enqueue_on(P->H, P->u, P->f, P->nrhs, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (rc == HTLR_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "htlr_plan: capture");
    } else {
        rc = cuda_fail(e, "htlr_plan: begin capture");
    }
    if (rc == HTLR_OK) {
        e = cudaGraphInstantiate(&P->exec, g, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "htlr_plan: instantiate");
    }
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (rc == HTLR_OK) {
        P->generation = P->H->generation;
        P->launches = P->H->last_launches;
    }
    return rc;
}

}  // namespace

extern "C" {

int htlr_plan_create(const htlr_handle *H, const double *u, double *f, int nrhs, htlr_plan **out)
{
    if (!out) return fail(HTLR_EINVAL, "htlr_plan_create: out must not be NULL");
    *out = nullptr;
    if (!handle_is_live(H)) return fail(HTLR_EINVAL, "htlr_plan_create: not a live HTLR handle");
    if (!u || !f || nrhs < 1) return fail(HTLR_EINVAL, "htlr_plan_create: bad u, f or nrhs");
    long long N = 1;
    for (int k = 0; k < H->d; ++k) N *= H->n;
    const char *ub = (const char *)u, *ue = (const char *)(u + N * nrhs);
    const char *fb = (const char *)f, *fe = (const char *)(f + N * nrhs);
    if (ub < fe && fb < ue) return fail(HTLR_EINVAL, "htlr_plan_create: u and f overlap");
    htlr_plan *P = new (std::nothrow) htlr_plan();
    if (!P) return fail(HTLR_ENOMEM, "htlr_plan_create: host allocation failed");
    P->H = H;
    P->u = u;
    P->f = f;
    P->nrhs = nrhs;
    int rc = capture(P);
    if (rc) {
        delete P;
        return rc;
    }
    *out = P;
    return HTLR_OK;
}

int htlr_plan_launch(htlr_plan *P)
{
    if (!P || !handle_is_live(P->H)) return fail(HTLR_EINVAL, "htlr_plan_launch: bad plan");
    if (P->generation != P->H->generation) {
        int rc = capture(P);
        if (rc) return rc;
    }
    cudaError_t e = cudaGraphLaunch(P->exec, P->H->stream);
    if (e != cudaSuccess) return cuda_fail(e, "htlr_plan_launch");
    const_cast<htlr_handle *>(P->H)->last_launches = P->launches;
    return HTLR_OK;
}

int htlr_plan_launches(const htlr_plan *P) { return P ? P->launches : -1; }

void htlr_plan_free(htlr_plan *P)
{
    if (!P) return;
    drop(P);
    delete P;
}

}  // extern "C"
