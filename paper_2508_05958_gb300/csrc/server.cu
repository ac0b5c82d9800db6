// Serving loop for second-kind solves a(x) u + K u = f (the inversion of eq. (1.1)) on
// resident HTLR operators, with continuous batching.  The paper has no serving layer;
// this is the request loop a solver service needs around Algorithms 1-2.
//
// One host thread owns the device work.  Requests wait in a FIFO until a slot and
// device memory are free; operators are constructed on first use (Algorithm 1) and stay
// resident until memory is needed, then the least recently used idle one is released.
// Every active request is a restarted GMRES(m) state machine (FP64 Arnoldi, classical
// Gram-Schmidt twice, Givens rotations on the host).  Each scheduler step advances every
// active request by one operator application: the requests of one operator that need the
// same handle are gathered into the columns of one multi-RHS HMultVec, so a request that
// arrives while others iterate joins the next step's batch and leaves as soon as it
// converges.  Different operators run on their own streams, so their steps overlap on
// the device.  In mixed mode each operator has two handles: an accurate one (df64) that
// defines the residual and a fast inner one (FP32 or tensor-core BF16X6) that builds the
// Krylov spaces; every restart is then one step of iterative refinement.
//
// All per-request vector work is done by batched kernels whose reductions use a fixed
// partition of the N rows, and the block stream computes each right-hand side
// independently of the others, so a request's result does not depend on which requests
// shared its batches.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "htlr_internal.h"

namespace htlr {
int matvec_enqueue(const htlr_handle *H, const double *u, double *f, int nrhs);
}  // namespace htlr

using namespace htlr;

namespace {

constexpr int kBlk = 152;      // row chunks of the batched reductions
constexpr int kThreads = 256;

int fail(int code, const char *msg)
{
    set_error(msg);
    return code;
}

// ---------------------------------------------------------------------------------
// batched vector kernels (one CTA row per request)
// ---------------------------------------------------------------------------------
struct DotDesc {           // out[out_off + j] = X_j . Y for j < cnt, X_j = X + j N
    const double *X;
    double *Y;
    int cnt;
    long long out_off;
};

__global__ void dots_partial_k(const DotDesc *__restrict__ D, long long N, int maxcnt,
                               double *__restrict__ part)
{
    __shared__ double red[kThreads];
    const DotDesc dd = D[blockIdx.y];
    const long long chunk = (N + kBlk - 1) / kBlk;
    const long long i0 = blockIdx.x * chunk, i1 = i0 + chunk < N ? i0 + chunk : N;
    for (int j = 0; j < dd.cnt; ++j) {
        const double *x = dd.X + (long long)j * N;
        double s = 0.0;
        for (long long i = i0 + threadIdx.x; i < i1; i += kThreads) s = fma(x[i], dd.Y[i], s);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int h = kThreads / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[((long long)blockIdx.y * kBlk + blockIdx.x) * maxcnt + j] = red[0];
        __syncthreads();
    }
}

__global__ void dots_final_k(const DotDesc *__restrict__ D, int n, int maxcnt,
                             const double *__restrict__ part, double *__restrict__ out)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * maxcnt) return;
    const int e = idx / maxcnt, j = idx % maxcnt;
    if (j >= D[e].cnt) return;
    double s = 0.0;
    for (int b = 0; b < kBlk; ++b) s += part[((long long)e * kBlk + b) * maxcnt + j];
    out[D[e].out_off + j] = s;
}

// Y -= sum_j X_j out[out_off + j]
__global__ void subcomb_k(const DotDesc *__restrict__ D, long long N, const double *__restrict__ out)
{
    const DotDesc dd = D[blockIdx.y];
    const double *c = out + dd.out_off;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        double s = dd.Y[i];
        for (int j = 0; j < dd.cnt; ++j) s -= dd.X[(long long)j * N + i] * c[j];
        dd.Y[i] = s;
    }
}

struct VecDesc {            // residual: dst = a - b (b may be null: 0)
    const double *a;        // scale:    dst = a * s
    const double *b;        // update:   dst += sum_j a_j c[j] (cnt terms, a_j = a + j N)
    double *dst;
    const double *c;
    double s;
    int cnt;
};

__global__ void resid_k(const VecDesc *__restrict__ D, long long N)
{
    const VecDesc v = D[blockIdx.y];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        v.dst[i] = v.a[i] - (v.b ? v.b[i] : 0.0);
}

__global__ void scale_k(const VecDesc *__restrict__ D, long long N)
{
    const VecDesc v = D[blockIdx.y];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        v.dst[i] = v.a[i] * v.s;
}

__global__ void update_k(const VecDesc *__restrict__ D, long long N)
{
    const VecDesc v = D[blockIdx.y];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x) {
        double s = v.dst[i];
        for (int j = 0; j < v.cnt; ++j) s = fma(v.a[(long long)j * N + i], v.c[j], s);
        v.dst[i] = s;
    }
}

// columns of the batch input: Ub[e N + i] = src_e[i]
__global__ void gather_k(const VecDesc *__restrict__ D, long long N, double *__restrict__ Ub)
{
    const VecDesc v = D[blockIdx.y];
    double *dst = Ub + (long long)blockIdx.y * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        dst[i] = v.a[i];
}

int grid_x(long long N) { return (int)std::min<long long>(152 * 4, (N + kThreads - 1) / kThreads); }

// ---------------------------------------------------------------------------------
// host state
// ---------------------------------------------------------------------------------
enum Phase { kResidual = 0, kArnoldi = 1 };

struct Request {
    long long id = 0;
    int op = 0;
    std::vector<double> f;
    double *u_host = nullptr;
    htlr_request_info info{};
    // device workspace: V ((m+1) N) | x | b | r
    double *ws = nullptr;
    size_t ws_bytes = 0;
    double *V = nullptr, *x = nullptr, *b = nullptr, *r = nullptr;
    int phase = kResidual;
    bool x_zero = true;
    int k = 0;
    double fn = 0.0, target = 0.0;
    std::vector<double> Hh, cs, sn, g;
    bool done = false;
    int slot = 0;  // batch position in the current step
};

struct Group {               // one handle of a resident operator and its batch buffers
    htlr_handle *H = nullptr;
    cudaStream_t s = nullptr;    // the operator's stream (not owned)
    double *Ub = nullptr, *Fb = nullptr;
    double *d_part = nullptr, *d_out = nullptr;
    DotDesc *d_dot = nullptr;
    VecDesc *d_vec = nullptr;
    double *d_coef = nullptr;
    // pinned host mirrors
    DotDesc *h_dot = nullptr;
    VecDesc *h_vec = nullptr;
    double *h_out = nullptr, *h_coef = nullptr;
    std::map<int, htlr_plan *> plans;
    std::vector<Request *> batch;  // this step
    int n_mv = 0;                  // entries with a matvec (first in batch)
};

struct Operator {
    htlr_operator_spec spec{};
    std::vector<double> a;
    long long N = 0;
    bool resident = false;
    cudaStream_t s = nullptr;  // both handles run on it, so their steps are ordered
    Group acc, inner;          // inner unused (H null) in FP64 mode
    size_t bytes = 0;
    long long last_used = 0;
    int active = 0;
    bool inflight = false;     // a step is on the operator's stream
    bool run_acc = false, run_inner = false;  // groups of that step
    long long steps = 0;
};

}  // namespace

struct htlr_server {
    htlr_server_options o{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;     // submitted, not yet seen by the loop
    std::list<Request *> pending;    // waiting for admission (loop thread only)
    std::vector<Request *> active;   // loop thread only
    std::map<long long, std::unique_ptr<Request>> reqs;
    std::vector<std::unique_ptr<Operator>> ops;  // guarded by mu (push_back may move it)
    std::vector<Operator *> view;                 // loop thread's copy of the pointers
    long long next_id = 1, step_no = 0;
    bool stop = false;
    size_t used = 0;
    htlr_server_stats st{};
    std::thread th;
    int S = 0;  // doubles per request in the small per-step arrays

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    void loop();
    void admit();
    int make_resident(Operator &op);
    int make_group(Operator &op, Group &g, int prec_far, int prec_near, int storage);
    void release(Operator &op);
    void release_group(Group &g);
    bool evict_one(const Operator *keep);
    void finish(Request *q, int err);
    int step();
    void enqueue_pre(Group &g, Operator &op, std::vector<Request *> &list, bool acc_handle);
    void host_post(Group &g, Operator &op);
};

namespace {

size_t ws_bytes(long long N, int m) { return sizeof(double) * (size_t)N * (size_t)(m + 4); }

template <class T>
int pinned(T **p, size_t count)
{
    cudaError_t e = cudaMallocHost((void **)p, sizeof(T) * (count ? count : 1));
    return e == cudaSuccess ? HTLR_OK : cuda_fail(e, "server: pinned buffer");
}

}  // namespace

void htlr_server::release_group(Group &g)
{
    for (auto &kv : g.plans) htlr_plan_free(kv.second);
    g.plans.clear();
    if (g.H) htlr_free(g.H);
    for (void *p : {(void *)g.Ub, (void *)g.Fb, (void *)g.d_part, (void *)g.d_out, (void *)g.d_dot,
                    (void *)g.d_vec, (void *)g.d_coef})
        if (p) cudaFree(p);
    for (void *p : {(void *)g.h_dot, (void *)g.h_vec, (void *)g.h_out, (void *)g.h_coef})
        if (p) cudaFreeHost(p);
    g = Group{};
}

void htlr_server::release(Operator &op)
{
    if (op.s) cudaStreamSynchronize(op.s);
    release_group(op.acc);
    release_group(op.inner);
    if (op.s) cudaStreamDestroy(op.s);
    op.s = nullptr;
    used -= std::min(used, op.bytes);
    op.bytes = 0;
    op.resident = false;
}

bool htlr_server::evict_one(const Operator *keep)
{
    Operator *victim = nullptr;
    for (Operator *p : view)
        if (p != keep && p->resident && p->active == 0 &&
            (!victim || p->last_used < victim->last_used))
            victim = p;
    if (!victim) return false;
    release(*victim);
    ++st.evictions;
    return true;
}

int htlr_server::make_group(Operator &op, Group &g, int prec_far, int prec_near, int storage)
{
    cudaError_t e;
    g.s = op.s;
    const htlr_operator_spec &sp = op.spec;
    htlr_kernel k{sp.kernel_type, sp.kscale, sp.kparam};
    htlr_grid grid{};
    grid.type = HTLR_GRID_UNIFORM;
    grid.a = op.a.empty() ? nullptr : op.a.data();
    const int B = o.max_batch, m = o.restart;
    const size_t bufs = 2 * sizeof(double) * (size_t)op.N * B;
    int rc = HTLR_ENOMEM;
    while (true) {
        htlr_options ho{};
        ho.storage = storage;
        ho.orth = -1;
        ho.stream = g.s;
        ho.far_precision = prec_far;
        ho.near_precision = prec_near;
        const size_t avail = o.hbm_budget > used + bufs ? o.hbm_budget - used - bufs : 0;
        ho.hbm_limit = avail ? avail : 1;
        rc = htlr_construct_ex(&g.H, &k, sp.d, sp.n, &grid, sp.leaf, sp.r, sp.eta, &ho);
        if (rc != HTLR_ENOMEM || !evict_one(&op)) break;
    }
    if (rc) return rc;
    ++st.constructions;
    htlr_stats hs{};
    htlr_info(g.H, &hs);
    op.bytes += hs.bytes_total + bufs;
    used += hs.bytes_total + bufs;
    if (o.autotune_ms > 0) {
        htlr_tune_result tr{};
        if ((rc = htlr_autotune(g.H, B, o.autotune_ms, &tr))) return rc;
    }
    const int maxcnt = m + 1;
    if ((e = device_malloc((void **)&g.Ub, sizeof(double) * op.N * B)) != cudaSuccess ||
        (e = device_malloc((void **)&g.Fb, sizeof(double) * op.N * B)) != cudaSuccess ||
        (e = device_malloc((void **)&g.d_part, sizeof(double) * (size_t)B * kBlk * maxcnt)) != cudaSuccess ||
        (e = device_malloc((void **)&g.d_out, sizeof(double) * (size_t)B * S)) != cudaSuccess ||
        (e = device_malloc((void **)&g.d_coef, sizeof(double) * (size_t)B * S)) != cudaSuccess ||
        (e = device_malloc((void **)&g.d_dot, sizeof(DotDesc) * (size_t)B * 3)) != cudaSuccess ||
        (e = device_malloc((void **)&g.d_vec, sizeof(VecDesc) * (size_t)B * 3)) != cudaSuccess)
        return cuda_fail(e, "server: batch buffers");
    if ((rc = pinned(&g.h_dot, (size_t)B * 3)) || (rc = pinned(&g.h_vec, (size_t)B * 3)) ||
        (rc = pinned(&g.h_out, (size_t)B * S)) || (rc = pinned(&g.h_coef, (size_t)B * S)))
        return rc;
    return HTLR_OK;
}

int htlr_server::make_resident(Operator &op)
{
    op.bytes = 0;
    const int storage = op.spec.storage;
    cudaError_t e = cudaStreamCreateWithFlags(&op.s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "server: stream");
    int rc;
    if (o.mixed) {
        rc = make_group(op, op.acc, HTLR_PREC_DF64, HTLR_PREC_DF64, storage);
        if (!rc) rc = make_group(op, op.inner, o.inner_precision, o.inner_precision, storage);
    } else {
        rc = make_group(op, op.acc, HTLR_PREC_FP64, HTLR_PREC_FP64, storage);
    }
    if (rc) {
        std::string keep = htlr_last_error();
        release(op);
        set_error(keep);
        return rc;
    }
    op.resident = true;
    st.bytes_peak = std::max(st.bytes_peak, (long long)used);
    return HTLR_OK;
}

void htlr_server::finish(Request *q, int err)
{
    Operator &op = *view[q->op];
    Group &g = op.acc;
    if (!err && q->u_host) {
        cudaError_t e = cudaMemcpyAsync(q->u_host, q->x, sizeof(double) * op.N,
                                        cudaMemcpyDeviceToHost, g.s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(g.s);
        if (e != cudaSuccess) err = HTLR_ECUDA;
    }
    if (q->ws) {
        cudaStreamSynchronize(op.s);
        cudaFree(q->ws);
        used -= std::min(used, q->ws_bytes);
        q->ws = nullptr;
    }
    if (op.active > 0 && q->info.status == HTLR_REQ_ACTIVE) --op.active;
    op.last_used = step_no;
    std::lock_guard<std::mutex> lk(mu);
    q->info.error = err;
    q->info.status = err ? HTLR_REQ_FAILED : HTLR_REQ_DONE;
    q->info.done_s = now();
    q->info.converged = !err && q->info.rel_residual <= o.tol;
    if (err) ++st.failed;
    else ++st.completed;
    cv_done.notify_all();
}

void htlr_server::admit()
{
    for (auto it = pending.begin(); it != pending.end() && (int)active.size() < o.max_active;) {
        Request *q = *it;
        Operator &op = *view[q->op];
        if (!op.resident) {
            int rc = make_resident(op);
            if (rc == HTLR_ENOMEM && !active.empty()) {  // may fit once others finish
                ++it;
                continue;
            }
            if (rc) {
                it = pending.erase(it);
                finish(q, rc);
                continue;
            }
        }
        const size_t need = ws_bytes(op.N, o.restart);
        while (used + need > o.hbm_budget && evict_one(&op)) {
        }
        if (used + need > o.hbm_budget) {
            if (active.empty() && op.active == 0) {
                it = pending.erase(it);
                set_error("server: request workspace does not fit the HBM budget");
                finish(q, HTLR_ENOMEM);
            } else {
                ++it;
            }
            continue;
        }
        cudaError_t e = device_malloc((void **)&q->ws, need);
        if (e != cudaSuccess) {
            it = pending.erase(it);
            finish(q, cuda_fail(e, "server: request workspace"));
            continue;
        }
        used += need;
        q->ws_bytes = need;
        st.bytes_peak = std::max(st.bytes_peak, (long long)used);
        const long long N = op.N;
        const int m = o.restart;
        q->V = q->ws;
        q->x = q->V + (size_t)(m + 1) * N;
        q->b = q->x + N;
        q->r = q->b + N;
        cudaMemsetAsync(q->x, 0, sizeof(double) * N, op.s);
        // from pageable memory: returns once f is staged, so the host copy can go
        cudaMemcpyAsync(q->b, q->f.data(), sizeof(double) * N, cudaMemcpyHostToDevice, op.s);
        std::vector<double>().swap(q->f);
        q->phase = kResidual;
        q->x_zero = true;
        q->Hh.assign((size_t)(m + 1) * m, 0.0);
        q->cs.assign(m, 0.0);
        q->sn.assign(m, 0.0);
        q->g.assign(m + 1, 0.0);
        {
            std::lock_guard<std::mutex> lk(mu);
            q->info.status = HTLR_REQ_ACTIVE;
            q->info.admit_s = now();
        }
        ++op.active;
        op.last_used = step_no;
        active.push_back(q);
        it = pending.erase(it);
    }
}

// Enqueue, for the requests of one group, the gather, the batched matvec and the
// reductions whose results the host needs, ending with their copy to pinned memory.
void htlr_server::enqueue_pre(Group &g, Operator &op, std::vector<Request *> &list, bool acc_handle)
{
    const long long N = op.N;
    const int m = o.restart, maxcnt = m + 1;
    g.batch.clear();
    // matvec entries first (their column in Ub / Fb is their slot)
    for (Request *q : list)
        if (!(q->phase == kResidual && q->x_zero)) g.batch.push_back(q);
    g.n_mv = (int)g.batch.size();
    for (Request *q : list)
        if (q->phase == kResidual && q->x_zero) g.batch.push_back(q);
    const int B = (int)g.batch.size();
    if (B == 0) return;
    (void)acc_handle;
    // descriptor regions at fixed offsets (multiples of max_batch): the post-step region
    // [2 MB, 3 MB) of h_vec may still be read by a pending copy of the previous step
    const int MB = o.max_batch;
    for (int i = 0; i < B; ++i) g.batch[i]->slot = i;
    // gather
    for (int i = 0; i < g.n_mv; ++i) {
        Request *q = g.batch[i];
        VecDesc v{};
        v.a = q->phase == kResidual ? q->x : q->V + (size_t)q->k * N;
        g.h_vec[i] = v;
    }
    cudaStream_t s = g.s;
    if (g.n_mv) {
        cudaMemcpyAsync(g.d_vec, g.h_vec, sizeof(VecDesc) * g.n_mv, cudaMemcpyHostToDevice, s);
        gather_k<<<dim3(grid_x(N), g.n_mv), kThreads, 0, s>>>(g.d_vec, N, g.Ub);
        int rc;
        if (o.use_graphs) {
            htlr_plan *&P = g.plans[g.n_mv];
            rc = P ? HTLR_OK : htlr_plan_create(g.H, g.Ub, g.Fb, g.n_mv, &P);
            if (!rc) rc = htlr_plan_launch(P);
        } else {
            rc = matvec_enqueue(g.H, g.Ub, g.Fb, g.n_mv);
        }
        if (rc) {
            for (Request *q : g.batch) q->done = true, q->info.error = rc;
            return;
        }
        ++st.batched_matvecs;
        st.matvec_columns += g.n_mv;
        st.max_batch_seen = std::max(st.max_batch_seen, g.n_mv);
        for (int i = 0; i < g.n_mv; ++i) ++g.batch[i]->info.matvecs;
    }
    // Arnoldi entries: CGS2 then the norm; residual entries: r = b - A x and its norm
    std::vector<int> arn, res;
    for (int i = 0; i < B; ++i) (g.batch[i]->phase == kArnoldi ? arn : res).push_back(i);
    auto w_of = [&](int i) { return g.Fb + (size_t)i * N; };
    const int na = (int)arn.size(), nr = (int)res.size();
    if (na) {
        for (int pass = 0; pass < 2; ++pass) {
            for (int a = 0; a < na; ++a) {
                Request *q = g.batch[arn[a]];
                g.h_dot[pass * MB + a] = DotDesc{q->V, w_of(arn[a]), q->k + 1,
                                                (long long)arn[a] * S + pass * maxcnt};
            }
        }
        for (int a = 0; a < na; ++a)
            g.h_dot[2 * MB + a] = DotDesc{w_of(arn[a]), w_of(arn[a]), 1,
                                         (long long)arn[a] * S + 2 * maxcnt};
        cudaMemcpyAsync(g.d_dot, g.h_dot, sizeof(DotDesc) * 3 * MB, cudaMemcpyHostToDevice, s);
        const int fin = (na * maxcnt + 255) / 256;
        for (int pass = 0; pass < 2; ++pass) {
            const DotDesc *D = g.d_dot + pass * MB;
            dots_partial_k<<<dim3(kBlk, na), kThreads, 0, s>>>(D, N, maxcnt, g.d_part);
            dots_final_k<<<fin, 256, 0, s>>>(D, na, maxcnt, g.d_part, g.d_out);
            subcomb_k<<<dim3(grid_x(N), na), kThreads, 0, s>>>(D, N, g.d_out);
        }
        dots_partial_k<<<dim3(kBlk, na), kThreads, 0, s>>>(g.d_dot + 2 * MB, N, maxcnt, g.d_part);
        dots_final_k<<<fin, 256, 0, s>>>(g.d_dot + 2 * MB, na, maxcnt, g.d_part, g.d_out);
    }
    if (nr) {
        VecDesc *hv = g.h_vec + MB;   // second third of the descriptor buffer
        for (int a = 0; a < nr; ++a) {
            Request *q = g.batch[res[a]];
            VecDesc v{};
            v.a = q->b;
            v.b = q->x_zero ? nullptr : w_of(res[a]);
            v.dst = q->r;
            hv[a] = v;
        }
        DotDesc *hd = g.h_dot + 2 * MB + na;
        for (int a = 0; a < nr; ++a) {
            Request *q = g.batch[res[a]];
            hd[a] = DotDesc{q->r, q->r, 1, (long long)res[a] * S + 2 * maxcnt};
        }
        cudaMemcpyAsync(g.d_vec + MB, hv, sizeof(VecDesc) * nr, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(g.d_dot + 2 * MB + na, hd, sizeof(DotDesc) * nr, cudaMemcpyHostToDevice, s);
        resid_k<<<dim3(grid_x(N), nr), kThreads, 0, s>>>(g.d_vec + MB, N);
        dots_partial_k<<<dim3(kBlk, nr), kThreads, 0, s>>>(g.d_dot + 2 * MB + na, N, maxcnt, g.d_part);
        dots_final_k<<<(nr * maxcnt + 255) / 256, 256, 0, s>>>(g.d_dot + 2 * MB + na, nr, maxcnt,
                                                            g.d_part, g.d_out);
    }
    cudaMemcpyAsync(g.h_out, g.d_out, sizeof(double) * (size_t)B * S, cudaMemcpyDeviceToHost, s);
}

// After the group's stream finished: advance every request's state machine on the host
// and enqueue the vector updates (next basis vector, solution update).
void htlr_server::host_post(Group &g, Operator &op)
{
    const long long N = op.N;
    const int m = o.restart, maxcnt = m + 1, B = (int)g.batch.size();
    if (B == 0) return;
    std::vector<VecDesc> sc, up;
    std::vector<double> coef;     // y vectors, S per entry slot
    coef.assign((size_t)B * S, 0.0);
    for (Request *q : g.batch) {
        if (q->done) continue;
        const double *out = g.h_out + (size_t)q->slot * S;
        auto &I = q->info;
        if (q->phase == kArnoldi) {
            const int k = q->k;
            double *hc = &q->Hh[(size_t)k * (m + 1)];
            for (int j = 0; j <= k; ++j) hc[j] = out[j] + out[maxcnt + j];
            const double hn = std::sqrt(std::max(0.0, out[2 * maxcnt]));
            hc[k + 1] = hn;
            for (int j = 0; j < k; ++j) {
                const double c0 = q->cs[j], s0 = q->sn[j];
                const double t = c0 * hc[j] + s0 * hc[j + 1];
                hc[j + 1] = -s0 * hc[j] + c0 * hc[j + 1];
                hc[j] = t;
            }
            const double a0 = hc[k], b0 = hc[k + 1], rr = std::hypot(a0, b0);
            const double c0 = rr > 0 ? a0 / rr : 1.0, s0 = rr > 0 ? b0 / rr : 0.0;
            q->cs[k] = c0;
            q->sn[k] = s0;
            hc[k] = rr;
            hc[k + 1] = 0.0;
            q->g[k + 1] = -s0 * q->g[k];
            q->g[k] = c0 * q->g[k];
            ++I.iterations;
            const bool end = std::fabs(q->g[k + 1]) <= q->target || k + 1 >= m || hn == 0.0 ||
                             rr == 0.0 || I.iterations >= o.max_iters;
            if (!end) {
                VecDesc v{};
                v.a = g.Fb + (size_t)q->slot * N;
                v.dst = q->V + (size_t)(k + 1) * N;
                v.s = 1.0 / hn;
                sc.push_back(v);
                q->k = k + 1;
            } else {
                // y = R^{-1} g (k + 1 terms), x += V y
                const int kk = k + 1;
                double *y = &coef[(size_t)q->slot * S];
                for (int i = kk - 1; i >= 0; --i) {
                    double v = q->g[i];
                    for (int j = i + 1; j < kk; ++j) v -= q->Hh[(size_t)j * (m + 1) + i] * y[j];
                    const double dg = q->Hh[(size_t)i * (m + 1) + i];
                    y[i] = dg != 0.0 ? v / dg : 0.0;
                }
                VecDesc v{};
                v.a = q->V;
                v.dst = q->x;
                v.cnt = kk;
                v.c = g.d_coef + (size_t)q->slot * S;
                up.push_back(v);
                q->phase = kResidual;
                q->x_zero = false;
            }
        } else {
            const double rn = std::sqrt(std::max(0.0, out[2 * maxcnt]));
            if (q->x_zero) q->fn = rn;       // r = f at x = 0
            I.rel_residual = q->fn > 0 ? rn / q->fn : 0.0;
            if (I.rel_residual <= o.tol || I.iterations >= o.max_iters || q->fn == 0.0) {
                q->done = true;
                continue;
            }
            if (!q->x_zero && o.mixed) ++I.refinements;
            std::fill(q->g.begin(), q->g.end(), 0.0);
            q->g[0] = rn;
            q->k = 0;
            q->target = o.mixed ? std::max(o.inner_tol * rn, 0.5 * o.tol * q->fn) : o.tol * q->fn;
            VecDesc v{};
            v.a = q->r;
            v.dst = q->V;
            v.s = 1.0 / rn;
            sc.push_back(v);
            q->phase = kArnoldi;
        }
    }
    cudaStream_t s = g.s;
    if (!up.empty()) {
        std::memcpy(g.h_coef, coef.data(), sizeof(double) * coef.size());
        cudaMemcpyAsync(g.d_coef, g.h_coef, sizeof(double) * coef.size(), cudaMemcpyHostToDevice, s);
    }
    const int nsc = (int)sc.size(), nup = (int)up.size();
    if (nsc + nup) {
        const int MB = o.max_batch;
        VecDesc *hv = g.h_vec + 2 * MB;
        for (int i = 0; i < nsc; ++i) hv[i] = sc[i];
        for (int i = 0; i < nup; ++i) hv[nsc + i] = up[i];
        cudaMemcpyAsync(g.d_vec + 2 * MB, hv, sizeof(VecDesc) * (nsc + nup), cudaMemcpyHostToDevice, s);
        if (nsc) scale_k<<<dim3(grid_x(N), nsc), kThreads, 0, s>>>(g.d_vec + 2 * MB, N);
        if (nup) update_k<<<dim3(grid_x(N), nup), kThreads, 0, s>>>(g.d_vec + 2 * MB + nsc, N);
    }
}

// One pass of the event loop: start a step on every idle operator that has active
// requests (its requests that need the same handle form one batched matvec), and finish
// the steps whose streams are idle (host side of GMRES, retirement).  Operators advance
// independently, so a slow operator does not hold back the others.
int htlr_server::step()
{
    bool progressed = false;
    for (int id = 0; id < (int)view.size(); ++id) {
        Operator &op = *view[id];
        if (!op.resident || op.active == 0 || op.inflight) continue;
        std::vector<Request *> la, li;
        for (Request *q : active) {
            if (q->op != id) continue;
            std::vector<Request *> &l = (o.mixed && q->phase == kArnoldi) ? li : la;
            if ((int)l.size() < o.max_batch) l.push_back(q);   // oldest first
        }
        if (la.empty() && li.empty()) continue;
        ++step_no;
        ++st.steps;
        op.last_used = step_no;
        op.run_acc = !la.empty();
        op.run_inner = !li.empty();
        if (op.run_acc) enqueue_pre(op.acc, op, la, true);
        if (op.run_inner) enqueue_pre(op.inner, op, li, false);
        op.inflight = true;
        progressed = true;
    }
    for (int id = 0; id < (int)view.size(); ++id) {
        Operator &op = *view[id];
        if (!op.inflight) continue;
        cudaError_t e = cudaStreamQuery(op.s);
        if (e == cudaErrorNotReady) continue;
        op.inflight = false;
        progressed = true;
        int err = e == cudaSuccess ? HTLR_OK : cuda_fail(e, "server: step");
        // the handles' device error words (bounded waits that gave up) are read every 32
        // steps of the operator and before any of its requests is delivered
        if (!err && ++op.steps % 32 == 0) {
            err = htlr_sync(op.acc.H);
            if (!err && op.inner.H) err = htlr_sync(op.inner.H);
        }
        if (!err) {
            if (op.run_acc) host_post(op.acc, op);
            if (op.run_inner) host_post(op.inner, op);
        }
        bool checked = false;
        for (size_t i = 0; i < active.size();) {
            Request *q = active[i];
            if (q->op != id || (!q->done && !err)) {
                ++i;
                continue;
            }
            if (!err && !checked) {
                err = htlr_sync(op.acc.H);
                if (!err && op.inner.H) err = htlr_sync(op.inner.H);
                checked = true;
            }
            active.erase(active.begin() + (long)i);
            finish(q, err ? err : q->info.error);
        }
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    return HTLR_OK;
}

void htlr_server::loop()
{
    cudaSetDevice(device);
    while (true) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active.empty() && pending.empty() && queue.empty()) {
                if (stop) {
                    view.clear();
                    for (auto &p : ops) view.push_back(p.get());
                    break;
                }
                cv_work.wait_for(lk, std::chrono::milliseconds(20));
            }
            view.clear();
            for (auto &p : ops) view.push_back(p.get());
            while (!queue.empty()) {
                pending.push_back(queue.front());
                queue.pop_front();
            }
            st.pending = (int)pending.size();
        }
        admit();
        if (active.empty()) continue;
        int rc = step();
        if (rc) {
            // a failed step fails its requests; the loop carries on with the others
            std::vector<Request *> act;
            act.swap(active);
            for (Request *q : act) finish(q, rc);
        }
        std::lock_guard<std::mutex> lk(mu);
        st.active = (int)active.size();
    }
    for (Operator *p : view)
        if (p->resident) release(*p);
}

extern "C" {

int htlr_server_create(const htlr_server_options *o, htlr_server **out)
{
    if (!out) return fail(HTLR_EINVAL, "htlr_server_create: out must not be NULL");
    *out = nullptr;
    htlr_server_options d{};
    d.hbm_budget = 0;
    d.max_active = 64;
    d.max_batch = 16;
    d.mixed = 1;
    d.inner_precision = HTLR_PREC_FP32;
    d.restart = 30;
    d.tol = 1e-10;
    d.inner_tol = 1e-4;
    d.max_iters = 3000;
    d.use_graphs = 1;
    d.autotune_ms = 0.0;
    const htlr_server_options &O = o ? *o : d;
    if (O.max_active < 1 || O.max_batch < 1 || O.max_batch > 64 || O.restart < 1 ||
        O.restart > 200 || !(O.tol > 0) || O.max_iters < 1 || (O.mixed != 0 && O.mixed != 1) ||
        (O.mixed && !(O.inner_tol > 0 && O.inner_tol < 1)) ||
        (O.mixed && O.inner_precision != HTLR_PREC_FP32 && O.inner_precision != HTLR_PREC_DF64 &&
         O.inner_precision != HTLR_PREC_BF16X6) ||
        !(O.autotune_ms >= 0))
        return fail(HTLR_EINVAL, "htlr_server_create: invalid options");
    htlr_server *S = new (std::nothrow) htlr_server();
    if (!S) return fail(HTLR_ENOMEM, "htlr_server_create: host allocation failed");
    S->o = O;
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) {
        delete S;
        return cuda_fail(e, "htlr_server_create: no device");
    }
    if (S->o.hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) {
            delete S;
            return cuda_fail(e, "htlr_server_create");
        }
        S->o.hbm_budget = (size_t)(0.8 * (double)fr);
    }
    S->S = 2 * (O.restart + 1) + 2;
    S->t0 = std::chrono::steady_clock::now();
    try {
        S->th = std::thread([S] { S->loop(); });
    } catch (...) {
        delete S;
        return fail(HTLR_ENOMEM, "htlr_server_create: cannot start the scheduler thread");
    }
    *out = S;
    return HTLR_OK;
}

int htlr_server_add_operator(htlr_server *S, const htlr_operator_spec *spec, int *op_id)
{
    if (!S || !spec || !op_id) return fail(HTLR_EINVAL, "htlr_server_add_operator: NULL argument");
    if (spec->d != 2 && spec->d != 3) return fail(HTLR_EINVAL, "htlr_server_add_operator: d must be 2 or 3");
    if (spec->leaf < 1 || spec->n < 2 || spec->n % spec->leaf || spec->r < 1)
        return fail(HTLR_EINVAL, "htlr_server_add_operator: bad n, leaf or r");
    if (spec->storage < HTLR_STORE_AUTO || spec->storage > HTLR_STORE_SHARED)
        return fail(HTLR_EINVAL, "htlr_server_add_operator: storage must be AUTO, STORED or SHARED");
    auto op = std::make_unique<Operator>();
    op->spec = *spec;
    op->N = 1;
    for (int k = 0; k < spec->d; ++k) op->N *= spec->n;
    if (spec->a) op->a.assign(spec->a, spec->a + op->N);
    op->spec.a = nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    // the loop thread reads `ops` only for operators that have requests, which are
    // submitted after this call returns; push_back may move the vector, so guard it
    S->ops.push_back(std::move(op));
    *op_id = (int)S->ops.size() - 1;
    return HTLR_OK;
}

int htlr_server_submit(htlr_server *S, int op_id, const double *f_host, double *u_host,
                       long long *req_id)
{
    if (!S || !f_host || !req_id) return fail(HTLR_EINVAL, "htlr_server_submit: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (op_id < 0 || op_id >= (int)S->ops.size())
        return fail(HTLR_EINVAL, "htlr_server_submit: unknown operator");
    if (S->stop) return fail(HTLR_EINVAL, "htlr_server_submit: server is shutting down");
    auto q = std::make_unique<Request>();
    q->id = S->next_id++;
    q->op = op_id;
    const long long N = S->ops[op_id]->N;
    q->f.assign(f_host, f_host + N);
    q->u_host = u_host;
    q->info.status = HTLR_REQ_QUEUED;
    q->info.submit_s = S->now();
    *req_id = q->id;
    S->queue.push_back(q.get());
    S->reqs[q->id] = std::move(q);
    ++S->st.submitted;
    S->cv_work.notify_all();
    return HTLR_OK;
}

int htlr_server_poll(htlr_server *S, long long req_id, htlr_request_info *info)
{
    if (!S || !info) return fail(HTLR_EINVAL, "htlr_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return fail(HTLR_EINVAL, "htlr_server_poll: unknown request");
    *info = it->second->info;
    return HTLR_OK;
}

int htlr_server_wait(htlr_server *S, long long req_id, double timeout_s, htlr_request_info *info)
{
    if (!S) return fail(HTLR_EINVAL, "htlr_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(req_id);
    if (it == S->reqs.end()) return fail(HTLR_EINVAL, "htlr_server_wait: unknown request");
    Request *q = it->second.get();
    auto ready = [&] { return q->info.status == HTLR_REQ_DONE || q->info.status == HTLR_REQ_FAILED; };
    if (timeout_s < 0) S->cv_done.wait(lk, ready);
    else S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready);
    if (info) *info = q->info;
    if (!ready()) return fail(HTLR_ETIMEOUT, "htlr_server_wait: timed out");
    return HTLR_OK;
}

int htlr_server_get_stats(htlr_server *S, htlr_server_stats *st)
{
    if (!S || !st) return fail(HTLR_EINVAL, "htlr_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *st = S->st;
    st->bytes_in_use = (long long)S->used;
    st->bytes_budget = (long long)S->o.hbm_budget;
    st->resident_operators = 0;
    for (auto &p : S->ops) st->resident_operators += p->resident ? 1 : 0;
    return HTLR_OK;
}

void htlr_server_destroy(htlr_server *S)
{
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    delete S;
}

}  // extern "C"
