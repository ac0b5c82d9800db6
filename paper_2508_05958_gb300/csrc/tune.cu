// Autotuner of the matvec's launch shapes.  The tunables are the ones that change the
// speed of HMultVec but not its result beyond rounding order:
//   - task_bytes: bytes of blocks one warp streams per task in the CUDA-core block stream
//     (more, shorter tasks balance better; fewer, longer ones write fewer partial sums);
//   - stream_ctas_per_sm, stream_threads: the stream's grid cap (152 x ctas) and CTA size;
//   - tc_stages: depth of the tensor-core kernel's shared-memory ring.
// Each candidate is timed with CUDA events on the handle's stream (one warm-up, then the
// median of a few matvecs on scratch vectors), by coordinate descent from the current
// settings, within a time budget.  The winner is applied to the handle and remembered in
// a process-wide table keyed by the operator's shape, so later operators of the same
// shape (the serving loop constructs many) take it without timing.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "htlr_internal.h"

namespace htlr {
int matvec_enqueue(const htlr_handle *H, const double *u, double *f, int nrhs);
bool handle_is_live(const htlr_handle *H);
}  // namespace htlr

using namespace htlr;

namespace {

struct Cfg {
    size_t task_bytes;
    int ctas, threads, stages;
};

std::mutex g_cache_mu;
std::map<std::string, Cfg> g_cache;

std::string shape_key(const htlr_handle *H, int nrhs)
{
    char buf[256];
    snprintf(buf, sizeof buf, "d%d n%d leaf%d p%d eta%.6g st%d far%d near%d t%d g%d k%d r%d",
             H->d, H->n, H->leaf, H->p, H->eta, H->storage, H->far_prec, H->near_prec,
             H->tensor, H->near_generated, H->kern.type, std::min(nrhs, H->nrc));
    return buf;
}

int apply(htlr_handle *H, const Cfg &c)
{
    if (!H->tc && c.task_bytes != H->task_bytes) {
        int rc = build_tasks(H, c.task_bytes, H->stream);
        if (rc) return rc;
    }
    H->stream_ctas_per_sm = c.ctas;
    H->stream_threads = c.threads;
    H->tc_stages_cap = c.stages;
    return HTLR_OK;
}

int fail(int code, const char *msg)
{
    set_error(msg);
    return code;
}

}  // namespace

extern "C" int htlr_autotune(htlr_handle *H, int nrhs, double budget_ms, htlr_tune_result *res)
{
    if (!handle_is_live(H)) return fail(HTLR_EINVAL, "htlr_autotune: not a live HTLR handle");
    if (nrhs < 1 || !(budget_ms >= 0)) return fail(HTLR_EINVAL, "htlr_autotune: bad nrhs or budget");
    htlr_tune_result out{};
    const std::string key = shape_key(H, nrhs);
    const Cfg start{H->task_bytes, H->stream_ctas_per_sm, H->stream_threads, H->tc_stages_cap};
    auto report = [&](const Cfg &c) {
        out.task_bytes = c.task_bytes;
        out.stream_ctas_per_sm = c.ctas;
        out.stream_threads = c.threads;
        out.tc_stages = c.stages;
        if (res) *res = out;
    };
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            int rc = apply(H, it->second);
            if (rc) return rc;
            out.from_cache = 1;
            report(it->second);
            return HTLR_OK;
        }
    }
    long long N = 1;
    for (int k = 0; k < H->d; ++k) N *= H->n;
    double *u = nullptr, *f = nullptr;
    cudaError_t e = device_malloc((void **)&u, sizeof(double) * N * nrhs);
    if (e == cudaSuccess) e = device_malloc((void **)&f, sizeof(double) * N * nrhs);
    if (e != cudaSuccess) {
        if (u) cudaFree(u);
        return cuda_fail(e, "htlr_autotune: scratch vectors");
    }
    cudaStream_t s = H->stream;
    cudaMemsetAsync(u, 0, sizeof(double) * N * nrhs, s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double spent = 0.0;
    int rc = HTLR_OK;
    // median device time of `reps` matvecs after one warm-up (ms)
    auto time_cfg = [&](const Cfg &c, int reps, float *ms) -> int {
        int r = apply(H, c);
        if (r) return r;
        if ((r = matvec_enqueue(H, u, f, nrhs))) return r;
        std::vector<float> t;
        for (int k = 0; k < reps; ++k) {
            cudaEventRecord(e0, s);
            if ((r = matvec_enqueue(H, u, f, nrhs))) return r;
            cudaEventRecord(e1, s);
            cudaError_t ee = cudaEventSynchronize(e1);
            if (ee != cudaSuccess) return cuda_fail(ee, "htlr_autotune: timing");
            float x = 0.f;
            cudaEventElapsedTime(&x, e0, e1);
            t.push_back(x);
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        spent += (reps + 1) * (double)*ms;
        ++out.candidates;
        return HTLR_OK;
    };
    Cfg best = start;
    float best_ms = 0.f;
    rc = time_cfg(start, 3, &best_ms);
    out.default_ms = best_ms;
    if (rc == HTLR_OK) {
        const int reps = 3;
        const double per = (reps + 1) * (double)best_ms;
        auto affordable = [&]() { return spent + per <= budget_ms; };
        auto try_cfg = [&](const Cfg &c) -> int {
            if (!affordable()) return HTLR_OK;
            float ms = 0.f;
            int r = time_cfg(c, reps, &ms);
            if (r) return r;
            if (ms < best_ms * 0.98f) {
                best_ms = ms;
                best = c;
            }
            return HTLR_OK;
        };
        if (!H->tc && !H->tasks.empty()) {
            // coordinate descent: task size, then grid cap, then CTA size
            for (size_t tb : {64u << 10, 128u << 10, 512u << 10, 1024u << 10}) {
                if (tb == start.task_bytes || rc) continue;
                Cfg c = best;
                c.task_bytes = tb;
                rc = try_cfg(c);
            }
            for (int ct : {4, 16, 2}) {
                if (ct == best.ctas || rc) continue;
                Cfg c = best;
                c.ctas = ct;
                rc = try_cfg(c);
            }
            for (int th : {128, 256}) {
                if (th == best.threads || rc) continue;
                Cfg c = best;
                c.threads = th;
                rc = try_cfg(c);
            }
        }
        if (H->tc) {
            for (int st : {2, 3, 4, 0}) {
                if (st == best.stages || rc) continue;
                Cfg c = best;
                c.stages = st;
                rc = try_cfg(c);
            }
        }
    }
    if (rc == HTLR_OK) rc = apply(H, best);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(u);
    cudaFree(f);
    if (rc) return rc;
    out.ms = best_ms;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        g_cache[key] = best;
    }
    report(best);
    return HTLR_OK;
}

extern "C" void htlr_autotune_clear_cache(void)
{
    std::lock_guard<std::mutex> g(g_cache_mu);
    g_cache.clear();
}
