// htlr_matvec_noalloc: HMultVec whose scratch lives in a fixed, statically allocated
// device array instead of buffers obtained with cudaMalloc.
//
// Who needs it: code that must not call the CUDA allocator when it applies an operator:
// a process whose device memory is already fully reserved by a pool or budget, a
// real-time or serving loop that cannot afford cudaMalloc/cudaFree (cudaFree waits for
// the whole device), or a caller that shares one constructed handle with other threads
// and wants its own scratch.  The scratch (per-level W and H tensors, the per-task
// partial results of the block stream and a copy of the task-kind table) is carved out
// of g_noalloc_scratch below.
//
// The array is part of the library image, so every GPU that loads the library holds it
// (kNoallocScratchBytes) until the process exits.  All calls share it: two calls whose
// work overlaps on the GPU (different streams, or different host threads without
// ordering) race and produce wrong results.  Every byte a call reads is written earlier
// in the same call, so nothing has to be cleared between calls.
#include <cstdio>
#include <vector>

#include "htlr_internal.h"

namespace htlr {

constexpr size_t kNoallocScratchBytes = 64ull << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

namespace {

// Device address of the static scratch on the current device.  It is looked up on every
// call (cudaGetSymbolAddress allocates nothing), so it stays right after the context has
// been reset or recreated.  The host-side symbol g_noalloc_scratch is only a stand-in and
// must never be passed to a kernel.
int scratch_address(unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    *out = static_cast<unsigned char *>(p);
    return HTLR_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

bool handle_is_live(const htlr_handle *H);
struct StageEvents;
int run_chunk(const htlr_handle *H, const KindDesc *d_kinds, double *part,
              const std::vector<double *> &W, const std::vector<double *> &Hs, const double *uc,
              double *fc, int nh, StageEvents *tev, cudaStream_t s);
int launch_near_gen_all(const htlr_handle *H, const double *uc, double *fc, int nh, cudaStream_t s);

int matvec_noalloc(const htlr_handle *H, const double *u, double *f, int nrhs)
{
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (cur != H->device) {
        set_error("htlr_matvec_noalloc: the handle's device is not the current device");
        return HTLR_EINVAL;
    }
    if (H->tc) {
        set_error("htlr_matvec_noalloc: operators with a BF16X6 (tensor-core) far field are "
                  "not supported; use htlr_matvec");
        return HTLR_EUNSUPPORTED;
    }
    // carve the scratch: kinds table, W and H per far level, task partials
    const int d = H->d, n = H->n, L = H->L;
    size_t off = 0;
    const size_t kinds_off = off;
    off += align256(sizeof(KindDesc) * H->kinds.size());
    std::vector<size_t> w_off(L + 1, 0), h_off(L + 1, 0);
    for (int lv = 1; lv <= L; ++lv) {
        const LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        size_t b = align256(sizeof(double) * (size_t)Lv.nbox * H->nrc * Lv.pd);
        w_off[lv] = off;
        off += b;
        h_off[lv] = off;
        off += b;
    }
    const size_t part_off = off;
    off += align256(sizeof(double) * (size_t)H->part_doubles);
    if (off > kNoallocScratchBytes) {
        char buf[200];
        snprintf(buf, sizeof buf,
                 "htlr_matvec_noalloc: this operator needs %zu bytes of scratch, above the static "
                 "maximum of %zu bytes; use htlr_matvec",
                 off, kNoallocScratchBytes);
        set_error(buf);
        return HTLR_ENOMEM;
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;

    // task kinds pointing at the scratch W tensors (copied from host memory)
    std::vector<KindDesc> kinds = H->kinds;
    for (int lv = 1; lv <= L; ++lv)
        if (H->lev[lv].nfar) kinds[lv].x = reinterpret_cast<const double *>(base + w_off[lv]);
    KindDesc *d_kinds = reinterpret_cast<KindDesc *>(base + kinds_off);
    cudaStream_t s = H->stream;
    e = cudaMemcpyAsync(d_kinds, kinds.data(), sizeof(KindDesc) * kinds.size(),
                        cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync (kinds)");
    double *part = reinterpret_cast<double *>(base + part_off);

    const long long N = [&] {
        long long v = 1;
        for (int k = 0; k < d; ++k) v *= n;
        return v;
    }();
    std::vector<double *> W(L + 1, nullptr), Hs(L + 1, nullptr);
    for (int lv = 1; lv <= L; ++lv) {
        if (H->lev[lv].nfar == 0) continue;
        W[lv] = reinterpret_cast<double *>(base + w_off[lv]);
        Hs[lv] = reinterpret_cast<double *>(base + h_off[lv]);
    }
    launch_near_gen_all(H, u, f, nrhs, s);
    for (int c0 = 0; c0 < nrhs; c0 += H->nrc) {
        const int nh = nrhs - c0 < H->nrc ? nrhs - c0 : H->nrc;
        run_chunk(H, d_kinds, part, W, Hs, u + (long long)c0 * N, f + (long long)c0 * N, nh,
                  nullptr, s);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "htlr_matvec_noalloc launch");
    return HTLR_OK;
}

}  // namespace htlr

extern "C" int htlr_matvec_noalloc(const htlr_handle *H, const double *u, double *f, int nrhs)
{
    if (!htlr::handle_is_live(H)) {
        htlr::set_error("not a live HTLR handle");
        return HTLR_EINVAL;
    }
    if (!u || !f) {
        htlr::set_error("u and f must not be NULL");
        return HTLR_EINVAL;
    }
    if (nrhs < 1) {
        htlr::set_error("nrhs must be >= 1");
        return HTLR_EINVAL;
    }
    long long N = 1;
    for (int k = 0; k < H->d; ++k) N *= H->n;
    const char *ub = (const char *)u, *ue = (const char *)(u + N * nrhs);
    const char *fb = (const char *)f, *fe = (const char *)(f + N * nrhs);
    if (ub < fe && fb < ue) {
        htlr::set_error("u and f must not overlap");
        return HTLR_EINVAL;
    }
    return htlr::matvec_noalloc(H, u, f, nrhs);
}
