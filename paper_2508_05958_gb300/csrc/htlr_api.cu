// C ABI of the HTLR library: argument checks, Construct (Algorithm 1) orchestration and
// HMultVec (Algorithm 2) orchestration.  Every step of the computation runs in the
// kernels of plan.cu, construct.cu and apply.cu; this file only plans, allocates and
// launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "htlr_internal.h"

namespace htlr {

static thread_local std::string g_err;
static std::mutex g_live_mu;
static std::set<const htlr_handle *> g_live;

void set_error(const std::string &msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char *what)
{
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return HTLR_ECUDA;
}

#define HTLR_CK(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

static std::atomic<long long> g_device_allocs{0};

cudaError_t device_malloc(void **p, size_t bytes)
{
    g_device_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(p, bytes);
}

static int fail(int code, const std::string &msg)
{
    set_error(msg);
    return code;
}

template <class T>
static int dalloc(htlr_handle *H, T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    cudaError_t e = device_malloc(&q, count * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
    H->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return HTLR_OK;
}

// Release one allocation made by dalloc (and forget it).
template <class T>
static void dfree(htlr_handle *H, T *&p)
{
    if (!p) return;
    for (size_t i = 0; i < H->allocs.size(); ++i)
        if (H->allocs[i] == (void *)p) {
            H->allocs.erase(H->allocs.begin() + (long)i);
            break;
        }
    cudaFree((void *)p);
    p = nullptr;
}

// Scratch allocations released at the end of construction.
struct Temps {
    std::vector<void *> p;
    ~Temps()
    {
        for (void *q : p) cudaFree(q);
    }
    template <class T>
    int alloc(T **out, size_t count)
    {
        *out = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = device_malloc(&q, count * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (temporary)");
        p.push_back(q);
        *out = static_cast<T *>(q);
        return HTLR_OK;
    }
};

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_q from Tricomi's
// asymptotic initial guesses; P_q' from the derivative recurrence
// P'_{j+1} = P'_{j-1} + (2j + 1) P_j.
static void gauss_legendre_host(int q, std::vector<double> &x, std::vector<double> &w)
{
    const double pi = 3.141592653589793238462643;
    x.assign(q, 0.0);
    w.assign(q, 0.0);
    for (int k = 1; k <= q; ++k) {
        double th = pi * (4.0 * k - 1.0) / (4.0 * q + 2.0);
        double z = (1.0 - (q - 1.0) / (8.0 * q * q * q)) * std::cos(th);
        double dp = 1.0;
        for (int it = 0; it < 64; ++it) {
            double pm1 = 1.0, p0 = z, dm1 = 0.0, d0 = 1.0;
            for (int j = 1; j < q; ++j) {
                double p1 = ((2.0 * j + 1.0) * z * p0 - j * pm1) / (j + 1.0);
                double d1 = dm1 + (2.0 * j + 1.0) * p0;
                pm1 = p0;
                p0 = p1;
                dm1 = d0;
                d0 = d1;
            }
            dp = d0;
            double step = p0 / d0;
            z -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        x[k - 1] = z;
        w[k - 1] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

static int ipow(int b, int e)
{
    int r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

// Decode a lexicographic box index of a level into its multi-index.
static void box_index(int box, int d, int level, int *b)
{
    int m = (1 << level) - 1;
    for (int k = 0; k < d; ++k) b[k] = (box >> (level * k)) & m;
    for (int k = d; k < 3; ++k) b[k] = 0;
}

struct Sizes {
    size_t cores = 0, near = 0, factors = 0, work = 0, lists = 0;
    size_t total() const { return cores + near + factors + work + lists; }
};

// Grouped tensor-core shape of Nd x Kd blocks (see tc_group.cu).
static TcgShape tcg_shape(int Nd, int Kd)
{
    TcgShape t;
    t.Kd = Kd;
    t.Nd = Nd;
    t.nch = (Kd + 15) / 16;
    // passes of at most kTcgMaxNw rows: two accumulator buffers of Nw columns fit in tensor
    // memory, and a drain thread holds Nw / 2 running sums in registers
    const int n16 = (Nd + 15) / 16 * 16;
    t.passes = (n16 + kTcgMaxNw - 1) / kTcgMaxNw;
    t.Nw = ((Nd + t.passes - 1) / t.passes + 15) / 16 * 16;
    t.Npad = t.Nw * t.passes;
    t.NGb = t.Npad / 8;
    t.core_elems = (long long)t.nch * 3 * t.NGb * 128;
    t.box_elems = (long long)3 * t.nch * (kTcRpMax / 8) * 128;
    return t;
}

// Class offset lists of one block list (rows = boxes of a level with nb1 per dimension,
// lexicographic): per parity class of the target box, the union of its rows' offsets
// sigma - tau with their block ids.  Valid only if every row of a class holds exactly
// the class offsets whose source lies inside the domain, each with one block id;
// returns false otherwise (the block list then stays on the per-row kernel).
static bool build_classes(int d, int nb1, const std::vector<int> &rowptr, const std::vector<int> &col,
                          const std::vector<int> &blk, std::vector<int4v> &out, int start[8],
                          int count[8])
{
    const long long nbox = d == 3 ? (long long)nb1 * nb1 * nb1 : (long long)nb1 * nb1;
    std::map<std::tuple<int, int, int>, int> cls[8];
    auto coords = [&](long long b, int &b1, int &b2, int &b3) {
        b1 = (int)(b % nb1);
        b2 = (int)((b / nb1) % nb1);
        b3 = d == 3 ? (int)(b / ((long long)nb1 * nb1)) : 0;
    };
    for (long long t = 0; t < nbox; ++t) {
        int b1, b2, b3;
        coords(t, b1, b2, b3);
        const int c = (b1 & 1) + 2 * (b2 & 1) + 4 * (b3 & 1);
        for (int e = rowptr[t]; e < rowptr[t + 1]; ++e) {
            int s1, s2, s3;
            coords(col[e], s1, s2, s3);
            auto key = std::make_tuple(s3 - b3, s2 - b2, s1 - b1);
            auto it = cls[c].find(key);
            if (it == cls[c].end()) cls[c][key] = blk[e];
            else if (it->second != blk[e]) return false;
        }
    }
    out.clear();
    for (int c = 0; c < 8; ++c) {
        start[c] = (int)out.size();
        count[c] = (int)cls[c].size();
        if (count[c] > 1024) return false;
        for (auto &kv : cls[c])
            out.push_back(int4v{std::get<2>(kv.first), std::get<1>(kv.first), std::get<0>(kv.first),
                                kv.second});
    }
    for (long long t = 0; t < nbox; ++t) {
        int b1, b2, b3;
        coords(t, b1, b2, b3);
        const int c = (b1 & 1) + 2 * (b2 & 1) + 4 * (b3 & 1);
        int inside = 0;
        for (int i = start[c]; i < start[c] + count[c]; ++i) {
            const int s1 = b1 + out[i].x, s2 = b2 + out[i].y, s3 = b3 + out[i].z;
            inside += s1 >= 0 && s1 < nb1 && s2 >= 0 && s2 < nb1 && s3 >= 0 && (d == 2 || s3 < nb1);
        }
        if (inside != rowptr[t + 1] - rowptr[t]) return false;
    }
    return true;
}

// Offsets of a class list with at least one source inside the domain for the group
// (b23, c1, j) of G targets (the work of that group in the grouped kernel).
static long long group_valid(int d, int nb1, int G, int b23, int c1, int j,
                             const std::vector<int4v> &cl, const int *cs, const int *cc)
{
    const int b2 = b23 % nb1, b3 = d == 3 ? b23 / nb1 : 0, t0 = c1 + 2 * j * G;
    const int c = c1 + 2 * (b2 & 1) + 4 * (b3 & 1);
    long long v = 0;
    for (int i = cs[c]; i < cs[c] + cc[c]; ++i) {
        const int s2 = b2 + cl[i].y, s3 = b3 + cl[i].z, lo = t0 + cl[i].x;
        v += s2 >= 0 && s2 < nb1 && (d == 2 || (s3 >= 0 && s3 < nb1)) && lo + 2 * (G - 1) >= 0 &&
             lo < nb1;
    }
    return v;
}

// Groups of a level for Rp right-hand sides, heaviest first (ties in index order).
static std::vector<int> group_order(int d, int lv, int Rp, const std::vector<int4v> &cl,
                                    const int *cs, const int *cc)
{
    const int nb1 = 1 << lv, G = 128 / Rp, nq = (nb1 / 2 + G - 1) / G;
    const int nb23 = d == 3 ? nb1 * nb1 : nb1;
    std::vector<long long> w((size_t)nb23 * 2 * nq);
    for (int b23 = 0; b23 < nb23; ++b23)
        for (int c1 = 0; c1 < 2; ++c1)
            for (int j = 0; j < nq; ++j)
                w[((size_t)b23 * 2 + c1) * nq + j] = group_valid(d, nb1, G, b23, c1, j, cl, cs, cc);
    std::vector<int> ord(w.size());
    for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return w[a] > w[b]; });
    return ord;
}

// CUDA-core stream tasks: runs of consecutive entries of one block row holding about
// `task_bytes` of blocks each (at least one entry), a partial-sum slot of nrc x ld
// doubles per task, and per row the index of its first task (the reductions sum a row's
// partials in task order).  Rebuilt in place by the autotuner; device tables are
// replaced and `generation` moves on.
int build_tasks(htlr_handle *H, size_t task_bytes, cudaStream_t s)
{
    const int d = H->d, L = H->L;
    const int rows_leaf = (int)ipow(H->leaf, d);
    std::vector<Task> tasks;
    long long part = 0;
    auto make_tasks = [&](int kind, const std::vector<int> &rowptr, int nrows, size_t blk_bytes,
                          int ld, std::vector<int> &row_task) {
        long long per = std::max<long long>(1, (long long)(task_bytes / blk_bytes));
        row_task.assign(nrows + 1, 0);
        for (int t = 0; t < nrows; ++t) {
            row_task[t] = (int)tasks.size();
            for (long long e = rowptr[t]; e < rowptr[t + 1]; e += per) {
                Task T;
                T.kind = kind;
                T.row = t;
                T.e0 = (int)e;
                T.e1 = (int)std::min<long long>(rowptr[t + 1], e + per);
                T.part = part;
                part += (long long)H->nrc * ld;
                tasks.push_back(T);
            }
        }
        row_task[nrows] = (int)tasks.size();
    };
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        if (H->tc)
            Lv.row_task_begin.assign(Lv.nbox + 1, (int)tasks.size());  // no CUDA-core tasks
        else
            make_tasks(lv, Lv.far_rowptr, Lv.nbox, (size_t)Lv.ld * Lv.pd * prec_bytes(H->far_prec),
                       Lv.ld, Lv.row_task_begin);
    }
    const int near_task0 = (int)tasks.size();
    if (!H->near_generated) {
        if (H->near_prec == kPrecBF16X6)
            H->near_row_task.assign((1 << (d * L)) + 1, (int)tasks.size());
        else
            make_tasks(L + 1, H->near_rowptr, 1 << (d * L),
                       (size_t)H->near_ld * rows_leaf * prec_bytes(H->near_prec), H->near_ld,
                       H->near_row_task);
    }
    // replace the device tables
    HTLR_CK(cudaStreamSynchronize(s));
    HTLR_CK(cudaStreamSynchronize(H->stream));
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        dfree(H, Lv.d_row_task);
        if (dalloc(H, &Lv.d_row_task, Lv.row_task_begin.size())) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(Lv.d_row_task, Lv.row_task_begin.data(),
                                sizeof(int) * Lv.row_task_begin.size(), cudaMemcpyHostToDevice, s));
    }
    if (!H->near_generated) {
        dfree(H, H->d_near_row_task);
        if (dalloc(H, &H->d_near_row_task, H->near_row_task.size())) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(H->d_near_row_task, H->near_row_task.data(),
                                sizeof(int) * H->near_row_task.size(), cudaMemcpyHostToDevice, s));
    }
    if (part > H->part_doubles || !H->d_part) {
        dfree(H, H->d_part);
        if (dalloc(H, &H->d_part, (size_t)part)) return HTLR_ECUDA;
        H->part_doubles = part;
    }
    dfree(H, H->d_tasks);
    if (dalloc(H, &H->d_tasks, tasks.size())) return HTLR_ECUDA;
    HTLR_CK(cudaMemcpyAsync(H->d_tasks, tasks.data(), sizeof(Task) * tasks.size(),
                            cudaMemcpyHostToDevice, s));
    HTLR_CK(cudaStreamSynchronize(s));
    H->tasks.swap(tasks);
    H->near_task0 = near_task0;
    H->task_bytes = task_bytes;
    ++H->generation;
    return HTLR_OK;
}

static int build(htlr_handle *H, const htlr_grid *grid, const htlr_options *o)
{
    const int d = H->d, n = H->n, leaf = H->leaf, p = H->p, L = H->L;
    const long long N = (long long)ipow(n, d);
    cudaStream_t s = H->stream;
    H->h = 1.0 / n;
    H->wgt = std::pow(H->h, d);
    Temps tmp;

    if (dalloc(H, &H->d_err, 1)) return HTLR_ECUDA;
    HTLR_CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), s));
    if (grid && grid->a) {
        if (dalloc(H, &H->d_a, (size_t)N)) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(H->d_a, grid->a, sizeof(double) * N, cudaMemcpyHostToDevice, s));
    }

    // ---- grid lines, cells and the 1-D boxes of every level (§2.2, Def. 3.3) ----
    std::vector<double> xs((size_t)d * n), es((size_t)d * (n + 1)), ws((size_t)d * n);
    for (int l = 0; l < d; ++l)
        for (int i = 0; i <= n; ++i) {
            if (H->tensor) {
                es[(size_t)l * (n + 1) + i] = grid->edges[(size_t)l * (n + 1) + i];
                if (i < n) xs[(size_t)l * n + i] = grid->coords[(size_t)l * n + i];
            } else {
                es[(size_t)l * (n + 1) + i] = i * H->h;
                if (i < n) xs[(size_t)l * n + i] = (i + 0.5) * H->h;
            }
        }
    for (int l = 0; l < d; ++l)
        for (int i = 0; i < n; ++i)
            ws[(size_t)l * n + i] = es[(size_t)l * (n + 1) + i + 1] - es[(size_t)l * (n + 1) + i];
    if (dalloc(H, &H->d_coords, xs.size()) || dalloc(H, &H->d_edges, es.size()) ||
        dalloc(H, &H->d_width, ws.size()))
        return HTLR_ECUDA;
    HTLR_CK(cudaMemcpyAsync(H->d_coords, xs.data(), sizeof(double) * xs.size(),
                            cudaMemcpyHostToDevice, s));
    HTLR_CK(cudaMemcpyAsync(H->d_edges, es.data(), sizeof(double) * es.size(),
                            cudaMemcpyHostToDevice, s));
    HTLR_CK(cudaMemcpyAsync(H->d_width, ws.data(), sizeof(double) * ws.size(),
                            cudaMemcpyHostToDevice, s));
    H->lev.assign(L + 1, LevelData());
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        const int nb1 = 1 << lv;
        const double side = std::ldexp(1.0, -lv);
        int maxc = 0;
        for (int l = 0; l < d; ++l) {
            Lv.first[l].assign(nb1, 0);
            Lv.cnt[l].assign(nb1, 0);
            // grid lines with coordinate in the half-open cell [k side, (k+1) side)
            int i = 0;
            for (int k = 0; k < nb1; ++k) {
                const double hi = (k + 1) * side;
                Lv.first[l][k] = i;
                while (i < n && (xs[(size_t)l * n + i] < hi || k == nb1 - 1)) ++i;
                Lv.cnt[l][k] = i - Lv.first[l][k];
                if (Lv.cnt[l][k] < 1)
                    return fail(HTLR_EINVAL, "a box of the cluster tree holds no grid line "
                                             "(every node must be non-empty, Def. 2.1)");
                maxc = std::max(maxc, Lv.cnt[l][k]);
            }
        }
        Lv.maxcnt = maxc;
    }
    {
        const LevelData &Ll = H->lev[L];
        int rows = 1;
        for (int l = 0; l < d; ++l) rows *= Ll.maxcnt;
        H->max_leaf_rows = rows;
    }
    HTLR_CK(cudaStreamSynchronize(s));

    // ---- Nystrom diagonal (eq. (1.4)) ----
    {
        std::vector<double> gx, gw;
        gauss_legendre_host(H->q, gx, gw);
        double *d_g = nullptr;
        if (tmp.alloc(&d_g, 2 * H->q + 1)) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(d_g, gx.data(), sizeof(double) * H->q, cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaMemcpyAsync(d_g + H->q, gw.data(), sizeof(double) * H->q,
                                cudaMemcpyHostToDevice, s));
        launch_diag(H->kern, d, H->h, H->q, d_g, d_g + H->q, d_g + 2 * H->q, s);
        HTLR_CK(cudaGetLastError());
        HTLR_CK(cudaMemcpyAsync(&H->diag, d_g + 2 * H->q, sizeof(double), cudaMemcpyDeviceToHost, s));
        HTLR_CK(cudaStreamSynchronize(s));
    }

    // ---- block cluster tree walk (Def. 2.4), level by level ----
    std::vector<int> prev_rowptr = {0, 1}, prev_col = {0};
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        Lv.level = lv;
        Lv.nbox1 = 1 << lv;
        Lv.nbox = 1 << (d * lv);
        Lv.nb = n >> lv;
        const int nbox = Lv.nbox;
        int *d_prow, *d_pcol, *d_cnt, *d_off, *d_fcol, *d_ncol;
        if (tmp.alloc(&d_prow, prev_rowptr.size()) || tmp.alloc(&d_pcol, prev_col.size()) ||
            tmp.alloc(&d_cnt, 2 * (size_t)nbox) || tmp.alloc(&d_off, 2 * (size_t)nbox))
            return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(d_prow, prev_rowptr.data(), sizeof(int) * prev_rowptr.size(),
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaMemcpyAsync(d_pcol, prev_col.data(), sizeof(int) * prev_col.size(),
                                cudaMemcpyHostToDevice, s));
        launch_walk(0, d, lv, H->eta, d_prow, d_pcol, d_cnt, d_cnt + nbox, nullptr, nullptr,
                    nullptr, nullptr, s);
        HTLR_CK(cudaGetLastError());
        std::vector<int> cnt(2 * (size_t)nbox);
        HTLR_CK(cudaMemcpyAsync(cnt.data(), d_cnt, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, s));
        HTLR_CK(cudaStreamSynchronize(s));
        std::vector<int> off(2 * (size_t)nbox);
        Lv.far_rowptr.assign(nbox + 1, 0);
        std::vector<int> near_rowptr(nbox + 1, 0);
        for (int t = 0; t < nbox; ++t) {
            Lv.far_rowptr[t + 1] = Lv.far_rowptr[t] + cnt[t];
            near_rowptr[t + 1] = near_rowptr[t] + cnt[nbox + t];
            off[t] = Lv.far_rowptr[t];
            off[nbox + t] = near_rowptr[t];
        }
        Lv.nfar = Lv.far_rowptr[nbox];
        long long nnear = near_rowptr[nbox];
        if (tmp.alloc(&d_fcol, Lv.nfar) || tmp.alloc(&d_ncol, nnear)) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(d_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice, s));
        launch_walk(1, d, lv, H->eta, d_prow, d_pcol, nullptr, nullptr, d_off, d_off + nbox,
                    d_fcol, d_ncol, s);
        HTLR_CK(cudaGetLastError());
        Lv.far_col.resize(Lv.nfar);
        std::vector<int> near_col(nnear);
        if (Lv.nfar)
            HTLR_CK(cudaMemcpyAsync(Lv.far_col.data(), d_fcol, sizeof(int) * Lv.nfar,
                                    cudaMemcpyDeviceToHost, s));
        if (nnear)
            HTLR_CK(cudaMemcpyAsync(near_col.data(), d_ncol, sizeof(int) * nnear,
                                    cudaMemcpyDeviceToHost, s));
        HTLR_CK(cudaStreamSynchronize(s));
        prev_rowptr.swap(near_rowptr);
        prev_col.swap(near_col);
    }
    H->near_rowptr = prev_rowptr;
    H->near_col = prev_col;
    H->nnear = (int64_t)H->near_col.size();

    // ---- per-level shapes and the storage decision ----
    const int rows_leaf = ipow(leaf, d);  // uniform leaves (tensor leaves are ragged)
    H->near_rows = rows_leaf;
    H->near_ld = round_up(rows_leaf, 32);
    const int want0 = o ? o->storage : HTLR_STORE_AUTO;
    // a TF32X3 near field is generated on the tensor cores: AUTO storage generates it
    H->near_generated = (H->tensor || want0 == HTLR_STORE_GENERATED ||
                         (want0 == HTLR_STORE_AUTO && H->near_prec == kPrecTF32X3)) ? 1 : 0;
    if (H->near_prec == kPrecTF32X3 && !H->near_generated)
        return fail(HTLR_EUNSUPPORTED, "a TF32X3 near field is generated (tensor grids, "
                                       "HTLR_STORE_GENERATED or AUTO storage)");
    if (!H->near_generated && H->near_ld / 32 > 16)
        return fail(HTLR_EUNSUPPORTED,
                    "stored dense leaf blocks above 512 points are not supported (use "
                    "HTLR_STORE_GENERATED)");
    if (H->max_leaf_rows > 1024)
        return fail(HTLR_EUNSUPPORTED, "leaf boxes above 1024 points are not supported");
    int first_far = -1;
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        if (first_far < 0) first_far = lv;
        Lv.pe = H->orth ? std::min(p, Lv.nb) : p;
        Lv.pd = ipow(Lv.pe, d);
        Lv.ld = round_up(Lv.pd, 32);
        if (Lv.ld / 32 > 16)
            return fail(HTLR_EUNSUPPORTED, "p_eff^d above 512 is not supported");
        Lv.tg = tcg_shape(Lv.pd, Lv.pd);
    }
    H->near_tg = tcg_shape(rows_leaf, rows_leaf);
    // tensor-core stream: the far field on the tensor cores, the near field on the tensor
    // cores too, generated, or held in FP64 / df64 / FP32 for the CUDA-core stream
    if (H->near_prec == kPrecBF16X6 && (H->far_prec != kPrecBF16X6 || H->near_generated))
        return fail(HTLR_EUNSUPPORTED, "a BF16X6 near field needs stored dense blocks and a "
                                       "BF16X6 far field");
    H->tc = (H->far_prec == kPrecBF16X6) ? 1 : 0;

    // unique offsets (tau - sigma) per level and for the inadmissible leaves
    auto offset_key = [&](int tau, int sig, int level) {
        int bt[3], bs[3];
        box_index(tau, d, level, bt);
        box_index(sig, d, level, bs);
        return std::make_tuple(bt[0] - bs[0], bt[1] - bs[1], bt[2] - bs[2]);
    };
    std::vector<std::vector<int>> shared_id(L + 1);
    std::vector<std::vector<std::tuple<int, int, int>>> shared_off(L + 1);
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        std::map<std::tuple<int, int, int>, int> ids;
        shared_id[lv].resize(Lv.nfar);
        for (int t = 0; t < Lv.nbox; ++t)
            for (int e = Lv.far_rowptr[t]; e < Lv.far_rowptr[t + 1]; ++e) {
                auto key = offset_key(t, Lv.far_col[e], lv);
                auto it = ids.find(key);
                int id;
                if (it == ids.end()) {
                    id = (int)shared_off[lv].size();
                    ids[key] = id;
                    shared_off[lv].push_back(key);
                } else {
                    id = it->second;
                }
                shared_id[lv][e] = id;
            }
    }
    std::vector<int> near_shared_id(H->nnear);
    std::vector<std::tuple<int, int, int>> near_shared_off;
    {
        std::map<std::tuple<int, int, int>, int> ids;
        const int nleaf = 1 << (d * L);
        for (int t = 0; t < nleaf; ++t)
            for (int e = H->near_rowptr[t]; e < H->near_rowptr[t + 1]; ++e) {
                auto key = offset_key(t, H->near_col[e], L);
                auto it = ids.find(key);
                int id;
                if (it == ids.end()) {
                    id = (int)near_shared_off.size();
                    ids[key] = id;
                    near_shared_off.push_back(key);
                } else {
                    id = it->second;
                }
                near_shared_id[e] = id;
            }
    }

    // tasks: runs of consecutive entries of one row, about kTaskBytes of blocks each
    const size_t kTaskBytes = 256 * 1024;
    H->nrc = H->tc ? kTcRpMax : 4;
    auto count_tasks = [&](const std::vector<int> &rowptr, int nrows, size_t blk_bytes) {
        long long per = std::max<long long>(1, (long long)(kTaskBytes / blk_bytes));
        long long nt = 0;
        for (int t = 0; t < nrows; ++t) {
            long long m = rowptr[t + 1] - rowptr[t];
            nt += (m + per - 1) / per;
        }
        return std::make_pair(nt, per);
    };
    Sizes sz_stored, sz_shared;
    long long part_doubles = 0, ntasks = 0;
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        size_t blk = H->tc ? (size_t)Lv.tg.core_elems * 2
                           : (size_t)Lv.ld * Lv.pd * prec_bytes(H->far_prec);
        // tensor-core tasks are whole block rows (one per row)
        auto ct = count_tasks(Lv.far_rowptr, Lv.nbox, H->tc ? 1 : blk);
        ntasks += ct.first;
        part_doubles += ct.first * (long long)H->nrc * Lv.ld;
        sz_stored.cores += blk * Lv.nfar;
        sz_shared.cores += blk * shared_off[lv].size();
        size_t fac = sizeof(double) * (H->tensor ? 2 * (size_t)d * n * p
                                                 : 2 * (size_t)Lv.nb * p + (size_t)p * p);
        size_t work = 2 * sizeof(double) * (size_t)Lv.nbox * H->nrc * Lv.pd;
        size_t lists = sizeof(int) * (2 * (size_t)Lv.nfar + 2 * ((size_t)Lv.nbox + 1));
        for (Sizes *z : {&sz_stored, &sz_shared}) {
            z->factors += fac;
            z->work += work;
            z->lists += lists;
        }
    }
    if (H->near_generated) {
        // no dense blocks: the per-point diagonal and the near lists only
        sz_stored.near = sz_shared.near = sizeof(double) * (size_t)N;
        size_t lists = sizeof(int) * ((size_t)H->nnear + (size_t)(1 << (d * L)) + 1);
        size_t work = sizeof(double) * part_doubles + sizeof(Task) * ntasks;
        for (Sizes *z : {&sz_stored, &sz_shared}) {
            z->lists += lists;
            z->work += work;
        }
    } else {
        size_t blk = H->near_prec == kPrecBF16X6
                         ? (size_t)H->near_tg.core_elems * 2
                         : (size_t)H->near_ld * rows_leaf * prec_bytes(H->near_prec);
        auto ct = count_tasks(H->near_rowptr, 1 << (d * L), H->near_prec == kPrecBF16X6 ? 1 : blk);
        ntasks += ct.first;
        part_doubles += ct.first * (long long)H->nrc * H->near_ld;
        sz_stored.near = blk * H->nnear;
        sz_shared.near = blk * near_shared_off.size();
        size_t lists = sizeof(int) * (2 * (size_t)H->nnear + 2 * ((size_t)(1 << (d * L)) + 1));
        size_t work = sizeof(double) * part_doubles + sizeof(Task) * ntasks;
        for (Sizes *z : {&sz_stored, &sz_shared}) {
            z->lists += lists;
            z->work += work;
        }
    }
    size_t limit = o ? o->hbm_limit : 0;
    if (limit == 0) {
        size_t fr = 0, tot = 0;
        HTLR_CK(cudaMemGetInfo(&fr, &tot));
        limit = (size_t)(0.9 * (double)fr);
    }
    int want = o ? o->storage : HTLR_STORE_AUTO;
    if (want == HTLR_STORE_GENERATED) want = HTLR_STORE_SHARED;  // cores per offset
    if (want == HTLR_STORE_AUTO) {
        if (H->tensor) want = HTLR_STORE_SHARED;
        else want = sz_stored.total() <= limit ? HTLR_STORE_STORED : HTLR_STORE_SHARED;
    }
    if (want != HTLR_STORE_STORED && want != HTLR_STORE_SHARED)
        return fail(HTLR_EINVAL, "options.storage must be AUTO, STORED, SHARED or GENERATED");
    if (H->tc && want == HTLR_STORE_STORED) {
        if (o && o->storage == HTLR_STORE_STORED)
            return fail(HTLR_EUNSUPPORTED,
                        "BF16X6 block lists are held one block per level and box offset "
                        "(SHARED or GENERATED storage), where the grouped tensor-core kernel "
                        "reads each block once for a group of targets; STORED blocks take "
                        "FP64, df64 or FP32");
        want = HTLR_STORE_SHARED;
    }
    const Sizes &sz = (want == HTLR_STORE_STORED) ? sz_stored : sz_shared;
    if (sz.total() > limit) {
        char buf[256];
        snprintf(buf, sizeof buf, "footprint %.3f GB exceeds the limit %.3f GB (storage %s)",
                 sz.total() / 1e9, limit / 1e9, want == HTLR_STORE_STORED ? "STORED" : "SHARED");
        return fail(HTLR_ENOMEM, buf);
    }
    H->storage = want;
    const bool stored = (want == HTLR_STORE_STORED);

    // ---- factors, cores, dense blocks (Algorithm 1) ----
    long long pdf = ipow(p, d);
    long long scratch_per = 2 * pdf * pdf;
    int nscr = (int)std::max<long long>(1, std::min<long long>(2 * 152, (512ll << 20) / (8 * scratch_per)));
    double *d_scratch = nullptr;
    if (first_far >= 0 && tmp.alloc(&d_scratch, (size_t)nscr * scratch_per)) return HTLR_ECUDA;
    // box geometry and factor offsets of every level (the leaf level is needed by the
    // output and the generated near field even without admissible blocks)
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        const int nb1 = 1 << lv;
        const int pe = Lv.nfar ? Lv.pe : p;
        size_t pool = 0;
        for (int l = 0; l < d; ++l) {
            Lv.uoff[l].assign(nb1, 0);
            Lv.voff[l].assign(nb1, 0);
            if (H->tensor)
                for (int k = 0; k < nb1; ++k) {
                    Lv.uoff[l][k] = Lv.voff[l][k] = (int)pool;
                    pool += (size_t)Lv.cnt[l][k] * pe;
                }
        }
        std::vector<int> geo((size_t)d * 4 * nb1);
        for (int l = 0; l < d; ++l)
            for (int k = 0; k < nb1; ++k) {
                geo[(size_t)l * 4 * nb1 + k] = Lv.first[l][k];
                geo[(size_t)l * 4 * nb1 + nb1 + k] = Lv.cnt[l][k];
                geo[(size_t)l * 4 * nb1 + 2 * nb1 + k] = Lv.uoff[l][k];
                geo[(size_t)l * 4 * nb1 + 3 * nb1 + k] = Lv.voff[l][k];
            }
        if (dalloc(H, &Lv.d_geo, geo.size())) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(Lv.d_geo, geo.data(), sizeof(int) * geo.size(),
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaStreamSynchronize(s));
        if (Lv.nfar == 0) continue;
        if (dalloc(H, &Lv.d_R, (size_t)p * p)) return HTLR_ECUDA;
        const double side = std::ldexp(1.0, -lv);
        if (H->tensor) {
            // per-box factors; the cell widths sit in V (no orthogonalisation)
            if (dalloc(H, &Lv.d_Upool, pool) || dalloc(H, &Lv.d_Vpool, pool)) return HTLR_ECUDA;
            launch_factor_tensor(d, n, lv, p, H->d_coords, H->d_width, Lv.d_geo, Lv.d_Upool,
                                 Lv.d_Vpool, s);
        } else {
            if (dalloc(H, &Lv.d_F, 2 * (size_t)Lv.nb * p)) return HTLR_ECUDA;
            launch_factor(Lv.nb, p, Lv.pe, side, H->h, H->orth, Lv.d_F, Lv.d_R, s);
            Lv.d_Upool = Lv.d_Vpool = Lv.d_F;
        }
        HTLR_CK(cudaGetLastError());
    }
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        const double side = std::ldexp(1.0, -lv);
        // core per block (STORED) or per offset (SHARED)
        std::vector<int> offs;
        if (stored) {
            Lv.far_core.resize(Lv.nfar);
            offs.resize(3 * (size_t)Lv.nfar);
            for (int t = 0; t < Lv.nbox; ++t)
                for (int e = Lv.far_rowptr[t]; e < Lv.far_rowptr[t + 1]; ++e) {
                    auto key = offset_key(t, Lv.far_col[e], lv);
                    offs[3 * (size_t)e] = std::get<0>(key);
                    offs[3 * (size_t)e + 1] = std::get<1>(key);
                    offs[3 * (size_t)e + 2] = std::get<2>(key);
                    Lv.far_core[e] = e;
                }
            Lv.ncores = Lv.nfar;
        } else {
            Lv.far_core = shared_id[lv];
            Lv.ncores = (int64_t)shared_off[lv].size();
            offs.resize(3 * (size_t)Lv.ncores);
            for (size_t c = 0; c < shared_off[lv].size(); ++c) {
                offs[3 * c] = std::get<0>(shared_off[lv][c]);
                offs[3 * c + 1] = std::get<1>(shared_off[lv][c]);
                offs[3 * c + 2] = std::get<2>(shared_off[lv][c]);
            }
        }
        int *d_offs = nullptr;
        if (tmp.alloc(&d_offs, offs.size())) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice, s));
        {
            // cores are formed in FP64, then kept as FP64, split in place into (hi, lo)
            // float pairs (df64), or converted to FP32
            const size_t nel = (size_t)Lv.ncores * Lv.ld * Lv.pd;
            double *dcore = nullptr;
            if (H->far_prec == kPrecFP32 || H->far_prec == kPrecBF16X6) {
                HTLR_CK(device_malloc((void **)&dcore, nel * sizeof(double)));
            } else if (dalloc(H, &dcore, nel)) {
                return HTLR_ECUDA;
            }
            // uniform grid: the weight h^d multiplies the core (Algorithm 1); tensor grid:
            // the cell widths are already in V
            launch_cores(H->kern, d, p, Lv.pe, Lv.ld, H->orth, side, H->tensor ? 1.0 : H->wgt,
                         Lv.d_R, Lv.ncores, d_offs, dcore, d_scratch, nscr, s);
            HTLR_CK(cudaGetLastError());
            Lv.d_cores = dcore;
            if (H->far_prec == kPrecDF64) launch_split_df64(dcore, nel, s);
            if (H->far_prec == kPrecFP32) {
                float *f32 = nullptr;
                int rc2 = dalloc(H, &f32, nel);
                if (rc2 == HTLR_OK) launch_to_fp32(dcore, f32, nel, s);
                cudaError_t e2 = cudaStreamSynchronize(s);
                cudaFree(dcore);
                if (rc2) return rc2;
                HTLR_CK(e2);
                Lv.d_cores = f32;
            }
            if (H->far_prec == kPrecBF16X6) {
                // packed split-BF16 chunks for the grouped tensor-core stream (one block per
                // offset): the level's offsets must form parity classes
                std::vector<int4v> cl;
                Lv.tg = tcg_shape(Lv.pd, Lv.pd);
                Lv.tcg = build_classes(d, 1 << lv, Lv.far_rowptr, Lv.far_col, Lv.far_core, cl,
                                       Lv.cls_start, Lv.cls_count);
                if (!Lv.tcg) {
                    cudaFree(dcore);
                    return fail(HTLR_EUNSUPPORTED, "BF16X6: the admissible offsets of a level do "
                                                   "not form parity classes");
                }
                Lv.h_cls = cl;
                if (dalloc(H, &Lv.d_cls, cl.size())) {
                    cudaFree(dcore);
                    return HTLR_ECUDA;
                }
                HTLR_CK(cudaMemcpyAsync(Lv.d_cls, cl.data(), sizeof(int4v) * cl.size(),
                                        cudaMemcpyHostToDevice, s));
                uint16_t *pk = nullptr;
                int rc2 = dalloc(H, &pk, (size_t)Lv.ncores * Lv.tg.core_elems);
                if (rc2 == HTLR_OK)
                    launch_tcg_pack_blocks(dcore, Lv.ncores, Lv.ld, Lv.pd, Lv.pd, Lv.tg.nch,
                                           Lv.tg.NGb, pk, s);
                cudaError_t e2 = cudaStreamSynchronize(s);
                cudaFree(dcore);
                if (rc2) return rc2;
                HTLR_CK(e2);
                Lv.d_cores = pk;
            }
            HTLR_CK(cudaGetLastError());
        }
        // lists
        if (dalloc(H, &Lv.d_far_col, Lv.nfar) || dalloc(H, &Lv.d_far_core, Lv.nfar) ||
            dalloc(H, &Lv.d_W, (size_t)Lv.nbox * H->nrc * Lv.pd) ||
            dalloc(H, &Lv.d_H, (size_t)Lv.nbox * H->nrc * Lv.pd))
            return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(Lv.d_far_col, Lv.far_col.data(), sizeof(int) * Lv.nfar,
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaMemcpyAsync(Lv.d_far_core, Lv.far_core.data(), sizeof(int) * Lv.nfar,
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaStreamSynchronize(s));  // offs / far_core host buffers go out of scope
    }
    // inadmissible leaves, generated: per-point diagonal and the near lists only
    if (H->near_generated) {
        if (dalloc(H, &H->d_diagpts, (size_t)N) || dalloc(H, &H->d_near_col, H->nnear) ||
            dalloc(H, &H->d_near_rowptr, H->near_rowptr.size()))
            return HTLR_ECUDA;
        if (H->tensor) {
            std::vector<double> gx, gw;
            gauss_legendre_host(H->q, gx, gw);
            double *d_g = nullptr;
            if (tmp.alloc(&d_g, 2 * (size_t)H->q)) return HTLR_ECUDA;
            HTLR_CK(cudaMemcpyAsync(d_g, gx.data(), sizeof(double) * H->q, cudaMemcpyHostToDevice, s));
            HTLR_CK(cudaMemcpyAsync(d_g + H->q, gw.data(), sizeof(double) * H->q,
                                    cudaMemcpyHostToDevice, s));
            launch_diag_points(H->kern, d, n, H->d_coords, H->d_edges, H->q, d_g, d_g + H->q,
                               H->d_diagpts, s);
            HTLR_CK(cudaGetLastError());
        } else {
            std::vector<double> dv((size_t)N, H->diag);  // the same integral at every point
            HTLR_CK(cudaMemcpyAsync(H->d_diagpts, dv.data(), sizeof(double) * N,
                                    cudaMemcpyHostToDevice, s));
            HTLR_CK(cudaStreamSynchronize(s));
        }
        HTLR_CK(cudaMemcpyAsync(H->d_near_col, H->near_col.data(), sizeof(int) * H->nnear,
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaMemcpyAsync(H->d_near_rowptr, H->near_rowptr.data(),
                                sizeof(int) * H->near_rowptr.size(), cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaStreamSynchronize(s));
        H->nnear_unique = 0;
    }
    // dense inadmissible leaves
    if (!H->near_generated) {
        std::vector<int> offs, taus;
        if (stored) {
            H->near_blk.resize(H->nnear);
            offs.resize(3 * (size_t)H->nnear);
            taus.resize(H->nnear);
            const int nleaf = 1 << (d * L);
            for (int t = 0; t < nleaf; ++t)
                for (int e = H->near_rowptr[t]; e < H->near_rowptr[t + 1]; ++e) {
                    auto key = offset_key(t, H->near_col[e], L);
                    offs[3 * (size_t)e] = std::get<0>(key);
                    offs[3 * (size_t)e + 1] = std::get<1>(key);
                    offs[3 * (size_t)e + 2] = std::get<2>(key);
                    taus[e] = t;
                    H->near_blk[e] = e;
                }
            H->nnear_unique = H->nnear;
        } else {
            H->near_blk = near_shared_id;
            H->nnear_unique = (int64_t)near_shared_off.size();
            offs.resize(3 * (size_t)H->nnear_unique);
            for (size_t c = 0; c < near_shared_off.size(); ++c) {
                offs[3 * c] = std::get<0>(near_shared_off[c]);
                offs[3 * c + 1] = std::get<1>(near_shared_off[c]);
                offs[3 * c + 2] = std::get<2>(near_shared_off[c]);
            }
        }
        int *d_offs = nullptr, *d_taus = nullptr;
        if (tmp.alloc(&d_offs, offs.size()) || tmp.alloc(&d_taus, taus.size())) return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(d_offs, offs.data(), sizeof(int) * offs.size(), cudaMemcpyHostToDevice, s));
        if (!taus.empty())
            HTLR_CK(cudaMemcpyAsync(d_taus, taus.data(), sizeof(int) * taus.size(),
                                    cudaMemcpyHostToDevice, s));
        if (dalloc(H, &H->d_near_col, H->nnear) || dalloc(H, &H->d_near_blk, H->nnear))
            return HTLR_ECUDA;
        const size_t nel = (size_t)H->nnear_unique * H->near_ld * rows_leaf;
        double *dnear = nullptr;
        if (H->near_prec == kPrecFP32 || H->near_prec == kPrecBF16X6) {
            HTLR_CK(device_malloc((void **)&dnear, nel * sizeof(double)));
        } else if (dalloc(H, &dnear, nel)) {
            return HTLR_ECUDA;
        }
        launch_near(H->kern, d, n, leaf, H->near_ld, H->h, H->wgt, H->diag,
                    stored ? H->d_a : nullptr, H->nnear_unique, d_offs, stored ? d_taus : nullptr,
                    dnear, s);
        HTLR_CK(cudaGetLastError());
        H->d_near = dnear;
        if (H->near_prec == kPrecDF64) launch_split_df64(dnear, nel, s);
        if (H->near_prec == kPrecFP32) {
            float *f32 = nullptr;
            int rc2 = dalloc(H, &f32, nel);
            if (rc2 == HTLR_OK) launch_to_fp32(dnear, f32, nel, s);
            cudaError_t e2 = cudaStreamSynchronize(s);
            cudaFree(dnear);
            if (rc2) return rc2;
            HTLR_CK(e2);
            H->d_near = f32;
        }
        if (H->near_prec == kPrecBF16X6) {
            // the diagonal entries (K_ii w_i, with a_i when folded) stay out of the split
            // blocks: out_kernel adds them to f in FP64
            std::vector<int> ids;
            const int nleaf = 1 << (d * L);
            for (int t = 0; t < nleaf; ++t)
                for (int e = H->near_rowptr[t]; e < H->near_rowptr[t + 1]; ++e)
                    if (H->near_col[e] == t) ids.push_back(H->near_blk[e]);
            std::sort(ids.begin(), ids.end());
            ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
            int *d_ids = nullptr;
            if (tmp.alloc(&d_ids, ids.size())) return HTLR_ECUDA;
            HTLR_CK(cudaMemcpyAsync(d_ids, ids.data(), sizeof(int) * ids.size(),
                                    cudaMemcpyHostToDevice, s));
            launch_zero_diag(dnear, H->near_ld, rows_leaf, d_ids, (int)ids.size(), s);
            std::vector<double> dv((size_t)N, H->diag);
            if (dalloc(H, &H->d_diagpts, (size_t)N)) return HTLR_ECUDA;
            HTLR_CK(cudaMemcpyAsync(H->d_diagpts, dv.data(), sizeof(double) * N,
                                    cudaMemcpyHostToDevice, s));
            HTLR_CK(cudaStreamSynchronize(s));
            std::vector<int4v> cl;
            H->near_tg = tcg_shape(rows_leaf, rows_leaf);
            H->near_tcg = build_classes(d, 1 << L, H->near_rowptr, H->near_col, H->near_blk, cl,
                                        H->near_cls_start, H->near_cls_count);
            if (!H->near_tcg) {
                cudaFree(dnear);
                return fail(HTLR_EUNSUPPORTED, "BF16X6: the inadmissible offsets of the leaves "
                                               "do not form parity classes");
            }
            H->h_near_cls = cl;
            if (dalloc(H, &H->d_near_cls, cl.size())) {
                cudaFree(dnear);
                return HTLR_ECUDA;
            }
            HTLR_CK(cudaMemcpyAsync(H->d_near_cls, cl.data(), sizeof(int4v) * cl.size(),
                                    cudaMemcpyHostToDevice, s));
            uint16_t *pk = nullptr;
            int rc2 = dalloc(H, &pk, (size_t)H->nnear_unique * H->near_tg.core_elems);
            if (rc2 == HTLR_OK)
                launch_tcg_pack_blocks(dnear, H->nnear_unique, H->near_ld, rows_leaf, rows_leaf,
                                       H->near_tg.nch, H->near_tg.NGb, pk, s);
            cudaError_t e2 = cudaStreamSynchronize(s);
            cudaFree(dnear);
            if (rc2) return rc2;
            HTLR_CK(e2);
            H->d_near = pk;
        }
        HTLR_CK(cudaGetLastError());
        HTLR_CK(cudaMemcpyAsync(H->d_near_col, H->near_col.data(), sizeof(int) * H->nnear,
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaMemcpyAsync(H->d_near_blk, H->near_blk.data(), sizeof(int) * H->nnear,
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaStreamSynchronize(s));
    }

    // ---- kinds (block lists per level + the near list); tasks follow ----
    H->kinds.assign(L + 2, KindDesc{});
    int max_cols = 1;
    for (int lv = 1; lv <= L; ++lv) {
        LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        KindDesc &K = H->kinds[lv];
        K.col = Lv.d_far_col;
        K.blk = Lv.d_far_core;
        K.blocks = Lv.d_cores;
        K.blk_stride = (long long)Lv.ld * Lv.pd;
        K.prec = H->far_prec;
        K.ld = Lv.ld;
        K.rows = Lv.pd;
        K.cols = Lv.pd;
        K.rpl = Lv.ld / 32;
        K.is_near = 0;
        K.x = Lv.d_W;
        K.x_box_stride = (long long)H->nrc * Lv.pd;
        max_cols = std::max(max_cols, Lv.pd);
    }
    if (!H->near_generated) {
        KindDesc &K = H->kinds[L + 1];
        K.col = H->d_near_col;
        K.blk = H->d_near_blk;
        K.blocks = H->d_near;
        K.blk_stride = (long long)H->near_ld * rows_leaf;
        K.prec = H->near_prec;
        K.ld = H->near_ld;
        K.rows = rows_leaf;
        K.cols = rows_leaf;
        K.rpl = H->near_ld / 32;
        K.is_near = 1;
        K.x = nullptr;
        K.x_box_stride = 0;
        max_cols = std::max(max_cols, rows_leaf);
    }
    // tensor-core stream: one task per non-empty block row, partials for kTcRpMax RHS
    if (H->tc) {
        long long ptc = 0;
        auto row_tasks = [&](int kind, const std::vector<int> &rowptr, int nrows, int ld,
                             std::vector<int> &row_task) {
            row_task.assign(nrows + 1, 0);
            for (int t = 0; t < nrows; ++t) {
                row_task[t] = (int)H->tasks_tc.size();
                if (rowptr[t + 1] > rowptr[t]) {
                    Task T;
                    T.kind = kind;
                    T.row = t;
                    T.e0 = rowptr[t];
                    T.e1 = rowptr[t + 1];
                    T.part = ptc;
                    ptc += (long long)kTcRpMax * ld;
                    H->tasks_tc.push_back(T);
                }
            }
            row_task[nrows] = (int)H->tasks_tc.size();
        };
        for (int lv = 1; lv <= L; ++lv) {
            LevelData &Lv = H->lev[lv];
            if (Lv.nfar == 0) continue;
            row_tasks(lv, Lv.far_rowptr, Lv.nbox, Lv.ld, Lv.row_task_tc);
            if (dalloc(H, &Lv.d_row_task_tc, Lv.row_task_tc.size()))
                return HTLR_ECUDA;
            {
                if (dalloc(H, &Lv.d_Wg, (size_t)Lv.nbox * Lv.tg.box_elems)) return HTLR_ECUDA;
                for (int k = 0; k < 3; ++k) {
                    if (tcg_encode_source_map(Lv.tmap[k].b, Lv.d_Wg, Lv.tg.nch, 16 << k, 1 << lv, d))
                        return fail(HTLR_ECUDA, "tensor map encoding failed");
                    std::vector<int> ord =
                        group_order(d, lv, 16 << k, Lv.h_cls, Lv.cls_start, Lv.cls_count);
                    if (dalloc(H, &Lv.d_order[k], ord.size())) return HTLR_ECUDA;
                    HTLR_CK(cudaMemcpyAsync(Lv.d_order[k], ord.data(), sizeof(int) * ord.size(),
                                            cudaMemcpyHostToDevice, s));
                    HTLR_CK(cudaStreamSynchronize(s));
                }
            }
            HTLR_CK(cudaMemcpyAsync(Lv.d_row_task_tc, Lv.row_task_tc.data(),
                                    sizeof(int) * Lv.row_task_tc.size(), cudaMemcpyHostToDevice, s));
        }
        if (H->near_prec == kPrecBF16X6) {
            row_tasks(L + 1, H->near_rowptr, 1 << (d * L), H->near_ld, H->near_row_task_tc);
            if (dalloc(H, &H->d_near_row_task_tc, H->near_row_task_tc.size())) return HTLR_ECUDA;
            {
                if (dalloc(H, &H->d_Ug, (size_t)(1 << (d * L)) * H->near_tg.box_elems))
                    return HTLR_ECUDA;
                for (int k = 0; k < 3; ++k) {
                    if (tcg_encode_source_map(H->near_tmap[k].b, H->d_Ug, H->near_tg.nch, 16 << k,
                                              1 << L, d))
                        return fail(HTLR_ECUDA, "tensor map encoding failed");
                    std::vector<int> ord = group_order(d, L, 16 << k, H->h_near_cls,
                                                       H->near_cls_start, H->near_cls_count);
                    if (dalloc(H, &H->d_near_order[k], ord.size())) return HTLR_ECUDA;
                    HTLR_CK(cudaMemcpyAsync(H->d_near_order[k], ord.data(), sizeof(int) * ord.size(),
                                            cudaMemcpyHostToDevice, s));
                    HTLR_CK(cudaStreamSynchronize(s));
                }
            }
            HTLR_CK(cudaMemcpyAsync(H->d_near_row_task_tc, H->near_row_task_tc.data(),
                                    sizeof(int) * H->near_row_task_tc.size(),
                                    cudaMemcpyHostToDevice, s));
        }
        if (dalloc(H, &H->d_tasks_tc, H->tasks_tc.size()) || dalloc(H, &H->d_part_tc, (size_t)ptc) ||
            dalloc(H, &H->d_grp_counter, (size_t)L + 2))
            return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(H->d_tasks_tc, H->tasks_tc.data(), sizeof(Task) * H->tasks_tc.size(),
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaStreamSynchronize(s));
    }
    // generated near field on the tensor cores: per leaf its first 16-source stage of
    // packed w u, and the (leaf, tile of near_tc_tile_rows() rows) items, heaviest first
    if (H->near_generated && H->near_prec == kPrecTF32X3) {
        const int nleaf = 1 << (d * L), m1 = (1 << L) - 1;
        const LevelData &Lf = H->lev[L];
        std::vector<int> stage0((size_t)nleaf + 1, 0), rows(nleaf);
        int max_rows = 0;
        for (int g = 0; g < nleaf; ++g) {
            int r = 1;
            for (int k = 0; k < d; ++k) r *= Lf.cnt[k][(g >> (L * k)) & m1];
            rows[g] = r;
            max_rows = std::max(max_rows, r);
            stage0[g + 1] = stage0[g] + (r + 15) / 16;
        }
        std::vector<long long> wgt;
        std::vector<int> it;
        for (int g = 0; g < nleaf; ++g) {
            long long st = 0;
            for (int e = H->near_rowptr[g]; e < H->near_rowptr[g + 1]; ++e)
                st += stage0[H->near_col[e] + 1] - stage0[H->near_col[e]];
            for (int tl = 0; tl * near_tc_tile_rows() < rows[g]; ++tl) {
                it.push_back(g);
                it.push_back(tl);
                wgt.push_back(st);
            }
        }
        std::vector<int> ord(wgt.size());
        for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return wgt[a] > wgt[b]; });
        std::vector<int> items(it.size());
        for (size_t i = 0; i < ord.size(); ++i) {
            items[2 * i] = it[2 * (size_t)ord[i]];
            items[2 * i + 1] = it[2 * (size_t)ord[i] + 1];
        }
        H->ntc_nitems = (int)ord.size();
        H->ntc_max_rows_pad = round_up(max_rows, 16);
        if (dalloc(H, &H->d_ntc_stage0, stage0.size()) || dalloc(H, &H->d_ntc_items, items.size()) ||
            dalloc(H, &H->d_ntc_wu, (size_t)stage0[nleaf] * 512) || dalloc(H, &H->d_ntc_counter, 1))
            return HTLR_ECUDA;
        HTLR_CK(cudaMemcpyAsync(H->d_ntc_stage0, stage0.data(), sizeof(int) * stage0.size(),
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaMemcpyAsync(H->d_ntc_items, items.data(), sizeof(int) * items.size(),
                                cudaMemcpyHostToDevice, s));
        HTLR_CK(cudaStreamSynchronize(s));
    }
    H->max_cols = max_cols;
    H->task_bytes = kTaskBytes;
    if (int rc = build_tasks(H, kTaskBytes, s)) return rc;
    if (dalloc(H, &H->d_kinds, H->kinds.size())) return HTLR_ECUDA;
    HTLR_CK(cudaMemcpyAsync(H->d_kinds, H->kinds.data(), sizeof(KindDesc) * H->kinds.size(),
                            cudaMemcpyHostToDevice, s));
    HTLR_CK(cudaStreamSynchronize(s));

    // ---- statistics ----
    htlr_stats &st = H->stats;
    std::memset(&st, 0, sizeof st);
    st.d = d;
    st.n = n;
    st.levels = L;
    st.p = p;
    st.storage = H->near_generated ? HTLR_STORE_GENERATED : H->storage;
    st.p_eff_leaf = H->orth ? std::min(p, leaf) : p;
    double paper = 0.0;
    for (int lv = 1; lv <= L; ++lv) {
        const LevelData &Lv = H->lev[lv];
        st.far_per_level[lv] = Lv.nfar;
        st.unique_cores += Lv.ncores;
        int pe = std::min(p, Lv.nb);
        paper += (double)Lv.nfar * (std::pow((double)pe, 2 * d) + 2.0 * d * Lv.nb * pe);
    }
    paper += (double)H->nnear * rows_leaf * (double)rows_leaf;
    st.near_blocks = H->nnear;
    {
        // point pairs of the near field: sum over inadmissible leaf pairs of |tau| |sigma|
        const LevelData &Ll = H->lev[L];
        auto pts = [&](int g) {
            long long c = 1;
            for (int k = 0; k < d; ++k) c *= Ll.cnt[k][(g >> (L * k)) & ((1 << L) - 1)];
            return c;
        };
        long long pairs = 0;
        for (int t = 0; t < (1 << (d * L)); ++t)
            for (int e = H->near_rowptr[t]; e < H->near_rowptr[t + 1]; ++e)
                pairs += pts(t) * pts(H->near_col[e]);
        st.near_point_pairs = pairs;
    }
    st.unique_near = H->nnear_unique;
    st.paper_storage_doubles = paper;
    st.bytes_cores = sz.cores;
    st.bytes_near = sz.near;
    st.bytes_factors = sz.factors;
    st.bytes_work = sz.work + sz.lists;
    st.bytes_total = sz.total();
    st.diag_value = H->diag;
    st.far_precision = H->far_prec;
    st.near_precision = H->near_prec;
    st.tc_grouped = H->near_tcg ? (int)(1u << 31) : 0;
    for (int lv = 1; lv <= L; ++lv)
        if (H->lev[lv].tcg) st.tc_grouped |= 1 << lv;
    return HTLR_OK;
}

static void destroy(htlr_handle *H)
{
    if (!H) return;
    for (void *q : H->allocs) cudaFree(q);
    if (H->d_stage_u) cudaFree(H->d_stage_u);
    if (H->d_stage_f) cudaFree(H->d_stage_f);
    H->allocs.clear();
    H->magic = kMagicDead;
    delete H;
}

static bool is_live(const htlr_handle *H)
{
    std::lock_guard<std::mutex> g(g_live_mu);
    return H && g_live.count(H) && H->magic == kMagicLive;
}

// Events bracketing the stages of one matvec (optional).
struct StageEvents {
    cudaEvent_t ev[2 * HTLR_NUM_STAGES];
    float ms[HTLR_NUM_STAGES];
};

bool handle_is_live(const htlr_handle *H) { return is_live(H); }

// The block stream of one RHS chunk: one launch when far and near blocks share a
// precision, else one launch per part.  Returns the number of launches.
int launch_streams(const htlr_handle *H, const KindDesc *d_kinds, const double *u, long long ldu,
                   int nh, double *part, cudaStream_t s)
{
    StreamArgs a;
    a.tasks = H->d_tasks;
    a.kinds = d_kinds;
    a.d = H->d;
    a.n = H->n;
    a.leaf = H->leaf;
    a.nl_level = leaf_level(H->n, H->leaf);
    a.u = u;
    a.ldu = ldu;
    a.nrhs = nh;
    a.max_cols = H->max_cols;
    a.part = part;
    a.err = H->d_err;
    a.streaming = H->storage == HTLR_STORE_STORED;
    a.stream = s;
    a.threads = H->stream_threads;
    a.ctas_per_sm = H->stream_ctas_per_sm;
    const int nt = (int)H->tasks.size();
    if (H->far_prec == H->near_prec) {
        a.t0 = 0;
        a.t1 = nt;
        launch_stream(H->far_prec, a);
        return 1;
    }
    a.t0 = 0;
    a.t1 = H->near_task0;
    launch_stream(H->far_prec, a);
    a.t0 = H->near_task0;
    a.t1 = nt;
    launch_stream(H->near_prec, a);
    return 2;
}

// Device view of a level's box geometry and factors.
LevelGeom level_geom(const htlr_handle *H, int lv)
{
    const LevelData &Lv = H->lev[lv];
    const int nb1 = 1 << lv;
    LevelGeom g{};
    for (int l = 0; l < 3; ++l) {
        const int *base = Lv.d_geo + (size_t)(l < H->d ? l : 0) * 4 * nb1;
        g.first[l] = base;
        g.cnt[l] = base + nb1;
        g.uoff[l] = base + 2 * nb1;
        g.voff[l] = base + 3 * nb1;
    }
    g.Upool = Lv.d_Upool;
    g.Vpool = Lv.d_Vpool;
    g.level = lv;
    g.pe = Lv.pe;
    g.pd = Lv.pd;
    g.maxcnt = Lv.maxcnt;
    return g;
}

// One RHS chunk of HMultVec (stages: up, stream [+ generated near], reduce, out) with the
// given scratch: W[lv], Hs[lv] per level, task partials, the kinds table.
// The generated near field for all right-hand sides at once (its kernel values are
// evaluated once per point pair and shared by up to 16 RHS per pass), written into f
// before the chunks add their far fields.
int launch_near_gen_all(const htlr_handle *H, const double *uc, double *fc, int nh, cudaStream_t s)
{
    if (!H->near_generated) return 0;
    const int d = H->d, n = H->n, L = H->L;
    const long long N = (long long)ipow(n, d);
    int launches = 0;
    if (H->near_prec == kPrecTF32X3) {
        // tensor cores: 16 right-hand sides per launch (packing of w u, then the product)
        NearTcArgs t{};
        t.k = H->kern;
        t.d = d;
        t.n = n;
        t.L = L;
        t.leafg = level_geom(H, L);
        t.coords = H->d_coords;
        t.width = H->d_width;
        t.diag = H->d_diagpts;
        t.a = H->d_a;
        t.rowptr = H->d_near_rowptr;
        t.col = H->d_near_col;
        t.stage0 = H->d_ntc_stage0;
        t.items = H->d_ntc_items;
        t.nitems = H->ntc_nitems;
        t.wu = H->d_ntc_wu;
        t.u = uc;
        t.ldu = N;
        t.f = fc;
        t.ldf = N;
        t.max_rows_pad = H->ntc_max_rows_pad;
        t.counter = H->d_ntc_counter;
        t.err = H->d_err;
        t.wait_cycles = H->tc_wait_cycles;
        for (int r0 = 0; r0 < nh; r0 += 16) {
            t.r0 = r0;
            t.nr = std::min(16, nh - r0);
            launch_near_tc(t, s);
            launches += 2;
        }
        return launches;
    }
    {
        NearGenArgs g{};
        g.k = H->kern;
        g.d = d;
        g.n = n;
        g.L = L;
        g.nrhs = nh;
        g.leafg = level_geom(H, L);
        g.coords = H->d_coords;
        g.width = H->d_width;
        g.diag = H->d_diagpts;
        g.a = H->d_a;
        g.rowptr = H->d_near_rowptr;
        g.col = H->d_near_col;
        g.u = uc;
        g.ldu = N;
        g.f = fc;
        g.ldf = N;
        g.max_rows = H->max_leaf_rows;
        launch_near_generated(H->near_prec, g, s);
        launches += (nh + 15) / 16;
    }
    return launches;
}

int run_chunk(const htlr_handle *H, const KindDesc *d_kinds, double *part,
              const std::vector<double *> &W, const std::vector<double *> &Hs, const double *uc,
              double *fc, int nh, StageEvents *tev, cudaStream_t s)
{
    const int d = H->d, n = H->n, L = H->L;
    const long long N = (long long)ipow(n, d);
    int launches = 0;
    auto mark = [&](int k) {
        if (tev) cudaEventRecord(tev->ev[k], s);
    };
    mark(0);
    for (int lv = 1; lv <= L; ++lv) {
        if (H->lev[lv].nfar == 0) continue;
        launch_up(d, n, level_geom(H, lv), uc, nh, N, H->nrc, W[lv], s, H->far_prec != kPrecFP64);
        ++launches;
    }
    mark(1);
    mark(2);
    if (H->tc) {
        // tensor-core stream: pack the source operands, then one grouped launch per
        // block list
        // grouped path: G = 128 / Rpg targets per MMA
        const int Rpg = nh <= 16 ? 16 : nh <= 32 ? 32 : 64, tmi = Rpg == 16 ? 0 : Rpg == 32 ? 1 : 2;
        auto tcg_launch = [&](const TcgShape &tg, const int4v *cls, const int *cs, const int *cc,
                              int lv, const int *row_task, const void *blocks, int ld,
                              const TmapBytes &tm, int *counter, const int *order) {
            TcgArgs g{};
            g.counter = counter;
            g.order = order;
            g.offs = reinterpret_cast<const int4 *>(cls);
            for (int c = 0; c < 8; ++c) {
                g.cls_start[c] = cs[c];
                g.cls_count[c] = cc[c];
            }
            g.d = d;
            g.nb1 = 1 << lv;
            g.G = 128 / Rpg;
            g.Rp = Rpg;
            g.nr = nh;
            g.nq = (g.nb1 / 2 + g.G - 1) / g.G;
            const long long nb23 = d == 3 ? (long long)g.nb1 * g.nb1 : g.nb1;
            g.ngroups = nb23 * 2 * g.nq;
            g.Nd = tg.Nd;
            g.nch = tg.nch;
            g.NGb = tg.NGb;
            g.Nw = tg.Nw;
            g.passes = tg.passes;
            g.blocks = static_cast<const uint16_t *>(blocks);
            g.core_elems = tg.core_elems;
            g.tasks = H->d_tasks_tc;
            g.row_task = row_task;
            g.part = H->d_part_tc;
            g.ld = ld;
            // copy rings within 200 KB of shared memory: the lead ring holds a segment's
            // stages until its leading products are issued (at least F slots, or the copies
            // of the segment's last stages would wait for its own leading products; two
            // segments where they fit); the cross ring takes the rest.  The segment length
            // fixes the summation order, so it is never changed by the ring depths (tuned)
            const size_t lb = tcg_lead_bytes(tg.Nw / 8), cb = tcg_cross_bytes(tg.Nw / 8);
            const size_t budget = 200 * 1024;
            int F = std::max(1, H->tc_seg_stages);
            while (F > 1 && (size_t)F * lb + 2 * cb > budget) --F;   // only for huge F
            if (F > kTcMaxLead) F = kTcMaxLead;
            int Sl = std::min(kTcMaxLead, 2 * F);
            while (Sl > F && (size_t)Sl * lb + 2 * cb > budget) --Sl;
            int Sc = (int)((budget - (size_t)Sl * lb) / cb);
            if (Sc > kTcMaxStages) Sc = kTcMaxStages;
            if (H->tc_stages_cap >= 2 && Sc > H->tc_stages_cap) Sc = H->tc_stages_cap;
            g.stages = Sc < 2 ? 2 : Sc;
            g.lead_stages = Sl;
            g.seg_stages = F;
            g.flush_segs = H->tc_flush_segs;
            int cols = 32;
            while (cols < 2 * tg.Nw) cols *= 2;   // two accumulator buffers
            g.tmem_cols = cols;
            g.err = H->d_err;
            g.wait_cycles = H->tc_wait_cycles;
            launch_tc_group(g, tm.b, s);
        };
        for (int lv = 1; lv <= L; ++lv) {
            const LevelData &Lv = H->lev[lv];
            if (Lv.nfar == 0) continue;
            launch_tcg_pack_x(W[lv], (long long)H->nrc * Lv.pd, Lv.pd, Lv.nbox, nh, Rpg,
                              Lv.tg.nch, 0, d, n, H->leaf, L, nullptr, 0, Lv.d_Wg, s);
            tcg_launch(Lv.tg, Lv.d_cls, Lv.cls_start, Lv.cls_count, lv, Lv.d_row_task_tc,
                       Lv.d_cores, Lv.ld, Lv.tmap[tmi], H->d_grp_counter + lv, Lv.d_order[tmi]);
            launches += 2;
        }
        if (H->near_prec == kPrecBF16X6) {
            launch_tcg_pack_x(nullptr, 0, H->near_rows, 1 << (d * L), nh, Rpg, H->near_tg.nch, 1,
                              d, n, H->leaf, L, uc, N, H->d_Ug, s);
            tcg_launch(H->near_tg, H->d_near_cls, H->near_cls_start, H->near_cls_count, L,
                       H->d_near_row_task_tc, H->d_near, H->near_ld, H->near_tmap[tmi],
                       H->d_grp_counter + L + 1, H->d_near_order[tmi]);
            launches += 2;
        }
    } else if (!H->tasks.empty()) {
        launches += launch_streams(H, d_kinds, uc, N, nh, part, s);
    }
    mark(3);
    mark(4);
    if (H->tc && H->near_prec != kPrecBF16X6 && !H->near_generated && !H->tasks.empty()) {
        // held near field on the CUDA cores beside a tensor-core far field, four right-hand
        // sides per pass (its partial-sum slots hold kTcRpMax RHS; pass r0 fills r0 .. r0+3)
        for (int r0 = 0; r0 < nh; r0 += 4)
            launches += launch_streams(H, d_kinds, uc + (long long)r0 * N, N, std::min(4, nh - r0),
                                       part + (long long)r0 * H->near_ld, s);
    }
    mark(5);
    mark(6);
    for (int lv = 1; lv <= L; ++lv) {
        const LevelData &Lv = H->lev[lv];
        if (Lv.nfar == 0) continue;
        if (H->tc)
            launch_reduce_far(Lv.nbox, Lv.pd, Lv.ld, H->nrc, nh, Lv.d_row_task_tc, H->d_tasks_tc,
                              H->d_part_tc, Hs[lv], s);
        else
            launch_reduce_far(Lv.nbox, Lv.pd, Lv.ld, H->nrc, nh, Lv.d_row_task, H->d_tasks, part,
                              Hs[lv], s);
        ++launches;
    }
    mark(7);
    mark(8);
    OutArgs oa{};
    oa.d = d;
    oa.n = n;
    oa.L = L;
    oa.nrc = H->nrc;
    oa.nrhs = nh;
    oa.leafg = level_geom(H, L);
    const bool near_tc = H->near_prec == kPrecBF16X6;
    oa.near_row_task = near_tc ? H->d_near_row_task_tc : H->d_near_row_task;
    oa.tasks = near_tc ? H->d_tasks_tc : H->d_tasks;
    oa.part = near_tc ? H->d_part_tc : part;
    oa.near_ld = H->near_ld;
    oa.a_add = (H->near_generated || (H->storage == HTLR_STORE_STORED && !near_tc)) ? nullptr
                                                                                     : H->d_a;
    oa.diag_add = near_tc ? H->d_diagpts : nullptr;
    oa.u = uc;
    oa.ldu = N;
    oa.near_in_f = H->near_generated;
    oa.ndown = 0;
    for (int lv = 1; lv <= L; ++lv) {
        if (H->lev[lv].nfar == 0) continue;
        oa.down[oa.ndown].g = level_geom(H, lv);
        oa.down[oa.ndown].H = Hs[lv];
        ++oa.ndown;
    }
    oa.f = fc;
    oa.ldf = N;
    launch_out(oa, H->max_leaf_rows, s, H->far_prec != kPrecFP64);
    ++launches;
    mark(9);
    if (tev)
        for (int st = 0; st < HTLR_NUM_STAGES; ++st) {
            cudaEventSynchronize(tev->ev[2 * st + 1]);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, tev->ev[2 * st], tev->ev[2 * st + 1]);
            tev->ms[st] += ms;
        }
    return launches;
}

static int enqueue_matvec(const htlr_handle *H, const double *u, double *f, int nrhs,
                          StageEvents *tev = nullptr, cudaStream_t on = nullptr);

// HMultVec for other parts of the library (GMRES): enqueue on the handle's stream.
int matvec_enqueue(const htlr_handle *H, const double *u, double *f, int nrhs)
{
    return enqueue_matvec(H, u, f, nrhs);
}

// The same sequence of launches on another stream (graph capture).
int matvec_enqueue_on(const htlr_handle *H, const double *u, double *f, int nrhs, cudaStream_t s)
{
    return enqueue_matvec(H, u, f, nrhs, nullptr, s);
}

static int enqueue_matvec(const htlr_handle *H, const double *u, double *f, int nrhs,
                          StageEvents *tev, cudaStream_t on)
{
    cudaStream_t st = on ? on : H->stream;
    const long long N = (long long)ipow(H->n, H->d);
    std::vector<double *> W(H->L + 1, nullptr), Hs(H->L + 1, nullptr);
    for (int lv = 1; lv <= H->L; ++lv) {
        W[lv] = H->lev[lv].d_W;
        Hs[lv] = H->lev[lv].d_H;
    }
    int launches = 0;
    if (H->near_generated) {
        if (tev) cudaEventRecord(tev->ev[4], st);
        launches += launch_near_gen_all(H, u, f, nrhs, st);
        if (tev) {
            cudaEventRecord(tev->ev[5], st);
            cudaEventSynchronize(tev->ev[5]);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, tev->ev[4], tev->ev[5]);
            tev->ms[2] += ms;
        }
    }
    for (int c0 = 0; c0 < nrhs; c0 += H->nrc) {
        const int nh = std::min(H->nrc, nrhs - c0);
        launches += run_chunk(H, H->d_kinds, H->d_part, W, Hs, u + (long long)c0 * N,
                              f + (long long)c0 * N, nh, tev, st);
    }
    const_cast<htlr_handle *>(H)->last_launches = launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "matvec launch");
    return HTLR_OK;
}

// Reads the handle's device error word after its stream has drained, clears it, and maps
// it to a status: a bounded wait that ran out is HTLR_ETIMEOUT, any other device check
// HTLR_EDEVICE.  Clearing on read reports each failure once and leaves the handle usable.
int check_device_error(const htlr_handle *H, const char *what)
{
    int err = 0;
    HTLR_CK(cudaMemcpy(&err, H->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!err) return HTLR_OK;
    HTLR_CK(cudaMemsetAsync(H->d_err, 0, sizeof(int), H->stream));
    HTLR_CK(cudaStreamSynchronize(H->stream));
    char buf[160];
    if (err == kDevTimeout) {
        snprintf(buf, sizeof buf,
                 "%s: a bounded device wait of a tensor-core kernel ran out (limit %lld SM "
                 "cycles); the results of that matvec are invalid",
                 what, (long long)H->tc_wait_cycles);
        return fail(HTLR_ETIMEOUT, buf);
    }
    snprintf(buf, sizeof buf, "%s: device check failed (code %d)", what, err);
    return fail(HTLR_EDEVICE, buf);
}

}  // namespace htlr

using namespace htlr;

extern "C" {

const char *htlr_last_error(void) { return g_err.c_str(); }

int htlr_construct_ex(htlr_handle **out, const htlr_kernel *k, int d, int n, const htlr_grid *grid,
                      int leaf, int r, double eta, const htlr_options *o)
{
    set_error("");
    if (!out) return fail(HTLR_EINVAL, "H must not be NULL");
    *out = nullptr;
    if (!k) return fail(HTLR_EINVAL, "kernel must not be NULL");
    if (k->type < HTLR_K_LOG || k->type > HTLR_K_CONST) return fail(HTLR_EINVAL, "unknown kernel type");
    if (!std::isfinite(k->scale) || !std::isfinite(k->param))
        return fail(HTLR_EINVAL, "kernel scale and param must be finite");
    if (k->type == HTLR_K_GAUSS && !(k->param > 0.0)) return fail(HTLR_EINVAL, "Gaussian sigma must be > 0");
    if (k->type == HTLR_K_POLY && (k->param < 0 || k->param > 16 || k->param != std::floor(k->param)))
        return fail(HTLR_EINVAL, "polynomial degree must be an integer in 0..16");
    if (d != 2 && d != 3) return fail(HTLR_EINVAL, "d must be 2 or 3");
    if (leaf < 1 || n < 2 || n % leaf) return fail(HTLR_EINVAL, "n must be a multiple of leaf");
    int ratio = n / leaf, L = 0;
    while ((1 << L) < ratio) ++L;
    if ((1 << L) != ratio || L < 1) return fail(HTLR_EINVAL, "n / leaf must be 2^L with L >= 1");
    if (L >= HTLR_MAX_LEVELS) return fail(HTLR_EINVAL, "too many levels");
    if (d * L > 30) return fail(HTLR_EINVAL, "too many boxes");
    if (r < 1 || r > kMaxP) return fail(HTLR_EINVAL, "r must be in 1..16");
    if (!std::isfinite(eta)) return fail(HTLR_EINVAL, "eta must be finite");
    const bool tensor = grid && grid->type == HTLR_GRID_TENSOR;
    if (grid && !tensor && grid->type != HTLR_GRID_UNIFORM)
        return fail(HTLR_EINVAL, "unknown grid type");
    if (tensor) {
        if (!grid->coords || !grid->edges)
            return fail(HTLR_EINVAL, "a tensor grid needs coords and edges");
        for (int l = 0; l < d; ++l) {
            const double *x = grid->coords + (size_t)l * n, *e = grid->edges + (size_t)l * (n + 1);
            if (e[0] != 0.0 || e[n] != 1.0)
                return fail(HTLR_EINVAL, "tensor grid: the cell edges must start at 0 and end at 1");
            for (int i = 0; i < n; ++i) {
                if (!(e[i] < e[i + 1]) || !(x[i] >= e[i] && x[i] <= e[i + 1]) ||
                    !std::isfinite(x[i]))
                    return fail(HTLR_EINVAL, "tensor grid: edges must increase and each "
                                             "coordinate must lie in its cell");
            }
        }
        if (o && o->orth == 1)
            return fail(HTLR_EUNSUPPORTED, "tensor grids use the interpolation factors "
                                           "without orthogonalisation (orth must be 0 or -1)");
    }
    int q = (o && o->quad_order > 0) ? o->quad_order : 16;
    if (q > 64) return fail(HTLR_EINVAL, "quad_order must be in 1..64");
    if (o && o->tc_segment < 0) return fail(HTLR_EINVAL, "tc_segment must be >= 0");
    if (o && o->tc_flush < 0) return fail(HTLR_EINVAL, "tc_flush must be >= 0");
    if (o && o->tc_wait_cycles < 0) return fail(HTLR_EINVAL, "tc_wait_cycles must be >= 0");
    if (o && (o->orth < -1 || o->orth > 1)) return fail(HTLR_EINVAL, "orth must be -1, 0 or 1");
    if (o && (o->far_precision < 0 || o->far_precision > 3 || o->near_precision < 0 ||
              o->near_precision > 4))
        return fail(HTLR_EINVAL, "precisions must be HTLR_PREC_FP64, _DF64, _FP32 or _BF16X6");

    htlr_handle *H = nullptr;
    try {
        H = new htlr_handle();
    } catch (const std::bad_alloc &) {
        return fail(HTLR_ENOMEM, "host allocation failed");
    }
    H->magic = kMagicLive;
    cudaGetDevice(&H->device);
    H->stream = o ? (cudaStream_t)o->stream : nullptr;
    H->kern = KernelDesc{k->type, k->scale, k->param};
    H->d = d;
    H->n = n;
    H->leaf = leaf;
    H->p = r;
    H->L = L;
    H->eta = eta;
    H->q = q;
    H->tensor = tensor ? 1 : 0;
    H->orth = (tensor || (o && o->orth == 0)) ? 0 : 1;
    H->far_prec = o ? o->far_precision : kPrecFP64;
    H->near_prec = o ? o->near_precision : kPrecFP64;
    if (o && o->tc_segment > 0) H->tc_seg_stages = o->tc_segment;
    if (o && o->tc_flush > 0) H->tc_flush_segs = o->tc_flush;
    if (o && o->tc_wait_cycles > 0) H->tc_wait_cycles = o->tc_wait_cycles;
    int rc;
    try {
        rc = build(H, grid, o);
    } catch (const std::bad_alloc &) {
        rc = fail(HTLR_ENOMEM, "host allocation failed");
    }
    if (rc != HTLR_OK) {
        std::string keep = g_err;
        destroy(H);
        set_error(keep);
        return rc;
    }
    {
        std::lock_guard<std::mutex> g(g_live_mu);
        g_live.insert(H);
    }
    *out = H;
    return HTLR_OK;
}

int htlr_construct(htlr_handle **out, const htlr_kernel *k, int d, int n, const htlr_grid *grid,
                   int leaf, int r, double eta)
{
    return htlr_construct_ex(out, k, d, n, grid, leaf, r, eta, nullptr);
}

int htlr_matvec(const htlr_handle *H, const double *u, double *f, int nrhs)
{
    if (!is_live(H)) return fail(HTLR_EINVAL, "not a live HTLR handle");
    if (!u || !f) return fail(HTLR_EINVAL, "u and f must not be NULL");
    if (nrhs < 1) return fail(HTLR_EINVAL, "nrhs must be >= 1");
    const long long N = (long long)ipow(H->n, H->d);
    const char *ub = (const char *)u, *ue = (const char *)(u + N * nrhs);
    const char *fb = (const char *)f, *fe = (const char *)(f + N * nrhs);
    if (ub < fe && fb < ue) return fail(HTLR_EINVAL, "u and f must not overlap");
    return enqueue_matvec(H, u, f, nrhs);
}

int htlr_matvec_timed(const htlr_handle *H, const double *u, double *f, int nrhs,
                      float *stage_ms)
{
    if (!is_live(H)) return fail(HTLR_EINVAL, "not a live HTLR handle");
    if (!u || !f || !stage_ms) return fail(HTLR_EINVAL, "u, f and stage_ms must not be NULL");
    if (nrhs < 1) return fail(HTLR_EINVAL, "nrhs must be >= 1");
    StageEvents tev;
    for (int k = 0; k < 2 * HTLR_NUM_STAGES; ++k) HTLR_CK(cudaEventCreate(&tev.ev[k]));
    for (int k = 0; k < HTLR_NUM_STAGES; ++k) tev.ms[k] = 0.f;
    int rc = enqueue_matvec(H, u, f, nrhs, &tev);
    cudaError_t e = cudaStreamSynchronize(H->stream);
    for (int k = 0; k < 2 * HTLR_NUM_STAGES; ++k) cudaEventDestroy(tev.ev[k]);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    for (int k = 0; k < HTLR_NUM_STAGES; ++k) stage_ms[k] = tev.ms[k];
    return check_device_error(H, "htlr_matvec_timed");
}

int htlr_matvec_host(htlr_handle *H, const double *u_host, double *f_host, int nrhs)
{
    if (!is_live(H)) return fail(HTLR_EINVAL, "not a live HTLR handle");
    if (!u_host || !f_host) return fail(HTLR_EINVAL, "u and f must not be NULL");
    if (nrhs < 1) return fail(HTLR_EINVAL, "nrhs must be >= 1");
    const size_t N = (size_t)ipow(H->n, H->d);
    size_t need = N * (size_t)nrhs;
    if (need > H->stage_cap) {
        if (H->d_stage_u) cudaFree(H->d_stage_u);
        if (H->d_stage_f) cudaFree(H->d_stage_f);
        H->d_stage_u = H->d_stage_f = nullptr;
        H->stage_cap = 0;
        HTLR_CK(device_malloc((void **)&H->d_stage_u, need * sizeof(double)));
        HTLR_CK(device_malloc((void **)&H->d_stage_f, need * sizeof(double)));
        H->stage_cap = need;
    }
    HTLR_CK(cudaMemcpyAsync(H->d_stage_u, u_host, need * sizeof(double), cudaMemcpyHostToDevice,
                            H->stream));
    int rc = enqueue_matvec(H, H->d_stage_u, H->d_stage_f, nrhs);
    if (rc) return rc;
    HTLR_CK(cudaMemcpyAsync(f_host, H->d_stage_f, need * sizeof(double), cudaMemcpyDeviceToHost,
                            H->stream));
    HTLR_CK(cudaStreamSynchronize(H->stream));
    return check_device_error(H, "htlr_matvec_host");
}

void htlr_free(htlr_handle *H)
{
    if (!H) return;
    {
        std::lock_guard<std::mutex> g(g_live_mu);
        if (!g_live.count(H)) {
            set_error("htlr_free: not a live HTLR handle (double free?)");
            return;
        }
        g_live.erase(H);
    }
    cudaStreamSynchronize(H->stream);
    destroy(H);
}

int htlr_info(const htlr_handle *H, htlr_stats *s)
{
    if (!is_live(H)) return fail(HTLR_EINVAL, "not a live HTLR handle");
    if (!s) return fail(HTLR_EINVAL, "stats pointer must not be NULL");
    *s = H->stats;
    return HTLR_OK;
}

int htlr_set_stream(htlr_handle *H, void *stream)
{
    if (!is_live(H)) return fail(HTLR_EINVAL, "not a live HTLR handle");
    H->stream = (cudaStream_t)stream;
    return HTLR_OK;
}

int htlr_sync(const htlr_handle *H)
{
    if (!is_live(H)) return fail(HTLR_EINVAL, "not a live HTLR handle");
    HTLR_CK(cudaStreamSynchronize(H->stream));
    return check_device_error(H, "htlr_sync");
}

int htlr_set_wait_limit(htlr_handle *H, long long cycles)
{
    if (!is_live(H)) return fail(HTLR_EINVAL, "not a live HTLR handle");
    if (cycles < 0) return fail(HTLR_EINVAL, "the wait limit must be >= 0");
    H->tc_wait_cycles = cycles > 0 ? cycles : 4000000000ll;
    ++H->generation;   // captured plans hold the old limit in their launch arguments
    return HTLR_OK;
}

long long htlr_device_allocations(void) { return g_device_allocs.load(std::memory_order_relaxed); }

double htlr_tensor_flops(const htlr_handle *H, int nrhs)
{
    if (!is_live(H) || nrhs < 1 || !H->tc) return 0.0;
    const int d = H->d, L = H->L;
    double total = 0.0;
    // grouped kernel: every (group, offset) with a source inside the domain, all chunks
    auto grouped = [&](const TcgShape &tg, const std::vector<int4v> &cl, const int *cs,
                       const int *cc, int lv, int Rpg) {
        const int nb1 = 1 << lv, G = 128 / Rpg, nq = (nb1 / 2 + G - 1) / G;
        const int nb23 = d == 3 ? nb1 * nb1 : nb1;
        long long pairs = 0;
        for (int b23 = 0; b23 < nb23; ++b23)
            for (int c1 = 0; c1 < 2; ++c1)
                for (int j = 0; j < nq; ++j) pairs += group_valid(d, nb1, G, b23, c1, j, cl, cs, cc);
        return (double)pairs * tg.nch * 6.0 * 2.0 * 128.0 * tg.Npad * 16.0;
    };
    for (int c0 = 0; c0 < nrhs; c0 += H->nrc) {
        const int nh = std::min(H->nrc, nrhs - c0);
        const int Rpg = nh <= 16 ? 16 : nh <= 32 ? 32 : 64;
        for (int lv = 1; lv <= L; ++lv) {
            const LevelData &Lv = H->lev[lv];
            if (Lv.nfar == 0) continue;
            total += grouped(Lv.tg, Lv.h_cls, Lv.cls_start, Lv.cls_count, lv, Rpg);
        }
        if (H->near_prec == kPrecBF16X6)
            total += grouped(H->near_tg, H->h_near_cls, H->near_cls_start, H->near_cls_count,
                             L, Rpg);
    }
    return total;
}

int htlr_last_launch_count(const htlr_handle *H)
{
    if (!is_live(H)) return -1;
    return H->last_launches;
}

}  // extern "C"
