// Internal declarations of the HTLR CUDA library (not part of the C ABI).
//
// Device data layout (uniform grid, natural point order i_1 + n i_2 + n^2 i_3):
//   * boxes of level l are numbered lexicographically, b_1 + 2^l b_2 + 4^l b_3;
//   * per level: one interpolation factor F_l (nb x pe, column-major) shared by every box
//     and dimension (the points sit at the same place in every box of a uniform grid),
//     orthonormal after the QR of Algorithm 1, and the triangular R_l (pe x p);
//   * admissible blocks of level l: CSR by target box tau (column = source box sigma,
//     core = index of the core tensor); a core is stored column-major [s][t] with
//     leading dimension ld = pd rounded up to 32 doubles (pd = pe^d), so every column
//     starts 256-byte aligned;
//   * inadmissible leaves: CSR by leaf tau, dense blocks [j][i] (leaf-local lexicographic
//     indices), same padding rule;
//   * matvec work arrays: W_l, H_l of shape [box][rhs][pd] for an RHS chunk.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/htlr.h"

namespace htlr {

constexpr uint64_t kMagicLive = 0x48544c52474233ull;
constexpr uint64_t kMagicDead = 0x64656164deadull;
constexpr int kMaxD = 3;
constexpr int kMaxP = 16;

// Device error codes written into the handle's error word.
enum DevErr : int { kDevOk = 0, kDevBadIndex = 1, kDevBadTask = 2, kDevTimeout = 3 };

// Arithmetic of a block list (same values as the public htlr_precision enum).
enum Prec : int { kPrecFP64 = 0, kPrecDF64 = 1, kPrecFP32 = 2, kPrecBF16X6 = 3, kPrecTF32X3 = 4 };

// Bytes of one block element in memory for a precision.
inline size_t prec_bytes(int prec) { return prec == kPrecFP32 ? 4 : 8; }

struct KernelDesc {
    int type;
    double scale;
    double param;
};

// One unit of streaming work: entries [e0, e1) of row `row` of list `kind`.
// kind 0..L: admissible blocks of that level; kind L+1: inadmissible leaves.
struct Task {
    int kind;
    int row;
    int e0, e1;
    long long part;  // offset of this task's partial result (doubles)
};

// Per-kind description used by the streaming kernel (kept in device memory).
struct KindDesc {
    const int *col;      // source box per entry
    const int *blk;      // block (core / dense) index per entry
    const void *blocks;  // double, float2 (hi, lo) or float elements, per `prec`
    long long blk_stride;  // elements between consecutive blocks (ld * cols)
    int prec;            // Prec of the blocks
    int ld;              // padded rows of a block
    int rows;            // real rows (pd_out)
    int cols;            // pd_in
    int rpl;             // rows per lane = ld / 32
    int is_near;         // 1: x gathered from u (natural order)
    const double *x;     // far: W of the level ([box][rhs][pd])
    long long x_box_stride;  // doubles per box in x (nrc * pd)
};

constexpr int kTcRpMax = 64;  // right-hand sides per tensor-core pass

// Grouped tensor-core form of a SHARED block list (tc_group.cu): blocks Nd x Kd packed
// as [chunk of 16 columns][split][row group][kcore][8][8], sources per box as
// [split][chunk][row group][kcore][8][8]; the block rows (N) in `passes` passes of Nw
// (Nw <= kTcgMaxNw: two accumulators of Nw columns fit in tensor memory, and each drain
// thread keeps Nw / 2 running sums in registers).
constexpr int kTcgMaxNw = 256;
struct TcgShape {
    int Kd = 0, Nd = 0, nch = 0, Npad = 0, NGb = 0, Nw = 0, passes = 0;
    long long core_elems = 0;    // bf16 elements per packed block
    long long box_elems = 0;     // bf16 elements per packed source box at 64 RHS
};
struct alignas(64) TmapBytes {   // an encoded CUtensorMap (128 bytes)
    unsigned char b[128];
};
struct int4v {                    // (o1, o2, o3, block id) of a class offset list
    int x, y, z, w;
};

struct LevelData {
    int level = 0, nb = 0, nbox1 = 0, nbox = 0, pe = 0, pd = 0, ld = 0;
    // tensor-core form (precision BF16X6): partial slots per target row
    std::vector<int> row_task_tc;
    int *d_row_task_tc = nullptr;
    int64_t nfar = 0;
    std::vector<int> far_rowptr, far_col, far_core;
    int *d_far_rowptr = nullptr, *d_far_col = nullptr, *d_far_core = nullptr;
    double *d_F = nullptr;      // uniform grid: nb x pe, the factor of every box
    double *d_R = nullptr;      // pe x p
    // box geometry along each dimension (1-D box k of this level), see LevelGeom
    std::vector<int> first[3], cnt[3], uoff[3], voff[3];
    int *d_geo = nullptr;       // device copy: first, cnt, uoff, voff for each dimension
    double *d_Upool = nullptr, *d_Vpool = nullptr;
    int maxcnt = 0;
    void *d_cores = nullptr;    // ncores x (ld * pd) elements of the far precision
    int64_t ncores = 0;
    double *d_W = nullptr, *d_H = nullptr;  // nbox x nrc x pd
    int task0 = 0, task1 = 0;               // task range (far) of this level
    std::vector<int> row_task_begin;        // per tau: first task; size nbox + 1
    int *d_row_task = nullptr;
    // grouped tensor-core path (SHARED storage): class offset lists, packed sources,
    // tensor maps of the sources for 16, 32 and 64 right-hand sides
    int tcg = 0;
    TcgShape tg;
    int cls_start[8] = {0}, cls_count[8] = {0};
    int4v *d_cls = nullptr;
    std::vector<int4v> h_cls;
    int *d_order[3] = {nullptr, nullptr, nullptr};  // group order for 16, 32, 64 RHS
    uint16_t *d_Wg = nullptr;
    TmapBytes tmap[3];
};

struct Plan;  // forward

}  // namespace htlr

struct htlr_handle {
    uint64_t magic = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    htlr::KernelDesc kern{};
    int d = 0, n = 0, leaf = 0, p = 0, L = 0, orth = 1, q = 16;
    double eta = 0.0;
    int storage = HTLR_STORE_STORED;
    int nrc = 1;  // RHS per chunk
    double h = 0.0, wgt = 0.0;  // grid step and quadrature weight h^d
    double diag = 0.0;          // K_ii h^d (uniform grid)
    double *d_a = nullptr;      // a(x) natural order or null
    int tensor = 0;             // 1: tensor (non-uniform) grid given by coordinates / edges
    int near_generated = 0;     // 1: inadmissible blocks recomputed in every matvec
    double *d_coords = nullptr, *d_width = nullptr, *d_edges = nullptr;  // d x n (n+1)
    double *d_diagpts = nullptr;  // per-point K_ii w_i (generated near field)
    int max_leaf_rows = 0;
    std::vector<htlr::LevelData> lev;  // levels 0..L
    // inadmissible leaves
    int64_t nnear = 0, nnear_unique = 0;
    std::vector<int> near_rowptr, near_col, near_blk;
    int *d_near_rowptr = nullptr, *d_near_col = nullptr, *d_near_blk = nullptr;
    void *d_near = nullptr;     // dense blocks, elements of the near precision
    int near_ld = 0, near_rows = 0;
    std::vector<int> near_row_task;  // per leaf: first task, size nleaf + 1
    int *d_near_row_task = nullptr;
    // streaming tasks
    std::vector<htlr::Task> tasks;
    htlr::Task *d_tasks = nullptr;
    htlr::KindDesc *d_kinds = nullptr;
    std::vector<htlr::KindDesc> kinds;
    double *d_part = nullptr;
    long long part_doubles = 0;
    int max_cols = 1;
    int far_prec = 0, near_prec = 0;
    int near_task0 = 0;  // first task of the inadmissible leaves
    // tensor-core stream (far_prec / near_prec BF16X6): row tasks, partials, near operand
    int tc = 0;
    std::vector<htlr::Task> tasks_tc;
    htlr::Task *d_tasks_tc = nullptr;
    double *d_part_tc = nullptr;
    int near_tcg = 0;                // grouped tensor-core path for the near field
    htlr::TcgShape near_tg;
    int near_cls_start[8] = {0}, near_cls_count[8] = {0};
    htlr::int4v *d_near_cls = nullptr;
    std::vector<htlr::int4v> h_near_cls;
    int *d_near_order[3] = {nullptr, nullptr, nullptr};
    int *d_grp_counter = nullptr;    // one per level + 1 (grouped tensor-core launches)
    // generated near field on the tensor cores (near_prec kPrecTF32X3)
    int *d_ntc_stage0 = nullptr;     // per leaf: first stage of its packed sources
    int *d_ntc_items = nullptr;      // (leaf, tile) pairs, heaviest first
    int ntc_nitems = 0, ntc_max_rows_pad = 0;
    float *d_ntc_wu = nullptr;       // packed w u, two TF32 terms, 16 RHS
    int *d_ntc_counter = nullptr;
    uint16_t *d_Ug = nullptr;
    htlr::TmapBytes near_tmap[3];
    std::vector<int> near_row_task_tc;
    int *d_near_row_task_tc = nullptr;
    int *d_err = nullptr;
    // host staging for htlr_matvec_host
    double *d_stage_u = nullptr, *d_stage_f = nullptr;
    size_t stage_cap = 0;
    int last_launches = 0;
    // launch tuning (autotuner): stream task size, CUDA-core stream CTAs per SM and
    // threads per CTA, tensor-core ring depth (0 = largest that fits); `generation`
    // changes whenever the device-side task tables are rebuilt (captured plans re-capture)
    size_t task_bytes = 256 * 1024;
    int stream_ctas_per_sm = 8, stream_threads = 256, tc_stages_cap = 0;
    int tc_seg_stages = 4;   // grouped tensor-core kernel: K stages per TMEM segment
    int tc_flush_segs = 32;  // grouped tensor-core kernel: segments per FP64 flush
    long long tc_wait_cycles = 4000000000ll;  // tensor-core kernels: bounded-wait limit
    int generation = 0;
    htlr_stats stats{};
    std::vector<void *> allocs;
};

namespace htlr {

// Error reporting (thread-local message).
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);
// Every device allocation the library makes goes through device_malloc, which counts
// them (htlr_device_allocations) so that a caller can check that an entry point
// allocated nothing.
cudaError_t device_malloc(void **p, size_t bytes);
// After the handle's stream has drained: read and clear its device error word
// (HTLR_ETIMEOUT for a bounded wait that ran out, HTLR_EDEVICE for other checks).
int check_device_error(const htlr_handle *H, const char *what);

// ---- plan.cu: block cluster tree walk -------------------------------------------
// Counts (pass 0) or fills (pass 1) the far and near lists of level `level` from the
// near list of level-1.  Boxes are lexicographic.  Strong admissibility when eta > 0.
void launch_walk(int pass, int d, int level, double eta, const int *d_prev_rowptr,
                 const int *d_prev_col, int *d_far_cnt, int *d_near_cnt,
                 const int *d_far_off, const int *d_near_off, int *d_far_col, int *d_near_col,
                 cudaStream_t s);

// ---- construct.cu -----------------------------------------------------------------
// Interpolation factor of a level (barycentric Lagrange on Chebyshev points) and, if
// orth, its economy QR; writes F (nb x pe) and R (pe x p; identity-padded if !orth).
void launch_factor(int nb, int p, int pe, double side, double h, int orth, double *d_F,
                   double *d_R, cudaStream_t s);
// Diagonal K_ii w_i on the uniform grid: int over the cell of k(center, y) dy.
void launch_diag(const KernelDesc &k, int d, double h, int q, const double *d_gx,
                 const double *d_gw, double *d_out, cudaStream_t s);
// Core tensors: for each core c, offset (tau - sigma) in boxes from d_off[c*3..]; writes
// wgt * k(xi_t, eta_s) transformed by R on all 2d modes, [s][t] with leading dim ld.
void launch_cores(const KernelDesc &k, int d, int p, int pe, int ld, int apply_r, double side,
                  double wgt, const double *d_R, int64_t ncores, const int *d_off,
                  double *d_cores, double *d_scratch, int nscratch_ctas, cudaStream_t s);
// Zero the diagonal entries of the dense blocks listed in d_ids.
void launch_zero_diag(double *blocks, int ld, int rows, const int *d_ids, int nids, cudaStream_t s);
// Precision conversions of finished blocks: in place to (hi, lo) float pairs, or into a
// separate FP32 array.
void launch_split_df64(double *d_buf, size_t count, cudaStream_t s);
void launch_to_fp32(const double *d_src, float *d_dst, size_t count, cudaStream_t s);
// Dense blocks of inadmissible leaves: block b between leaves with offset d_off[b*3..]
// (tau - sigma) and, for STORED, target leaf d_tau[b] (to add a on the diagonal).
void launch_near(const KernelDesc &k, int d, int n, int leaf, int ld, double h, double wgt,
                 double diag, const double *d_a, int64_t nblk, const int *d_off,
                 const int *d_tau, double *d_blocks, cudaStream_t s);

// ---- apply.cu -------------------------------------------------------------------
// Arguments of one launch of the block stream over tasks [t0, t1), all of one precision.
// streaming = true marks the blocks as read once per matvec (evict-first loads).
struct StreamArgs {
    const Task *tasks;
    int t0, t1;
    const KindDesc *kinds;
    int d, n, leaf, nl_level;
    const double *u;
    long long ldu;
    int nrhs;
    int max_cols;
    double *part;
    int *err;
    bool streaming;
    cudaStream_t stream;
    int threads = 256;     // 128 or 256 (one warp per task)
    int ctas_per_sm = 8;   // grid cap: 152 x ctas_per_sm
};
void launch_stream_fp64(const StreamArgs &a);
void launch_stream_df64(const StreamArgs &a);
void launch_stream_fp32(const StreamArgs &a);
void launch_stream(int prec, const StreamArgs &a);
// (Re)build the CUDA-core stream tasks of H for a task size in bytes (htlr_api.cu).
int build_tasks(htlr_handle *H, size_t task_bytes, cudaStream_t s);
// Level of the leaves: n = leaf * 2^nl_level.
int leaf_level(int n, int leaf);
void launch_reduce_far(int nbox, int pd, int ld, int nrc, int nrhs_here, const int *d_row_task,
                       const Task *d_tasks, const double *d_part, double *d_H, cudaStream_t s);
// Geometry of the boxes of one level along each dimension (device arrays indexed by the
// 1-D box index k < 2^level): grid lines [first, first + cnt) of the box, and where its
// target factor U (cnt x pe) and source factor V (cnt x pe), column-major, start in the
// factor pools.  On a uniform grid every box of a level points at the same factor.
struct LevelGeom {
    const int *first[3];
    const int *cnt[3];
    const int *uoff[3];
    const int *voff[3];
    const double *Upool;
    const double *Vpool;
    int level, pe, pd, maxcnt;
};
struct DownLevel {
    LevelGeom g;
    const double *H;
};
// df64: float-pair arithmetic on the FP32 pipe (used unless the far field is FP64).
void launch_up(int d, int n, const LevelGeom &g, const double *u, int nrhs_here, long long ldu,
               int nrc, double *d_W, cudaStream_t s, bool df64);
// out: f_tau = base + sum over far levels of H_anc x_l U_l (rows of the leaf).  The base
// is the sum of the leaf's dense-block task partials [+ a u] (near_in_f = 0), or the
// value already in f written by the generated near field (near_in_f = 1).
struct OutArgs {
    int d, n, L, nrc, nrhs;
    LevelGeom leafg;             // geometry of the leaf level (first / cnt only)
    const int *near_row_task;    // per leaf: task range of its dense blocks
    const Task *tasks;
    const double *part;
    int near_ld;
    const double *a_add;         // add a(x) u when the dense blocks do not hold it
    const double *diag_add;      // add K_ii w_i u_i (per point) when the blocks do not hold it
    const double *u;
    long long ldu;
    int near_in_f;
    int ndown;
    DownLevel down[HTLR_MAX_LEVELS];
    double *f;
    long long ldf;
};
void launch_out(const OutArgs &a, int max_rows, cudaStream_t s, bool df64);
// Generated near field: f_tau = sum over the leaf's near list of K(x_i, y_j) w_j u_j (j != i)
// + (diag_i + a_i) u_i, kernel values recomputed in every call.  prec: kPrecFP64 or
// kPrecFP32 (coordinates taken relative to the target leaf before rounding).
struct NearGenArgs {
    KernelDesc k;
    int d, n, L, nrhs;
    LevelGeom leafg;
    const double *coords;  // d * n
    const double *width;   // d * n cell widths
    const double *diag;    // N values: K_ii w_i
    const double *a;       // N values or null
    const int *rowptr, *col;
    const double *u;
    long long ldu;
    double *f;
    long long ldf;
    int max_rows;
};
void launch_near_generated(int prec, const NearGenArgs &a, cudaStream_t s);
// ---- near_tc.cu: generated near field on the tensor cores (kPrecTF32X3) ----
// The same product as NearGenArgs for 16 right-hand sides (r0 .. r0 + nr - 1): kernel
// values generated per pair into tensor memory as two TF32 terms, times w_j u_j packed as
// two TF32 terms per source (`wu`, refilled by the launch), kind::tf32 MMAs.
struct NearTcArgs {
    KernelDesc k;
    int d, n, L;
    LevelGeom leafg;
    const double *coords;  // d * n
    const double *width;   // d * n cell widths
    const double *diag;    // N values: K_ii w_i
    const double *a;       // N values or null
    const int *rowptr, *col;
    const int *stage0;     // per leaf: first 16-source stage of its packed sources (nleaf + 1)
    const int *items;      // (leaf, 128-row tile) pairs, heaviest first
    int nitems;
    float *wu;             // stage0[nleaf] x 512 floats
    const double *u;
    long long ldu;
    double *f;
    long long ldf;
    int r0, nr;
    int max_rows_pad;      // largest leaf, rounded up to 16 points
    int *counter;          // next item (reset before each launch)
    int *err;
    long long wait_cycles;
};
void launch_near_tc(const NearTcArgs &a, cudaStream_t s);
// Rows of one near_tc item (a tile of a leaf's rows, taken by one warpgroup).
int near_tc_tile_rows();
// ---- tc_group.cu: grouped tensor-core stream for SHARED block lists ----
struct TcgArgs {
    const int4 *offs;                  // class offset lists (o1, o2, o3, block id)
    int cls_start[8], cls_count[8];
    int d, nb1;                        // dimension, boxes per dimension at this level
    int G, Rp, nr;                     // targets per group (G Rp = 128), padded / real RHS
    int nq;                            // groups along one parity line of dimension 1
    long long ngroups;
    int Nd, nch, NGb, Nw, passes;
    const uint16_t *blocks;
    long long core_elems;
    const Task *tasks;
    const int *row_task;
    double *part;
    int ld;
    int stages, lead_stages, tmem_cols;  // cross and lead copy-ring depths
    int *err;
    int *counter;                      // next group (reset to 0 before each launch)
    const int *order;                  // groups, heaviest first
    int seg_stages;                    // K stages per TMEM segment (fresh accumulator)
    int flush_segs;                    // segments summed in FP32 before the FP64 flush
    long long wait_cycles;             // limit of each bounded wait (SM clock cycles)
};
void launch_tcg_pack_blocks(const double *src, long long nblk, int ld, int Nd, int Kd, int nch,
                            int NGb, uint16_t *dst, cudaStream_t s);
void launch_tcg_pack_x(const double *W, long long w_box_stride, int Kd, int nbox, int nr, int Rp,
                       int nch, int is_near, int d, int n, int leaf, int L, const double *u,
                       long long ldu, uint16_t *dst, cudaStream_t s);
// Shared-memory bytes of one slot of the lead ring (a1, b1) and of the cross ring (a2, a3,
// b2, b3) of the grouped kernel for Nw = 8 NGw block rows per pass.
size_t tcg_lead_bytes(int NGw);
size_t tcg_cross_bytes(int NGw);
void launch_tc_group(const TcgArgs &a, const void *tmap, cudaStream_t s);
int tcg_encode_source_map(void *tmap_out, const uint16_t *base, int nch, int Rp, int nb1, int d);
constexpr int kTcMaxStages = 8;   // deepest cross copy ring of the tensor-core kernel
constexpr int kTcMaxLead = 16;    // deepest lead copy ring

// Tensor grids: factors of every (level, dim, box), U(i, mu) = L_mu(x_i) and
// V(i, mu) = L_mu(x_i) w_i on the Chebyshev points of the box's geometric cell.
// geo: the level's device geometry array, per dimension [first | cnt | uoff | voff], each
// 2^level ints.
void launch_factor_tensor(int d, int n, int level, int p, const double *coords,
                          const double *width, const int *geo, double *Upool, double *Vpool,
                          cudaStream_t s);
// Tensor grids: K_ii w_i = int over the cell of point i of k(x_i, y) dy for every point.
void launch_diag_points(const KernelDesc &k, int d, int n, const double *coords,
                        const double *edges, int q, const double *gx, const double *gw,
                        double *diag, cudaStream_t s);

}  // namespace htlr
