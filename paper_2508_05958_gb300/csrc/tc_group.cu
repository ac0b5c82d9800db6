// Tensor-core block stream for SHARED operators, grouped by target (tcgen05, sm_103a).
//
// With SHARED storage every admissible block of a level with the same box offset
// o = sigma - tau is the same matrix B_o (and likewise for the inadmissible leaves), so
// the products B_o X_{tau+o} of several targets tau can read B_o once.  Per level, the
// targets of one parity class (b_1 mod 2, b_2 mod 2, b_3 mod 2) have the same offsets,
// except where tau + o leaves the domain.  A group is G same-parity targets along
// dimension 1, tau_k = tau_0 + 2k e_1, and the kernel forms the transposed products
//
//     Y^T[(k, r), t] += sum_s X_{tau_k + o}[s, r] B_o[t, s]      (every offset o),
//
// an MMA with M = G x Rp = 128 rows (target, right-hand side), N = the block's rows and
// K = its columns, FP32 accumulation in TMEM.  One CTA owns a group for all of its
// offsets, so Y_tau is complete when it is written: no partial sums across CTAs.
//
// Operands (three-way BF16 split, the six products a_i b_j with i + j <= 2):
//   A = the source tensors X_{tau_k + o} of the G targets: one 5-D TMA tensor load per
//       split gathers them, because the sources of a group sit at stride 2 boxes along
//       dimension 1 (the tensor is the packed source array viewed as
//       [b_23][q][c_1][split, chunk, row group][128 elements], b_1 = 2q + c_1); sources
//       outside the domain read zeros;
//   B = B_o, packed at construction chunk by chunk, one bulk copy per stage.
// Both in the canonical K-major layout without swizzle: 8-row groups 256 bytes apart
// (SBO), the two 8-column core matrices of a 16-column chunk 128 bytes apart (LBO).
//
// Roles (10 warps):
//   * one thread of warp 1 issues the copies into an S-stage ring as soon as a stage is
//     free ("empty" mbarrier, committed by the MMAs that read it);
//   * one thread of warp 0 waits for each stage ("full" mbarrier, completed by the
//     copies' byte count) and issues its MMAs;
//   * warps 2..9 drain the accumulator.
// Accumulation is segmented, because the tensor cores' FP32 accumulation loses about
// 2e-8 relative per accumulated MMA, with a bias, so the error grows with the number of
// MMAs summed in one accumulator (7.6e-4 over a whole c3 row).  Every `seg_stages`
// stages the MMA thread commits the segment and switches to the other of two TMEM
// accumulator buffers (N <= 256 columns each; wider block lists are done in two passes
// over N).  The drain warps read the finished buffer with tcgen05.ld, add it to FP32
// sums held in their registers (two warps per TMEM lane quadrant, half the columns
// each), and release the buffer.  The drain of one segment overlaps the MMAs of the
// next.  At the end of a pass the sums are written as the FP64 partials of the group's
// rows.
// Groups are taken heaviest first from an atomic counter over a host-sorted order, so
// the SMs finish together.  Every wait is bounded (A.wait_cycles SM cycles): on timeout
// the kernel records kDevTimeout, waits (with the long default limit) for the copies and
// MMAs it has issued, frees TMEM and returns.
#include <cuda.h>

#include "tc_common.cuh"

namespace htlr {

using namespace tcc;

namespace {

constexpr int kGThreads = 320;        // MMA warp, copy warp, eight drain warps
constexpr int kDrainThreads = 256;
constexpr int kMaxDrainChunks = 16;   // 8-column chunks per drain thread (Nw <= 256)
constexpr int kMaxGroupOffsets = 1024;

}  // namespace

// ---------------------------------------------------------------------------------
// Construction: pack FP64 blocks ([s][t], leading dimension ld, Nd x Kd) into
// [chunk][split][row group (NGb)][kcore (2)][8][8] split-BF16 elements.
// ---------------------------------------------------------------------------------
__global__ void tcg_pack_blocks_kernel(const double *__restrict__ src, long long nblk, int ld,
                                       int Nd, int Kd, int nch, int NGb, uint16_t *__restrict__ dst)
{
    const long long per_chunk = (long long)kSplits * NGb * 128;
    const long long per_blk = per_chunk * nch;
    const long long total = per_blk * nblk;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long b = idx / per_blk;
        long long rem = idx % per_blk;
        const int ch = (int)(rem / per_chunk);
        rem %= per_chunk;
        const int split = (int)(rem / (NGb * 128));
        rem %= NGb * 128;
        const int gn = (int)(rem / 128), o = (int)(rem % 128);
        const int c = o / 64, row = (o % 64) / 8, e = o % 8;
        const int t = gn * 8 + row, s = ch * 16 + c * 8 + e;
        const double x =
            (t < Nd && s < Kd) ? src[b * (long long)ld * Kd + (long long)s * ld + t] : 0.0;
        dst[idx] = bf16_split(x, split);
    }
}

void launch_tcg_pack_blocks(const double *src, long long nblk, int ld, int Nd, int Kd, int nch,
                            int NGb, uint16_t *dst, cudaStream_t s)
{
    if (nblk > 0)
        tcg_pack_blocks_kernel<<<152 * 8, 256, 0, s>>>(src, nblk, ld, Nd, Kd, nch, NGb, dst);
}

// ---------------------------------------------------------------------------------
// Per matvec: pack the source operand per box as [split][chunk][row group (Rp / 8)]
// [kcore (2)][8][8]: far field W [box][r][pd] (FP64), near field u gathered per leaf.
// Rows r >= nr and columns s >= Kd are zero.
// ---------------------------------------------------------------------------------
__global__ void tcg_pack_x_kernel(const double *__restrict__ W, long long w_box_stride, int Kd,
                                  int nbox, int nr, int Rp, int nch, int is_near, int d, int n,
                                  int leaf, int L, const double *__restrict__ u, long long ldu,
                                  uint16_t *__restrict__ dst)
{
    const int NGa = Rp / 8;
    const long long per_split = (long long)nch * NGa * 128;
    const long long per_box = kSplits * per_split;
    const long long total = per_box * nbox;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long box = idx / per_box;
        long long rem = idx % per_box;
        const int split = (int)(rem / per_split);
        rem %= per_split;
        const int ch = (int)(rem / (NGa * 128));
        rem %= NGa * 128;
        const int g = (int)(rem / 128), o = (int)(rem % 128);
        const int c = o / 64, row = (o % 64) / 8, e = o % 8;
        const int r = g * 8 + row, s = ch * 16 + c * 8 + e;
        double x = 0.0;
        if (r < nr && s < Kd) {
            if (is_near) {
                const int nl1 = 1 << L;
                long long nat = 0, str = 1;
                int ss = s;
                for (int k = 0; k < d; ++k) {
                    const int bk = (int)((box >> (L * k)) & (nl1 - 1));
                    nat += (long long)(bk * leaf + ss % leaf) * str;
                    ss /= leaf;
                    str *= n;
                }
                x = u[nat + ldu * r];
            } else {
                x = W[box * w_box_stride + (long long)r * Kd + s];
            }
        }
        dst[idx] = bf16_split(x, split);
    }
}

void launch_tcg_pack_x(const double *W, long long w_box_stride, int Kd, int nbox, int nr, int Rp,
                       int nch, int is_near, int d, int n, int leaf, int L, const double *u,
                       long long ldu, uint16_t *dst, cudaStream_t s)
{
    tcg_pack_x_kernel<<<152 * 8, 256, 0, s>>>(W, w_box_stride, Kd, nbox, nr, Rp, nch, is_near, d,
                                              n, leaf, L, u, ldu, dst);
}

// ---------------------------------------------------------------------------------
// The grouped stream.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kGThreads, 1)
    tc_group_kernel(const __grid_constant__ CUtensorMap tmap, TcgArgs A)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full_bar[kTcMaxStages], empty_bar[kTcMaxStages];
    __shared__ uint64_t seg_full[2], seg_empty[2], done_bar;
    __shared__ uint32_t tmem_holder, consumed;
    __shared__ volatile int abort_flag;
    __shared__ int n_valid, cur_group;
    __shared__ short valid_idx[kMaxGroupOffsets];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = A.stages, G = A.G, Rp = A.Rp, NGa = Rp / 8, nch = A.nch, NGb = A.NGb;
    const int Nw = A.Nw, NGw = Nw / 8, passes = A.passes;
    const long long F = A.seg_stages;                           // stages per segment
    const uint32_t a_split_bytes = 128u * 16u * 2u;             // 128 rows x 16 columns
    const uint32_t a_bytes = kSplits * a_split_bytes;
    const uint32_t b_split_bytes = (uint32_t)NGw * 256u;        // Nw rows x 16 columns
    const uint32_t b_bytes = kSplits * b_split_bytes;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&seg_full[b], 1);
            mbar_init(&seg_empty[b], kDrainThreads);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(A.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;
    // D f32, A and B bf16, both K-major, N = Nw, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Nw >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);
    const uint32_t lbo = 128, sbo = 256;
    const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
    const int nb1 = A.nb1;
    // drain warps 2..9: TMEM lane quadrant warp % 4 (accumulator row m), and one half of
    // the Nw columns of a pass each; their running sums stay in registers
    const bool drainer = warp >= 2;
    const int m = ((warp & 3) << 5) + lane;
    const int half = (warp - 2) >> 2;
    const int my_cols = Nw / 2, my_c0 = half * my_cols;   // a multiple of 8
    const int nck = my_cols / 8;                          // <= kMaxDrainChunks
    // counters run across groups
    uint32_t it_p = 0;       // loads issued (producer, tid 32)
    uint32_t it_c = 0;       // stages consumed (MMA thread, tid 0)
    uint32_t sc_m = 0;       // segments committed (MMA thread)
    uint32_t sc_d = 0;       // segments drained (drain threads)
    int done_pending = 0;
    uint32_t done_ph = 0;
    bool ok = true;

    while (true) {
        // next group, heaviest first (dynamic: an atomic counter over a host-sorted order)
        if (tid == 0) cur_group = atomicAdd(A.counter, 1);
        __syncthreads();
        const long long gi = cur_group;
        if (gi >= A.ngroups) break;
        const long long grp = A.order[gi];
        // group -> (b23, c1, j): tau_0 = (c1 + 2 j G, b2, b3)
        const int j = (int)(grp % A.nq);
        const long long rest = grp / A.nq;
        const int c1 = (int)(rest % 2);
        const int b23 = (int)(rest / 2);
        const int b2 = b23 % nb1, b3 = A.d == 3 ? b23 / nb1 : 0;
        const int t0b1 = c1 + 2 * j * G;
        const int cls = c1 + 2 * (b2 & 1) + 4 * (b3 & 1);
        const int4 *offs = A.offs + A.cls_start[cls];
        const int noff = A.cls_count[cls];
        // offsets with at least one source inside the domain (warp 0, in list order)
        if (warp == 0) {
            int cnt = 0;
            for (int base = 0; base < noff; base += 32) {
                const int i = base + lane;
                bool v = false;
                if (i < noff) {
                    const int4 o = offs[i];
                    const int s2 = b2 + o.y, s3 = b3 + o.z, lo = t0b1 + o.x;
                    v = s2 >= 0 && s2 < nb1 && (A.d == 2 || (s3 >= 0 && s3 < nb1)) &&
                        lo + 2 * (G - 1) >= 0 && lo < nb1;
                }
                const unsigned msk = __ballot_sync(0xffffffffu, v);
                if (v) valid_idx[cnt + __popc(msk & ((1u << lane) - 1u))] = (short)i;
                cnt += __popc(msk);
            }
            if (lane == 0) n_valid = cnt;
        }
        __syncthreads();
        const long long total = (long long)n_valid * nch;          // stages per pass
        const long long nseg = (total + F - 1) / F;                 // segments per pass
        if (tid == 32 && total > 0) {
            // producer: refill a stage as soon as the MMAs that read it are done
            for (int ps = 0; ps < passes && !abort_flag; ++ps)
                for (long long q = 0; q < total; ++q, ++it_p) {
                    const int s = (int)(it_p % S);
                    if (it_p >= (uint32_t)S &&
                        !mbar_wait(&empty_bar[s], ((it_p / S) - 1) & 1, A.wait_cycles, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    const int4 o = offs[valid_idx[(int)(q / nch)]];
                    const int ch = (int)(q % nch);
                    const int s0 = t0b1 + o.x;                 // b_1 of the first source
                    const int sc1 = s0 & 1;                    // (two's complement: also < 0)
                    const int sq0 = (s0 - sc1) / 2;
                    const int sb23 = (b2 + o.y) + nb1 * (b3 + o.z);
                    unsigned char *st = sm + (size_t)s * stage_bytes;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                     smem_u32(&full_bar[s])),
                                 "r"(stage_bytes)
                                 : "memory");
                    for (int a = 0; a < kSplits; ++a)
                        tensor_load_5d(st + a * a_split_bytes, &tmap, 0, (a * nch + ch) * NGa, sc1,
                                       sq0, sb23, &full_bar[s]);
                    const uint16_t *gb = A.blocks + (long long)o.w * A.core_elems +
                                         (long long)ch * (kSplits * NGb * 128);
                    if (passes == 1) {
                        bulk_load(st + a_bytes, gb, b_bytes, &full_bar[s]);
                    } else {
                        for (int b = 0; b < kSplits; ++b)
                            bulk_load(st + a_bytes + b * b_split_bytes,
                                      gb + (long long)b * NGb * 128 + (long long)ps * NGw * 128,
                                      b_split_bytes, &full_bar[s]);
                    }
                }
        }
        if (tid == 0 && total > 0) {
            // MMA issue: the six split products into the segment's accumulator buffer
            for (int ps = 0; ps < passes && !abort_flag; ++ps)
                for (long long q = 0; q < total; ++q, ++it_c) {
                    const long long qs = q % F;
                    const uint32_t buf = sc_m & 1;
                    if (qs == 0) {
                        // the buffer's previous segment must be drained before it is reset
                        if (sc_m >= 2 &&
                            !mbar_wait(&seg_empty[buf], ((sc_m >> 1) - 1) & 1, A.wait_cycles, &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                    }
                    const int s = (int)(it_c % S);
                    if (!mbar_wait(&full_bar[s], (it_c / S) & 1, A.wait_cycles, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    const uint32_t a_base = smem_u32(sm + (size_t)s * stage_bytes);
                    const uint32_t b_base = a_base + a_bytes;
                    for (int pr = 0; pr < 6; ++pr) {
                        const uint32_t accumulate = (qs == 0 && pr == 0) ? 0u : 1u;
                        mma_bf16(tmem + buf * (uint32_t)Nw,
                                 smem_desc(a_base + pa[pr] * a_split_bytes, lbo, sbo),
                                 smem_desc(b_base + pb[pr] * b_split_bytes, lbo, sbo), idesc,
                                 accumulate);
                    }
                    mma_commit(&empty_bar[s]);
                    if (qs == F - 1 || q == total - 1) {
                        mma_commit(&seg_full[buf]);
                        ++sc_m;
                    }
                }
            consumed = it_c;
        }
        if (drainer) {
            // accumulator row m = k Rp + r: target tau_k = tau_0 + 2k e_1, RHS r
            const int k = m / Rp, r = m % Rp;
            const int tb1 = t0b1 + 2 * k;
            double *out = nullptr;
            if (tb1 < nb1 && r < A.nr) {
                const int tau = tb1 + nb1 * b23;
                const int ta = A.row_task[tau];
                if (A.row_task[tau + 1] > ta) out = A.part + A.tasks[ta].part + (long long)r * A.ld;
            }
            for (int ps = 0; ps < passes; ++ps) {
                float acc[kMaxDrainChunks * 8];
#pragma unroll
                for (int i = 0; i < kMaxDrainChunks * 8; ++i) acc[i] = 0.f;
                for (long long sg = 0; sg < nseg; ++sg, ++sc_d) {
                    const uint32_t buf = sc_d & 1;
                    if (!mbar_wait(&seg_full[buf], (sc_d >> 1) & 1, A.wait_cycles, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                           buf * (uint32_t)Nw + (uint32_t)my_c0;
#pragma unroll
                    for (int c = 0; c < kMaxDrainChunks; ++c) {
                        if (c < nck) {
                            uint32_t v[8];
                            asm volatile(
                                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]),
                                  "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
                                : "r"(tbase + (uint32_t)(8 * c)));
                            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                            for (int jj = 0; jj < 8; ++jj) acc[8 * c + jj] += __uint_as_float(v[jj]);
                        }
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                     smem_u32(&seg_empty[buf]))
                                 : "memory");
                }
                if (abort_flag) break;
                if (out) {
                    const int col0 = ps * Nw + my_c0;
#pragma unroll
                    for (int i = 0; i < kMaxDrainChunks * 8; ++i)
                        if (i < my_cols && col0 + i < A.Nd) out[col0 + i] = (double)acc[i];
                }
            }
        }
        __syncthreads();
        if (abort_flag) {
            ok = false;
            break;
        }
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(A.err, (int)kDevTimeout);
            // every MMA issued by this CTA finishes before TMEM is released
            mma_commit(&done_bar);
            ++done_pending;
            for (; done_pending > 0; --done_pending) {
                mbar_wait(&done_bar, done_ph);
                done_ph ^= 1;
            }
        }
        if (tid == 32) {
            // every copy issued into shared memory lands before the CTA exits
            for (uint32_t it = consumed; it < it_p; ++it)
                mbar_wait(&full_bar[it % S], (it / S) & 1);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(A.tmem_cols));
}

size_t tcg_stage_bytes(int NGw) { return (size_t)kSplits * 128 * 16 * 2 + (size_t)kSplits * NGw * 256; }

void launch_tc_group(const TcgArgs &a, const void *tmap, cudaStream_t s)
{
    if (a.ngroups <= 0) return;
    cudaMemsetAsync(a.counter, 0, sizeof(int), s);
    const size_t smem = tcg_stage_bytes(a.Nw / 8) * a.stages;
    cudaFuncSetAttribute(tc_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = a.ngroups < 152 ? (int)a.ngroups : 152;
    tc_group_kernel<<<grid, kGThreads, smem, s>>>(*static_cast<const CUtensorMap *>(tmap), a);
}

// ---------------------------------------------------------------------------------
// Host: the tensor map of a packed source array for Rp right-hand sides at a level with
// nb1 boxes per dimension: [b23][q][c1][split, chunk, row group][128 elements].
// ---------------------------------------------------------------------------------
namespace {
using EncodeFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                              const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                              const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                              CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encode_fn()
{
    static EncodeFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}
}  // namespace

int tcg_encode_source_map(void *tmap_out, const uint16_t *base, int nch, int Rp, int nb1, int d)
{
    EncodeFn fn = encode_fn();
    if (!fn) return HTLR_ECUDA;
    const int NGa = Rp / 8;
    const int G = 128 / Rp;
    const cuuint64_t box_elems = (cuuint64_t)kSplits * nch * NGa * 128;
    const cuuint64_t nb23 = d == 3 ? (cuuint64_t)nb1 * nb1 : (cuuint64_t)nb1;
    cuuint64_t dims[5] = {128, (cuuint64_t)kSplits * nch * NGa, 2, (cuuint64_t)(nb1 / 2), nb23};
    cuuint64_t strides[4] = {256, box_elems * 2, box_elems * 4, box_elems * 2 * nb1};
    cuuint32_t box[5] = {128, (cuuint32_t)NGa, 1, (cuuint32_t)G, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = fn(static_cast<CUtensorMap *>(tmap_out), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5,
                    const_cast<uint16_t *>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? HTLR_OK : HTLR_ECUDA;
}

}  // namespace htlr
