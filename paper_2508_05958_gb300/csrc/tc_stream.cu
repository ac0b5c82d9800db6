// Tensor-core block stream for many right-hand sides (tcgen05, sm_103a).
//
// For a block row tau of a block list (admissible blocks of one level, or the
// inadmissible leaves), Y_tau = sum_sigma B_{tau sigma} X_sigma with X_sigma the
// contracted source tensor W_sigma (or u_sigma) for Rp right-hand sides: a sum of dense
// GEMMs M = rows, K = cols, N = Rp, accumulated in tensor memory (TMEM).
//
// Arithmetic: three-way BF16 split.  Every operand x is held as x1 + x2 + x3 with
// x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2) (24 significant bits); the
// product keeps the six terms a_i b_j with i + j <= 4 (a1b1, a1b2, a2b1, a1b3, a2b2,
// a3b1), each a tcgen05.mma kind::f16 with FP32 accumulation.  The dropped terms are
// below 2^-24 relative: an FP32-class contraction at BF16 tensor-core rate.
//
// Data path: blocks are packed at construction into the canonical K-major layout of the
// MMA shared-memory descriptors (8 x 16-byte core matrices, no swizzle), chunk by chunk
// of kc columns, the three splits and every 128-row M-tile of a chunk contiguous; the
// source tensors are packed the same way each matvec.  One elected thread moves each
// chunk with bulk asynchronous copies (cp.async.bulk, completion on an mbarrier), issues
// the MMAs and commits them to the stage's "empty" mbarrier; S stages keep copies ahead
// of the tensor core.  After the row, the four warps read the accumulator with
// tcgen05.ld and write an FP64 partial for the usual fixed-order reduction.  Every wait
// is bounded (A.wait_cycles SM cycles): on timeout the kernel records kDevTimeout, waits
// (with the long default limit) for the copies and MMAs it issued, frees TMEM and returns.
#include "tc_common.cuh"

namespace htlr {

using namespace tcc;

namespace {

constexpr int kTcM = 128;
constexpr int kTcThreads = 128;

}  // namespace

// ---------------------------------------------------------------------------------
// Construction: pack FP64 blocks ([s][t], leading dimension ld, `rows` x `cols`) into
// the split-BF16 chunked layout.  Per block: nchunks chunks; per chunk [split][mtile]
// sub-tiles of 128 x kc, canonical layout: element (m, k) at (m / 8) * 64 + (k / 8) *
// 1024 + (m % 8) * 8 + k % 8 (SBO 128 bytes, LBO 2048 bytes).
// ---------------------------------------------------------------------------------
__global__ void tc_pack_blocks_kernel(const double *__restrict__ src, long long nblk, int ld,
                                      int rows, int cols, int mtiles, int kc, int nchunks,
                                      uint16_t *__restrict__ dst)
{
    const long long sub = (long long)kTcM * kc;             // elements per sub-tile
    const long long chunk = (long long)kSplits * mtiles * sub;
    const long long per_blk = chunk * nchunks;
    const long long total = per_blk * nblk;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long b = idx / per_blk;
        long long rem = idx % per_blk;
        const int c = (int)(rem / chunk);
        rem %= chunk;
        const int split = (int)(rem / (mtiles * sub));
        rem %= mtiles * sub;
        const int mt = (int)(rem / sub);
        const int o = (int)(rem % sub);
        const int kcore = o / 1024, g = (o % 1024) / 64, r = (o % 64) / 8, e = o % 8;
        const int t = mt * kTcM + g * 8 + r, s = c * kc + kcore * 8 + e;
        const double x =
            (t < rows && s < cols) ? src[b * (long long)ld * cols + (long long)s * ld + t] : 0.0;
        dst[idx] = bf16_split(x, split);
    }
}

void launch_tc_pack_blocks(const double *src, long long nblk, int ld, int rows, int cols,
                           int mtiles, int kc, int nchunks, uint16_t *dst, cudaStream_t s)
{
    if (nblk > 0)
        tc_pack_blocks_kernel<<<152 * 8, 256, 0, s>>>(src, nblk, ld, rows, cols, mtiles, kc,
                                                      nchunks, dst);
}

// ---------------------------------------------------------------------------------
// Per matvec: pack the source operand.  Far field: W [box][r][pd] (FP64) -> per box
// nchunks x [split][Rp x kc canonical].  Near field: u gathered per leaf (natural order).
// ---------------------------------------------------------------------------------
__global__ void tc_pack_x_kernel(const double *__restrict__ W, long long w_box_stride, int pd,
                                 int nbox, int nr, int Rp, int kc, int nchunks, int is_near,
                                 int d, int n, int leaf, int L, const double *__restrict__ u,
                                 long long ldu, uint16_t *__restrict__ dst)
{
    const long long sub = (long long)Rp * kc;
    const long long chunk = kSplits * sub;
    const long long per_box = chunk * nchunks;
    const long long total = per_box * nbox;
    const int lbo_e = (Rp / 8) * 64;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long box = idx / per_box;
        long long rem = idx % per_box;
        const int c = (int)(rem / chunk);
        rem %= chunk;
        const int split = (int)(rem / sub);
        const int o = (int)(rem % sub);
        const int kcore = o / lbo_e, g = (o % lbo_e) / 64, r = (o % 64) / 8, e = o % 8;
        const int rr = g * 8 + r, s = c * kc + kcore * 8 + e;
        double x = 0.0;
        if (rr < nr && s < pd) {
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
                x = u[nat + ldu * rr];
            } else {
                x = W[box * w_box_stride + (long long)rr * pd + s];
            }
        }
        dst[idx] = bf16_split(x, split);
    }
}

void launch_tc_pack_x(const double *W, long long w_box_stride, int pd, int nbox, int nr, int Rp,
                      int kc, int nchunks, int is_near, int d, int n, int leaf, int L,
                      const double *u, long long ldu, uint16_t *dst, cudaStream_t s)
{
    tc_pack_x_kernel<<<152 * 8, 256, 0, s>>>(W, w_box_stride, pd, nbox, nr, Rp, kc, nchunks,
                                             is_near, d, n, leaf, L, u, ldu, dst);
}

// ---------------------------------------------------------------------------------
// The stream.  Tasks are whole block rows of one kind; grid-stride over tasks, one CTA
// of 128 threads per SM (TMEM: mtiles * Rp columns).
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kTcThreads, 1) tc_stream_kernel(TcArgs A)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full_bar[kTcMaxStages], empty_bar[kTcMaxStages], done_bar;
    __shared__ uint32_t tmem_holder;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = A.stages, mtiles = A.mtiles, kc = A.kc, Rp = A.Rp;
    const uint32_t sub_a = (uint32_t)(kTcM * kc * 2);   // bytes of one A sub-tile
    const uint32_t sub_b = (uint32_t)(Rp * kc * 2);     // bytes of one B sub-tile
    const uint32_t a_chunk_bytes = kSplits * mtiles * sub_a;
    const uint32_t b_chunk_bytes = kSplits * sub_b;
    const uint32_t stage_bytes = a_chunk_bytes + b_chunk_bytes;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
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
    // instruction descriptor: D f32, A and B bf16, both K-major, N = Rp, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Rp >> 3) << 17) |
                           ((uint32_t)(kTcM >> 4) << 24);
    const uint32_t a_lbo = 16 * 128, a_sbo = 128;
    const uint32_t b_lbo = (uint32_t)(Rp / 8) * 128, b_sbo = 128;
    // the six products a_i b_j with i + j <= 2 (0-based)
    const int pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
    // per-stage phase bookkeeping (thread 0 only); bit s of `loaded`: a copy into stage s
    // whose completion has not been observed; of `pending`: MMAs committed to empty_bar[s]
    // whose completion has not been observed
    uint32_t full_ph = 0, empty_ph = 0, pending = 0, loaded = 0;
    uint32_t done_ph = 0;
    int done_out = 0;           // thread 0: commits to done_bar not yet observed
    __shared__ int row_ok;
    bool ok = true;
    const long long lim = A.wait_cycles;

    for (int t = A.t0 + blockIdx.x; t < A.t1 && ok; t += gridDim.x) {
        const Task T = A.tasks[t];
        const int ne = T.e1 - T.e0;
        const long long total = (long long)ne * A.nchunks;
        if (tid == 0 && total > 0) {
            auto load = [&](long long q) -> bool {
                const int s = (int)(q % S);
                if (pending & (1u << s)) {  // the MMAs that read this stage must be done
                    if (!mbar_wait(&empty_bar[s], (empty_ph >> s) & 1, lim)) return false;
                    empty_ph ^= 1u << s;
                    pending &= ~(1u << s);
                }
                const int e = T.e0 + (int)(q / A.nchunks), c = (int)(q % A.nchunks);
                const uint16_t *ga = A.blocks + (long long)A.blk[e] * A.blk_elems +
                                     (long long)c * (a_chunk_bytes / 2);
                const uint16_t *gb = A.x + (long long)A.col[e] * A.x_box_elems +
                                     (long long)c * (b_chunk_bytes / 2);
                unsigned char *st = sm + (size_t)s * stage_bytes;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                 smem_u32(&full_bar[s])),
                             "r"(stage_bytes)
                             : "memory");
                bulk_load(st, ga, a_chunk_bytes, &full_bar[s]);
                bulk_load(st + a_chunk_bytes, gb, b_chunk_bytes, &full_bar[s]);
                loaded |= 1u << s;
                return true;
            };
            for (long long q = 0; q < total && q < S && ok; ++q) ok = load(q);
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (long long q = 0; q < total && ok; ++q) {
                const int s = (int)(q % S);
                if (!mbar_wait(&full_bar[s], (full_ph >> s) & 1, lim)) {
                    ok = false;
                    break;
                }
                full_ph ^= 1u << s;
                loaded &= ~(1u << s);
                const uint32_t a_base = smem_u32(sm + (size_t)s * stage_bytes);
                const uint32_t b_base = a_base + a_chunk_bytes;
                for (int mt = 0; mt < mtiles; ++mt) {
                    const uint32_t d_tmem = tmem + (uint32_t)(mt * Rp);
                    for (int j = 0; j < kc / 16; ++j) {
                        for (int pr = 0; pr < 6; ++pr) {
                            const uint32_t a_addr =
                                a_base + (uint32_t)(pa[pr] * mtiles + mt) * sub_a + 2 * j * a_lbo;
                            const uint32_t b_addr = b_base + (uint32_t)pb[pr] * sub_b + 2 * j * b_lbo;
                            const uint32_t accumulate = (q == 0 && j == 0 && pr == 0) ? 0u : 1u;
                            mma_bf16(d_tmem, smem_desc(a_addr, a_lbo, a_sbo),
                                     smem_desc(b_addr, b_lbo, b_sbo), idesc, accumulate);
                        }
                    }
                }
                mma_commit(&empty_bar[s]);
                pending |= 1u << s;
                // refill the stage of the previous chunk (its MMAs were queued earlier, so
                // the tensor core always has the current chunk to work on meanwhile)
                if (q >= 1 && q - 1 + S < total) ok = load(q - 1 + S);
            }
            if (ok) {
                // the row's MMAs: one commit, observed by thread 0 alone
                mma_commit(&done_bar);
                done_out = 1;
                if (mbar_wait(&done_bar, done_ph, lim)) {
                    done_ph ^= 1;
                    done_out = 0;
                } else {
                    ok = false;
                }
            }
            row_ok = ok ? 1 : 0;
        }
        if (tid == 0 && total == 0) row_ok = 1;
        __syncthreads();
        const int rok = row_ok;
        __syncthreads();   // every thread has read row_ok before thread 0 writes it again
        if (!rok) {
            ok = false;
            break;
        }
        if (total == 0) continue;
        asm volatile("tcgen05.fence::after_thread_sync;");
        {
            // accumulator rows: warp w holds lanes 32 w .. 32 w + 31 of every M-tile
            double *out = A.part + T.part;
            for (int mt = 0; mt < mtiles; ++mt) {
                const int row = mt * kTcM + warp * 32 + lane;
                for (int c0 = 0; c0 < Rp; c0 += 8) {
                    uint32_t r[8];
                    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mt * Rp + c0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                          "=r"(r[6]), "=r"(r[7])
                        : "r"(taddr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                    if (row < A.rows)
                        for (int jj = 0; jj < 8; ++jj)
                            if (c0 + jj < A.nr)
                                out[(long long)(c0 + jj) * A.ld + row] = (double)__uint_as_float(r[jj]);
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    if (!ok) {
        if (tid == 0) {
            atomicExch(A.err, (int)kDevTimeout);
            // clean-up with the long default limit: every MMA this CTA issued finishes
            // (one commit covers them all) and every copy it issued lands before TMEM and
            // shared memory are released
            if (!done_out) {
                mma_commit(&done_bar);
                done_out = 1;
            }
            mbar_wait(&done_bar, done_ph);
            for (int s = 0; s < S; ++s)
                if (pending & (1u << s)) mbar_wait(&empty_bar[s], (empty_ph >> s) & 1);
            for (int s = 0; s < S; ++s)
                if (loaded & (1u << s)) mbar_wait(&full_bar[s], (full_ph >> s) & 1);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(A.tmem_cols));
}

size_t tc_stage_bytes(int mtiles, int kc, int Rp)
{
    return (size_t)kSplits * mtiles * kTcM * kc * 2 + (size_t)kSplits * Rp * kc * 2;
}

void launch_tc_stream(const TcArgs &a, cudaStream_t s)
{
    const int ntasks = a.t1 - a.t0;
    if (ntasks <= 0) return;
    const size_t smem = tc_stage_bytes(a.mtiles, a.kc, a.Rp) * a.stages;
    cudaFuncSetAttribute(tc_stream_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = ntasks < 152 ? ntasks : 152;
    tc_stream_kernel<<<grid, kTcThreads, smem, s>>>(a);
}

}  // namespace htlr
