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
// accumulator buffers (N <= 256 columns each; wider block lists are done in several
// passes over N).  The drain warps read the finished buffer with tcgen05.ld, add it to FP32
// sums held in their registers (two warps per TMEM lane quadrant, half the columns
// each), and release the buffer.  The drain of one segment overlaps the MMAs of the
// next.  At the end of a pass the sums are written as the FP64 partials of the group's
// rows.
// Work items, one pass of one group each, are taken heaviest first from an atomic counter
// over a host-sorted order, so the SMs finish together.  Every wait is bounded (A.wait_cycles SM cycles): on timeout
// the kernel records kDevTimeout, waits (with the long default limit) for the copies and
// MMAs it has issued, frees TMEM and returns.
#include <cuda.h>

#include "tc_common.cuh"

namespace htlr {

using namespace tcc;

namespace {

constexpr int kGThreads = 320;        // MMA warp, copy warp, eight drain warps
constexpr int kDrainThreads = 256;
constexpr int kMaxDrainChunks = kTcgMaxNw / 16;   // 8-column chunks per drain thread
constexpr int kLdBatch = 1;           // tensor-memory loads in flight per drain thread
constexpr int kMaxGroupOffsets = 1024;

}  // namespace

// FP32 -> FP64 by integer operations (the FP64 pipe is slow on this part); zero and
// subnormal inputs give signed zero, infinities and NaN keep their class.
__device__ __forceinline__ double widen_f32(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xFFu;
    const unsigned long long sign = (unsigned long long)(b & 0x80000000u) << 32;
    const unsigned long long man = (unsigned long long)(b & 0x7FFFFFu) << 29;
    unsigned long long bits = sign | ((unsigned long long)(e + 896u) << 52) | man;
    bits = e == 0u ? sign : bits;
    bits = e == 0xFFu ? (sign | 0x7FF0000000000000ull | man) : bits;
    return __longlong_as_double((long long)bits);
}

// L2 policy for the partial rows: kept in L2 ahead of streamed data, so that the
// periodic additions of a row find it there instead of in DRAM.
__device__ __forceinline__ uint64_t l2_evict_last()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// *p += v in FP64 at L2, without waiting for it (the owner thread is the only writer).
__device__ __forceinline__ void red_add_f64(double *p, double v, uint64_t pol)
{
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void st_f64_hint(double *p, double v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol)
                 : "memory");
}

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
// Three-way BF16 split of x from one rounding to FP32: x ~ h = a1 + a2 + a3 exactly,
// |x - h| <= 2^-24 |x|; the splits themselves are exact FP32 subtractions.
__device__ __forceinline__ void bf16_split3_f32(double x, uint16_t &s1, uint16_t &s2, uint16_t &s3)
{
    const float h = __double2float_rn(x);
    const __nv_bfloat16 a1 = __float2bfloat16_rn(h);
    const float r1 = __fsub_rn(h, __bfloat162float(a1));
    const __nv_bfloat16 a2 = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(a2));
    s1 = __bfloat16_as_ushort(a1);
    s2 = __bfloat16_as_ushort(a2);
    s3 = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

// One thread per element of the packed tile layout of one box (grid.y = box): reads its
// source value once (W [box][r][Kd] for the far field, u gathered from natural order for
// the near field), writes its three split terms at the same position of the three split
// planes.  Consecutive threads cover 8 columns x 4 rows of a core matrix pair, so the
// reads come in 64-byte runs and each split's writes are contiguous.
__global__ void __launch_bounds__(256) tcg_pack_x_kernel(
    const double *__restrict__ W, long long w_box_stride, int Kd, int nbox, int nr, int Rp,
    int nch, int is_near, int d, int n, int leaf, int L, const double *__restrict__ u,
    long long ldu, uint16_t *__restrict__ dst)
{
    const int NGa = Rp / 8;
    const int per_split = nch * NGa * 128;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= per_split) return;
    const int ch = idx / (NGa * 128);
    const int rem = idx - ch * (NGa * 128);
    const int g = rem >> 7, o = rem & 127;
    const int c = o >> 6, row = (o >> 3) & 7, e = o & 7;
    const int r = g * 8 + row, s = ch * 16 + c * 8 + e;
    for (long long box = blockIdx.y; box < nbox; box += gridDim.y) {
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
        uint16_t s1, s2, s3;
        bf16_split3_f32(x, s1, s2, s3);
        uint16_t *out = dst + box * (long long)kSplits * per_split + idx;
        out[0] = s1;
        out[per_split] = s2;
        out[2 * per_split] = s3;
    }
}

void launch_tcg_pack_x(const double *W, long long w_box_stride, int Kd, int nbox, int nr, int Rp,
                       int nch, int is_near, int d, int n, int leaf, int L, const double *u,
                       long long ldu, uint16_t *dst, cudaStream_t s)
{
    const int per_split = nch * (Rp / 8) * 128;
    dim3 grid((per_split + 255) / 256, nbox < 65535 ? nbox : 65535);
    tcg_pack_x_kernel<<<grid, 256, 0, s>>>(W, w_box_stride, Kd, nbox, nr, Rp, nch, is_near, d, n,
                                           leaf, L, u, ldu, dst);
}

// ---------------------------------------------------------------------------------
// The grouped stream.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kGThreads, 1)
    tc_group_kernel(const __grid_constant__ CUtensorMap tmap, TcgArgs A)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    // two copy rings: the lead ring holds a1 and b1 of a stage until the segment's leading
    // products are issued; the cross ring holds a2, a3, b2, b3 and is released as soon as
    // the stage's cross products are done.  full_bar (per cross slot) completes when all
    // of a stage's copies have landed
    __shared__ uint64_t full_bar[kTcMaxStages], cross_empty[kTcMaxStages];
    __shared__ uint64_t lead_empty[kTcMaxLead];
    __shared__ uint64_t seg_full[2], seg_empty[2], done_bar;
    __shared__ uint32_t tmem_holder, consumed;
    __shared__ volatile int abort_flag;
    __shared__ int n_valid, cur_group;
    __shared__ short valid_idx[kMaxGroupOffsets];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Sc = A.stages, Sl = A.lead_stages;
    const int G = A.G, Rp = A.Rp, NGa = Rp / 8, nch = A.nch, NGb = A.NGb;
    const int Nw = A.Nw, NGw = Nw / 8, passes = A.passes;
    const long long F = A.seg_stages;                           // stages per segment
    const uint32_t a_split_bytes = 128u * 16u * 2u;             // 128 rows x 16 columns
    const uint32_t b_split_bytes = (uint32_t)NGw * 256u;        // Nw rows x 16 columns
    const uint32_t lead_bytes = a_split_bytes + b_split_bytes;  // a1, b1
    const uint32_t cross_bytes = 2u * lead_bytes;               // a2, a3, b2, b3
    const uint32_t stage_bytes = lead_bytes + cross_bytes;
    unsigned char *const cross_ring = sm + (size_t)Sl * lead_bytes;
    if (tid == 0) {
        for (int s = 0; s < Sc; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&cross_empty[s], 1);
        }
        for (int s = 0; s < Sl; ++s) mbar_init(&lead_empty[s], 1);
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
    // ring positions, carried incrementally (no divisions in the issue loops): slot
    // index, lap parity and "first lap" of the cross and lead rings, per role
    int pc = 0, pl = 0;                      // producer: next cross / lead slot
    uint32_t pc_lap = 0, pl_lap = 0;         // producer: lap parity of those slots
    bool pc_first = true, pl_first = true;   // producer: slot not used before
    int mc = 0, ml = 0;                      // MMA thread: next cross / lead slot
    uint32_t mc_lap = 0;                     // MMA thread: lap parity of the cross slot
    uint32_t sc_m = 0;       // segments committed (MMA thread)
    uint32_t sc_d = 0;       // segments drained (drain threads)
    int done_pending = 0;
    uint32_t done_ph = 0;
    bool ok = true;

    while (true) {
        // next work item, heaviest first (dynamic: an atomic counter over a host-sorted
        // order).  An item is one pass over N of one group: the passes of a group write
        // disjoint columns of its partial rows, so they run on different CTAs, which
        // doubles the items of two-pass block lists (levels with few groups fill the SMs)
        if (tid == 0) cur_group = atomicAdd(A.counter, 1);
        __syncthreads();
        const long long gi = cur_group;
        if (gi >= A.ngroups * passes) break;
        const long long grp = A.order[gi / passes];
        const int ps_lo = (int)(gi % passes), ps_hi = ps_lo + 1;   // this item's pass
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
            // producer: stage it_p goes to cross slot it_p % Sc and lead slot it_p % Sl, each
            // refilled once the MMAs that read its previous stage are done
            for (int ps = ps_lo; ps < ps_hi && !abort_flag; ++ps) {
                int oi = 0, ch = 0;                    // offset (in valid order) and chunk
                for (long long q = 0; q < total; ++q, ++it_p) {
                    const int c = pc, l = pl;
                    if (!pc_first &&
                        !mbar_wait(&cross_empty[c], pc_lap ^ 1u, A.wait_cycles, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    if (!pl_first &&
                        !mbar_wait(&lead_empty[l], pl_lap ^ 1u, A.wait_cycles, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    if (++pc == Sc) {
                        pc = 0;
                        pc_lap ^= 1u;
                        pc_first = false;
                    }
                    if (++pl == Sl) {
                        pl = 0;
                        pl_lap ^= 1u;
                        pl_first = false;
                    }
                    const int4 o = offs[valid_idx[oi]];
                    const int chc = ch;
                    if (++ch == nch) {
                        ch = 0;
                        ++oi;
                    }
                    const int s0 = t0b1 + o.x;                 // b_1 of the first source
                    const int sc1 = s0 & 1;                    // (two's complement: also < 0)
                    const int sq0 = (s0 - sc1) / 2;
                    const int sb23 = (b2 + o.y) + nb1 * (b3 + o.z);
                    unsigned char *ld = sm + (size_t)l * lead_bytes;
                    unsigned char *cr = cross_ring + (size_t)c * cross_bytes;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                                     smem_u32(&full_bar[c])),
                                 "r"(stage_bytes)
                                 : "memory");
                    // A splits: a1 to the lead slot, a2 and a3 to the cross slot
                    tensor_load_5d(ld, &tmap, 0, chc * NGa, sc1, sq0, sb23, &full_bar[c]);
                    for (int a = 1; a < kSplits; ++a)
                        tensor_load_5d(cr + (a - 1) * a_split_bytes, &tmap, 0, (a * nch + chc) * NGa,
                                       sc1, sq0, sb23, &full_bar[c]);
                    // B splits (block B_o, chunk ch, this pass's rows): b1 to the lead slot, b2
                    // and b3 to the cross slot (contiguous when the block is one pass wide)
                    const uint16_t *gb = A.blocks + (long long)o.w * A.core_elems +
                                         (long long)chc * (kSplits * NGb * 128) +
                                         (long long)ps * NGw * 128;
                    bulk_load(ld + a_split_bytes, gb, b_split_bytes, &full_bar[c]);
                    if (passes == 1) {
                        bulk_load(cr + 2 * a_split_bytes, gb + (long long)NGb * 128,
                                  2 * b_split_bytes, &full_bar[c]);
                    } else {
                        for (int b = 1; b < kSplits; ++b)
                            bulk_load(cr + 2 * a_split_bytes + (b - 1) * b_split_bytes,
                                      gb + (long long)b * NGb * 128, b_split_bytes, &full_bar[c]);
                    }
                }
            }
        }
        if (tid == 0 && total > 0) {
            // MMA issue, segment by segment: a segment is F consecutive stages accumulated
            // in one TMEM buffer, started fresh.  Each stage's cross products (a3b1, a2b2,
            // a1b3, a2b1, a1b2) are issued as soon as it lands, and its cross slot released;
            // the leading products a1b1 of the segment come last, once the accumulator holds
            // the small cross terms only, so that its truncation acts on few additions of
            // full magnitude
            // shared-memory descriptors as a base plus (byte offset >> 4): the address field
            // is the low 14 bits (addresses below 256 KB), so offsets add without carry
            const uint64_t d0 = smem_desc(smem_u32(sm), lbo, sbo);
            const uint32_t a16 = a_split_bytes >> 4, b16 = b_split_bytes >> 4;
            const uint32_t lead16 = lead_bytes >> 4, cross16 = cross_bytes >> 4;
            const uint32_t cring16 = (uint32_t)((size_t)Sl * lead_bytes) >> 4;
            for (int ps = ps_lo; ps < ps_hi && !abort_flag; ++ps)
                for (long long q0 = 0; q0 < total; q0 += F) {
                    const int nq = (int)(total - q0 < F ? total - q0 : F);
                    const uint32_t buf = sc_m & 1;
                    const uint32_t dt = tmem + buf * (uint32_t)Nw;
                    // the buffer's previous segment must be drained before it is reset
                    if (sc_m >= 2 &&
                        !mbar_wait(&seg_empty[buf], ((sc_m >> 1) - 1) & 1, A.wait_cycles, &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const int ml0 = ml;                      // lead slot of the segment's first stage
                    bool landed = true;
                    for (int i = 0; i < nq; ++i) {
                        if (!mbar_wait(&full_bar[mc], mc_lap, A.wait_cycles, &abort_flag)) {
                            landed = false;
                            break;
                        }
                        ++it_c;
                        const uint64_t dl = d0 + (uint64_t)((uint32_t)ml * lead16);   // a1 | b1
                        const uint64_t dc = d0 + (uint64_t)(cring16 + (uint32_t)mc * cross16);
                        // a2 = dc, a3 = dc + a16, b2 = dc + 2 a16, b3 = dc + 2 a16 + b16;
                        // a1 = dl, b1 = dl + a16
                        mma_bf16(dt, dc + a16, dl + a16, idesc, i == 0 ? 0u : 1u);     // a3 b1
                        mma_bf16(dt, dc, dc + 2 * a16, idesc, 1u);                      // a2 b2
                        mma_bf16(dt, dl, dc + 2 * a16 + b16, idesc, 1u);                // a1 b3
                        mma_bf16(dt, dc, dl + a16, idesc, 1u);                          // a2 b1
                        mma_bf16(dt, dl, dc + 2 * a16, idesc, 1u);                      // a1 b2
                        mma_commit(&cross_empty[mc]);
                        if (++mc == Sc) {
                            mc = 0;
                            mc_lap ^= 1u;
                        }
                        if (++ml == Sl) ml = 0;
                    }
                    if (!landed) {
                        abort_flag = 1;
                        break;
                    }
                    for (int i = 0, l = ml0; i < nq; ++i) {
                        const uint64_t dl = d0 + (uint64_t)((uint32_t)l * lead16);
                        mma_bf16(dt, dl, dl + a16, idesc, 1u);                          // a1 b1
                        mma_commit(&lead_empty[l]);
                        if (++l == Sl) l = 0;
                    }
                    mma_commit(&seg_full[buf]);
                    ++sc_m;
                }
            consumed = it_c;
        }
        if (drainer) {
            // accumulator row m = k Rp + r: target tau_k = tau_0 + 2k e_1, RHS r.  Its FP64
            // partial row in global memory, or null for padding rows (looked up again at each
            // flush rather than held in registers through the drain loop)
            auto row_out = [&]() -> double * {
                const int k = m / Rp, r = m % Rp;
                const int tb1 = t0b1 + 2 * k;
                if (tb1 >= nb1 || r >= A.nr) return nullptr;
                const int tau = tb1 + nb1 * b23;
                const int ta = A.row_task[tau];
                if (A.row_task[tau + 1] <= ta) return nullptr;
                return A.part + A.tasks[ta].part + (long long)r * A.ld;
            };
            const int FL = A.flush_segs;
            for (int ps = ps_lo; ps < ps_hi; ++ps) {
                // FP32 sums of the drained segments; every FL segments (and after the last
                // one) they go to the row's FP64 partial: stored by the first flush of the
                // pass, then added by fire-and-forget L2 reductions, so the drain never waits
                // on memory
                for (long long g0 = 0; g0 < nseg && !abort_flag; g0 += FL) {
                    const long long g1 = g0 + FL < nseg ? g0 + FL : nseg;
                    float acc[kMaxDrainChunks * 8];
#pragma unroll
                    for (int i = 0; i < kMaxDrainChunks * 8; ++i) acc[i] = 0.f;
                    for (long long sg = g0; sg < g1; ++sg, ++sc_d) {
                        const uint32_t buf = sc_d & 1;
                        if (!mbar_wait(&seg_full[buf], (sc_d >> 1) & 1, A.wait_cycles, &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint32_t tbase = tmem + ((uint32_t)((warp & 3) * 32) << 16) +
                                               buf * (uint32_t)Nw + (uint32_t)my_c0;
                        // kLdBatch 8-column loads in flight, then one wait
#pragma unroll
                        for (int c0 = 0; c0 < kMaxDrainChunks; c0 += kLdBatch) {
                            if (c0 < nck) {
                                uint32_t v[kLdBatch][8];
#pragma unroll
                                for (int cc = 0; cc < kLdBatch; ++cc)
                                    if (c0 + cc < nck)
                                        asm volatile(
                                            "tcgen05.ld.sync.aligned.32x32b.x8.b32 "
                                            "{%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                            : "=r"(v[cc][0]), "=r"(v[cc][1]), "=r"(v[cc][2]),
                                              "=r"(v[cc][3]), "=r"(v[cc][4]), "=r"(v[cc][5]),
                                              "=r"(v[cc][6]), "=r"(v[cc][7])
                                            : "r"(tbase + (uint32_t)(8 * (c0 + cc))));
                                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                                for (int cc = 0; cc < kLdBatch; ++cc)
                                    if (c0 + cc < nck)
#pragma unroll
                                        for (int jj = 0; jj < 8; ++jj)
                                            acc[8 * (c0 + cc) + jj] += __uint_as_float(v[cc][jj]);
                            }
                        }
                        asm volatile("tcgen05.fence::before_thread_sync;");
                        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                         smem_u32(&seg_empty[buf]))
                                     : "memory");
                    }
                    if (abort_flag) break;
                    double *o = row_out();
                    if (o) {
                        const int col0 = ps * Nw + my_c0;
                        const int lim = min(my_cols, A.Nd - col0);
                        o += col0;
                        const uint64_t pol = l2_evict_last();
                        if (g0 > 0) {
#pragma unroll
                            for (int i = 0; i < kMaxDrainChunks * 8; ++i)
                                if (i < lim) red_add_f64(o + i, widen_f32(acc[i]), pol);
                        } else {
#pragma unroll
                            for (int i = 0; i < kMaxDrainChunks * 8; ++i)
                                if (i < lim) st_f64_hint(o + i, widen_f32(acc[i]), pol);
                        }
                    }
                }
                if (abort_flag) break;
                double *o = row_out();
                if (nseg == 0 && o) {
                    // a pass without segments: the row's partial is zero
                    const int col0 = ps * Nw + my_c0;
                    for (int i = 0; i < my_cols; ++i)
                        if (col0 + i < A.Nd) o[col0 + i] = 0.0;
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
                mbar_wait(&full_bar[it % Sc], (it / Sc) & 1);
        }
        __syncthreads();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(A.tmem_cols));
}

size_t tcg_lead_bytes(int NGw) { return (size_t)128 * 16 * 2 + (size_t)NGw * 256; }
size_t tcg_cross_bytes(int NGw) { return 2 * tcg_lead_bytes(NGw); }

void launch_tc_group(const TcgArgs &a, const void *tmap, cudaStream_t s)
{
    if (a.ngroups <= 0) return;
    cudaMemsetAsync(a.counter, 0, sizeof(int), s);
    const size_t smem = tcg_lead_bytes(a.Nw / 8) * a.lead_stages + tcg_cross_bytes(a.Nw / 8) * a.stages;
    cudaFuncSetAttribute(tc_group_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const long long items = a.ngroups * a.passes;   // (group, pass) work items
    const int grid = items < 152 ? (int)items : 152;
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
