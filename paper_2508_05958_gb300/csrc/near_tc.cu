// Generated near field on the tensor cores (tcgen05, sm_103a): the inadmissible leaves of
// Algorithm 2 with the kernel values recomputed per point pair (eq. (4.1)), 16 right-hand
// sides at a time:
//
//   f_i = sum_{sigma near tau} sum_{j in sigma, j != i} k(x_i, y_j) (s w_j u_j)
//         + (K_ii w_i + a_i) u_i,                                       i in tau,
//
// with s the kernel's scale and w_j the cell measure of source j.  Per (target leaf, tile
// of 128 rows) this is the MMA  D[i, r] += A[i, j] B[j, r]  with M = 128 rows, N = 16
// right-hand sides and K = the near sources, 16 per stage:
//   A = the kernel values, computed in FP32 by the thread that owns row i (one thread per
//       tensor-memory lane) and written straight into tensor memory (tcgen05.st) as two
//       TF32 terms: a1 = k rounded to TF32 (nearest), a2 = k - a1, exact in FP32, of
//       which the tensor cores read the leading 11 bits;
//   B = s w_j u_j, packed once per launch as two TF32 terms per source (b1 = nearest,
//       b2 = nearest of the rest), leaf by leaf and 16 sources per stage, in the
//       canonical K-major layout without swizzle: 8-row groups (right-hand sides) 256
//       bytes apart, the two 4-column core matrices of an 8-column K step 128 bytes apart.
// Three products a2 b1, a1 b2, a1 b1 per K step (kind::tf32, M 128, N 16, K 8; a2 b2 is
// below 2^-22 relative and dropped), FP32 accumulation in tensor memory.
//
// The arithmetic is the generation: about ten FP32-pipe instructions and one or two SFU
// operations per pair, against the 16 multiply-adds per pair that move to the tensor
// cores.  Coordinates are taken relative to the target leaf's corner in FP64 before the
// rounding to FP32 (as in the CUDA-core generated near field), so neighbouring points keep
// accurate distances.
//
// Accumulation, as in the grouped tensor-core kernel: the tensor cores truncate every
// addition to the FP32 accumulator, so a segment of kSegStages stages starts in a fresh
// accumulator with the small cross products of all its stages, and only then adds the
// leading products a1 b1; the generating threads read the finished segment back
// (tcgen05.ld), add it to FP32 sums in registers, and add those to FP64 sums in shared
// memory every kFlushSegs segments.
//
// CTA: four warpgroups of generating threads, each with its own MMA warp, one CTA per
// SM.  A warpgroup takes (leaf, tile) items from an atomic counter (heaviest first) and
// streams the sources of the leaf's near list: it stages their coordinates in shared
// memory, then per stage generates A into one of three tensor-memory slots while the
// stage's B is copied (cp.async) into the matching shared-memory slot, and hands the
// stage to its MMA thread one stage later (the stores and the copy complete meanwhile).
// The MMA thread issues the stage's products and frees a slot by a commit once the MMAs
// that read it are done.  One MMA thread per warpgroup, not one per CTA: issuing the
// small MMAs (N = 16) of four warpgroups from one thread held the generation back by a
// third.  Tensor memory: 512 columns, 128 per warpgroup (three A slots of 32 columns, two
// accumulators of 16).
// Every wait is bounded (wait_cycles); on timeout the CTA records kDevTimeout, lets its
// MMAs finish, frees tensor memory and returns.
#include <type_traits>

#include "tc_common.cuh"
#include "near_gen_impl.cuh"

namespace htlr {

using namespace tcc;

namespace {

constexpr int kSlots = 3;                       // A (tensor memory) and B (shared) slots
// rows per generating thread (tiles per warpgroup); two, with two warpgroups, measured
// slower than one with four: the generation needs warps more than per-thread parallelism
constexpr int kR = 1;
constexpr int kWG = 4 / kR;                     // generating warpgroups per CTA
constexpr int kGenThreads = 128 * kWG;
constexpr int kThreads = kGenThreads + 32 * kWG;   // + one MMA warp per warpgroup
constexpr int kAccCol = 32 * kSlots;            // accumulators after the A slots of a tile
constexpr int kTileCols = kAccCol + 32;         // tensor-memory columns of a tile
constexpr int kWgCols = kTileCols * kR;         // tensor-memory columns of a warpgroup
constexpr int kSegStages = 2;                   // stages per accumulation segment (< kSlots)
constexpr int kFlushSegs = 16;                  // segments summed in FP32 per FP64 flush
constexpr int kRhs = 16;
constexpr uint32_t kStageBytes = 2048;          // B of one stage: 2 terms x 2 K steps x 512 B
constexpr int kInfoFirst = 1, kInfoLast = 2, kInfoExit = 4;

static_assert(kSegStages < kSlots, "a segment's slots must leave one slot free");
static_assert(kWG * kWgCols <= 512, "tensor memory holds 512 columns");

// x rounded to TF32 (10 fraction bits), to nearest with ties away from zero: add half a
// unit of the 11th significant bit to the magnitude and clear the 13 low bits.  Exact for
// every finite x below the largest finite TF32 value; the rest, x - tf32(x), is exact in
// FP32.
__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    return (__float_as_uint(x) + 0x1000u) & 0xFFFFE000u;
}

// (x.x - y.x, x.y - y.y), one packed FP32 instruction
__device__ __forceinline__ float2 sub2(float2 x, float2 y)
{
    unsigned long long p, q, r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(x.x), "f"(x.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(q) : "f"(y.x), "f"(y.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(p), "l"(q));
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}

__device__ __forceinline__ void named_sync(int id)
{
    asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

// D[tmem] (+)= A[tmem] x B[smem], kind::tf32
__device__ __forceinline__ void mma_tf32_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b,
                                            uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&v)[8])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr),
                 "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                 "r"(v[7]));
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

}  // namespace

// ---------------------------------------------------------------------------------
// B operand: s w_j u_j[r0 + r] of every source, leaf by leaf (sources in the leaf's own
// order, padded with zeros to whole stages of 16), as two TF32 terms.  One CTA per leaf.
// Element (j, r, term) of a leaf sits in stage j / 16 at float offset
//   term * 256 + ks * 128 + (r / 8) * 64 + (kk / 4) * 32 + (r % 8) * 4 + kk % 4,
// with kk = j % 16 % 8 and ks = j % 16 / 8 (the K step of the stage).
// ---------------------------------------------------------------------------------
__global__ void near_tc_pack_kernel(NearTcArgs A)
{
    const int leaf = blockIdx.x, d = A.d, n = A.n;
    int f[3], c[3];
    leaf_box(A.leafg, d, A.L, leaf, f, c);
    const int rows = c[0] * c[1] * c[2];
    const int s0 = A.stage0[leaf], nst = A.stage0[leaf + 1] - s0;
    const int per_rhs = nst * 16;
    float *dst = A.wu + (size_t)s0 * 512;
    for (int e = threadIdx.x; e < per_rhs * kRhs; e += blockDim.x) {
        const int r = e / per_rhs, j = e % per_rhs;
        float v = 0.f;
        if (j < rows && r < A.nr) {
            const int j1 = j % c[0], j23 = j / c[0], j2 = j23 % c[1], j3 = j23 / c[1];
            const int gj[3] = {f[0] + j1, f[1] + j2, f[2] + j3};
            long long na = 0, str = 1;
            double w = 1.0;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (k < d) {
                    w *= A.width[(long long)k * n + gj[k]];
                    na += (long long)gj[k] * str;
                    str *= n;
                }
            v = (float)(A.k.scale * w * A.u[na + A.ldu * (A.r0 + r)]);
        }
        const uint32_t b1 = tf32_rna(v);
        const uint32_t b2 = tf32_rna(v - __uint_as_float(b1));
        const int st = j >> 4, kk16 = j & 15, ks = kk16 >> 3, kk = kk16 & 7;
        const int off = ks * 128 + (r >> 3) * 64 + (kk >> 2) * 32 + (r & 7) * 4 + (kk & 3);
        float *p = dst + (size_t)st * 512 + off;
        p[0] = __uint_as_float(b1);
        p[256] = __uint_as_float(b2);
    }
}

// ---------------------------------------------------------------------------------
// Kernel values of the thread's kR rows x (relative to the target leaf's corner, scaled by
// coord_scale) against 8 sources (one K step), as two TF32 terms each; the sources'
// coordinates are loaded once for all rows.  c holds, per group of four sources, -y_1 (4
// floats), -y_2, -y_3.  SELF: source j0 + jj == row i gives 0 (the diagonal K_ii w_i is
// added apart).
// ---------------------------------------------------------------------------------
template <int KT, bool SELF>
__device__ __forceinline__ void gen_half(const KParams &kp, int d, const float *__restrict__ c,
                                         const float (&xr)[kR][3], const int (&i)[kR], int j0,
                                         uint32_t (&a1)[kR][8], uint32_t (&a2)[kR][8])
{
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const float4 Y0 = *reinterpret_cast<const float4 *>(c + 12 * q);
        const float4 Y1 = *reinterpret_cast<const float4 *>(c + 12 * q + 4);
        const float4 Y2 = *reinterpret_cast<const float4 *>(c + 12 * q + 8);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 y0 = h ? make_float2(Y0.z, Y0.w) : make_float2(Y0.x, Y0.y);
            const float2 y1 = h ? make_float2(Y1.z, Y1.w) : make_float2(Y1.x, Y1.y);
            const float2 y2 = h ? make_float2(Y2.z, Y2.w) : make_float2(Y2.x, Y2.y);
            const int jj = 4 * q + 2 * h;
#pragma unroll
            for (int m = 0; m < kR; ++m) {
                const float2 dx = __fadd2_rn(make_float2(xr[m][0], xr[m][0]), y0);
                const float2 dy = __fadd2_rn(make_float2(xr[m][1], xr[m][1]), y1);
                const float2 dz = __fadd2_rn(make_float2(xr[m][2], xr[m][2]), y2);
                float2 r2 = __fmul2_rn(dx, dx);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                float2 kv;
                if constexpr (KT == HTLR_K_EXP_R) {
                    const float2 r =
                        __fmul2_rn(r2, make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y)));
                    kv = make_float2(ex2_approx(-r.x), ex2_approx(-r.y));
                } else {
                    kv.x = kv_eval<float, KT>(kp, d, r2.x, dx.x, dy.x, dz.x);
                    kv.y = kv_eval<float, KT>(kp, d, r2.y, dx.y, dy.y, dz.y);
                }
                if constexpr (SELF) {
                    kv.x = j0 + jj == i[m] ? 0.f : kv.x;
                    kv.y = j0 + jj + 1 == i[m] ? 0.f : kv.y;
                }
                const uint32_t h0 = tf32_rna(kv.x), h1 = tf32_rna(kv.y);
                const float2 rem = sub2(kv, make_float2(__uint_as_float(h0), __uint_as_float(h1)));
                a1[m][jj] = h0;
                a1[m][jj + 1] = h1;
                a2[m][jj] = __float_as_uint(rem.x);
                a2[m][jj + 1] = __float_as_uint(rem.y);
            }
        }
    }
}

template <int KT>
__global__ void __launch_bounds__(kThreads, 1) near_tc_kernel(NearTcArgs A)
{
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ __align__(8) uint64_t afull[kWG][kSlots], sfree[kWG][kSlots], segfull[kWG][2];
    __shared__ __align__(8) uint64_t done_bar[kWG];
    __shared__ int info[kWG][kSlots];
    __shared__ int cur_item[kWG];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_word;
    volatile int *const abortp = &abort_word;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int d = A.d, n = A.n, L = A.L;
    const int coord_floats = A.max_rows_pad / 4 * 12;
    const uint32_t wg_bytes = (uint32_t)coord_floats * 4u + kSlots * kStageBytes;
    if (tid == 0) {
        for (int w = 0; w < kWG; ++w) {
            for (int s = 0; s < kSlots; ++s) {
                mbar_init(&afull[w][s], 128);
                mbar_init(&sfree[w][s], 1);
            }
            mbar_init(&segfull[w][0], 1);
            mbar_init(&segfull[w][1], 1);
        }
        for (int w = 0; w < kWG; ++w) mbar_init(&done_bar[w], 1);
        abort_word = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kGenThreads / 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_holder;

    if (tid >= kGenThreads) {
        // ---------------- the MMA thread of warpgroup g ----------------
        const int g = (tid - kGenThreads) >> 5;
        if ((tid & 31) == 0) {
            const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) |
                                   ((uint32_t)(kRhs >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            const uint32_t ring = smem_u32(sm) + (uint32_t)coord_floats * 4u + (uint32_t)g * wg_bytes;
            uint32_t ms = 0, mseg = 0;
            int nst_seg = 0;
            while (true) {
                const int a = (int)(ms % kSlots);
                if (!mbar_wait(&afull[g][a], (ms / kSlots) & 1, A.wait_cycles, abortp)) {
                    *abortp = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int fl = *reinterpret_cast<volatile int *>(&info[g][a]);
                ++ms;
                if (fl & kInfoExit) break;
                const uint32_t buf = mseg & 1;
                const uint64_t bd = smem_desc(ring + (uint32_t)a * kStageBytes, 128, 256);
#pragma unroll
                for (int m = 0; m < kR; ++m) {   // tile m: columns g kWgCols + kTileCols m
                    const uint32_t tt = tmem + (uint32_t)(g * kWgCols + kTileCols * m);
                    const uint32_t dt = tt + kAccCol + 16u * buf, ta = tt + 32u * a;
                    mma_tf32_ts(dt, ta + 16, bd, idesc, (fl & kInfoFirst) ? 0u : 1u);   // a2 b1
                    mma_tf32_ts(dt, ta, bd + 64, idesc, 1u);                            // a1 b2
                    mma_tf32_ts(dt, ta + 24, bd + 32, idesc, 1u);                       // a2 b1
                    mma_tf32_ts(dt, ta + 8, bd + 96, idesc, 1u);                        // a1 b2
                }
                ++nst_seg;
                if (fl & kInfoLast) {
#pragma unroll
                    for (int k = 0; k < kSegStages; ++k)
                        if (k < nst_seg) {
                            const int sa = (a + kSlots - nst_seg + 1 + k) % kSlots;
                            const uint64_t bd1 = smem_desc(ring + (uint32_t)sa * kStageBytes, 128, 256);
#pragma unroll
                            for (int m = 0; m < kR; ++m) {
                                const uint32_t tt = tmem + (uint32_t)(g * kWgCols + kTileCols * m);
                                const uint32_t dt = tt + kAccCol + 16u * buf, ta1 = tt + 32u * sa;
                                mma_tf32_ts(dt, ta1, bd1, idesc, 1u);           // a1 b1
                                mma_tf32_ts(dt, ta1 + 8, bd1 + 32, idesc, 1u);  // a1 b1
                            }
                        }
#pragma unroll
                    for (int k = 0; k < kSegStages; ++k)
                        if (k < nst_seg) mma_commit(&sfree[g][(a + kSlots - nst_seg + 1 + k) % kSlots]);
                    mma_commit(&segfull[g][buf]);
                    ++mseg;
                    nst_seg = 0;
                }
            }
            mma_commit(&done_bar[g]);
            mbar_wait(&done_bar[g], 0);
        }
        __syncwarp();
    } else {
        // ------- generating warpgroup g: rows t + 128 m (m < kR) of its tile -------
        const int g = warp >> 2, t = tid & 127, q = warp & 3;
        float *const cxyz = reinterpret_cast<float *>(sm + (size_t)g * wg_bytes);
        unsigned char *const bring = sm + (size_t)g * wg_bytes + (size_t)coord_floats * 4;
        // FP64 sums: row slot m, RHS r of thread tid at s64[(m * kRhs + r) * kGenThreads]
        double *const s64 = reinterpret_cast<double *>(sm + (size_t)kWG * wg_bytes) + tid;
        const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(g * kWgCols);
        KParams kp;
        kp.scale = A.k.scale;
        kp.param = A.k.param;
        kp.inv2s2 = A.k.type == HTLR_K_GAUSS ? 1.0 / (2.0 * A.k.param * A.k.param) : 0.0;
        kp.deg = (int)A.k.param;
        const double cs = coord_scale<float>(A.k.type, A.k.param);
        uint32_t s = 0;      // stages of this warpgroup (all items)
        uint32_t cseg = 0;   // segments started
        uint32_t dseg = 0;   // segments drained
        int nflush = 0;
        float acc[kR][kRhs];
        auto flush = [&]() {
#pragma unroll
            for (int m = 0; m < kR; ++m)
#pragma unroll
                for (int r = 0; r < kRhs; ++r) {
                    s64[(m * kRhs + r) * kGenThreads] += (double)acc[m][r];
                    acc[m][r] = 0.f;
                }
            nflush = 0;
        };
        // Reads the finished accumulator of segment dseg into the FP32 sums.
        auto drain = [&]() {
            const uint32_t buf = dseg & 1;
            if (!mbar_wait(&segfull[g][buf], (dseg >> 1) & 1, A.wait_cycles, abortp)) *abortp = 1;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int m = 0; m < kR; ++m) {
                uint32_t v[16];
                tmem_ld16(tbase + kTileCols * m + kAccCol + 16u * buf, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int r = 0; r < kRhs; ++r) acc[m][r] += __uint_as_float(v[r]);
            }
            ++dseg;
            if (++nflush == kFlushSegs) flush();
            asm volatile("tcgen05.fence::before_thread_sync;");
        };
        while (true) {
            // next item; the decision (stop on abort) is the warpgroup's, taken by one thread
            if (t == 0) cur_item[g] = *abortp ? A.nitems : atomicAdd(A.counter, 1);
            named_sync(1 + g);
            const int it = cur_item[g];
            named_sync(1 + g);
            if (it >= A.nitems) break;
            const int tau = A.items[2 * it], tile = A.items[2 * it + 1];
            int tf[3], tcn[3];
            leaf_box(A.leafg, d, L, tau, tf, tcn);
            const int rows = tcn[0] * tcn[1] * tcn[2];
            double lo[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                lo[k] = k < d ? ldexp((double)((tau >> (L * k)) & ((1 << L) - 1)), -L) : 0.0;
            // rows past the leaf evaluate a far-away dummy point (finite, never written)
            int i[kR];
            float xr[kR][3];
            long long nat[kR];
#pragma unroll
            for (int m = 0; m < kR; ++m) {
                i[m] = tile * 128 * kR + 128 * m + t;
                xr[m][0] = xr[m][1] = xr[m][2] = 4.f;
                nat[m] = -1;
                if (i[m] < rows) {
                    const int j1 = i[m] % tcn[0], j23 = i[m] / tcn[0], j2 = j23 % tcn[1], j3 = j23 / tcn[1];
                    const int gi[3] = {tf[0] + j1, tf[1] + j2, tf[2] + j3};
                    long long na = 0, str = 1;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        xr[m][k] = 0.f;
                        if (k < d) {
                            xr[m][k] = (float)((A.coords[(long long)k * n + gi[k]] - lo[k]) * cs);
                            na += (long long)gi[k] * str;
                            str *= n;
                        }
                    }
                    nat[m] = na;
                }
#pragma unroll
                for (int r = 0; r < kRhs; ++r) {
                    acc[m][r] = 0.f;
                    s64[(m * kRhs + r) * kGenThreads] = 0.0;
                }
            }
            nflush = 0;
            const int e0 = A.rowptr[tau], e1 = A.rowptr[tau + 1];
            // A stage is handed to the MMA thread one stage late: its tensor-memory stores and
            // its B copy (cp.async, global to shared) complete while the next stage's first K
            // step is generated.  publish() waits for them (all but the newest copy group when
            // `newest_pending`), arrives on the slot's mbarrier and, at the first stage of a
            // segment, drains the item's previous segment.
            bool pend = false;
            int pend_a = 0, pend_fl = 0;
            auto publish = [&](bool newest_pending) {
                if (newest_pending) asm volatile("cp.async.wait_group 1;" ::: "memory");
                else asm volatile("cp.async.wait_group 0;" ::: "memory");
                asm volatile("tcgen05.wait::st.sync.aligned;");
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                if (t == 0) info[g][pend_a] = pend_fl;
                mbar_arrive(&afull[g][pend_a]);
                pend = false;
                if (pend_fl & kInfoFirst) {
                    if (cseg > dseg) drain();
                    ++cseg;
                }
            };
            int seg_pos = 0;
            for (int e = e0; e < e1; ++e) {
                const int sg = A.col[e];
                int sf[3], scn[3];
                leaf_box(A.leafg, d, L, sg, sf, scn);
                const int cols = scn[0] * scn[1] * scn[2];
                const int nst = A.stage0[sg + 1] - A.stage0[sg];
                const float *bsrc = A.wu + (size_t)A.stage0[sg] * 512 + 4 * t;
                // the source leaf's coordinates relative to the target leaf's corner, negated;
                // the padding up to whole stages sits far away (its B is zero)
                named_sync(1 + g);
                for (int j = t; j < nst * 16; j += 128) {
                    float y[3] = {8.f, 8.f, 8.f};
                    if (j < cols) {
                        const int j1 = j % scn[0], j23 = j / scn[0], j2 = j23 % scn[1], j3 = j23 / scn[1];
                        const int gj[3] = {sf[0] + j1, sf[1] + j2, sf[2] + j3};
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            y[k] = k < d ? (float)((A.coords[(long long)k * n + gj[k]] - lo[k]) * cs) : 0.f;
                    }
                    const int qq = j >> 2, l = j & 3;
                    cxyz[12 * qq + l] = -y[0];
                    cxyz[12 * qq + 4 + l] = -y[1];
                    cxyz[12 * qq + 8 + l] = -y[2];
                }
                named_sync(1 + g);
                const bool self = sg == tau;
                for (int ls = 0; ls < nst; ++ls, ++s) {
                    const bool first = seg_pos == 0;
                    const bool last = seg_pos == kSegStages - 1 || (e == e1 - 1 && ls == nst - 1);
                    const int a = (int)(s % kSlots);
                    const uint32_t use = s / kSlots;
                    // the slot's previous stage (three back) is in a committed segment
                    if (use > 0 && !mbar_wait(&sfree[g][a], (use - 1) & 1, A.wait_cycles, abortp))
                        *abortp = 1;
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n cp.async.commit_group;" ::"r"(
                                     smem_u32(bring + a * kStageBytes + 16 * t)),
                                 "l"(bsrc + (size_t)ls * 512)
                                 : "memory");
                    const uint32_t col = tbase + 32u * a;
                    const float *cst = cxyz + 48 * ls;
                    auto body = [&](auto self_c) {
                        constexpr bool SELF = decltype(self_c)::value;
                        uint32_t a1[kR][8], a2[kR][8];
                        gen_half<KT, SELF>(kp, d, cst, xr, i, 16 * ls, a1, a2);
                        if (pend) publish(true);
#pragma unroll
                        for (int m = 0; m < kR; ++m) {
                            tmem_st8(col + kTileCols * m, a1[m]);
                            tmem_st8(col + kTileCols * m + 16u, a2[m]);
                        }
                        gen_half<KT, SELF>(kp, d, cst + 24, xr, i, 16 * ls + 8, a1, a2);
#pragma unroll
                        for (int m = 0; m < kR; ++m) {
                            tmem_st8(col + kTileCols * m + 8u, a1[m]);
                            tmem_st8(col + kTileCols * m + 24u, a2[m]);
                        }
                    };
                    if (self) body(std::true_type{});
                    else body(std::false_type{});
                    pend = true;
                    pend_a = a;
                    pend_fl = (first ? kInfoFirst : 0) | (last ? kInfoLast : 0);
                    seg_pos = last ? 0 : seg_pos + 1;
                }
            }
            if (pend) publish(false);
            while (dseg < cseg) drain();   // the item's last segment
            flush();
#pragma unroll
            for (int m = 0; m < kR; ++m) {
                if (nat[m] < 0) continue;
                const double dg = A.diag[nat[m]] + (A.a ? A.a[nat[m]] : 0.0);
                for (int r = 0; r < A.nr; ++r) {
                    const long long c0 = A.r0 + r;
                    A.f[nat[m] + A.ldf * c0] =
                        s64[(m * kRhs + r) * kGenThreads] + dg * A.u[nat[m] + A.ldu * c0];
                }
            }
        }
        // tell the MMA thread that this warpgroup is done
        {
            const int a = (int)(s % kSlots);
            const uint32_t use = s / kSlots;
            if (use > 0 && !mbar_wait(&sfree[g][a], (use - 1) & 1, A.wait_cycles, abortp))
                *abortp = 1;
            if (t == 0) info[g][a] = kInfoExit;
            mbar_arrive(&afull[g][a]);
        }
    }
    __syncthreads();
    if (tid == 0 && *abortp) atomicExch(A.err, (int)kDevTimeout);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == kGenThreads / 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <int KT>
static void launch_kt(const NearTcArgs &a, size_t smem, int grid, cudaStream_t s)
{
    cudaFuncSetAttribute(near_tc_kernel<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    near_tc_kernel<KT><<<grid, kThreads, smem, s>>>(a);
}

int near_tc_tile_rows() { return 128 * kR; }

void launch_near_tc(const NearTcArgs &a, cudaStream_t s)
{
    if (a.nitems <= 0) return;
    const int nleaf = 1 << (a.d * a.L);
    near_tc_pack_kernel<<<nleaf, 256, 0, s>>>(a);
    cudaMemsetAsync(a.counter, 0, sizeof(int), s);
    const size_t wg_bytes = (size_t)a.max_rows_pad * 12 + kSlots * kStageBytes;
    // at least 116 KB, so that one CTA (and its 512 tensor-memory columns) fills an SM
    size_t smem = kWG * wg_bytes + (size_t)kR * kRhs * kGenThreads * sizeof(double);
    if (smem < 116 * 1024) smem = 116 * 1024;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int want = (a.nitems + kWG - 1) / kWG;
    const int grid = want < sms ? want : sms;
    switch (a.k.type) {
    case HTLR_K_LOG: launch_kt<HTLR_K_LOG>(a, smem, grid, s); break;
    case HTLR_K_INV_R: launch_kt<HTLR_K_INV_R>(a, smem, grid, s); break;
    case HTLR_K_EXP_R: launch_kt<HTLR_K_EXP_R>(a, smem, grid, s); break;
    case HTLR_K_GAUSS: launch_kt<HTLR_K_GAUSS>(a, smem, grid, s); break;
    case HTLR_K_POLY: launch_kt<HTLR_K_POLY>(a, smem, grid, s); break;
    default: launch_kt<HTLR_K_CONST>(a, smem, grid, s); break;
    }
}

}  // namespace htlr
