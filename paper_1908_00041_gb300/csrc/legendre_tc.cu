// Split-precision Legendre stage on tcgen05 tensor cores (precision FAVEST_BF16X6).
//
// Per order mu and parity p the Legendre stage is a dense product:
//   forward : Q[rows, n]   = sum_j  Lam[rows, j] * Fb[j, n]      (rows = l - mu of parity p)
//   adjoint : S_p[j, n]    = sum_r  Lam[r, j]   * g[r, n]
// Lam (the recurrence values, run in double-float arithmetic) is produced by a generator
// kernel and stored as three bf16 pieces (hi + mid + lo = the value rounded to FP32); g carries three
// bf16 pieces as well, and Fb (FP32 records from the forward DFT) is split into three pieces
// by converter warps of the forward GEMM as it is loaded.  The GEMM kernels form 6 of the 9
// piece products (those with combined weight >= 2^-16 of the leading one).  Because the tensor core
// accumulates in FP32 with truncation (products below one ulp of the running sum are
// dropped), the leading hi*hi product is accumulated in a fresh TMEM buffer for each
// K-chunk of 32 and added to an FP32 register sum (round-to-nearest) by the epilogue;
// the five correction products, 2^-8 smaller, accumulate in TMEM over the whole K.
//
// One work item is a 128 x N output tile (N = 256 columns, i.e. 32 fields, or 128 for
// small batches) over its whole K range, in K-chunks of 32.  Operand tiles in global
// memory are pre-arranged so that one K-chunk of one piece is a contiguous block in the
// shared-memory core-matrix layout (see tc.cuh):
//   forward A (Lam, M = rows, K = j, MN-major): [K/8 groups][M/8 groups][8 j][8 rows]  8 KB
//   adjoint A (Lam^T, M = j, K = rows, K-major): [M/8][K/8][8 j][8 rows]               8 KB
//   B (pieces of Fb or g, K x N, MN-major):     [K/8][N/8][8 k][8 n]           K32 x N x 2 B
#include "favest_internal.h"
#include "recurrence.cuh"
#include "tc.cuh"
#include "bf16_split.cuh"

#include <cuda_bf16.h>

namespace favest {

namespace {

constexpr int kGenThreads = 128;
constexpr int kChunkK = kGemmChunkK;              // K depth of one operand chunk (32)
constexpr int kTileM = 128;
constexpr int kPieceBytes = kTileM * kChunkK * 2;  // 8 KB: one bf16 piece of an A chunk
constexpr int kPieces = 3;
constexpr int kChunkBytes = kPieces * kPieceBytes;  // 24 KB

// Two FP32 values -> three bf16x2 words (pieces hi, mid, lo; f0 in the low halves), split
// exactly with round-to-nearest: hi = bf16(f), mid = bf16(f - hi), lo = bf16(f - hi - mid).
// One conversion instruction rounds both values of a piece.
__device__ __forceinline__ unsigned bf2_bits(__nv_bfloat162 v)
{
    unsigned u;
    memcpy(&u, &v, 4);
    return u;
}

__device__ __forceinline__ void split3x2(float f0, float f1, unsigned &h, unsigned &m, unsigned &l)
{
    const __nv_bfloat162 bh = __floats2bfloat162_rn(f0, f1);
    const float2 fh = __bfloat1622float2(bh);
    const float r0 = f0 - fh.x, r1 = f1 - fh.y;
    const __nv_bfloat162 bm = __floats2bfloat162_rn(r0, r1);
    const float2 fm = __bfloat1622float2(bm);
    const __nv_bfloat162 bl = __floats2bfloat162_rn(r0 - fm.x, r1 - fm.y);
    h = bf2_bits(bh);
    m = bf2_bits(bm);
    l = bf2_bits(bl);
}

// Rows r0 .. r0 + 15 of the NJ chains of one thread (r0 a multiple of 16).  Word k of parity
// p holds rows 4k + p (low half) and 4k + 2 + p (high half) of the block, so each value waits
// in fprev for its partner two rows on and the pair is split by split3x2.  kEdge: the block
// holds row 0 (the start value, no step) or rows past the order's last (emitted as zero);
// the checks are warp-uniform, and the blocks in between run without them.
template <int kGenJ, bool kEdge>
__device__ __forceinline__ void gen_block16(const float2 *__restrict__ As, int r0, int nrow,
                                            const bool (&act)[kGenJ], const bool (&live)[kGenJ],
                                            const Df (&x)[kGenJ], Df (&y1)[kGenJ], Df (&y2)[kGenJ],
                                            unsigned (&pk)[kGenJ][2][3][4])
{
    float fprev[kGenJ][2];
#pragma unroll
    for (int w = 0; w < 16; ++w) {
        const int r = r0 + w;
        float f[kGenJ];
        if (!kEdge || r < nrow) {
            const float2 av = __ldg(As + r);
            const Df a{av.x, av.y};
#pragma unroll
            for (int i = 0; i < kGenJ; ++i) {
                f[i] = 0.f;
                if (!act[i]) continue;                     // no work for inactive chains
                if (!kEdge || r > 0) {
                    const Df yl = df_step(a, x[i], y1[i], y2[i]);
                    y2[i] = y1[i];
                    y1[i] = yl;
                }
                f[i] = live[i] ? y1[i].h : 0.f;
            }
        } else {
#pragma unroll
            for (int i = 0; i < kGenJ; ++i) f[i] = 0.f;
        }
        const int p = w & 1, k = w >> 2;
#pragma unroll
        for (int i = 0; i < kGenJ; ++i) {
            if ((w & 2) == 0) fprev[i][p] = f[i];
            else split3x2(fprev[i][p], f[i], pk[i][p][0][k], pk[i][p][1][k], pk[i][p][2][k]);
        }
    }
}

// Generator: 128 threads per CTA arranged as (128 / lt) orders x lt latitudes (lt = 32,
// 64 or 128, a multiple of the warp so each warp runs one order); a CTA covers mb such
// order groups in turn.  A thread runs the scaled recurrences of one order (double-float
// FP32 pairs, recurrence.cuh) at NJ (1 or 2) latitudes lt apart (the block covers NJ lt
// consecutive latitudes) over all rows l = mu..L+1, interleaved step by step: each step of
// a recurrence depends on the one before, so independent chains in the same thread keep
// more work in flight per warp (at the price of registers and of fewer, longer blocks for
// small grids).  The high part of each value, its FP32 rounding, is split into the pieces.
// Per parity it packs 8 consecutive rows into one 16-byte core-matrix row per piece.
// (lt, mb) is the block shape the autotuner picks per degree.  Latitudes below jc0 (the
// order's turning bound rounded down to a K-chunk: every value there is below 1e-13) and
// padding latitudes are not stored; their operand positions were zeroed when the plan was
// created.
// Output: the one Legendre layout both GEMM directions read, [piece][row block][JP][8 rows]:
// the 16-byte unit of the 8 rows rp .. rp + 7 of parity p at latitude j goes to
//   lam + piece * rb_total JP 16 + ((lam_rb[mu*2+p] + rp / 8) JP + j) 16,
// so a warp (32 consecutive latitudes) stores 512 consecutive bytes per piece.
template <int kGenJ>
__device__ __forceinline__ void gen_order(unsigned char *__restrict__ lam, const int *__restrict__ lam_rb,
                                          long long rb_total, const float2 *__restrict__ xdf, const double *__restrict__ sj,
                                          const double *__restrict__ cmu, const float2 *__restrict__ Adf, int L,
                                          int J, int JP, int mu, const int (&jv)[kGenJ], int jc0)
{
    const int nrow = L + 2 - mu;
    const float2 *As = Adf + tab_off(L, mu);    // recurrence multipliers of this order (double-float)

    bool act[kGenJ];
    bool any = false;
#pragma unroll
    for (int i = 0; i < kGenJ; ++i) {
        act[i] = jv[i] < J && jv[i] >= jc0;
        any |= act[i];
    }
    if (!any) return;
    Df y1[kGenJ], y2[kGenJ], x[kGenJ];
    int c[kGenJ];
#pragma unroll
    for (int i = 0; i < kGenJ; ++i) {
        y1[i] = Df{0.f, 0.f};
        y2[i] = Df{0.f, 0.f};
        c[i] = 1 << 20;                            // inactive chains stay silent
        x[i] = Df{0.f, 0.f};
        if (act[i]) {
            const float2 xv = __ldg(xdf + jv[i]);
            x[i] = Df{xv.x, xv.y};
            sectoral_start_df(cmu[mu], sj[jv[i]], mu, y1[i], c[i]);
        }
    }
    const int nrow_p0 = (nrow + 1) / 2, nrow_p1 = nrow / 2;
    int rbase[2];
#pragma unroll
    for (int p = 0; p < 2; ++p) rbase[p] = __ldg(lam_rb + mu * 2 + p);

    unsigned pk[kGenJ][2][kPieces][4];   // [chain][parity][piece][4 x 2 bf16]
    for (int r0 = 0; r0 < nrow; r0 += 16) {
        if (r0 + 16 < nrow) {                          // the next block's multipliers into L1
            asm volatile("prefetch.L1 [%0];" ::"l"(As + r0 + 16));
            asm volatile("prefetch.L1 [%0];" ::"l"(As + min(r0 + 31, nrow - 1)));
        }
        bool live[kGenJ];
#pragma unroll
        for (int i = 0; i < kGenJ; ++i) live[i] = c[i] == 0;
        if (r0 > 0 && r0 + 16 <= nrow) gen_block16<kGenJ, false>(As, r0, nrow, act, live, x, y1, y2, pk);
        else gen_block16<kGenJ, true>(As, r0, nrow, act, live, x, y1, y2, pk);
#pragma unroll
        for (int i = 0; i < kGenJ; ++i) renorm_df(y1[i], y2[i], c[i]);   // growth over 16 rows stays below 2^26
        // flush: rows r0/2 .. r0/2+7 of each parity
        const int rp = r0 >> 1;                        // multiple of 8
#pragma unroll
        for (int i = 0; i < kGenJ; ++i) {
            const int j = jv[i];
#pragma unroll
            for (int p = 0; p < 2; ++p) {
                const int np = p ? nrow_p1 : nrow_p0;
                if (act[i] && rp < np) {
                    const size_t unit = ((size_t)(rbase[p] + rp / 8) * JP + j) * 16;
#pragma unroll
                    for (int q = 0; q < kPieces; ++q) {
                        uint4 v = make_uint4(pk[i][p][q][0], pk[i][p][q][1], pk[i][p][q][2], pk[i][p][q][3]);
                        *reinterpret_cast<uint4 *>(lam + (size_t)q * rb_total * JP * 16 + unit) = v;
                    }
                }
            }
        }
    }
}

template <int kGenJ>
__global__ void __launch_bounds__(kGenThreads) k_gen_lambda(
    unsigned char *__restrict__ lam, const int *__restrict__ lam_rb, long long rb_total,
    const float2 *__restrict__ xdf, const double *__restrict__ sj,
    const double *__restrict__ cmu, const float2 *__restrict__ Adf, const int *__restrict__ jcmin, int L, int J,
    int JP, int lt, int mb)
{
    const int olanes = kGenThreads / lt;
    const int jblocks = (JP + kGenJ * lt - 1) / (kGenJ * lt);
    const int jb = blockIdx.x % jblocks, og = blockIdx.x / jblocks;
    int jv[kGenJ];
#pragma unroll
    for (int i = 0; i < kGenJ; ++i) jv[i] = (jb * kGenJ + i) * lt + threadIdx.x % lt;
    for (int k = 0; k < mb; ++k) {
        const int mu = (og * mb + k) * olanes + threadIdx.x / lt;   // uniform in the warp
        if (mu > L) break;
        gen_order<kGenJ>(lam, lam_rb, rb_total, xdf, sj, cmu, Adf, L, J, JP, mu, jv, __ldg(jcmin + mu));
    }
}

// ---------------------------------------------------------------------------
// Persistent GEMM: every item computes out[rows 0..127][cols 0..N-1] =
//   sum_{c < nk} A_c * B_c  (three bf16 pieces each, 6 products)
// Warp 0 loads operand chunks with TMA (boxes of whole 512-byte rows), warp 1 issues the
// MMAs, warps 4.. drain TMEM (each a 32-lane quadrant and 128 columns; warps 2-3 idle, so
// that the roles sit in whole warpgroups for the register split).  This kernel serves the
// adjoint (K-major Legendre operand, bf16 piece operands); the forward runs k_tc_gemm_f.
// TMEM: columns [0, N) hold the hi*hi product of the current K-chunk (drained into FP32
// register sums after every chunk), columns [N, 2N) accumulate the five correction
// products over the whole item.  Per chunk the MMA warp issues the corrections first,
// which gives the epilogue time to drain the previous chunk's hi*hi columns.
// ---------------------------------------------------------------------------
constexpr int kStages = 3;
constexpr uint32_t kTmemCols = 512;

constexpr int kEpiCols = 128;       // TMEM columns drained by one epilogue warp

template <int N>
constexpr int gemm_threads() { return 128 + 32 * 4 * (N / kEpiCols); }

__device__ __forceinline__ void set_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

// Polls of an mbarrier before a wait gives up (about a second).
constexpr uint32_t kWaitPolls = 1u << 26;

// Wait that also gives up after `limit` polls, or when another role aborted (abort may be
// null: the drain waits of the abort path itself, which only the limit ends).
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 1023) == 1023 && abort && *abort) return false;
    }
    return false;
}

// Work items are handed out at run time: the producer thread of each CTA takes the next
// item index from a device counter (sched[0]) and publishes it in a ring of kItemSlots
// shared-memory slots; every consumer role reads the indices from the ring in the same
// order and releases a slot once it has read it.  A taken index at or past the item count
// is published as -1, which ends every role's loop.  A CTA takes the next listed item as
// soon as it is free (greedy list scheduling), so the load stays balanced whatever the
// host's order, and the host lists items that share an operand next to each other (they
// then run at the same time on the CTAs that free up together), heavier groups first.
// The last CTA to finish resets sched[0..1] for the next launch.
constexpr int kItemSlots = 4;

struct ItemRing {
    int q[kItemSlots];
    uint64_t full[kItemSlots], empty[kItemSlots];
};

__device__ __forceinline__ void item_ring_init(ItemRing &R, int consumers)
{
    for (int s = 0; s < kItemSlots; ++s) {
        tc::mbar_init(&R.full[s], 1);
        tc::mbar_init(&R.empty[s], consumers);
    }
}

// producer: publishes the n-th index of this CTA into slot n % kItemSlots; false if the
// wait for the slot gave up
__device__ __forceinline__ bool item_publish(ItemRing &R, uint32_t n, int *sched, int nitems, volatile int *abort,
                                             uint32_t limit, int &it)
{
    const int s = n % kItemSlots;
    if (!wait_or_abort(&R.empty[s], ((n / kItemSlots) & 1) ^ 1, abort, limit)) return false;
    it = atomicAdd(sched, 1);
    if (it >= nitems) it = -1;
    R.q[s] = it;
    tc::mbar_arrive(&R.full[s]);     // release: the index is visible to the slot's waiters
    return true;
}

// consumer: waits for the n-th index (false if the wait gave up); the caller releases the
// slot with item_release once every thread of its role has read it
__device__ __forceinline__ bool item_take(ItemRing &R, uint32_t n, volatile int *abort, uint32_t limit, int &it)
{
    const int s = n % kItemSlots;
    if (!wait_or_abort(&R.full[s], (n / kItemSlots) & 1, abort, limit)) return false;
    it = *reinterpret_cast<volatile int *>(&R.q[s]);
    return true;
}

__device__ __forceinline__ void item_release(ItemRing &R, uint32_t n) { tc::mbar_arrive(&R.empty[n % kItemSlots]); }

// after the CTA's last item (called by the producer thread, after the final barrier): the
// last CTA of the launch resets the counters; every CTA has taken its last index by then
__device__ __forceinline__ void item_sched_done(int *sched)
{
    __threadfence();
    if (atomicAdd(sched + 1, 1) == (int)gridDim.x - 1) {
        sched[0] = 0;
        sched[1] = 0;
        __threadfence();
    }
}

template <int N>
struct GemmSmem {
    unsigned char a[kStages][kChunkBytes];
    unsigned char b[kStages][kPieces * kChunkK * N * 2];
    uint64_t full[kStages], empty[kStages];
    uint64_t dmain_full, dmain_empty, dcorr_full, dcorr_empty;
    uint64_t drain;            // abort path: completion of the MMA warp's last issued MMAs
    ItemRing ring;
    uint32_t tmem_base;
    int abort;
};

template <int N>
__global__ void __launch_bounds__(gemm_threads<N>(), 1) k_tc_gemm(
    const GemmGroup *__restrict__ groups, const TcItem *__restrict__ items, int nitems, int a_mn_major,
    int *__restrict__ status, int *__restrict__ sched, uint32_t poll_limit, int skip_loads)
{
    constexpr int kEpiWarps = 4 * (N / kEpiCols);   // 4 lane quadrants x N / 128 column parts
    constexpr int kPieceB = kChunkK * N * 2;        // bytes of one B piece per chunk
    constexpr int kChunkB = kPieces * kPieceB;
    extern __shared__ __align__(1024) unsigned char sm_raw[];
    GemmSmem<N> &S = *reinterpret_cast<GemmSmem<N> *>(sm_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tc::tmem_alloc(&S.tmem_base, kTmemCols);
    if (threadIdx.x == 32) {
        for (int s = 0; s < kStages; ++s) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.empty[s], 1);
        }
        tc::mbar_init(&S.dmain_full, 1);
        tc::mbar_init(&S.dmain_empty, kEpiWarps);
        tc::mbar_init(&S.dcorr_full, 1);
        tc::mbar_init(&S.dcorr_empty, kEpiWarps);
        tc::mbar_init(&S.drain, 1);
        item_ring_init(S.ring, 1 + kEpiWarps);        // consumers: the MMA thread, the epilogue warps
        S.abort = 0;
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem_base;
    volatile int *abort = &S.abort;

    if (warp < 4) {
      // registers: launched at 168 per thread (384 threads); warpgroup 0 (producer, MMA
      // issuer, two idle warps) drops to 56 and the two epilogue warpgroups rise to 224, which
      // their 128 FP32 running sums per thread need: 128 x 56 + 256 x 224 = 384 x 168
      if constexpr (N == 256) tc::setmaxnreg_dec<56>();
      if (warp == 0) {
        // ---------------- producer ----------------
        // (skip_loads: failure-path self-test -- nothing is loaded, so the MMA and epilogue
        // waits must run out, report FAVEST_ETIMEOUT and return)
        if (lane == 0) {
            uint32_t phase = 0;                     // bit s: parity of stage s's next use
            uint32_t issued = 0;                    // bit s: stage s has been loaded at least once
            int stage = 0;
            for (uint32_t n = 0; !*abort; ++n) {
                int it;
                if (!item_publish(S.ring, n, sched, nitems, abort, poll_limit, it)) {
                    set_status(status, FAVEST_ETIMEOUT);
                    *abort = 1;
                    break;
                }
                if (it < 0) break;
                if (skip_loads) continue;
                const TcItem I = items[it];
                // the group's tensor maps live in global memory (generic addresses)
                const CUtensorMap *tmap_a = &groups[I.group].tmap_a, *tmap_b = &groups[I.group].tmap_b;
                for (int c = 0; c < I.nk; ++c) {
                    if (!wait_or_abort(&S.empty[stage], ((phase >> stage) & 1) ^ 1, abort, poll_limit)) {
                        set_status(status, FAVEST_ETIMEOUT);
                        *abort = 1;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&S.full[stage], kChunkBytes + kChunkB);
                    // the Legendre chunk: a 4-D box of the one layout; the coefficient operand
                    // buffer is a 2-D array of 512-byte rows: a chunk is a box of whole rows
                    // starting at its byte offset / 512
                    tc::tma_load_4d(S.a[stage], tmap_a, 0, I.ay + c * I.ady, I.az + c * I.adz, 0, &S.full[stage]);
                    tc::tma_load_2d(S.b[stage], tmap_b, 0, (int)((I.b_off + (long long)c * I.b_stride) >> 9),
                                    &S.full[stage]);
                    phase ^= 1u << stage;
                    issued |= 1u << stage;
                    stage = (stage + 1) % kStages;
                }
            }
            // On abort, loads this warp issued may still be in flight: wait (bounded) until
            // each stage's last load has landed, so that no copy writes this CTA's shared
            // memory after the CTA has exited.  A load completes on its own; only a broken
            // barrier could make this wait run out, and then nothing better can be done.
            if (*abort)
                for (int s = 0; s < kStages; ++s)
                    if (issued & (1u << s)) wait_or_abort(&S.full[s], ((phase >> s) & 1) ^ 1, nullptr, poll_limit);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kTileM, N, a_mn_major, 1) | (1u << 7) | (1u << 10);
            uint32_t phase = 0, main_use = 0, corr_use = 0;
            int stage = 0;
            const uint32_t dmain = tmem, dcorr = tmem + N;
            // A, per piece [K/8 or M/8 row blocks][latitudes][8 rows] (the box of the one
            // Legendre layout): MN-major (forward, [M/8 = 16][K = 32]): K-groups 128 B apart,
            // M-blocks 512 B, K-step (2 groups) 256 B; K-major (adjoint, [K/8 = 4][M = 128]):
            // M-groups 128 B apart, K-groups 2048 B, K-step 4096 B.  (Descriptor: leading
            // byte offset = K-direction stride, stride byte offset = M/N-direction stride.)
            // B: MN-major, K-groups of N/8 x 128 B.
            const uint32_t a_step = a_mn_major ? 256u : 4096u;
            const uint32_t a_lbo = a_mn_major ? 128u : 2048u, a_sbo = a_mn_major ? 512u : 128u;
            constexpr uint32_t b_step = 2 * (N / 8) * 128, b_lbo = (N / 8) * 128;
            for (uint32_t n = 0; !*abort; ++n) {
                int it;
                if (!item_take(S.ring, n, abort, poll_limit, it)) {
                    set_status(status, FAVEST_ETIMEOUT);
                    *abort = 1;
                    break;
                }
                item_release(S.ring, n);
                if (it < 0) break;
                const TcItem I = items[it];
                if (!wait_or_abort(&S.dcorr_empty, (corr_use & 1) ^ 1, abort, poll_limit)) {
                    set_status(status, FAVEST_ETIMEOUT);
                    *abort = 1;
                    break;
                }
                for (int c = 0; c < I.nk; ++c) {
                    if (!wait_or_abort(&S.full[stage], (phase >> stage) & 1, abort, poll_limit)) {
                        set_status(status, FAVEST_ETIMEOUT);
                        *abort = 1;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(S.a[stage]), b0 = tc::smem_u32(S.b[stage]);
                    // corrections (weights 2^-8 and 2^-16 of hi*hi) accumulate over the item
#pragma unroll
                    for (int s = 0; s < kChunkK / 16; ++s) {
                        const uint32_t as = a0 + s * a_step, bs = b0 + s * b_step;
                        const uint64_t A0 = tc::sdesc(as, a_lbo, a_sbo);
                        const uint64_t A1 = tc::sdesc(as + kPieceBytes, a_lbo, a_sbo);
                        const uint64_t A2 = tc::sdesc(as + 2 * kPieceBytes, a_lbo, a_sbo);
                        const uint64_t B0 = tc::sdesc(bs, b_lbo, 128);
                        const uint64_t B1 = tc::sdesc(bs + kPieceB, b_lbo, 128);
                        const uint64_t B2 = tc::sdesc(bs + 2 * kPieceB, b_lbo, 128);
                        tc::mma_f16(dcorr, A0, B1, idesc, (c > 0 || s > 0) ? 1u : 0u);
                        tc::mma_f16(dcorr, A1, B0, idesc, 1);
                        tc::mma_f16(dcorr, A0, B2, idesc, 1);
                        tc::mma_f16(dcorr, A1, B1, idesc, 1);
                        tc::mma_f16(dcorr, A2, B0, idesc, 1);
                    }
                    // hi*hi of this chunk into the drained main columns
                    if (!wait_or_abort(&S.dmain_empty, (main_use & 1) ^ 1, abort, poll_limit)) {
                        set_status(status, FAVEST_ETIMEOUT);
                        *abort = 1;
                        break;
                    }
                    tc::fence_after_sync();
#pragma unroll
                    for (int s = 0; s < kChunkK / 16; ++s)
                        tc::mma_f16(dmain, tc::sdesc(a0 + s * a_step, a_lbo, a_sbo),
                                    tc::sdesc(b0 + s * b_step, b_lbo, 128), idesc, s > 0);
                    tc::mma_commit(&S.empty[stage]);
                    tc::mma_commit(&S.dmain_full);
                    phase ^= 1u << stage;
                    main_use++;
                    stage = (stage + 1) % kStages;
                }
                if (*abort) break;
                tc::mma_commit(&S.dcorr_full);
                corr_use++;
            }
            // On abort, MMAs issued before it may still be running: wait (bounded) for all of
            // them before the TMEM they write is released below.
            if (*abort) {
                tc::mma_commit(&S.drain);
                wait_or_abort(&S.drain, 0, nullptr, poll_limit);
            }
        }
      }
    } else {
      if constexpr (N == 256) tc::setmaxnreg_inc<224>();
        // ------ epilogue (warp w >= 4: TMEM lane quadrant w % 4, columns 128 * ((w-4) / 4) ..) ------
        const int quad = warp & 3;
        const int part = (warp - 4) >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t main_use = 0, corr_use = 0;
        float acc[kEpiCols];
        for (uint32_t n = 0; !*abort; ++n) {
            int it = -1;
            const bool got = __all_sync(0xffffffffu, item_take(S.ring, n, abort, poll_limit, it));
            if (!got) {
                set_status(status, FAVEST_ETIMEOUT);
                *abort = 1;
                break;
            }
            __syncwarp();
            if (lane == 0) item_release(S.ring, n);
            if (it < 0) break;
            const int nk = __ldg(&items[it].nk);   // the rest of the item is read at the end
#pragma unroll
            for (int i = 0; i < kEpiCols; ++i) acc[i] = 0.f;
            bool ok = true;
            for (int c = 0; c < nk; ++c) {
                if (!wait_or_abort(&S.dmain_full, main_use & 1, abort, poll_limit)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t col0 = tmem + lane_base + part * kEpiCols;
#pragma unroll
                for (int q = 0; q < kEpiCols / 16; ++q) {
                    float v[16];
                    tc::tmem_ld16(col0 + q * 16, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[q * 16 + i] += v[i];
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.dmain_empty);
                main_use++;
            }
            if (!ok || !wait_or_abort(&S.dcorr_full, corr_use & 1, abort, poll_limit)) {
                set_status(status, FAVEST_ETIMEOUT);
                *abort = 1;
                break;
            }
            tc::fence_after_sync();
#pragma unroll
            for (int q = 0; q < kEpiCols / 16; ++q) {
                float v[16];
                tc::tmem_ld16(tmem + lane_base + N + part * kEpiCols + q * 16, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[q * 16 + i] += v[i];
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.dcorr_empty);
            corr_use++;
            if (row < __ldg(&items[it].rows)) {
                // 8 columns per field: this warp writes fields part*16 .. part*16+15 of the tile
                const long long col_gs = __ldg(&items[it].col_gs);
                // rows come in groups of 4 consecutive 32-byte records; out_ld = group stride
                float *dst = groups[__ldg(&items[it].group)].out + __ldg(&items[it].out_off) + (long long)(row >> 2) * __ldg(&items[it].out_ld) +
                             (row & 3) * 8 + (long long)(part * (kEpiCols / 8)) * col_gs;
#pragma unroll
                for (int g = 0; g < kEpiCols / 8; ++g) {
                    float4 *d4 = reinterpret_cast<float4 *>(dst + g * col_gs);
                    d4[0] = make_float4(acc[8 * g], acc[8 * g + 1], acc[8 * g + 2], acc[8 * g + 3]);
                    d4[1] = make_float4(acc[8 * g + 4], acc[8 * g + 5], acc[8 * g + 6], acc[8 * g + 7]);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
    if (threadIdx.x == 0) item_sched_done(sched);
}

// ---------------------------------------------------------------------------
// Forward GEMM with an FP32 field operand.  The forward DFT stores its spectra as FP32
// records ([parity][8 floats] per latitude, field group and order, 64 bytes), so a K-chunk
// of the field operand arrives through TMA as rows of 32 bytes (8 floats), a third of the
// rows and two thirds of the bytes of three bf16 pieces.  Converter warps split it in shared
// memory into the three bf16 pieces the MMAs read (the same split the DFT made before, so
// results are bitwise unchanged); the element order of the FP32 box, [K/8][N/8][8 k][8 n],
// is already the pieces' core-matrix order.
// Warps, by warpgroup (the register split below acts on whole warpgroups): 0 producer (TMA of
// the Legendre chunk and the FP32 field chunk) and 1 MMA issuer (2, 3 idle); 4..7 converters;
// 8..15 epilogue (lane quadrant warp % 4, column half (warp - 8) / 4).
// Per stage (three of 72 KB): full (TMA landed) -> converters -> ready (pieces written) ->
// MMA -> empty.  Registers: launched at 128 per thread (512 threads); warpgroup 0 (producer,
// MMA) drops to 56, the converters to 104 (their rows in registers) and the two epilogue
// warpgroups rise to 176, which the epilogue's 128 FP32 running sums per thread need:
// 128 x 56 + 128 x 104 + 256 x 176 = 512 x 128.
// ---------------------------------------------------------------------------
constexpr int kFStages = 3;
constexpr int kConvWarps = 4;
constexpr int kFThreads = 512;
constexpr int kConvRows = kChunkK * 256 / 8 / (32 * kConvWarps);   // 8-float rows per converter thread (N = 256)

// OR of a flag over the converter warps, at named barrier 1 (a barrier for all of them)
__device__ __forceinline__ bool conv_any(uint32_t flag)
{
    uint32_t any;
    asm volatile("{\n\t.reg .pred q, p;\n\t"
                 "setp.ne.u32 q, %1, 0;\n\t"
                 "bar.red.or.pred p, 1, %2, q;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(any)
                 : "r"(flag), "n"(32 * kConvWarps)
                 : "memory");
    return any != 0;
}

template <int N>
struct GemmSmemF {
    unsigned char a[kFStages][kChunkBytes];
    unsigned char b[kFStages][kPieces * kChunkK * N * 2];   // FP32 chunk lands in its first 2/3
    uint64_t full[kFStages], ready[kFStages], empty[kFStages];
    uint64_t dmain_full, dmain_empty, dcorr_full, dcorr_empty;
    uint64_t drain;
    ItemRing ring;
    uint32_t tmem_base;
    int abort;
};

template <int N>
__global__ void __launch_bounds__(kFThreads, 1) k_tc_gemm_f(
    const GemmGroup *__restrict__ groups, const TcItem *__restrict__ items, int nitems, int *__restrict__ status,
    int *__restrict__ sched, uint32_t poll_limit)
{
    constexpr int kEpiWarps = 4 * (N / kEpiCols);
    constexpr int kPieceB = kChunkK * N * 2;
    constexpr int kChunkBF = kChunkK * N * 4;       // FP32 field chunk (first 2/3 of a piece buffer)
    extern __shared__ __align__(1024) unsigned char sm_raw_f[];
    GemmSmemF<N> &S = *reinterpret_cast<GemmSmemF<N> *>(sm_raw_f);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tc::tmem_alloc(&S.tmem_base, kTmemCols);
    if (threadIdx.x == 32) {
        for (int s = 0; s < kFStages; ++s) {
            tc::mbar_init(&S.full[s], 1);
            tc::mbar_init(&S.ready[s], kConvWarps);
            tc::mbar_init(&S.empty[s], 1);
        }
        tc::mbar_init(&S.dmain_full, 1);
        tc::mbar_init(&S.dmain_empty, kEpiWarps);
        tc::mbar_init(&S.dcorr_full, 1);
        tc::mbar_init(&S.dcorr_empty, kEpiWarps);
        tc::mbar_init(&S.drain, 1);
        item_ring_init(S.ring, 1 + kConvWarps + kEpiWarps);   // the MMA thread, converter and epilogue warps
        S.abort = 0;
        tc::mbar_fence_init();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = S.tmem_base;
    volatile int *abort = &S.abort;
    const int wg = warp >> 2;

    if (wg == 0) {
      tc::setmaxnreg_dec<56>();
      if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            uint32_t phase = 0, issued = 0;
            int stage = 0;
            for (uint32_t n = 0; !*abort; ++n) {
                int it;
                if (!item_publish(S.ring, n, sched, nitems, abort, poll_limit, it)) {
                    set_status(status, FAVEST_ETIMEOUT);
                    *abort = 1;
                    break;
                }
                if (it < 0) break;
                const TcItem I = items[it];
                const CUtensorMap *tmap_a = &groups[I.group].tmap_a, *tmap_b = &groups[I.group].tmap_b;
                for (int c = 0; c < I.nk; ++c) {
                    if (!wait_or_abort(&S.empty[stage], ((phase >> stage) & 1) ^ 1, abort, poll_limit)) {
                        set_status(status, FAVEST_ETIMEOUT);
                        *abort = 1;
                        break;
                    }
                    tc::mbar_arrive_expect_tx(&S.full[stage], kChunkBytes + kChunkBF);
                    tc::tma_load_4d(S.a[stage], tmap_a, 0, I.ay + c * I.ady, I.az + c * I.adz, 0, &S.full[stage]);
                    tc::tma_load_5d(S.b[stage], tmap_b, I.bx, I.bw, 0, I.by, (kChunkK / 8) * (I.bk + c),
                                    &S.full[stage]);
                    phase ^= 1u << stage;
                    issued |= 1u << stage;
                    stage = (stage + 1) % kFStages;
                }
            }
            // on abort: let this warp's loads land before the CTA can exit (bounded)
            if (*abort)
                for (int s = 0; s < kFStages; ++s)
                    if (issued & (1u << s)) wait_or_abort(&S.full[s], ((phase >> s) & 1) ^ 1, nullptr, poll_limit);
        }
      } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_f16(kTileM, N, 1, 1) | (1u << 7) | (1u << 10);
            uint32_t phase = 0, main_use = 0, corr_use = 0;
            int stage = 0;
            const uint32_t dmain = tmem, dcorr = tmem + N;
            // A MN-major, per piece [M/8 = 16 row blocks][K = 32 latitudes][8 rows]: K-groups
            // 128 B apart, M-blocks 512 B (leading byte offset = K-direction stride)
            constexpr uint32_t a_step = 256u, a_lbo = 128u, a_sbo = 512u;
            constexpr uint32_t b_step = 2 * (N / 8) * 128, b_lbo = (N / 8) * 128;
            for (uint32_t n = 0; !*abort; ++n) {
                int it;
                if (!item_take(S.ring, n, abort, poll_limit, it)) {
                    set_status(status, FAVEST_ETIMEOUT);
                    *abort = 1;
                    break;
                }
                item_release(S.ring, n);
                if (it < 0) break;
                const TcItem I = items[it];
                if (!wait_or_abort(&S.dcorr_empty, (corr_use & 1) ^ 1, abort, poll_limit)) {
                    set_status(status, FAVEST_ETIMEOUT);
                    *abort = 1;
                    break;
                }
                for (int c = 0; c < I.nk; ++c) {
                    if (!wait_or_abort(&S.ready[stage], (phase >> stage) & 1, abort, poll_limit)) {
                        set_status(status, FAVEST_ETIMEOUT);
                        *abort = 1;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(S.a[stage]), b0 = tc::smem_u32(S.b[stage]);
#pragma unroll
                    for (int s = 0; s < kChunkK / 16; ++s) {
                        const uint32_t as = a0 + s * a_step, bs = b0 + s * b_step;
                        const uint64_t A0 = tc::sdesc(as, a_lbo, a_sbo);
                        const uint64_t A1 = tc::sdesc(as + kPieceBytes, a_lbo, a_sbo);
                        const uint64_t A2 = tc::sdesc(as + 2 * kPieceBytes, a_lbo, a_sbo);
                        const uint64_t B0 = tc::sdesc(bs, b_lbo, 128);
                        const uint64_t B1 = tc::sdesc(bs + kPieceB, b_lbo, 128);
                        const uint64_t B2 = tc::sdesc(bs + 2 * kPieceB, b_lbo, 128);
                        tc::mma_f16(dcorr, A0, B1, idesc, (c > 0 || s > 0) ? 1u : 0u);
                        tc::mma_f16(dcorr, A1, B0, idesc, 1);
                        tc::mma_f16(dcorr, A0, B2, idesc, 1);
                        tc::mma_f16(dcorr, A1, B1, idesc, 1);
                        tc::mma_f16(dcorr, A2, B0, idesc, 1);
                    }
                    if (!wait_or_abort(&S.dmain_empty, (main_use & 1) ^ 1, abort, poll_limit)) {
                        set_status(status, FAVEST_ETIMEOUT);
                        *abort = 1;
                        break;
                    }
                    tc::fence_after_sync();
#pragma unroll
                    for (int s = 0; s < kChunkK / 16; ++s)
                        tc::mma_f16(dmain, tc::sdesc(a0 + s * a_step, a_lbo, a_sbo),
                                    tc::sdesc(b0 + s * b_step, b_lbo, 128), idesc, s > 0);
                    tc::mma_commit(&S.empty[stage]);
                    tc::mma_commit(&S.dmain_full);
                    phase ^= 1u << stage;
                    main_use++;
                    stage = (stage + 1) % kFStages;
                }
                if (*abort) break;
                tc::mma_commit(&S.dcorr_full);
                corr_use++;
            }
            if (*abort) {
                tc::mma_commit(&S.drain);
                wait_or_abort(&S.drain, 0, nullptr, poll_limit);
            }
        }
      }
    } else if (wg == 1) {
        tc::setmaxnreg_dec<104>();
        // ---------------- converters: FP32 field chunk -> three bf16 pieces, in place ----------------
        // The FP32 rows (8 floats, 32 bytes) occupy the first 2/3 of the stage's piece buffer and
        // the pieces (16 bytes per row each) all of it, so every converter thread first reads
        // its rows into registers and the converter warps meet at a named barrier before any
        // piece is written.
        constexpr int kRows = kChunkK * N / 8 / (32 * kConvWarps);
        static_assert(kRows * 32 * kConvWarps * 8 == kChunkK * N && kRows <= kConvRows, "converter rows");
        // Each thread waits on the stage on its own, so whether a chunk goes ahead is agreed
        // at the named barrier itself (an OR over the converter threads of "my wait gave up"):
        // every converter thread then passes the same number of barriers and leaves together.
        // The item indices are agreed the same way.
        const int ct = threadIdx.x - 128;                // 0 .. 32 * kConvWarps - 1
        uint32_t phase = 0;
        int stage = 0;
        bool ok = true;
        for (uint32_t n = 0; ok; ++n) {
            int it = -1;
            const uint32_t take_gave_up = item_take(S.ring, n, abort, poll_limit, it) ? 0u : 1u;
            if (conv_any(take_gave_up)) { ok = false; break; }
            __syncwarp();
            if (lane == 0) item_release(S.ring, n);
            if (it < 0) break;
            const int nk = __ldg(&items[it].nk);
            for (int c = 0; c < nk; ++c) {
                const uint32_t gave_up =
                    wait_or_abort(&S.full[stage], (phase >> stage) & 1, abort, poll_limit) ? 0u : 1u;
                const float4 *src = reinterpret_cast<const float4 *>(S.b[stage]);
                uint4 *dst = reinterpret_cast<uint4 *>(S.b[stage]);
                float4 v4[kRows][2];
                if (!gave_up) {
#pragma unroll
                    for (int k = 0; k < kRows; ++k) {
                        const int r = ct + k * 32 * kConvWarps;
                        v4[k][0] = src[2 * r];
                        v4[k][1] = src[2 * r + 1];
                    }
                }
                if (conv_any(gave_up)) { ok = false; break; }
                // row r: 8 consecutive floats -> 16 bytes of each piece at the same position
#pragma unroll
                for (int k = 0; k < kRows; ++k) {
                    const int r = ct + k * 32 * kConvWarps;
                    const float v[8] = {v4[k][0].x, v4[k][0].y, v4[k][0].z, v4[k][0].w,
                                        v4[k][1].x, v4[k][1].y, v4[k][1].z, v4[k][1].w};
                    uint4 pc[3];
                    pack_row3(v, pc);
#pragma unroll
                    for (int q = 0; q < kPieces; ++q) dst[q * (kPieceB / 16) + r] = pc[q];
                }
                tc::fence_proxy_async_smem();            // the MMAs read the pieces through the async proxy
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.ready[stage]);
                phase ^= 1u << stage;
                stage = (stage + 1) % kFStages;
            }
        }
        if (!ok) {
            set_status(status, FAVEST_ETIMEOUT);
            *abort = 1;
        }
    } else {
      tc::setmaxnreg_inc<176>();
      if (warp - 8 < kEpiWarps) {
        // ------ epilogue (lane quadrant warp % 4, columns 128 * ((warp - 8) / 4) ..) ------
        const int quad = warp & 3;
        const int part = (warp - 8) >> 2;
        const int row = quad * 32 + lane;
        const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
        uint32_t main_use = 0, corr_use = 0;
        float acc[kEpiCols];
        for (uint32_t n = 0; !*abort; ++n) {
            int it = -1;
            const bool got = __all_sync(0xffffffffu, item_take(S.ring, n, abort, poll_limit, it));
            if (!got) {
                set_status(status, FAVEST_ETIMEOUT);
                *abort = 1;
                break;
            }
            __syncwarp();
            if (lane == 0) item_release(S.ring, n);
            if (it < 0) break;
            const int nk = __ldg(&items[it].nk);
#pragma unroll
            for (int i = 0; i < kEpiCols; ++i) acc[i] = 0.f;
            bool ok = true;
            for (int c = 0; c < nk; ++c) {
                if (!wait_or_abort(&S.dmain_full, main_use & 1, abort, poll_limit)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t col0 = tmem + lane_base + part * kEpiCols;
#pragma unroll
                for (int q = 0; q < kEpiCols / 16; ++q) {
                    float v[16];
                    tc::tmem_ld16(col0 + q * 16, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[q * 16 + i] += v[i];
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&S.dmain_empty);
                main_use++;
            }
            if (!ok || !wait_or_abort(&S.dcorr_full, corr_use & 1, abort, poll_limit)) {
                set_status(status, FAVEST_ETIMEOUT);
                *abort = 1;
                break;
            }
            tc::fence_after_sync();
#pragma unroll
            for (int q = 0; q < kEpiCols / 16; ++q) {
                float v[16];
                tc::tmem_ld16(tmem + lane_base + N + part * kEpiCols + q * 16, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[q * 16 + i] += v[i];
            }
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&S.dcorr_empty);
            corr_use++;
            if (row < __ldg(&items[it].rows)) {
                const long long col_gs = __ldg(&items[it].col_gs);
                float *dst = groups[__ldg(&items[it].group)].out + __ldg(&items[it].out_off) +
                             (long long)(row >> 2) * __ldg(&items[it].out_ld) + (row & 3) * 8 +
                             (long long)(part * (kEpiCols / 8)) * col_gs;
#pragma unroll
                for (int g = 0; g < kEpiCols / 8; ++g) {
                    float4 *d4 = reinterpret_cast<float4 *>(dst + g * col_gs);
                    d4[0] = make_float4(acc[8 * g], acc[8 * g + 1], acc[8 * g + 2], acc[8 * g + 3]);
                    d4[1] = make_float4(acc[8 * g + 4], acc[8 * g + 5], acc[8 * g + 6], acc[8 * g + 7]);
                }
            }
        }
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
    if (threadIdx.x == 0) item_sched_done(sched);
}

template <int N>
cudaError_t launch_gemm_f(const GemmGroup *groups, const TcItem *items, int nitems, int *status, int num_sms,
                          cudaStream_t s)
{
    const size_t smem = sizeof(GemmSmemF<N>) + 1024;
    auto k = k_tc_gemm_f<N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = nitems < num_sms ? nitems : num_sms;
    if (grid <= 0) return cudaSuccess;
    k<<<grid, kFThreads, smem, s>>>(groups, items, nitems, status, gemm_sched(status, true), kWaitPolls);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_gemm_n(const GemmGroup *groups, const TcItem *items, int nitems, int a_mn_major, int *status,
                          int num_sms, cudaStream_t s, uint32_t poll_limit = kWaitPolls, int skip_loads = 0)
{
    const size_t smem = sizeof(GemmSmem<N>) + 1024;
    auto k = k_tc_gemm<N>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = nitems < num_sms ? nitems : num_sms;
    if (grid <= 0) return cudaSuccess;
    k<<<grid, gemm_threads<N>(), smem, s>>>(groups, items, nitems, a_mn_major, status,
                                           gemm_sched(status, a_mn_major != 0), poll_limit, skip_loads);
    return cudaGetLastError();
}

}  // namespace

template <int NJ>
void launch_gen_t(const Plan &p, int lt, int mb, cudaStream_t s)
{
    const int olanes = kGenThreads / lt;
    const int ogroups = (p.L + 1 + olanes * mb - 1) / (olanes * mb);
    const int grid = ((p.JP + NJ * lt - 1) / (NJ * lt)) * ogroups;
    k_gen_lambda<NJ><<<grid, kGenThreads, 0, s>>>((unsigned char *)p.d_lam, p.d_lam_rb, p.lam_rb_total, p.d_xdf,
                                                  p.d_sin, p.d_cmu, p.d_Adf, p.d_jcmin, p.L, p.J, p.JP, lt, mb);
}

cudaError_t launch_gen_lambda_shape(const Plan &p, int layouts, int lt, int mb, int nj, cudaStream_t s)
{
    // one layout serves both directions: every request writes it
    if (lt != 32 && lt != 64 && lt != 128) return cudaErrorInvalidValue;
    if (layouts != kGenFwd && layouts != kGenAdj && layouts != kGenBoth) return cudaErrorInvalidValue;
    if (nj == 1) launch_gen_t<1>(p, lt, mb, s);
    else if (nj == 2) launch_gen_t<2>(p, lt, mb, s);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_gen_lambda(const Plan &p, int layouts, cudaStream_t s)
{
    return launch_gen_lambda_shape(p, layouts, p.gen_lt, p.gen_mb, p.gen_nj, s);
}

cudaError_t launch_tc_gemm_items(int gemm_n, const GemmGroup *groups, const TcItem *items, int nitems,
                                 int a_mn_major, int *status, int num_sms, cudaStream_t s)
{
    // the forward items (MN-major Legendre operand) read the FP32 field operand
    if (a_mn_major)
        return gemm_n == 256 ? launch_gemm_f<256>(groups, items, nitems, status, num_sms, s)
                             : launch_gemm_f<128>(groups, items, nitems, status, num_sms, s);
    return gemm_n == 256 ? launch_gemm_n<256>(groups, items, nitems, a_mn_major, status, num_sms, s)
                         : launch_gemm_n<128>(groups, items, nitems, a_mn_major, status, num_sms, s);
}

cudaError_t launch_gemm_selftest(const Plan &p, uint32_t poll_limit, cudaStream_t s)
{
    // one adjoint item, nothing loaded
    return p.gemm_n == 256 ? launch_gemm_n<256>(p.d_ggroups, p.d_items_a, 1, 0, p.d_status, p.num_sms, s, poll_limit, 1)
                           : launch_gemm_n<128>(p.d_ggroups, p.d_items_a, 1, 0, p.d_status, p.num_sms, s, poll_limit, 1);
}

cudaError_t launch_tc_gemm(const Plan &p, bool fwd, cudaStream_t s)
{
    return launch_tc_gemm_items(p.gemm_n, p.d_ggroups, fwd ? p.d_items_f : p.d_items_a,
                                fwd ? p.n_items_f : p.n_items_a, fwd ? 1 : 0, p.d_status, p.num_sms, s);
}

}  // namespace favest
