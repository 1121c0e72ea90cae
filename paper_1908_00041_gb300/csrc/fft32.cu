// Longitude DFT stage of the split-precision path (FP32 arithmetic, FP64-derived
// twiddles rounded to FP32).  One CTA per (field b, folded latitude j) handles the four
// rings theta/phi x (j, nlat-1-j) (real fields: see k_rfft_fwd_bf16):
//   forward: T -> FFT -> weighted equatorial fold F+- = omega_j (F_j +- F_j') -> FP32
//            records staged per warp and stored into the tensor-core GEMM's field-operand
//            layout by bulk asynchronous copies (the GEMM splits them into bf16 pieces).
//   inverse: streams the even/odd Legendre sums E, O of every order through shared memory
//            (TMA boxes), forms G_j = (E + O) / sin(theta_j), G_j' = (E - O) / sin(theta_j),
//            inverse FFT whose last stage stores to global memory.
// Power-of-two lengths run register radix-16 butterflies (forward: decimation in frequency
// with the first stage fed from global memory; inverse: its transpose); other lengths a
// generic mixed-radix decimation in frequency with a digit-reversal table.  At n = 2048
// (L = 1023) complex fields take k_fft_fwd_sw / k_fft_inv_sw instead: rings brought in by
// bulk copies, an XOR-swizzled layout in place of the padding, records to and from
// registers without staging.  Every stage reads its twiddles from per-stage tables in
// [q][k] order, so that a warp's threads read consecutive entries.
#include "favest_internal.h"
#include "bf16_split.cuh"
#include "fft_device.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace favest {

namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <bool INV>
__device__ __forceinline__ float2 twf(const float2 *__restrict__ tw, int q)
{
    float2 t = __ldg(tw + q);
    return INV ? make_float2(t.x, -t.y) : t;
}

// In-place decimation-in-frequency FFT of `nr` rings of n points stored back to back.
// Stage s (radix R, block length Nb, h = Nb/R): for every block and k < h the R points
// x[k + t h] are replaced by their R-point DFT, output q scaled by w_Nb^{q k}.  Frequency m
// ends at position perm[m] (mixed-radix digit reversal, precomputed on the host).  Each
// butterfly reads and writes the same addresses, and the butterflies of a stage touch
// disjoint positions, so one buffer suffices.
// Radices 2 and 4, and the odd primes 3..13: one thread per butterfly, its R points in
// registers and the R roots of unity w_R^j loaded once per stage.  Primes from 17 up: a
// Bluestein convolution on the radix-16 engine (dif_stage_bluestein, after the engine).
// The output twiddle exponent q k n/Nb is below n (q < R, k < Nb/R): no reduction is needed.

// Butterfly index -> (ring, block, k) without integer division: q = floor(x / d) for
// 0 <= x < 2^15 and 1 <= d <= 4096 as the high word of x * m, m = floor((2^32 - 1) / d) + 1
// (ceil(2^32 / d) unless d is a power of two, then exact): the excess x (m d - 2^32) / 2^32
// stays below 1 while x d < 2^32, which these ranges (x < 4 rings * 1024, d <= 2048) keep.
struct Recip {
    unsigned m;
    int d;
};
__device__ __forceinline__ Recip recip(int d) { return Recip{0xffffffffu / (unsigned)d + 1u, d}; }
__device__ __forceinline__ int rdiv(int x, Recip r) { return r.d == 1 ? x : (int)__umulhi((unsigned)x, r.m); }

// Odd prime R: with w_R^j = (c_j, y_j) and w_R^{-j} = (c_j, -y_j), the pairs r, R - r give
//   out_q     = v_0 + sum_{r=1}^{H} [c_{qr} (v_r + v_{R-r}) + i y_{qr} (v_r - v_{R-r})] = A_q + i B_q,
//   out_{R-q} = A_q - i B_q,   H = (R - 1) / 2,
// 4 H^2 real multiply-adds per butterfly instead of R (R - 1) complex ones.
// twS: the stage's twiddles in [q][k] order (entry q h + k = w_n^(q k n / Nb))
template <int R, bool INV>
__device__ __forceinline__ void dif_stage_small(float2 *x, const float2 *__restrict__ tw,
                                                const float2 *__restrict__ twS, int n, int Nb, int nr)
{
    constexpr int H = (R - 1) / 2;
    const int h = Nb / R, nbf = n / R, rstep = n / R;
    float2 wr[H + 1];                                  // w_R^j = w_n^{j n / R}, j <= H
#pragma unroll
    for (int j = 1; j <= H; ++j) wr[j] = twf<INV>(tw, j * rstep);
    const Recip rn = recip(nbf), rh = recip(h);
    for (int t = threadIdx.x; t < nbf * nr; t += blockDim.x) {
        const int ring = rdiv(t, rn), i = t - ring * nbf;
        const int blk = rdiv(i, rh), k = i - blk * h;
        float2 *xr = x + ring * n + blk * Nb + k;
        const float2 v0 = xr[0];
        float2 sm[H], df[H];
        float2 out0 = v0;
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const float2 a = xr[r * h], b = xr[(R - r) * h];
            sm[r - 1] = caddf(a, b);
            df[r - 1] = csubf(a, b);
            out0 = caddf(out0, sm[r - 1]);
        }
        xr[0] = out0;
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            float2 A = v0, Bq = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                // w_R^{qr}: index e = qr mod R, and w_R^e = conj(w_R^{R-e}) above H
                const int e = (q * r) % R;
                const float wc = e <= H ? wr[e].x : wr[R - e].x;
                const float ws = e <= H ? wr[e].y : -wr[R - e].y;
                A.x = fmaf(wc, sm[r - 1].x, A.x);
                A.y = fmaf(wc, sm[r - 1].y, A.y);
                Bq.x = fmaf(ws, df[r - 1].x, Bq.x);
                Bq.y = fmaf(ws, df[r - 1].y, Bq.y);
            }
            const float2 op = make_float2(A.x - Bq.y, A.y + Bq.x);     // A + i B
            const float2 om = make_float2(A.x + Bq.y, A.y - Bq.x);     // A - i B
            xr[q * h] = cmulf(op, twf<INV>(twS + k, q * h));
            xr[(R - q) * h] = cmulf(om, twf<INV>(twS + k, (R - q) * h));
        }
    }
}

// Power-of-two lengths n = 2^LOG2N (64..4096): in-place decimation in frequency with
// radix-16 butterflies held in registers, then one last radix-2^r stage (r = LOG2N mod 4,
// or 16 when that is 0).  The last stage has no twiddles and writes its outputs back in
// natural frequency order, so no digit-reversal table is needed on either side.  All
// index arithmetic is shifts and masks.  Shared memory holds one padding complex after
// every 16, which makes every stage's accesses (stride 1, 8 or 16 complexes across a
// half-warp) and the natural-order write free of bank conflicts.
// ---------------------------------------------------------------------------
constexpr int kFftThreads = 256;

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// cos and sin of 2 pi j / 16
__host__ __device__ constexpr float cos16(int j)
{
    constexpr float t[16] = {1.f, 0.92387953251128674f, 0.70710678118654752f, 0.38268343236508977f,
                             0.f, -0.38268343236508977f, -0.70710678118654752f, -0.92387953251128674f,
                             -1.f, -0.92387953251128674f, -0.70710678118654752f, -0.38268343236508977f,
                             0.f, 0.38268343236508977f, 0.70710678118654752f, 0.92387953251128674f};
    return t[j & 15];
}
__host__ __device__ constexpr float sin16(int j) { return cos16(j + 12); }

template <int R>
struct Log2c { static constexpr int v = R == 2 ? 1 : R == 4 ? 2 : R == 8 ? 3 : 4; };

// R-point DFT in registers by radix-2 decimation in frequency (forward: exp(-2 pi i qt/R),
// inverse: exp(+...)); output q ends in v[bitrev(q)]
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R])
{
#pragma unroll
    for (int s = R / 2; s >= 1; s >>= 1) {
#pragma unroll
        for (int g = 0; g < R; g += 2 * s) {
#pragma unroll
            for (int j = 0; j < s; ++j) {
                const float2 a = v[g + j], b = v[g + j + s];
                v[g + j] = caddf(a, b);
                const float2 d = csubf(a, b);
                const int e = j * (16 / (2 * s));        // w_{2s}^j = w_16^e
                if (e == 0) {
                    v[g + j + s] = d;
                } else if (e == 4) {                     // -i (forward) or +i (inverse)
                    v[g + j + s] = INV ? make_float2(-d.y, d.x) : make_float2(d.y, -d.x);
                } else {
                    const float c = cos16(e), sn = INV ? sin16(e) : -sin16(e);
                    v[g + j + s] = make_float2(fmaf(c, d.x, -sn * d.y), fmaf(c, d.y, sn * d.x));
                }
            }
        }
    }
}

__host__ __device__ constexpr int bitrev(int x, int bits)
{
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

// one in-place radix-16 stage at block length NB over nr rings; kTab: tw is the stage's
// [q][k] table (entry q h + k = w_n^(q k n / NB)), else the plain w_n^i table
template <int LOG2N, int NB, bool INV, bool kTab = false>
__device__ __forceinline__ void dif_stage16(float2 *x, const float2 *__restrict__ tw, int nr)
{
    constexpr int n = 1 << LOG2N, R = 16;
    constexpr int h = NB / R, ts = n / NB, nbf = n / R;
    for (int t = threadIdx.x; t < nbf * nr; t += kFftThreads) {
        const int ring = t >> (LOG2N - 4);
        const int i = t & (nbf - 1);
        const int k = i & (h - 1);
        const int base = ring * n + (i - k) * R + k;     // block (i / h) * NB, offset k
        float2 v[R];
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = x[padi(base + q * h)];
        dft_reg<R, INV>(v);
        x[padi(base)] = v[0];
#pragma unroll
        for (int q = 1; q < R; ++q)
            x[padi(base + q * h)] = cmulf(v[bitrev(q, 4)], twf<INV>(tw, kTab ? q * h + k : q * k * ts));
    }
    __syncthreads();
}

// last stage (h = 1, no twiddles): blocks of RL consecutive points; output q of block blk
// is frequency m = nibble_reverse(blk) + q * n / RL, stored back at position m.  All of a
// ring's blocks are read before any of its points is rewritten.
template <int LOG2N, int RL, bool INV>
__device__ __forceinline__ void dif_last(float2 *x, int nr)
{
    constexpr int n = 1 << LOG2N, LB = Log2c<RL>::v;
    constexpr int nblk = n / RL, ndig = (LOG2N - LB) / 4;
    static_assert(nblk <= kFftThreads && (LOG2N - LB) % 4 == 0, "unsupported length");
    constexpr int rings_per_round = kFftThreads / nblk;
    const int t = threadIdx.x;
    for (int r0 = 0; r0 < nr; r0 += rings_per_round) {
        const int ring = r0 + t / nblk, blk = t & (nblk - 1);
        const bool act = t < nblk * rings_per_round && ring < nr;
        float2 v[RL];
        if (act) {
#pragma unroll
            for (int q = 0; q < RL; ++q) v[q] = x[padi(ring * n + blk * RL + q)];
            dft_reg<RL, INV>(v);
        }
        __syncthreads();
        if (act) {
            int m0 = 0;
#pragma unroll
            for (int d = 0; d < ndig; ++d) m0 |= ((blk >> (4 * d)) & 15) << (4 * (ndig - 1 - d));
#pragma unroll
            for (int q = 0; q < RL; ++q) x[padi(ring * n + m0 + q * nblk)] = v[bitrev(q, LB)];
        }
        __syncthreads();
    }
}

// Bluestein stage of a prime radix R >= 17 (stage st of the plan): Bluestein's identity
// q t = (q^2 + t^2 - (q - t)^2) / 2 turns each R-point DFT into a cyclic convolution,
//   out_q = c_q sum_t (x_t c_t) conj(c_{q-t}),   c_t = exp(-i pi t^2 / R),
// done at power-of-two length M >= 2R - 1 in the CTA's shared-memory scratch, P butterflies
// side by side per round: M <= 4096 runs both FFTs on the radix-16 engine above (natural order
// in and out, padded layout), the product with the precomputed spectrum of conj(c) (scaled by
// 1/M) between them; M = 8192 (R > 2048) uses radix-2 passes, a decimation in frequency
// (natural in, bit-reversed out), the spectrum stored bit-reversed, and a decimation in time
// with conjugate twiddles (bit-reversed in, natural out).  The inverse transform is the
// conjugate of the forward one of the conjugated input.  A round reads all its points before
// any is rewritten, and the butterflies of a stage touch disjoint positions.  FP32 error of the
// stage about 2e-7 of its largest output for R up to 2251 (checked on the host against a
// library FFT before the kernel was written).
template <int LG, bool INV>
__device__ __forceinline__ void fft_p2_smem(float2 *x, const float2 *__restrict__ tw, int nr)
{
    constexpr int n16 = LG / 4, rem = LG % 4, nfull = rem ? n16 : n16 - 1;
    static_assert(nfull >= 1 && nfull <= 2, "radix-16 engine lengths 2^5 .. 2^12");
    dif_stage16<LG, (1 << LG), INV>(x, tw, nr);
    if constexpr (nfull >= 2) dif_stage16<LG, (1 << LG) / 16, INV>(x, tw, nr);
    dif_last<LG, (rem ? (1 << rem) : 16), INV>(x, nr);
}

struct BlueStage {
    int n, R, Nb, nr, P;
    const float2 *ch, *sp, *tm;
    __device__ __forceinline__ int base_of(int bi) const
    {
        const int h = Nb / R, nbf = n / R;
        const int ring = bi / nbf, i = bi - ring * nbf;
        const int blk = i / h, k = i - blk * h;
        return ring * n + blk * Nb + k;
    }
};

template <int LG, bool INV>
__device__ __noinline__ void bluestein_rounds(float2 *x, const float2 *__restrict__ tw, const BlueStage b, float2 *sc)
{
    constexpr int M = 1 << LG;
    const int R = b.R, h = b.Nb / b.R, ts = b.n / b.Nb, nbf = b.n / b.R, total = nbf * b.nr;
    for (int b0 = 0; b0 < total; b0 += b.P) {
        const int np = total - b0 < b.P ? total - b0 : b.P;
        for (int idx = threadIdx.x; idx < np * M; idx += blockDim.x) {
            const int bb = idx >> LG, t = idx & (M - 1);
            float2 v = make_float2(0.f, 0.f);
            if (t < R) {
                float2 xv = x[b.base_of(b0 + bb) + t * h];
                if (INV) xv.y = -xv.y;
                v = cmulf(xv, __ldg(b.ch + t));
            }
            sc[padi(idx)] = v;
        }
        __syncthreads();
        fft_p2_smem<LG, false>(sc, b.tm, np);
        for (int idx = threadIdx.x; idx < np * M; idx += blockDim.x)
            sc[padi(idx)] = cmulf(sc[padi(idx)], __ldg(b.sp + (idx & (M - 1))));
        __syncthreads();
        fft_p2_smem<LG, true>(sc, b.tm, np);
        for (int idx = threadIdx.x; idx < np * R; idx += blockDim.x) {
            const int bb = idx / R, q = idx - bb * R;
            const int bi = b0 + bb;
            const int k = (bi - (bi / nbf) * nbf) % h;
            float2 v = cmulf(sc[padi((bb << LG) + q)], __ldg(b.ch + q));
            if (INV) v.y = -v.y;
            x[b.base_of(bi) + q * h] = cmulf(v, twf<INV>(tw, q * k * ts));
        }
        __syncthreads();
    }
}

// M = 8192: radix-2 passes (the engine stops at 2^12)
template <bool INV>
__device__ __noinline__ void bluestein_rounds_r2(float2 *x, const float2 *__restrict__ tw, const BlueStage b, int lg,
                                                 float2 *sc)
{
    const int M = 1 << lg, hm = M >> 1;
    const int R = b.R, h = b.Nb / b.R, ts = b.n / b.Nb, nbf = b.n / b.R, total = nbf * b.nr;
    for (int b0 = 0; b0 < total; b0 += b.P) {
        const int np = total - b0 < b.P ? total - b0 : b.P;
        for (int idx = threadIdx.x; idx < np * M; idx += blockDim.x) {
            const int bb = idx >> lg, t = idx & (M - 1);
            float2 v = make_float2(0.f, 0.f);
            if (t < R) {
                float2 xv = x[b.base_of(b0 + bb) + t * h];
                if (INV) xv.y = -xv.y;
                v = cmulf(xv, __ldg(b.ch + t));
            }
            sc[idx] = v;
        }
        __syncthreads();
        for (int lgs = lg - 1; lgs >= 0; --lgs) {          // half-block s = 2^lgs
            const int s = 1 << lgs;
            for (int u = threadIdx.x; u < np * hm; u += blockDim.x) {
                const int uu = u & (hm - 1), j = uu & (s - 1);
                const int i0 = ((u >> (lg - 1)) << lg) + ((uu >> lgs) << (lgs + 1)) + j;
                const float2 a = sc[i0], c = sc[i0 + s];
                sc[i0] = caddf(a, c);
                sc[i0 + s] = cmulf(csubf(a, c), __ldg(b.tm + (j << (lg - 1 - lgs))));
            }
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < np * M; idx += blockDim.x)
            sc[idx] = cmulf(sc[idx], __ldg(b.sp + (idx & (M - 1))));
        __syncthreads();
        for (int lgs = 0; lgs < lg; ++lgs) {
            const int s = 1 << lgs;
            for (int u = threadIdx.x; u < np * hm; u += blockDim.x) {
                const int uu = u & (hm - 1), j = uu & (s - 1);
                const int i0 = ((u >> (lg - 1)) << lg) + ((uu >> lgs) << (lgs + 1)) + j;
                float2 w = __ldg(b.tm + (j << (lg - 1 - lgs)));
                w.y = -w.y;
                const float2 a = sc[i0], c = cmulf(sc[i0 + s], w);
                sc[i0] = caddf(a, c);
                sc[i0 + s] = csubf(a, c);
            }
            __syncthreads();
        }
        for (int idx = threadIdx.x; idx < np * R; idx += blockDim.x) {
            const int bb = idx / R, q = idx - bb * R;
            const int bi = b0 + bb;
            const int k = (bi - (bi / nbf) * nbf) % h;
            float2 v = cmulf(sc[(bb << lg) + q], __ldg(b.ch + q));
            if (INV) v.y = -v.y;
            x[b.base_of(bi) + q * h] = cmulf(v, twf<INV>(tw, q * k * ts));
        }
        __syncthreads();
    }
}

// The rounds are out of line: inlined into the generic DFT kernels (128 registers at two CTAs
// per SM) the engine code made them spill.
template <bool INV>
__device__ __forceinline__ void dif_stage_bluestein(float2 *x, const float2 *__restrict__ tw, int n, int R, int Nb,
                                                 int nr, int lg, int P, const float2 *ch, const float2 *sp,
                                                 const float2 *tm, float2 *sc)
{
    const BlueStage b{n, R, Nb, nr, P, ch, sp, tm};
    switch (lg) {
    case 5: bluestein_rounds<5, INV>(x, tw, b, sc); break;
    case 6: bluestein_rounds<6, INV>(x, tw, b, sc); break;
    case 7: bluestein_rounds<7, INV>(x, tw, b, sc); break;
    case 8: bluestein_rounds<8, INV>(x, tw, b, sc); break;
    case 9: bluestein_rounds<9, INV>(x, tw, b, sc); break;
    case 10: bluestein_rounds<10, INV>(x, tw, b, sc); break;
    case 11: bluestein_rounds<11, INV>(x, tw, b, sc); break;
    case 12: bluestein_rounds<12, INV>(x, tw, b, sc); break;
    default: bluestein_rounds_r2<INV>(x, tw, b, lg, sc); break;
    }
}

// sc: the Bluestein scratch (FftPlan::blue_scratch bytes) when the plan has such stages;
// BLUE = false compiles without the Bluestein branch (plans whose radices are all <= 13)
// st0: the first stage to run (the stages before it already done, see first_stage_global)
template <bool INV, bool BLUE>
__device__ void dif_f32(float2 *x, const float2 *__restrict__ tw, const RadixPlanArg &rp, int nr, float2 *sc,
                        int st0 = 0)
{
    const int n = rp.n;
    int Nb = n;
    for (int st = 0; st < st0; ++st) Nb /= rp.radix[st];
    for (int st = st0; st < rp.nstages; ++st) {
        const int R = rp.radix[st];
        const int h = Nb / R;
        const int nbf = n / R;
        if (R == 3) {
            dif_stage_small<3, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 5) {
            dif_stage_small<5, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 7) {
            dif_stage_small<7, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 11) {
            dif_stage_small<11, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 13) {
            dif_stage_small<13, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (BLUE && R != 2 && R != 4) {         // primes >= 17 (build_bluestein marks them all)
            dif_stage_bluestein<INV>(x, tw, n, R, Nb, nr, rp.blue_lg[st], rp.blue_P[st], rp.blue_chirp + rp.blue_off[st],
                                     rp.blue_spec + rp.blue_moff[st], rp.blue_tw + rp.blue_moff[st], sc);
        } else {
            const float2 *twS = tw + rp.tw_off[st];
            const Recip rn = recip(nbf), rh = recip(h);
            for (int t = threadIdx.x; t < nbf * nr; t += blockDim.x) {
                const int ring = rdiv(t, rn), i = t - ring * nbf;
                const int blk = rdiv(i, rh), k = i - blk * h;
                float2 *xr = x + ring * n + blk * Nb + k;
                if (R == 4) {
                    const float2 v0 = xr[0], v1 = xr[h], v2 = xr[2 * h], v3 = xr[3 * h];
                    const float2 s02 = caddf(v0, v2), d02 = csubf(v0, v2);
                    const float2 s13 = caddf(v1, v3), d13 = csubf(v1, v3);
                    const float2 rot = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
                    xr[0] = caddf(s02, s13);
                    xr[h] = cmulf(caddf(d02, rot), twf<INV>(twS, h + k));
                    xr[2 * h] = cmulf(csubf(s02, s13), twf<INV>(twS, 2 * h + k));
                    xr[3 * h] = cmulf(csubf(d02, rot), twf<INV>(twS, 3 * h + k));
                } else {
                    const float2 v0 = xr[0], v1 = xr[h];
                    xr[0] = caddf(v0, v1);
                    xr[h] = cmulf(csubf(v0, v1), twf<INV>(twS, h + k));
                }
            }
        }
        __syncthreads();
        Nb = h;
    }
}

// Decimation in time, the transpose of dif_f32 (the DFT matrix is symmetric): with the
// decimation-in-frequency transform written as F = P S_{S-1} .. S_1 S_0 (stage S_s:
// butterflies, then the output twiddles; P: the digit-reversal gather), F = F^T =
// S_0^T .. S_{S-1}^T P^T, where P^T scatters frequency m to position perm[m] and S_s^T
// multiplies the same twiddles into a butterfly's inputs before the same R-point DFT.
// dit_f32 runs S_{S-1}^T .. S_{st_end}^T in place; last_stage_global runs S_0^T (radix 2 or
// 4, block length n), whose outputs k + q h are in natural order, straight to global memory.
// Radices 2, 4 and the odd primes 3..13 (plans without Bluestein stages).
template <int R, bool INV>
__device__ __forceinline__ void dit_stage_small(float2 *x, const float2 *__restrict__ tw,
                                                const float2 *__restrict__ twS, int n, int Nb, int nr)
{
    constexpr int H = (R - 1) / 2;
    const int h = Nb / R, nbf = n / R, rstep = n / R;
    float2 wr[H + 1];                                  // w_R^j, j <= H
#pragma unroll
    for (int j = 1; j <= H; ++j) wr[j] = twf<INV>(tw, j * rstep);
    const Recip rn = recip(nbf), rh = recip(h);
    for (int t = threadIdx.x; t < nbf * nr; t += blockDim.x) {
        const int ring = rdiv(t, rn), i = t - ring * nbf;
        const int blk = rdiv(i, rh), k = i - blk * h;
        float2 *xr = x + ring * n + blk * Nb + k;
        const float2 v0 = xr[0];
        float2 sm[H], df[H];
        float2 out0 = v0;
#pragma unroll
        for (int r = 1; r <= H; ++r) {
            const float2 a = cmulf(xr[r * h], twf<INV>(twS, r * h + k));
            const float2 b = cmulf(xr[(R - r) * h], twf<INV>(twS, (R - r) * h + k));
            sm[r - 1] = caddf(a, b);
            df[r - 1] = csubf(a, b);
            out0 = caddf(out0, sm[r - 1]);
        }
        xr[0] = out0;
#pragma unroll
        for (int q = 1; q <= H; ++q) {
            float2 A = v0, Bq = make_float2(0.f, 0.f);
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                const int e = (q * r) % R;
                const float wc = e <= H ? wr[e].x : wr[R - e].x;
                const float ws = e <= H ? wr[e].y : -wr[R - e].y;
                A.x = fmaf(wc, sm[r - 1].x, A.x);
                A.y = fmaf(wc, sm[r - 1].y, A.y);
                Bq.x = fmaf(ws, df[r - 1].x, Bq.x);
                Bq.y = fmaf(ws, df[r - 1].y, Bq.y);
            }
            xr[q * h] = make_float2(A.x - Bq.y, A.y + Bq.x);         // A + i B
            xr[(R - q) * h] = make_float2(A.x + Bq.y, A.y - Bq.x);   // A - i B
        }
    }
}

// radix-4 / radix-2 butterflies of a decimation-in-time stage on inputs v (twiddled)
template <bool INV>
__device__ __forceinline__ void dft4(float2 (&v)[4])
{
    const float2 s02 = caddf(v[0], v[2]), d02 = csubf(v[0], v[2]);
    const float2 s13 = caddf(v[1], v[3]), d13 = csubf(v[1], v[3]);
    const float2 rot = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
    v[0] = caddf(s02, s13);
    v[1] = caddf(d02, rot);
    v[2] = csubf(s02, s13);
    v[3] = csubf(d02, rot);
}

template <bool INV>
__device__ void dit_f32(float2 *x, const float2 *__restrict__ tw, const RadixPlanArg &rp, int nr, int st_end)
{
    const int n = rp.n;
    for (int st = rp.nstages - 1; st >= st_end; --st) {
        int Nb = n;
        for (int s2 = 0; s2 < st; ++s2) Nb /= rp.radix[s2];
        const int R = rp.radix[st];
        if (R == 3) {
            dit_stage_small<3, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 5) {
            dit_stage_small<5, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 7) {
            dit_stage_small<7, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 11) {
            dit_stage_small<11, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else if (R == 13) {
            dit_stage_small<13, INV>(x, tw, tw + rp.tw_off[st], n, Nb, nr);
        } else {
            const int h = Nb / R, nbf = n / R;
            const float2 *twS = tw + rp.tw_off[st];
            const Recip rn = recip(nbf), rh = recip(h);
            for (int t = threadIdx.x; t < nbf * nr; t += blockDim.x) {
                const int ring = rdiv(t, rn), i = t - ring * nbf;
                const int blk = rdiv(i, rh), k = i - blk * h;
                float2 *xr = x + ring * n + blk * Nb + k;
                if (R == 4) {
                    float2 v[4] = {xr[0], cmulf(xr[h], twf<INV>(twS, h + k)), cmulf(xr[2 * h], twf<INV>(twS, 2 * h + k)),
                                   cmulf(xr[3 * h], twf<INV>(twS, 3 * h + k))};
                    dft4<INV>(v);
#pragma unroll
                    for (int q = 0; q < 4; ++q) xr[q * h] = v[q];
                } else {
                    const float2 v0 = xr[0], v1 = cmulf(xr[h], twf<INV>(twS, h + k));
                    xr[0] = caddf(v0, v1);
                    xr[h] = csubf(v0, v1);
                }
            }
        }
        __syncthreads();
    }
}

// S_0^T (radix R1 = 4 or 2, block length n, h = n / R1) from shared memory to sink.store:
// butterfly k of ring r writes the natural-order points k + q h, so across a warp every
// store covers consecutive positions.
template <int R1, bool INV, typename Sink>
__device__ void last_stage_global(const float2 *x, const float2 *__restrict__ tw, int n, int nr, const Sink &sink)
{
    const int h = n / R1;
    const Recip rh = recip(h);
    for (int t = threadIdx.x; t < h * nr; t += kFftThreads) {
        const int ring = rdiv(t, rh), k = t - ring * h;
        const float2 *xr = x + ring * n + k;
        const auto rw = sink.row(ring);
        if constexpr (R1 == 4) {
            float2 v[4] = {xr[0], cmulf(xr[h], twf<INV>(tw, k)), cmulf(xr[2 * h], twf<INV>(tw, 2 * k)),
                           cmulf(xr[3 * h], twf<INV>(tw, 3 * k))};
            dft4<INV>(v);
#pragma unroll
            for (int q = 0; q < 4; ++q) sink.store(rw, k + q * h, v[q]);
        } else {
            const float2 v0 = xr[0], v1 = cmulf(xr[h], twf<INV>(tw, k));
            sink.store(rw, k, caddf(v0, v1));
            sink.store(rw, k + h, csubf(v0, v1));
        }
    }
}

template <bool INV, typename Sink>
__device__ __forceinline__ void last_stage_global(const float2 *x, const float2 *__restrict__ tw,
                                                  const RadixPlanArg &rp, int nr, const Sink &sink)
{
    if (rp.radix[0] == 4)
        last_stage_global<4, INV>(x, tw, rp.n, nr, sink);
    else
        last_stage_global<2, INV>(x, tw, rp.n, nr, sink);
}

// Full transform of nr rings, natural order in and out, by the factorisation
//   radix-16 at block length n, [radix-16 at n/16,] radix-2^r blocks (dif_last),
// with the first radix-16 stage fed straight from global memory: src.row(r) locates ring r
// and src.load(row, i) returns its point i.  tw: w_n^i (i < n), then the two radix-16 stages'
// twiddles in [q][k] order (n and n / 16 entries), so that a warp reads them contiguously.  Each thread keeps the 16 inputs of two
// butterflies in registers (32 independent loads in flight; across a warp every load covers
// consecutive addresses), so the input needs no pass through shared memory.
template <int LOG2N, bool INV, typename Src>
__device__ void fft_p2_from_global(float2 *x, const float2 *__restrict__ tw, int nr, const Src &src)
{
    constexpr int n = 1 << LOG2N, n16 = LOG2N / 4, rem = LOG2N % 4, R = 16, h = n / R;
    constexpr int nfull = rem ? n16 : n16 - 1;
    static_assert(nfull >= 1 && nfull <= 2, "a first radix-16 stage is required");
    constexpr int kPer = 2;
    for (int t0 = threadIdx.x; t0 < h * nr; t0 += kPer * kFftThreads) {
        float2 v[kPer][R];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int t = t0 + u * kFftThreads;
            if (t < h * nr) {
                const auto rw = src.row(t >> (LOG2N - 4));
                const int k = t & (h - 1);
#pragma unroll
                for (int q = 0; q < R; ++q) v[u][q] = src.load(rw, k + q * h);
            }
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int t = t0 + u * kFftThreads;
            if (t < h * nr) {
                const int ring = t >> (LOG2N - 4), k = t & (h - 1);
                dft_reg<R, INV>(v[u]);
                const int base = ring * n + k;
                x[padi(base)] = v[u][0];
#pragma unroll
                for (int q = 1; q < R; ++q)
                    x[padi(base + q * h)] = cmulf(v[u][bitrev(q, 4)], twf<INV>(tw + n, q * h + k));
            }
        }
    }
    __syncthreads();
    if constexpr (nfull >= 2) dif_stage16<LOG2N, n / 16, INV, true>(x, tw + n + n, nr);
    dif_last<LOG2N, (rem ? (1 << rem) : 16), INV>(x, nr);
}

// The forward DFT's B-operand records (64 bytes per order: parity x 8 floats) are staged per
// warp in shared memory: the records of a warp's 32 consecutive orders are 2 KB of
// consecutive bytes in global memory, which a direct per-thread store would touch at a
// 64-byte stride.  One lane hands the staged block to
// a bulk asynchronous copy (shared -> global), so the copy takes no load/store-unit
// instructions; before the warp stages its next records it waits until the copy has read
// the staging buffer.
constexpr int kRecUint4 = 4;                               // 16-byte chunks per record
constexpr int kStageBytes = (kFftThreads / 32) * 32 * kRecUint4 * 16;   // 16 KB

// 8 floats of one parity as two 16-byte chunks of a record
__device__ __forceinline__ void pack_row_f32(const float (&v)[8], uint4 (&out)[2])
{
    out[0] = make_uint4(__float_as_uint(v[0]), __float_as_uint(v[1]), __float_as_uint(v[2]), __float_as_uint(v[3]));
    out[1] = make_uint4(__float_as_uint(v[4]), __float_as_uint(v[5]), __float_as_uint(v[6]), __float_as_uint(v[7]));
}

__device__ __forceinline__ void bulk_wait_read()
{
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

// stage -> global: nrec records (16-byte aligned addresses, 64 nrec bytes)
__device__ __forceinline__ void flush_records(unsigned char *__restrict__ dst, const uint4 *stg, int nrec, int lane)
{
    // the generic-proxy writes of the staging buffer become visible to the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (lane == 0 && nrec > 0) {
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                     "r"((uint32_t)__cvta_generic_to_shared(stg)), "r"(nrec * kRecUint4 * 16)
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
}

// before the staging buffer is written again (and before the block exits)
__device__ __forceinline__ void staging_free(int lane)
{
    if (lane == 0) bulk_wait_read();
    __syncwarp();
}

// Records of the orders mu0 + lane (valid lanes; nrec of them from mu0 on) at dst = the
// record of mu0: staged per warp and handed to one bulk copy (LOG2N >= 0), or (LOG2N < 0)
// stored from registers, two 32-byte stores (a whole sector each) per lane.
__device__ __forceinline__ void st_v8(unsigned char *p, const uint4 (&v)[2])
{
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(v[0].x), "r"(v[0].y),
                 "r"(v[0].z), "r"(v[0].w), "r"(v[1].x), "r"(v[1].y), "r"(v[1].z), "r"(v[1].w)
                 : "memory");
}

template <int LOG2N>
__device__ __forceinline__ void put_records(unsigned char *__restrict__ dst, uint4 *stg, int lane, bool valid,
                                            int nrec, const uint4 (&rec_p)[2], const uint4 (&rec_m)[2])
{
    if constexpr (LOG2N < 0) {
        if (valid) {
            st_v8(dst + (size_t)lane * 64, rec_p);
            st_v8(dst + (size_t)lane * 64 + 32, rec_m);
        }
    } else {
        staging_free(lane);                          // the previous round's copy has read it
        if (valid) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                stg[lane * kRecUint4 + q] = rec_p[q];
                stg[lane * kRecUint4 + 2 + q] = rec_m[q];
            }
        }
        flush_records(dst, stg, nrec, lane);
    }
}

// One 32-byte load (a whole sector per lane) through the read-only path; p 32-byte aligned.
__device__ __forceinline__ void ldg_v8(const float4 *p, float4 &a, float4 &b)
{
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
                 : "l"(p));
}

constexpr int kInvOrders = 2;    // orders per thread whose inverse-DFT inputs are loaded at once
                                 // (4 measured slower at n = 2048 and spill at 3 blocks per SM)

// bytes of the DFT buffer of 4 rings of n points (padded for the power-of-two engine)
template <int LOG2N>
__host__ __device__ constexpr int fft_smem_bytes(int n)
{
    return (LOG2N > 0 ? 4 * n + 4 * n / 16 : 4 * n) * 8;
}

// Blocks per SM the DFT kernels are compiled for.  At 3 (85 registers) the n = 2048
// instantiations spill about 128 bytes per thread in the first radix-16 stage; they get
// the 111 registers they need at 2 (inverse DFT at L = 1023: 1.05 -> 0.79 ms), and the
// forward kernel's 24 KB record staging allows only 2 of them per SM there anyway.  The
// generic lengths (LOG2N = 0) hold radix-13 butterflies and their roots in registers.
template <int LOG2N>
__host__ __device__ constexpr int fft_blocks_per_sm() { return LOG2N == 12 ? 1 : (LOG2N == 11 || LOG2N == 0) ? 2 : 3; }
// LOG2N: 6..12 the power-of-two engine at n = 2^LOG2N; 0 the generic stages with Bluestein
// stages for primes from 17 up (record staging after the DFT); -1 the generic stages with
// radices <= 13 only, compiled for three blocks per SM: the four rings (64 KB at n = 2002)
// are then the whole shared-memory block, the forward kernel storing its records straight
// from registers (put_records).

// Inverse-side engine: the transpose of fft_p2_from_global's factorisation (the DFT matrix is
// symmetric, so the stages taken in reverse order, each transposed, give the same
// transform).  dit_first reads the natural-order points nibble_reverse(blk) + q n / RL and
// writes block blk's RL outputs consecutively; each radix-16 stage multiplies its inputs
// by the twiddles before the butterfly; the last stage (block length n) produces the
// outputs in natural order, thread k holding points k + q n / 16, and hands them to
// sink.store(ring, position, value) instead of shared memory: across a warp each store
// covers consecutive positions.
template <int LOG2N, int RL, bool INV>
__device__ __forceinline__ void dit_first(float2 *x, int nr)
{
    constexpr int n = 1 << LOG2N, LB = Log2c<RL>::v;
    constexpr int nblk = n / RL, ndig = (LOG2N - LB) / 4;
    static_assert(nblk <= kFftThreads && (LOG2N - LB) % 4 == 0, "unsupported length");
    constexpr int rings_per_round = kFftThreads / nblk;
    const int t = threadIdx.x;
    for (int r0 = 0; r0 < nr; r0 += rings_per_round) {
        const int ring = r0 + t / nblk, blk = t & (nblk - 1);
        const bool act = t < nblk * rings_per_round && ring < nr;
        float2 v[RL];
        if (act) {
            int m0 = 0;
#pragma unroll
            for (int d = 0; d < ndig; ++d) m0 |= ((blk >> (4 * d)) & 15) << (4 * (ndig - 1 - d));
#pragma unroll
            for (int q = 0; q < RL; ++q) v[q] = x[padi(ring * n + m0 + q * nblk)];
            dft_reg<RL, INV>(v);
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int q = 0; q < RL; ++q) x[padi(ring * n + blk * RL + q)] = v[bitrev(q, LB)];
        }
        __syncthreads();
    }
}

// transposed radix-16 stage at block length NB (twiddles, then butterfly), in place; tw is
// the stage's [q][k] table
template <int LOG2N, int NB, bool INV>
__device__ __forceinline__ void dit_stage16(float2 *x, const float2 *__restrict__ tw, int nr)
{
    constexpr int n = 1 << LOG2N, R = 16;
    constexpr int h = NB / R, nbf = n / R;
    for (int t = threadIdx.x; t < nbf * nr; t += kFftThreads) {
        const int ring = t >> (LOG2N - 4);
        const int i = t & (nbf - 1);
        const int k = i & (h - 1);
        const int base = ring * n + (i - k) * R + k;
        float2 v[R];
        v[0] = x[padi(base)];
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmulf(x[padi(base + q * h)], twf<INV>(tw, q * h + k));
        dft_reg<R, INV>(v);
#pragma unroll
        for (int q = 0; q < R; ++q) x[padi(base + q * h)] = v[bitrev(q, 4)];
    }
    __syncthreads();
}

// full transform of nr rings held in natural order in shared memory, outputs to sink (tw as
// for fft_p2_from_global)
template <int LOG2N, bool INV, typename Sink>
__device__ void fft_p2_to_global(float2 *x, const float2 *__restrict__ tw, int nr, const Sink &sink)
{
    constexpr int n = 1 << LOG2N, n16 = LOG2N / 4, rem = LOG2N % 4, R = 16, h = n / R;
    constexpr int nfull = rem ? n16 : n16 - 1;
    static_assert(nfull >= 1 && nfull <= 2, "a radix-16 stage of block length n is required");
    dit_first<LOG2N, (rem ? (1 << rem) : 16), INV>(x, nr);
    if constexpr (nfull >= 2) dit_stage16<LOG2N, n / 16, INV>(x, tw + n + n, nr);
    for (int t = threadIdx.x; t < h * nr; t += kFftThreads) {
        const int ring = t >> (LOG2N - 4), k = t & (h - 1);
        float2 v[R];
        v[0] = x[padi(ring * n + k)];
#pragma unroll
        for (int q = 1; q < R; ++q) v[q] = cmulf(x[padi(ring * n + k + q * h)], twf<INV>(tw + n, q * h + k));
        dft_reg<R, INV>(v);
        const auto rw = sink.row(ring);
#pragma unroll
        for (int q = 0; q < R; ++q) sink.store(rw, k + q * h, v[bitrev(q, 4)]);
    }
}

// ring sources of the forward kernels: complex rows (T_th, T_ph of one field), or the
// packed z = T_th + i T_ph of a real field (zero for the missing second field of a pair)
struct ComplexRows {
    const float2 *th, *ph;
    size_t fb;
    int j, jm, n;
    __device__ __forceinline__ const float2 *row(int ring) const
    {
        return ((ring & 1) ? ph : th) + fb + (size_t)(ring < 2 ? j : jm) * n;
    }
    __device__ __forceinline__ float2 load(const float2 *r, int i) const { return __ldg(r + i); }
};
struct RealPairRows {
    const float *th, *ph;
    const long long *toff;
    int q, B, nlat, j, jm, n;
    struct Row { const float *th, *ph; bool ok; };
    __device__ __forceinline__ Row row(int ring) const
    {
        const int bf = 2 * q + (ring & 1);
        if (bf >= B) return {th, ph, false};
        const size_t off = (toff ? (size_t)toff[bf] : (size_t)bf * nlat * n) + (size_t)(ring < 2 ? j : jm) * n;
        return {th + off, ph + off, true};
    }
    __device__ __forceinline__ float2 load(const Row &r, int i) const
    {
        return r.ok ? make_float2(__ldg(r.th + i), __ldg(r.ph + i)) : make_float2(0.f, 0.f);
    }
};

// Generic lengths: the first decimation-in-frequency stage fed straight from global memory
// through src (as fft_p2_from_global does for powers of two).  n = 2(L+1) is even, so the
// factorisation (4s first, then a 2) always starts with radix R1 = 4 or 2; block length n,
// h = n / R1, butterfly k of ring r takes the points k + q h and writes them back scaled
// by w_n^{q k}.  kPer butterflies per thread have their loads in flight together.  Returns
// after a barrier; dif_f32 continues from stage 1.
template <int R1, bool INV, typename Src>
__device__ void first_stage_global(float2 *x, const float2 *__restrict__ tw, int n, int nr, const Src &src)
{
    constexpr int kPer = 1;      // measured: 2 or 4 butterflies per thread spill at 80 registers and run slower
    const int h = n / R1;
    const Recip rh = recip(h);
    for (int t0 = threadIdx.x; t0 < h * nr; t0 += kPer * kFftThreads) {
        float2 v[kPer][R1];
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int t = t0 + u * kFftThreads;
            if (t < h * nr) {
                const int ring = rdiv(t, rh), k = t - ring * h;
                const auto rw = src.row(ring);
#pragma unroll
                for (int q = 0; q < R1; ++q) v[u][q] = src.load(rw, k + q * h);
            }
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u) {
            const int t = t0 + u * kFftThreads;
            if (t < h * nr) {
                const int ring = rdiv(t, rh), k = t - ring * h;
                float2 *xr = x + ring * n + k;
                if constexpr (R1 == 4) {
                    const float2 s02 = caddf(v[u][0], v[u][2]), d02 = csubf(v[u][0], v[u][2]);
                    const float2 s13 = caddf(v[u][1], v[u][3]), d13 = csubf(v[u][1], v[u][3]);
                    const float2 rot = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
                    xr[0] = caddf(s02, s13);
                    xr[h] = cmulf(caddf(d02, rot), twf<INV>(tw, k));
                    xr[2 * h] = cmulf(csubf(s02, s13), twf<INV>(tw, 2 * k));
                    xr[3 * h] = cmulf(csubf(d02, rot), twf<INV>(tw, 3 * k));
                } else {
                    xr[0] = caddf(v[u][0], v[u][1]);
                    xr[h] = cmulf(csubf(v[u][0], v[u][1]), twf<INV>(tw, k));
                }
            }
        }
    }
    __syncthreads();
}

template <bool INV, typename Src>
__device__ __forceinline__ void first_stage_global(float2 *x, const float2 *__restrict__ tw, const RadixPlanArg &rp,
                                                   int nr, const Src &src)
{
    if (rp.radix[0] == 4)
        first_stage_global<4, INV>(x, tw, rp.n, nr, src);
    else
        first_stage_global<2, INV>(x, tw, rp.n, nr, src);
}

// ring sinks of the inverse kernels, the counterparts of the sources above
struct ComplexRowsOut {
    float2 *th, *ph;
    size_t fb;
    int j, jm, n;
    __device__ __forceinline__ float2 *row(int ring) const
    {
        return ((ring & 1) ? ph : th) + fb + (size_t)(ring < 2 ? j : jm) * n;
    }
    __device__ __forceinline__ void store(float2 *r, int i, float2 v) const { r[i] = v; }
};
struct RealPairRowsOut {
    float *th, *ph;
    const long long *toff;
    int q, B, nlat, j, jm, n;
    struct Row { float *th, *ph; bool ok; };
    __device__ __forceinline__ Row row(int ring) const
    {
        const int bf = 2 * q + (ring & 1);
        if (bf >= B) return {th, ph, false};
        const size_t off = (toff ? (size_t)toff[bf] : (size_t)bf * nlat * n) + (size_t)(ring < 2 ? j : jm) * n;
        return {th + off, ph + off, true};
    }
    __device__ __forceinline__ void store(const Row &r, int i, float2 v) const
    {
        if (r.ok) {
            r.th[i] = v.x;
            r.ph[i] = v.y;
        }
    }
};

// grid: B * J CTAs (field-major); shared: 4 * n float2 (+ padding for LOG2N > 0) and the
// record staging.  LOG2N > 0 selects the power-of-two engine, 0 the generic one.
template <int LOG2N>
__global__ void __launch_bounds__(kFftThreads, fft_blocks_per_sm<LOG2N>()) k_fft_fwd_bf16(
    const float2 *__restrict__ Tth, const float2 *__restrict__ Tph, unsigned char *__restrict__ Fb,
    RadixPlanArg rp, const float2 *__restrict__ tw, const int *__restrict__ perm,
    const float *__restrict__ omega, int L, int nlat, int J, int has_eq, int nf,
    const long long *__restrict__ toff)
{
    extern __shared__ float4 sm_f4[];
    float2 *buf = reinterpret_cast<float2 *>(sm_f4);
    const int n = rp.n;
    const int b = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;    // rings: (th, j), (ph, j), (th, j'), (ph, j')
    const int jm = nlat - 1 - j;
    const size_t fb = toff ? (size_t)toff[b] : (size_t)b * nlat * n;   // field b's plane
    if constexpr (LOG2N > 0) {
        fft_p2_from_global<LOG2N, false>(buf, tw, nr, ComplexRows{Tth, Tph, fb, j, jm, n});
    }
    if constexpr (LOG2N <= 0) {
        // generic lengths: the first stage reads the rings, the others run in shared memory
        first_stage_global<false>(buf, tw, rp, nr, ComplexRows{Tth, Tph, fb, j, jm, n});
        dif_f32<false, LOG2N == 0>(buf, tw, rp, nr,
                                   reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(sm_f4) +
                                                              fft_smem_bytes<LOG2N>(n)),
                                   1);
    }
    const float w = omega[j];
    // Fb[j/8][field][j%8][mu][parity][8 floats]: this CTA's block is contiguous over mu (the
    // tensor-core GEMM splits the values into bf16 pieces as it loads them)
    unsigned char *dst_base = Fb + ((((size_t)(j / 8) * nf + b) * 8 + (j % 8)) * (L + 1)) * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint4 *stg = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(sm_f4) + fft_smem_bytes<LOG2N>(n)) +
                 warp * 32 * kRecUint4;
    for (int mu0 = warp * 32; mu0 <= L; mu0 += blockDim.x) {
        const int mu = mu0 + lane;
        uint4 rec_p[2], rec_m[2];
        if (mu <= L) {
            float vp[8], vm[8];
            // n % 8 = c*4 + s*2 + im ; s = 0: +mu (bin mu), s = 1: -mu (bin n - mu, or 0 at mu = 0)
#pragma unroll
            for (int sgn = 0; sgn < 2; ++sgn) {
                const int bin = (sgn == 0 || mu == 0) ? mu : n - mu;
                const int pos = LOG2N > 0 ? bin : __ldg(perm + bin);
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i0 = c * n + pos, i1 = (2 + c) * n + pos;
                    const float2 a = buf[LOG2N > 0 ? padi(i0) : i0];
                    const float2 z = eq ? make_float2(0.f, 0.f) : buf[LOG2N > 0 ? padi(i1) : i1];
                    const int base = c * 4 + sgn * 2;
                    vp[base] = w * (a.x + z.x);
                    vp[base + 1] = w * (a.y + z.y);
                    vm[base] = eq ? 0.f : w * (a.x - z.x);
                    vm[base + 1] = eq ? 0.f : w * (a.y - z.y);
                }
            }
            pack_row_f32(vp, rec_p);
            pack_row_f32(vm, rec_m);
        }
        const int nrec = L + 1 - mu0 < 32 ? L + 1 - mu0 : 32;
        put_records<LOG2N>(dst_base + (size_t)mu0 * 64, stg, lane, mu <= L, nrec, rec_p, rec_m);
    }
    if (LOG2N >= 0) staging_free(lane);              // shared memory stays until the copies read it
}

// ---------------------------------------------------------------------------
// n = 2048 (L = 1023), complex fields: the transform above with the four rings brought
// into shared memory by bulk asynchronous copies, so that no registers wait on loads in
// flight and a CTA's copy proceeds while the other CTAs on the SM compute.  The copies
// write whole rows, so the 64 KB ring buffer carries no padding: the first stage writes
// point i of a ring to position swz(i) instead (its low three bits XORed with bits 4-6,
// bit 3 with bit 7), which leaves every later access of the factorisation -- radix 16 at
// block length 128, radix 8 at 8, the digit-reversed natural-order write, the bins read
// for the records -- free of bank conflicts (enumerated on the host: test_dft_swizzle.py).  swz
// changes only the low four bits, so the first stage's writes stay within the 16-point
// groups its warp has read.  Records leave from registers as two 32-byte stores per order.
// ---------------------------------------------------------------------------
constexpr int kSwN = 2048;
constexpr int kSwSmem = 4 * kSwN * 8 + 16;   // four rings and the copy's barrier
constexpr int kSwBlocksPerSm = 2;

__device__ __forceinline__ int swz(int a) { return a ^ ((a >> 4) & 7) ^ (((a >> 7) & 1) << 3); }

__global__ void __launch_bounds__(kFftThreads, kSwBlocksPerSm) k_fft_fwd_sw(
    const float2 *__restrict__ Tth, const float2 *__restrict__ Tph, unsigned char *__restrict__ Fb,
    const float2 *__restrict__ tw, const float *__restrict__ omega, int L, int nlat, int J, int has_eq, int nf,
    const long long *__restrict__ toff, int *status)
{
    constexpr int n = kSwN;
    extern __shared__ float4 sm_f4[];
    float2 *X = reinterpret_cast<float2 *>(sm_f4);
    uint64_t *bar = reinterpret_cast<uint64_t *>(X + 4 * n);
    const int b = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;    // rings: (th, j), (ph, j), (th, j'), (ph, j')
    const int jm = nlat - 1 - j;
    const size_t fb = toff ? (size_t)toff[b] : (size_t)b * nlat * n;
    if (fb & 1) {                 // a row that does not start on 16 bytes cannot be copied
        if (threadIdx.x == 0) atomicCAS(status, 0, FAVEST_EINVAL);
        return;
    }
    if (threadIdx.x == 0) {
        tc::mbar_init(bar, 1);
        tc::mbar_fence_init();
        tc::mbar_arrive_expect_tx(bar, nr * n * 8);
        for (int r = 0; r < nr; ++r)
            tc::bulk_g2s(X + r * n, ((r & 1) ? Tph : Tth) + fb + (size_t)(r < 2 ? j : jm) * n, n * 8, bar);
    }
    __syncthreads();              // the barrier is initialised before anyone waits on it
    if (!tc::mbar_wait(bar, 0)) atomicCAS(status, 0, FAVEST_ETIMEOUT);

    // radix 16 at block length n: rows in natural order, outputs to swz positions
    const float2 *twA = tw + n, *twB = tw + 2 * n;
    for (int t = threadIdx.x; t < 128 * nr; t += kFftThreads) {    // whole warps per ring
        const int k = t & 127;
        float2 *xr = X + (t >> 7) * n;
        float2 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = xr[k + 128 * q];
        dft_reg<16, false>(v);
        __syncwarp();             // the warp's reads are done before its writes
        xr[swz(k)] = v[0];
#pragma unroll
        for (int q = 1; q < 16; ++q) xr[swz(k + 128 * q)] = cmulf(v[bitrev(q, 4)], twf<false>(twA, q * 128 + k));
    }
    __syncthreads();
    // radix 16 at block length 128
    for (int t = threadIdx.x; t < 128 * nr; t += kFftThreads) {
        const int i = t & 127, k = i & 7, base = (i >> 3) * 128 + k;
        float2 *xr = X + (t >> 7) * n;
        float2 v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = xr[swz(base + 8 * q)];
        dft_reg<16, false>(v);
        xr[swz(base)] = v[0];
#pragma unroll
        for (int q = 1; q < 16; ++q) xr[swz(base + 8 * q)] = cmulf(v[bitrev(q, 4)], twf<false>(twB, q * 8 + k));
    }
    __syncthreads();
    // radix 8 on blocks of 8 consecutive points, outputs to natural order (frequency
    // nibble_reverse(blk) + 256 q); two rings per round, two blocks per thread
    for (int r0 = 0; r0 < nr; r0 += 2) {
        float2 v[2][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int idx = threadIdx.x + u * kFftThreads, blk = idx & 255;
            const float2 *xr = X + (r0 + (idx >> 8)) * n;
#pragma unroll
            for (int q = 0; q < 8; ++q) v[u][q] = xr[swz(blk * 8 + q)];
            dft_reg<8, false>(v[u]);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int idx = threadIdx.x + u * kFftThreads, blk = idx & 255;
            float2 *xr = X + (r0 + (idx >> 8)) * n;
            const int m0 = ((blk & 15) << 4) | (blk >> 4);
#pragma unroll
            for (int q = 0; q < 8; ++q) xr[swz(m0 + 256 * q)] = v[u][bitrev(q, 3)];
        }
    }
    __syncthreads();

    // weighted fold and records, as in k_fft_fwd_bf16
    const float w = omega[j];
    unsigned char *dst_base = Fb + ((((size_t)(j / 8) * nf + b) * 8 + (j % 8)) * (L + 1)) * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int mu0 = warp * 32; mu0 <= L; mu0 += blockDim.x) {
        const int mu = mu0 + lane;
        if (mu > L) continue;
        float vp[8], vm[8];
#pragma unroll
        for (int sgn = 0; sgn < 2; ++sgn) {
            const int bin = swz((sgn == 0 || mu == 0) ? mu : n - mu);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const float2 a = X[c * n + bin];
                const float2 z = eq ? make_float2(0.f, 0.f) : X[(2 + c) * n + bin];
                const int base = c * 4 + sgn * 2;
                vp[base] = w * (a.x + z.x);
                vp[base + 1] = w * (a.y + z.y);
                vm[base] = eq ? 0.f : w * (a.x - z.x);
                vm[base + 1] = eq ? 0.f : w * (a.y - z.y);
            }
        }
        uint4 rec_p[2], rec_m[2];
        pack_row_f32(vp, rec_p);
        pack_row_f32(vm, rec_m);
        st_v8(dst_base + (size_t)mu * 64, rec_p);
        st_v8(dst_base + (size_t)mu * 64 + 32, rec_m);
    }
}

// The inverse kernels' sum records: the 32-byte records of latitude j (parities 0 and 1)
// for every order mu, from S32[group][JP/4][L+1][parity][4][8].  For power-of-two lengths
// they stream through shared memory in TMA boxes of kInvChunk orders ([order][parity][8],
// 16 KB), two buffers deep: the next box is in flight while each thread spreads one order
// of the current one onto its frequency bins.  Other lengths (or a shared-memory block
// not aligned for the TMA) read them with 256-bit loads, kInvOrders orders per thread at
// a time.  put(mu, ev, ov) receives the even- and odd-parity sums of order mu.
constexpr int kInvStageBytes = 2 * kInvChunk * 64 + 16;      // two boxes and their barriers

template <int LOG2N, typename Put>
__device__ __forceinline__ void stream_records(const float *__restrict__ S32, const CUtensorMap *tmap,
                                               unsigned char *stage, int *status, int grp, int j, int L, int JP,
                                               Put put)
{
    const bool tma = LOG2N > 0 && (__cvta_generic_to_shared(stage) & 127) == 0;   // uniform
    if (tma) {
        uint64_t *bars = reinterpret_cast<uint64_t *>(stage + 2 * kInvChunk * 64);
        const int nch = (L + kInvChunk) / kInvChunk;             // boxes covering orders 0..L
        if (threadIdx.x == 0) {
            tc::mbar_init(&bars[0], 1);
            tc::mbar_init(&bars[1], 1);
            tc::mbar_fence_init();
        }
        __syncthreads();
        auto issue = [&](int c) {
            tc::mbar_arrive_expect_tx(&bars[c & 1], kInvChunk * 64);
            tc::tma_load_5d(stage + (c & 1) * kInvChunk * 64, tmap, 8 * (j & 3), 0, c * kInvChunk, j >> 2, grp,
                            &bars[c & 1]);
        };
        if (threadIdx.x == 0) issue(0);
        for (int c = 0; c < nch; ++c) {
            // box c + 1 refills the buffer that box c - 1 used (released by the barrier below)
            if (threadIdx.x == 0 && c + 1 < nch) issue(c + 1);
            if (!tc::mbar_wait(&bars[c & 1], (c >> 1) & 1)) atomicCAS(status, 0, FAVEST_ETIMEOUT);
            const float4 *rec = reinterpret_cast<const float4 *>(stage + (c & 1) * kInvChunk * 64);
            for (int i = threadIdx.x; i < kInvChunk; i += blockDim.x) {
                const int mu = c * kInvChunk + i;
                if (mu > L) break;
                const float4 e0 = rec[4 * i], e1 = rec[4 * i + 1], o0 = rec[4 * i + 2], o1 = rec[4 * i + 3];
                const float ev[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
                const float ov[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
                put(mu, ev, ov);
            }
            __syncthreads();
        }
        return;
    }
    for (int mu0 = threadIdx.x; mu0 <= L; mu0 += kInvOrders * blockDim.x) {
        // kInvOrders orders per iteration: their loads are issued before any is used
        float4 ld[kInvOrders][4];
#pragma unroll
        for (int h = 0; h < kInvOrders; ++h) {
            const int mu = mu0 + h * blockDim.x;
            if (mu <= L) {
                const float4 *e = reinterpret_cast<const float4 *>(
                    S32 + ((((size_t)grp * (JP / 4) + (j >> 2)) * (L + 1) + mu) * 2) * 32 + (j & 3) * 8);
                const float4 *o = e + 8;                 // parity 1: the next 4 x 8 floats
                ldg_v8(e, ld[h][0], ld[h][1]);
                ldg_v8(o, ld[h][2], ld[h][3]);
            }
        }
#pragma unroll
        for (int h = 0; h < kInvOrders; ++h) {
            const int mu = mu0 + h * blockDim.x;
            if (mu > L) break;
            const float ev[8] = {ld[h][0].x, ld[h][0].y, ld[h][0].z, ld[h][0].w,
                                 ld[h][1].x, ld[h][1].y, ld[h][1].z, ld[h][1].w};
            const float ov[8] = {ld[h][2].x, ld[h][2].y, ld[h][2].z, ld[h][2].w,
                                 ld[h][3].x, ld[h][3].y, ld[h][3].z, ld[h][3].w};
            put(mu, ev, ov);
        }
    }
    __syncthreads();
}

// The even/odd sums of ring j, order mu: the polar patch's (its own buffer
// polS[group][pol_jc][pol_muc][parity][8], written next to the GEMM) for the pairs it
// recomputed -- rings j < pol_jc, orders 1 <= mu < pol_muc whose tile of 32 starts below
// lim, the bound of the last ring of j's pair -- else the GEMM's, as streamed.
__device__ __forceinline__ void polar_or_gemm(const float *__restrict__ polS, int lim, int muc, size_t base, int mu,
                                              const float (&ev_in)[8], const float (&ov_in)[8], float (&ev)[8],
                                              float (&ov)[8])
{
    if (polS && mu >= 1 && mu < muc && (mu & ~31) < lim) {
        const float4 *src = reinterpret_cast<const float4 *>(polS + (base + mu) * 16);
        const float4 v0 = __ldg(src), v1 = __ldg(src + 1), v2 = __ldg(src + 2), v3 = __ldg(src + 3);
        ev[0] = v0.x; ev[1] = v0.y; ev[2] = v0.z; ev[3] = v0.w;
        ev[4] = v1.x; ev[5] = v1.y; ev[6] = v1.z; ev[7] = v1.w;
        ov[0] = v2.x; ov[1] = v2.y; ov[2] = v2.z; ov[3] = v2.w;
        ov[4] = v3.x; ov[5] = v3.y; ov[6] = v3.z; ov[7] = v3.w;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            ev[k] = ev_in[k];
            ov[k] = ov_in[k];
        }
    }
}

// grid: B * J; S32 = [field][JP/4][L+1][parity][4][8] fp32; shared 4 * n float2 (+ padding)
// and, for power-of-two n, the record stream's two boxes
template <int LOG2N>
__global__ void __launch_bounds__(kFftThreads, fft_blocks_per_sm<LOG2N>()) k_fft_inv_bf16(
    const float *__restrict__ S32, const __grid_constant__ CUtensorMap tmap_s, float2 *__restrict__ Tth,
    float2 *__restrict__ Tph, RadixPlanArg rp, const float2 *__restrict__ tw, const int *__restrict__ perm,
    const float2 *__restrict__ isc, int L, int nlat, int J, int has_eq, int JP, const long long *__restrict__ toff,
    int *status, const float *__restrict__ polS, const int *__restrict__ plim, int pol_jc, int pol_muc)
{
    extern __shared__ float4 sm_i4[];
    float2 *buf = reinterpret_cast<float2 *>(sm_i4);
    const int n = rp.n;
    const int b = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;
    // 1/sin(theta_j), times the point weight of rings j and nlat-1-j (equal) for the
    // weighted adjoint (isc[j] = (scale, weight))
    const float2 sc2 = __ldg(isc + j);
    const float is = sc2.x, w0 = sc2.y;
    // every bin but n/2 is written below (n = 2(L+1): orders 0..L at bins mu and n - mu);
    // the decimation-in-time variant (LOG2N < 0) takes bin m at position perm[m]
    if (threadIdx.x < nr) {
        const int i = threadIdx.x * n + (LOG2N < 0 ? __ldg(perm + n / 2) : n / 2);
        buf[LOG2N > 0 ? padi(i) : i] = make_float2(0.f, 0.f);
    }
    const bool polar = j < pol_jc;
    const int plim_j = polar ? __ldg(plim + ((j | 1) < pol_jc ? (j | 1) : pol_jc - 1)) : 0;
    const size_t pbase = ((size_t)b * (polar ? pol_jc : 0) + j) * pol_muc;
    auto put = [&](int mu, const float (&ev_in)[8], const float (&ov_in)[8]) {
        float ev[8], ov[8];
        polar_or_gemm(polar ? polS : nullptr, plim_j, pol_muc, pbase, mu, ev_in, ov_in, ev, ov);
        // order 0 arrives already divided by sin(theta) (synthesised on lambda^1)
        const float sc = mu == 0 ? w0 : is;
        const int pp = LOG2N < 0 ? __ldg(perm + mu) : mu;
        const int pm = LOG2N < 0 ? (mu == 0 ? 0 : __ldg(perm + n - mu)) : n - mu;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int sgn = 0; sgn < 2; ++sgn) {
                if (mu == 0 && sgn == 1) continue;
                const int bin = sgn ? pm : pp;
                const int k = c * 4 + sgn * 2;
                const int i0 = c * n + bin, i1 = (2 + c) * n + bin;
                buf[LOG2N > 0 ? padi(i0) : i0] = make_float2((ev[k] + ov[k]) * sc, (ev[k + 1] + ov[k + 1]) * sc);
                if (!eq)
                    buf[LOG2N > 0 ? padi(i1) : i1] = make_float2((ev[k] - ov[k]) * sc, (ev[k + 1] - ov[k + 1]) * sc);
            }
        }
    };
    stream_records<LOG2N>(S32, &tmap_s, reinterpret_cast<unsigned char *>(sm_i4) + fft_smem_bytes<LOG2N>(n), status, b,
                          j, L, JP, put);
    const int jm = nlat - 1 - j;
    const size_t fb = toff ? (size_t)toff[b] : (size_t)b * nlat * n;
    if constexpr (LOG2N > 0) {
        fft_p2_to_global<LOG2N, true>(buf, tw, nr, ComplexRowsOut{Tth, Tph, fb, j, jm, n});
    } else if constexpr (LOG2N < 0) {
        dit_f32<true>(buf, tw, rp, nr, 1);
        last_stage_global<true>(buf, tw, rp, nr, ComplexRowsOut{Tth, Tph, fb, j, jm, n});
    } else {
        dif_f32<true, LOG2N == 0>(buf, tw, rp, nr,
                      reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(sm_i4) + fft_smem_bytes<LOG2N>(n)));
        const int n2 = n / 2;
        const Recip rn2 = recip(n2);
        for (int idx = threadIdx.x; idx < nr * n2; idx += blockDim.x) {
            const int ring = rdiv(idx, rn2), k2 = idx - ring * n2;
            const float2 v0 = buf[ring * n + __ldg(perm + 2 * k2)];
            const float2 v1 = buf[ring * n + __ldg(perm + 2 * k2 + 1)];
            float2 *dst = (ring & 1) ? Tph : Tth;
            const int jj = (ring < 2) ? j : jm;
            reinterpret_cast<float4 *>(dst + fb + (size_t)jj * n)[k2] = make_float4(v0.x, v0.y, v1.x, v1.y);
        }
    }
}

// ---------------------------------------------------------------------------
// n = 2048 (L = 1023), complex fields, inverse: the transpose of k_fft_fwd_sw.  The sum
// records stream through shared memory in TMA boxes as in k_fft_inv_bf16, but a thread
// takes one component (theta or phi) of one order: its two 16-byte chunks (even and odd
// parity) are read in an order that alternates every two orders, which makes each
// quarter-warp's loads cover all 32 banks (the one-order-per-thread reads of 64-byte
// records met four-way conflicts).  The bins go to the swizzled layout of k_fft_fwd_sw,
// with ring r shifted by 8 r complexes so that the theta and phi bins of the
// same orders fall on different banks; the transposed stages then read and write without
// conflicts, and the last stage stores rows from registers.
// ---------------------------------------------------------------------------
constexpr int kSwRingsFloat2 = 4 * kSwN + 24;                     // ring r shifted by 8 r
constexpr int kSwInvSmem = kSwRingsFloat2 * 8 + 128 + 2 * kInvChunk * 64 + 16;

__device__ __forceinline__ float2 *sw_ring(float2 *X, int r) { return X + r * (kSwN + 8); }

__global__ void __launch_bounds__(kFftThreads, 2) k_fft_inv_sw(
    const __grid_constant__ CUtensorMap tmap_s, float2 *__restrict__ Tth, float2 *__restrict__ Tph,
    const float2 *__restrict__ tw, const float2 *__restrict__ isc, int L, int nlat, int J, int has_eq,
    const long long *__restrict__ toff, int *status, const float *__restrict__ polS,
    const int *__restrict__ plim, int pol_jc, int pol_muc)
{
    constexpr int n = kSwN;
    extern __shared__ float4 sm_i4[];
    float2 *X = reinterpret_cast<float2 *>(sm_i4);
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(X + kSwRingsFloat2);
    unsigned char *stage = reinterpret_cast<unsigned char *>(X + kSwRingsFloat2) + (((s0 + 127) & ~127u) - s0);
    uint64_t *bars = reinterpret_cast<uint64_t *>(stage + 2 * kInvChunk * 64);
    const int b = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;
    const float2 sc2 = __ldg(isc + j);      // 1/sin(theta_j) and the point weight (order 0)
    const float is = sc2.x, w0 = sc2.y;
    if (threadIdx.x < nr) sw_ring(X, threadIdx.x)[swz(n / 2)] = make_float2(0.f, 0.f);   // the unused bin
    const bool polar = j < pol_jc;
    const int plim_j = polar ? __ldg(plim + ((j | 1) < pol_jc ? (j | 1) : pol_jc - 1)) : 0;
    const size_t pbase = ((size_t)b * (polar ? pol_jc : 0) + j) * pol_muc;

    const int nch = (L + kInvChunk) / kInvChunk;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    auto issue = [&](int c) {
        tc::mbar_arrive_expect_tx(&bars[c & 1], kInvChunk * 64);
        tc::tma_load_5d(stage + (c & 1) * kInvChunk * 64, &tmap_s, 8 * (j & 3), 0, c * kInvChunk, j >> 2, b,
                        &bars[c & 1]);
    };
    if (threadIdx.x == 0) issue(0);
    for (int c = 0; c < nch; ++c) {
        if (threadIdx.x == 0 && c + 1 < nch) issue(c + 1);   // refills the buffer box c - 1 used
        if (!tc::mbar_wait(&bars[c & 1], (c >> 1) & 1)) atomicCAS(status, 0, FAVEST_ETIMEOUT);
        const float4 *rec = reinterpret_cast<const float4 *>(stage + (c & 1) * kInvChunk * 64);
        for (int tsk = threadIdx.x; tsk < 2 * kInvChunk; tsk += kFftThreads) {
            const int r = tsk >> 1, comp = tsk & 1, mu = c * kInvChunk + r;
            if (mu > L) break;
            const int p0 = (r >> 1) & 1;                      // which parity is read first
            const float4 u0 = rec[r * 4 + p0 * 2 + comp], u1 = rec[r * 4 + (p0 ^ 1) * 2 + comp];
            float4 e = p0 ? u1 : u0, o = p0 ? u0 : u1;        // even / odd sums, (+mu, -mu)
            if (polar && mu >= 1 && mu < pol_muc && (mu & ~31) < plim_j) {
                const float4 *src = reinterpret_cast<const float4 *>(polS + (pbase + mu) * 16);
                e = __ldg(src + comp);
                o = __ldg(src + 2 + comp);
            }
            const float sc = mu == 0 ? w0 : is;    // order 0 arrives divided by sin(theta)
            float2 *r0 = sw_ring(X, comp), *r1 = sw_ring(X, 2 + comp);
            const int bp = swz(mu);
            r0[bp] = make_float2((e.x + o.x) * sc, (e.y + o.y) * sc);
            if (!eq) r1[bp] = make_float2((e.x - o.x) * sc, (e.y - o.y) * sc);
            if (mu != 0) {
                const int bm = swz(n - mu);
                r0[bm] = make_float2((e.z + o.z) * sc, (e.w + o.w) * sc);
                if (!eq) r1[bm] = make_float2((e.z - o.z) * sc, (e.w - o.w) * sc);
            }
        }
        __syncthreads();
    }

    // radix 8 (transposed last stage of the forward factorisation): natural-order points
    // nibble_reverse(blk) + 256 q to block blk; two rings per round, two blocks per thread
    for (int r0 = 0; r0 < nr; r0 += 2) {
        float2 v[2][8];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int idx = threadIdx.x + u * kFftThreads, blk = idx & 255;
            const float2 *xr = sw_ring(X, r0 + (idx >> 8));
            const int m0 = ((blk & 15) << 4) | (blk >> 4);
#pragma unroll
            for (int q = 0; q < 8; ++q) v[u][q] = xr[swz(m0 + 256 * q)];
            dft_reg<8, true>(v[u]);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int idx = threadIdx.x + u * kFftThreads, blk = idx & 255;
            float2 *xr = sw_ring(X, r0 + (idx >> 8));
#pragma unroll
            for (int q = 0; q < 8; ++q) xr[swz(blk * 8 + q)] = v[u][bitrev(q, 3)];
        }
    }
    __syncthreads();
    // transposed radix 16 at block length 128 (twiddles, then butterfly)
    const float2 *twA = tw + n, *twB = tw + 2 * n;
    for (int t = threadIdx.x; t < 128 * nr; t += kFftThreads) {
        const int i = t & 127, k = i & 7, base = (i >> 3) * 128 + k;
        float2 *xr = sw_ring(X, t >> 7);
        float2 v[16];
        v[0] = xr[swz(base)];
#pragma unroll
        for (int q = 1; q < 16; ++q) v[q] = cmulf(xr[swz(base + 8 * q)], twf<true>(twB, q * 8 + k));
        dft_reg<16, true>(v);
#pragma unroll
        for (int q = 0; q < 16; ++q) xr[swz(base + 8 * q)] = v[bitrev(q, 4)];
    }
    __syncthreads();
    // transposed radix 16 at block length n: natural-order outputs k + 128 q stored as rows
    const int jm = nlat - 1 - j;
    const size_t fb = toff ? (size_t)toff[b] : (size_t)b * nlat * n;
    for (int t = threadIdx.x; t < 128 * nr; t += kFftThreads) {
        const int ring = t >> 7, k = t & 127;
        const float2 *xr = sw_ring(X, ring);
        float2 v[16];
        v[0] = xr[swz(k)];
#pragma unroll
        for (int q = 1; q < 16; ++q) v[q] = cmulf(xr[swz(k + 128 * q)], twf<true>(twA, q * 128 + k));
        dft_reg<16, true>(v);
        float2 *dst = ((ring & 1) ? Tph : Tth) + fb + (size_t)(ring < 2 ? j : jm) * n;
#pragma unroll
        for (int q = 0; q < 16; ++q) dst[k + 128 * q] = v[bitrev(q, 4)];
    }
}

// ---------------------------------------------------------------------------
// Real fields.  A real field's two components are packed into one complex ring
// z = T_th + i T_ph, whose spectrum Z gives both component spectra (T_th, T_ph real):
//   F_th(m) = (Z(m) + conj Z(-m)) / 2,   F_ph(m) = (Z(m) - conj Z(-m)) / (2 i),
// of which only m >= 0 is kept (F(-m) = conj F(m)).  One CTA takes the fields 2q and
// 2q+1 at the folded latitude pair (j, nlat-1-j): four complex rings, the same shared
// memory and transform count as one complex field.  The B-operand record of the pair
// holds columns c*4 + f*2 + (re, im) for component c and field f of the pair, at +mu.
// For power-of-two nphi the first radix-16 stage reads the rows itself (float loads, a warp
// covering 128 consecutive bytes per load); other lengths stage them with float2 loads.
// ---------------------------------------------------------------------------
template <int V>
__device__ __forceinline__ void load_v(const float *p, float (&v)[V])
{
    if constexpr (V == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = t.x; v[1] = t.y;
    }
}

template <int V>
__device__ __forceinline__ void store_v(float *p, const float (&v)[V])
{
    if constexpr (V == 4) *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

// grid: ceil(B / 2) * J CTAs (pair-major); shared as for the complex kernel
template <int LOG2N>
__global__ void __launch_bounds__(kFftThreads, fft_blocks_per_sm<LOG2N>()) k_rfft_fwd_bf16(
    const float *__restrict__ Tth, const float *__restrict__ Tph, unsigned char *__restrict__ Fb,
    RadixPlanArg rp, const float2 *__restrict__ tw, const int *__restrict__ perm,
    const float *__restrict__ omega, int L, int nlat, int J, int has_eq, int nf, int B,
    const long long *__restrict__ toff)
{
    extern __shared__ float4 sm_r4[];
    float2 *buf = reinterpret_cast<float2 *>(sm_r4);
    const int n = rp.n;
    const int q = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;    // rings: (2q, j), (2q+1, j), (2q, j'), (2q+1, j')
    const int jm = nlat - 1 - j;
    if constexpr (LOG2N > 0)
        fft_p2_from_global<LOG2N, false>(buf, tw, nr, RealPairRows{Tth, Tph, toff, q, B, nlat, j, jm, n});
    if constexpr (LOG2N <= 0) {
        // generic lengths: the first stage reads the rings, the others run in shared memory
        first_stage_global<false>(buf, tw, rp, nr, RealPairRows{Tth, Tph, toff, q, B, nlat, j, jm, n});
        dif_f32<false, LOG2N == 0>(buf, tw, rp, nr,
                                   reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(sm_r4) +
                                                              fft_smem_bytes<LOG2N>(n)),
                                   1);
    }
    const float w = 0.5f * omega[j];             // the 1/2 of the component split folded in
    unsigned char *dst_base = Fb + ((((size_t)(j / 8) * nf + q) * 8 + (j % 8)) * (L + 1)) * 64;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint4 *stg = reinterpret_cast<uint4 *>(reinterpret_cast<unsigned char *>(sm_r4) + fft_smem_bytes<LOG2N>(n)) +
                 warp * 32 * kRecUint4;
    for (int mu0 = warp * 32; mu0 <= L; mu0 += blockDim.x) {
        const int mu = mu0 + lane;
        uint4 rec_p[2], rec_m[2];
        if (mu <= L) {
            const int bp = mu, bm = mu == 0 ? 0 : n - mu;
            const int pp = LOG2N > 0 ? bp : __ldg(perm + bp), pm = LOG2N > 0 ? bm : __ldg(perm + bm);
            float vp[8], vm[8];
#pragma unroll
            for (int f = 0; f < 2; ++f) {
                const int e0 = f * n + pp, e1 = f * n + pm, e2 = (2 + f) * n + pp, e3 = (2 + f) * n + pm;
                const float2 a = buf[LOG2N > 0 ? padi(e0) : e0], a2 = buf[LOG2N > 0 ? padi(e1) : e1];
                const float2 z = eq ? make_float2(0.f, 0.f) : buf[LOG2N > 0 ? padi(e2) : e2];
                const float2 z2 = eq ? make_float2(0.f, 0.f) : buf[LOG2N > 0 ? padi(e3) : e3];
                // 2 F_th = Z(m) + conj Z(-m), 2 F_ph = -i (Z(m) - conj Z(-m)), rings j and j'
                const float tjx = a.x + a2.x, tjy = a.y - a2.y, pjx = a.y + a2.y, pjy = a2.x - a.x;
                const float tkx = z.x + z2.x, tky = z.y - z2.y, pkx = z.y + z2.y, pky = z2.x - z.x;
                vp[f * 2] = w * (tjx + tkx);
                vp[f * 2 + 1] = w * (tjy + tky);
                vp[4 + f * 2] = w * (pjx + pkx);
                vp[4 + f * 2 + 1] = w * (pjy + pky);
                vm[f * 2] = eq ? 0.f : w * (tjx - tkx);
                vm[f * 2 + 1] = eq ? 0.f : w * (tjy - tky);
                vm[4 + f * 2] = eq ? 0.f : w * (pjx - pkx);
                vm[4 + f * 2 + 1] = eq ? 0.f : w * (pjy - pky);
            }
            pack_row_f32(vp, rec_p);
            pack_row_f32(vm, rec_m);
        }
        const int nrec = L + 1 - mu0 < 32 ? L + 1 - mu0 : 32;
        put_records<LOG2N>(dst_base + (size_t)mu0 * 64, stg, lane, mu <= L, nrec, rec_p, rec_m);
    }
    if (LOG2N >= 0) staging_free(lane);              // shared memory stays until the copies read it
}

// Real fields, inverse: for field f of the pair, the spectrum of z = T_th + i T_ph is
//   Z(m) = G_th(m) + i G_ph(m),  Z(-m) = conj G_th(m) + i conj G_ph(m)   (m >= 1),
//   Z(0) = Re G_th(0) + i Re G_ph(0),
// so one inverse transform per field and ring yields both real components.
template <int LOG2N>
__global__ void __launch_bounds__(kFftThreads, fft_blocks_per_sm<LOG2N>()) k_rfft_inv_bf16(
    const float *__restrict__ S32, const __grid_constant__ CUtensorMap tmap_s, float *__restrict__ Tth,
    float *__restrict__ Tph, RadixPlanArg rp, const float2 *__restrict__ tw, const int *__restrict__ perm,
    const float2 *__restrict__ isc, int L, int nlat, int J, int has_eq, int JP, int B,
    const long long *__restrict__ toff, int *status, const float *__restrict__ polS, const int *__restrict__ plim,
    int pol_jc, int pol_muc)
{
    extern __shared__ float4 sm_s4[];
    float2 *buf = reinterpret_cast<float2 *>(sm_s4);
    constexpr int V = 2;
    const int n = rp.n;
    const int q = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;
    const float2 sc2 = __ldg(isc + j);
    const float is = sc2.x, w0 = sc2.y;
    // every bin but n/2 is written below (at position perm[m] for LOG2N < 0, as above)
    if (threadIdx.x < nr) {
        const int i = threadIdx.x * n + (LOG2N < 0 ? __ldg(perm + n / 2) : n / 2);
        buf[LOG2N > 0 ? padi(i) : i] = make_float2(0.f, 0.f);
    }
    const bool polar = j < pol_jc;
    const int plim_j = polar ? __ldg(plim + ((j | 1) < pol_jc ? (j | 1) : pol_jc - 1)) : 0;
    const size_t pbase = ((size_t)q * (polar ? pol_jc : 0) + j) * pol_muc;
    auto put = [&](int mu, const float (&ev_in)[8], const float (&ov_in)[8]) {
        float ev[8], ov[8];
        polar_or_gemm(polar ? polS : nullptr, plim_j, pol_muc, pbase, mu, ev_in, ov_in, ev, ov);
        const float sc = mu == 0 ? w0 : is;
        const int pp = LOG2N < 0 ? __ldg(perm + mu) : mu;
        const int pm = LOG2N < 0 ? (mu == 0 ? 0 : __ldg(perm + n - mu)) : n - mu;
#pragma unroll
        for (int f = 0; f < 2; ++f) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                if (side == 1 && eq) continue;
                const float sg = side ? -1.f : 1.f;   // ring j: E + O, ring j': E - O
                const int kt = f * 2, kp = 4 + f * 2;
                const float gtx = (ev[kt] + sg * ov[kt]) * sc, gty = (ev[kt + 1] + sg * ov[kt + 1]) * sc;
                const float gpx = (ev[kp] + sg * ov[kp]) * sc, gpy = (ev[kp + 1] + sg * ov[kp + 1]) * sc;
                const int rb = (2 * side + f) * n;
                if (mu == 0) {
                    const int i0 = rb + pp;
                    buf[LOG2N > 0 ? padi(i0) : i0] = make_float2(gtx, gpx);
                } else {
                    const int i0 = rb + pp, i1 = rb + pm;
                    buf[LOG2N > 0 ? padi(i0) : i0] = make_float2(gtx - gpy, gty + gpx);
                    buf[LOG2N > 0 ? padi(i1) : i1] = make_float2(gtx + gpy, gpx - gty);
                }
            }
        }
    };
    stream_records<LOG2N>(S32, &tmap_s, reinterpret_cast<unsigned char *>(sm_s4) + fft_smem_bytes<LOG2N>(n), status, q,
                          j, L, JP, put);
    const int jm = nlat - 1 - j;
    if constexpr (LOG2N > 0) {
        fft_p2_to_global<LOG2N, true>(buf, tw, nr, RealPairRowsOut{Tth, Tph, toff, q, B, nlat, j, jm, n});
        return;
    }
    if constexpr (LOG2N < 0) {
        dit_f32<true>(buf, tw, rp, nr, 1);
        last_stage_global<true>(buf, tw, rp, nr, RealPairRowsOut{Tth, Tph, toff, q, B, nlat, j, jm, n});
        return;
    }
    dif_f32<true, LOG2N == 0>(buf, tw, rp, nr,
                  reinterpret_cast<float2 *>(reinterpret_cast<unsigned char *>(sm_s4) + fft_smem_bytes<LOG2N>(n)));
    const int nv = n / V;
    const Recip rnv = recip(nv);
    for (int idx = threadIdx.x; idx < nr * nv; idx += blockDim.x) {
        const int ring = rdiv(idx, rnv), kv = idx - ring * nv;
        const int bf = 2 * q + (ring & 1);
        if (bf >= B) continue;
        float th[V], ph[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const float2 z = buf[ring * n + __ldg(perm + kv * V + i)];
            th[i] = z.x;
            ph[i] = z.y;
        }
        const size_t fb = toff ? (size_t)toff[bf] : (size_t)bf * nlat * n;
        const size_t off = fb + (size_t)(ring < 2 ? j : jm) * n + (size_t)kv * V;
        store_v<V>(Tth + off, th);
        store_v<V>(Tph + off, ph);
    }
}

}  // namespace

template <int LOG2N>
cudaError_t launch_fwd_t(const Plan &p, const void *Tth, const void *Tph, cudaStream_t s)
{
    RadixPlanArg rp = make_radix_arg(p.fft);
    // record staging after the DFT; the Bluestein scratch (during the DFT) shares its space
    const size_t blue = p.fft.blue_scratch;
    const size_t smem = (size_t)fft_smem_bytes<LOG2N>(p.nphi) + (LOG2N < 0 ? 0 : blue > kStageBytes ? blue : kStageBytes);
    if (p.real) {
        auto k = k_rfft_fwd_bf16<LOG2N>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<p.ncg * p.J, kFftThreads, smem, s>>>((const float *)Tth, (const float *)Tph, (unsigned char *)p.d_Fb,
                                                 rp, p.fft.tw32, p.d_perm,
                                                 p.unit_weights ? p.d_omega_unit32 : p.d_omega32, p.L, p.nlat,
                                                 p.J, p.has_eq, p.nf, p.B, p.d_toff);
        return cudaGetLastError();
    }
    if constexpr (LOG2N == 11) {
        // whole rows by bulk copies: both planes 16-byte aligned (row starts then are, field
        // offsets being even)
        if ((((uintptr_t)Tth | (uintptr_t)Tph) & 15) == 0) {
            cudaFuncSetAttribute(k_fft_fwd_sw, cudaFuncAttributeMaxDynamicSharedMemorySize, kSwSmem);
            k_fft_fwd_sw<<<p.B * p.J, kFftThreads, kSwSmem, s>>>(
                (const float2 *)Tth, (const float2 *)Tph, (unsigned char *)p.d_Fb, p.fft.tw32,
                p.unit_weights ? p.d_omega_unit32 : p.d_omega32, p.L, p.nlat, p.J, p.has_eq, p.nf, p.d_toff,
                p.d_status);
            return cudaGetLastError();
        }
    }
    auto k = k_fft_fwd_bf16<LOG2N>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<p.B * p.J, kFftThreads, smem, s>>>((const float2 *)Tth, (const float2 *)Tph, (unsigned char *)p.d_Fb, rp,
                                   p.fft.tw32, p.d_perm, p.unit_weights ? p.d_omega_unit32 : p.d_omega32, p.L,
                                   p.nlat, p.J, p.has_eq, p.nf, p.d_toff);
    return cudaGetLastError();
}

template <int LOG2N>
cudaError_t launch_inv_t(const Plan &p, void *Tth, void *Tph, cudaStream_t s)
{
    RadixPlanArg rp = make_radix_arg(p.fft);
    const size_t blue = p.fft.blue_scratch;
    const size_t smem = (size_t)fft_smem_bytes<LOG2N>(p.nphi) + (LOG2N > 0 ? kInvStageBytes : blue);
    if (p.real) {
        auto k = k_rfft_inv_bf16<LOG2N>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<p.ncg * p.J, kFftThreads, smem, s>>>((const float *)p.d_S32, p.tmap_s32, (float *)Tth, (float *)Tph, rp,
                                                 p.fft.tw32, p.d_perm, p.d_isc32 + (p.adj_weighted ? p.J : 0),
                                                 p.L, p.nlat, p.J, p.has_eq, p.JP, p.B, p.d_toff, p.d_status,
                                                 p.d_polS, p.d_pol_lim, p.pol_jc, p.pol_muc);
        return cudaGetLastError();
    }
    if constexpr (LOG2N == 11) {
        cudaFuncSetAttribute(k_fft_inv_sw, cudaFuncAttributeMaxDynamicSharedMemorySize, kSwInvSmem);
        k_fft_inv_sw<<<p.B * p.J, kFftThreads, kSwInvSmem, s>>>(
            p.tmap_s32, (float2 *)Tth, (float2 *)Tph, p.fft.tw32, p.d_isc32 + (p.adj_weighted ? p.J : 0), p.L,
            p.nlat, p.J, p.has_eq, p.d_toff, p.d_status, p.d_polS, p.d_pol_lim, p.pol_jc, p.pol_muc);
        return cudaGetLastError();
    }
    auto k = k_fft_inv_bf16<LOG2N>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<p.B * p.J, kFftThreads, smem, s>>>((const float *)p.d_S32, p.tmap_s32, (float2 *)Tth, (float2 *)Tph, rp,
                                   p.fft.tw32, p.d_perm, p.d_isc32 + (p.adj_weighted ? p.J : 0), p.L, p.nlat,
                                   p.J, p.has_eq, p.JP, p.d_toff, p.d_status, p.d_polS, p.d_pol_lim, p.pol_jc,
                                   p.pol_muc);
    return cudaGetLastError();
}

cudaError_t launch_fft_fwd_bf16(const Plan &p, const void *Tth, const void *Tph, cudaStream_t s)
{
    switch (p.fft_log2n) {
    case 6: return launch_fwd_t<6>(p, Tth, Tph, s);
    case 7: return launch_fwd_t<7>(p, Tth, Tph, s);
    case 8: return launch_fwd_t<8>(p, Tth, Tph, s);
    case 9: return launch_fwd_t<9>(p, Tth, Tph, s);
    case 10: return launch_fwd_t<10>(p, Tth, Tph, s);
    case 11: return launch_fwd_t<11>(p, Tth, Tph, s);
    case 12: return launch_fwd_t<12>(p, Tth, Tph, s);
    default: return p.fft.blue_scratch ? launch_fwd_t<0>(p, Tth, Tph, s) : launch_fwd_t<-1>(p, Tth, Tph, s);
    }
}

cudaError_t launch_fft_inv_bf16(const Plan &p, void *Tth, void *Tph, cudaStream_t s)
{
    switch (p.fft_log2n) {
    case 6: return launch_inv_t<6>(p, Tth, Tph, s);
    case 7: return launch_inv_t<7>(p, Tth, Tph, s);
    case 8: return launch_inv_t<8>(p, Tth, Tph, s);
    case 9: return launch_inv_t<9>(p, Tth, Tph, s);
    case 10: return launch_inv_t<10>(p, Tth, Tph, s);
    case 11: return launch_inv_t<11>(p, Tth, Tph, s);
    case 12: return launch_inv_t<12>(p, Tth, Tph, s);
    default: return p.fft.blue_scratch ? launch_inv_t<0>(p, Tth, Tph, s) : launch_inv_t<-1>(p, Tth, Tph, s);
    }
}

}  // namespace favest
