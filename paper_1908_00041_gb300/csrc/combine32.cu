// Coefficient-side stages of the split-precision path (same formulas as combine.cu):
//   combine  : FP32 scalar sums Q (tensor-core GEMM output, rows l - mu, 8 columns per
//              column group: component c, sign s of m, re/im) -> a_lm, b_lm (complex64)
//   uncombine: a_lm, b_lm (complex64) -> scaled scalar coefficients g, written as three
//              bf16 pieces in the tensor-core B-operand layout (K-chunks of 32 rows by
//              N = 128 or 256 columns).
// Real fields (REAL = true): a column group is a pair of fields 2q, 2q+1 at m = +mu, in the
// slots the complex layout gives to m = +mu and m = -mu; coefficients are stored for
// m >= 0 only, at l(l+1)/2 - 1 + m of a field's KR = L(L+3)/2.
#include "favest_internal.h"
#include "bf16_split.cuh"

namespace favest {

namespace {


constexpr int kCT = 32;          // orders and degrees per combine tile
constexpr int kCTRows = kCT + 2;  // degrees l0 - 1 .. l0 + 32 (one-row halo each side)

// Tiled combine.  grid.x enumerates the tiles (order block ob <= degree block lb) of
// the (l >= mu) triangle, grid.y the field.  Phase 1 stages, for the tile's 32 orders
// and the degrees l0-1 .. l0+32, the 32-byte sum records of Q = [field][ntab rows][8]
// (rows of order mu from tab_off(L, mu): l = mu, mu+2, .. then l = mu+1, ..) in shared
// memory.  Phase 2: warp w takes degrees l0 + w, l0 + w + 8, ..; lane = order, so the
// stores of a_{l,+mu} (ascending) and a_{l,-mu} (descending) are contiguous runs.
template <bool REAL>
__global__ void __launch_bounds__(256) k_combine_bf16(const float *__restrict__ Q, float2 *__restrict__ a,
                                                      float2 *__restrict__ bo, const float *__restrict__ P,
                                                      const float *__restrict__ M, const float *__restrict__ R,
                                                      int L, int K, const long long *__restrict__ coff, int B,
                                                      float ps)
{
    // [order][(degree - (l0 - 1)) * 2 + half]; the odd row length (69 x 16 B) spreads the
    // lanes (orders) of a quarter-warp over distinct bank groups
    __shared__ float4 qs[kCT][kCTRows * 2 + 1];
    // the tile's P, M, R coefficients [table][order][degree - l0], rows padded to 33 so that
    // the lanes (orders) of phase 2 read distinct banks; staged by coalesced loads (degrees
    // of one order are consecutive in the tables) instead of one scattered load per lane
    __shared__ float pmr[3][kCT][kCT + 1];
    // tile index -> (ob, lb), lb >= ob, row-major over lb
    int t = blockIdx.x, lb = 0;
    while (t > lb) {
        t -= lb + 1;
        ++lb;
    }
    const int ob = t;
    const int mu0 = ob * kCT, l0 = lb * kCT;
    const int bi = blockIdx.y;
    const size_t cb = (coff && !REAL) ? (size_t)coff[bi] : (size_t)bi * K;
    const float *qb = Q + (size_t)bi * tab_off(L, L + 1) * 8;
    // phase 1: records (order i, degree l0 - 1 + d), d = 0 .. 33, for l in [mu, L+1]; all of a
    // thread's loads are issued before any is stored
    constexpr int kE = kCT * kCTRows * 2, kPer = (kE + 255) / 256;
    float4 v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = threadIdx.x + u * 256;
        const int half = e & 1, d = (e >> 1) % kCTRows, i = (e >> 1) / kCTRows;
        const int mu = mu0 + i, l = l0 - 1 + d;
        v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < kE && mu <= L && l >= mu && l <= L + 1) {
            const int r = l - mu, n0 = (L + 3 - mu) / 2;
            const float4 *src = reinterpret_cast<const float4 *>(
                qb + (tab_off(L, mu) + ((r & 1) ? n0 : 0) + (r >> 1)) * 8);
            v[u] = __ldg(src + half);
        }
    }
    constexpr int kT = kCT * kCT, kTPer = 3 * kT / 256;
    float tv[kTPer];
#pragma unroll
    for (int u = 0; u < kTPer; ++u) {
        const int e = threadIdx.x + u * 256, tab = e / kT, i = (e % kT) / kCT, dl = e % kCT;
        const int mu = mu0 + i, l = l0 + dl;
        tv[u] = 0.f;
        if (mu <= L && l >= 1 && l <= L && l >= mu) {
            const float *src = tab == 0 ? P : tab == 1 ? M : R;
            tv[u] = __ldg(src + tab_off(L, mu) + (l - mu));
        }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = threadIdx.x + u * 256;
        if (e < kE) qs[(e >> 1) / kCTRows][((e >> 1) % kCTRows) * 2 + (e & 1)] = v[u];
    }
#pragma unroll
    for (int u = 0; u < kTPer; ++u) {
        const int e = threadIdx.x + u * 256;
        pmr[e / kT][(e % kT) / kCT][e % kCT] = tv[u];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int mu = mu0 + lane;
    for (int l = l0 + warp; l < l0 + kCT; l += 8) {
        if (l < 1 || l > L || mu > l) continue;
        const int d = l - (l0 - 1);
        const float Pl = pmr[0][lane][l - l0], Ml = pmr[1][lane][l - l0], Rl = pmr[2][lane][l - l0];
        const bool has_m = l > mu;
        const float4 q1a = qs[lane][(d + 1) * 2], q1b = qs[lane][(d + 1) * 2 + 1];
        const float4 q0a = qs[lane][d * 2], q0b = qs[lane][d * 2 + 1];
        const float4 qma = qs[lane][(d - 1) * 2], qmb = qs[lane][(d - 1) * 2 + 1];
        const float q1[8] = {q1a.x, q1a.y, q1a.z, q1a.w, q1b.x, q1b.y, q1b.z, q1b.w};
        const float q0[8] = {q0a.x, q0a.y, q0a.z, q0a.w, q0b.x, q0b.y, q0b.z, q0b.w};
        const float qm[8] = {qma.x, qma.y, qma.z, qma.w, qmb.x, qmb.y, qmb.z, qmb.w};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (!REAL && mu == 0 && s == 1) continue;
            if (REAL && 2 * bi + s >= B) continue;
            const int m = (!REAL && s) ? -mu : mu;
            const float sg = (!REAL && s && (mu & 1)) ? -1.f : 1.f;
            const float Rm = Rl * (float)m;
            // th: cols s*2 + {0,1}; ph: 4 + s*2 + {0,1}
            const int ct = s * 2, cp = 4 + s * 2;
            const float tmx = has_m ? qm[ct] : 0.f, tmy = has_m ? qm[ct + 1] : 0.f;
            const float pmx = has_m ? qm[cp] : 0.f, pmy = has_m ? qm[cp + 1] : 0.f;
            const float ax = sg * fmaf(Pl, q1[ct], fmaf(-Ml, tmx, Rm * q0[cp + 1]));
            const float ay = sg * fmaf(Pl, q1[ct + 1], fmaf(-Ml, tmy, -Rm * q0[cp]));
            const float bx = sg * fmaf(Pl, q1[cp], fmaf(-Ml, pmx, -Rm * q0[ct + 1]));
            const float by = sg * fmaf(Pl, q1[cp + 1], fmaf(-Ml, pmy, Rm * q0[ct]));
            const size_t k = REAL ? (coff ? (size_t)coff[2 * bi + s] : (size_t)(2 * bi + s) * K) +
                                        (size_t)l * (l + 1) / 2 - 1 + mu
                                  : cb + (size_t)l * l + l + m - 1;
            // real fields, transpose for the real inner product: orders m > 0 doubled
            const float sc = (REAL && mu > 0) ? ps : 1.f;
            a[k] = make_float2(sc * ax, sc * ay);
            bo[k] = make_float2(sc * bx, sc * by);
        }
    }
}

constexpr int kUS = 4 * (kCT + 1) + 1;  // shared row stride (float2, odd) of the uncombine tile

// Tiled uncombine.  grid.x enumerates the tiles (order block ob <= row block lb) of the
// (l' >= mu) triangle of rows l' = mu..L+1, grid.y the field.  Phase 1 stages the
// coefficients a, b of orders +-mu, mu in the tile, at degrees l0-1 .. l0+32 (coalesced
// over the order); phase 2: warp w takes orders mu0 + w, + 8, ..; lane = row l' = l0 + lane,
// so the 16-byte rows it writes into the tensor-core B layout (8 consecutive rows of a
// parity per 128-byte core-matrix block) are contiguous.
// Order 0 is special: sin(theta) d_theta lambda_l^0 vanishes at the poles, so forming
// G(j, 0) as (sum_l lambda_l^0 g_l) / sin(theta_j) would amplify rounding errors near
// the poles by 1/sin(theta_1).  Instead d_theta lambda_l^0 = sqrt(l(l+1)) lambda_l^1 gives
//   G_th(j, 0) = sum_l a_l0 lambda_l^1(theta_j),  G_ph(j, 0) = sum_l b_l0 lambda_l^1(theta_j)
// with no division: order 0 is synthesised on the order-1 Legendre tiles (rows l = 1..L+1)
// and the inverse FFT stage skips the 1/sin(theta) factor for it.
template <bool REAL>
__global__ void __launch_bounds__(256) k_uncombine_bf16(const float2 *__restrict__ a, const float2 *__restrict__ b,
                                                        unsigned char *__restrict__ gb,
                                                        const long long *__restrict__ g_off,
                                                        const float *__restrict__ P, const float *__restrict__ M,
                                                        const float *__restrict__ R, const float *__restrict__ k1tab,
                                                        int L, int K, int N, const long long *__restrict__ coff, int B,
                                                        float ps)
{
    // cs[(l - (l0 - 1)) * kUS + q * (kCT + 1) + order], q = (a+, a-, b+, b-); real fields:
    // (a of field 2q, a of 2q+1, b of 2q, b of 2q+1), all at m = +mu
    __shared__ float2 cs[kCTRows * kUS];
    int t = blockIdx.x, lb = 0;
    while (t > lb) {
        t -= lb + 1;
        ++lb;
    }
    const int ob = t;
    const int mu0 = ob * kCT, l0 = lb * kCT;
    const int bi = blockIdx.y;
    const size_t cb = (coff && !REAL) ? (size_t)coff[bi] : (size_t)bi * K;
    // all of a thread's loads are issued before any is stored
    constexpr int kE = kCTRows * 4 * kCT, kPer = (kE + 255) / 256;
    float2 v[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = threadIdx.x + u * 256;
        const int i = e % kCT, q = (e / kCT) & 3, d = e / (4 * kCT);
        const int mu = mu0 + i, l = l0 - 1 + d;
        v[u] = make_float2(0.f, 0.f);
        if (e >= kE) continue;
        if (REAL) {
            const int bf = 2 * bi + (q & 1);
            if (l >= 1 && l <= L && mu <= l && bf < B) {
                const size_t fcb = coff ? (size_t)coff[bf] : (size_t)bf * K;
                v[u] = __ldg(((q & 2) ? b : a) + fcb + (size_t)l * (l + 1) / 2 - 1 + mu);
            }
        } else {
            const int m = (q & 1) ? -mu : mu;
            if (l >= 1 && l <= L && mu <= l && !(mu == 0 && (q & 1)))
                v[u] = __ldg(((q & 2) ? b : a) + cb + (size_t)l * l + l + m - 1);
        }
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int e = threadIdx.x + u * 256;
        if (e >= kE) continue;
        const int i = e % kCT, q = (e / kCT) & 3, d = e / (4 * kCT);
        float2 x = v[u];
        if (REAL && mu0 + i > 0) x = make_float2(ps * x.x, ps * x.y);   // real transpose: m > 0 halved
        cs[d * kUS + q * (kCT + 1) + i] = x;
    }
    __syncthreads();
    constexpr int KC = kGemmChunkK;
    const int fpt = N / 8;                        // fields per column tile
    const int nt = bi / fpt, bg = bi % fpt;
    const long long piece = (long long)KC * N * 2, chunk = 3 * piece;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = l0 + lane;                      // this thread's row degree
    const int d = l - (l0 - 1);
    for (int i = warp; i < kCT; i += 8) {
        const int mu = mu0 + i;
        if (mu > L) break;
        const int lmin = mu == 0 ? 1 : mu;        // first row of this order's tiles
        if (l < lmin || l > L + 1) continue;
        const int r = l - lmin;
        const int nrow = L + 2 - lmin;
        const int nka = (r & 1) ? (nrow / 2 + KC - 1) / KC : ((nrow + 1) / 2 + KC - 1) / KC;
        float v[8];
        if (mu == 0) {
            // the order-1 tiles hold lambda_l^1 / kappa_l^(1)
            const float k1 = (l <= L) ? k1tab[l] : 0.f;
            const float2 a0 = cs[d * kUS + 0 * (kCT + 1) + i], b0 = cs[d * kUS + 2 * (kCT + 1) + i];
            v[0] = k1 * a0.x; v[1] = k1 * a0.y; v[2] = 0.f; v[3] = 0.f;
            v[4] = k1 * b0.x; v[5] = k1 * b0.y; v[6] = 0.f; v[7] = 0.f;
            if (REAL) {   // the pair's second field in the slots of m = -0
                const float2 a1 = cs[d * kUS + 1 * (kCT + 1) + i], b1 = cs[d * kUS + 3 * (kCT + 1) + i];
                v[2] = k1 * a1.x; v[3] = k1 * a1.y;
                v[6] = k1 * b1.x; v[7] = k1 * b1.y;
            }
        } else {
            const long long t0 = tab_off(L, mu);
            const float Pm = (r > 0) ? P[t0 + r - 1] : 0.f;
            const float Mp = (l + 1 <= L) ? M[t0 + r + 1] : 0.f;
            const float Rr = (l <= L) ? R[t0 + r] : 0.f;
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int m = (!REAL && s) ? -mu : mu;
                const float sg = (!REAL && s && (mu & 1)) ? -1.f : 1.f;
                const float Rl = Rr * (float)m;
                const float2 am1 = cs[(d - 1) * kUS + s * (kCT + 1) + i];
                const float2 ap1 = cs[(d + 1) * kUS + s * (kCT + 1) + i];
                const float2 bm1 = cs[(d - 1) * kUS + (2 + s) * (kCT + 1) + i];
                const float2 bp1 = cs[(d + 1) * kUS + (2 + s) * (kCT + 1) + i];
                const float2 a0 = cs[d * kUS + s * (kCT + 1) + i];
                const float2 b0 = cs[d * kUS + (2 + s) * (kCT + 1) + i];
                v[s * 2 + 0] = sg * fmaf(Pm, am1.x, fmaf(-Mp, ap1.x, Rl * b0.y));
                v[s * 2 + 1] = sg * fmaf(Pm, am1.y, fmaf(-Mp, ap1.y, -Rl * b0.x));
                v[4 + s * 2 + 0] = sg * fmaf(Pm, bm1.x, fmaf(-Mp, bp1.x, -Rl * a0.y));
                v[4 + s * 2 + 1] = sg * fmaf(Pm, bm1.y, fmaf(-Mp, bp1.y, Rl * a0.x));
            }
        }
        const int p = r & 1, rp = r >> 1;
        const int kc = rp / KC, rr = rp % KC;
        // chunk [K/8][N/8][8 k][8 n]: row group rr/8, column group = this field
        unsigned char *dst = gb + g_off[mu * 2 + p] + ((long long)nt * nka + kc) * chunk +
                             (long long)(rr / 8) * (fpt * 128) + bg * 128 + (rr % 8) * 16;
        uint4 w[3];
        pack_row3(v, w);
#pragma unroll
        for (int q = 0; q < 3; ++q) *reinterpret_cast<uint4 *>(dst + q * piece) = w[q];
    }
}

}  // namespace

cudaError_t launch_combine_bf16(const Plan &p, void *a, void *b, cudaStream_t s)
{
    const int K = p.real ? p.L * (p.L + 3) / 2 : p.L * p.L + 2 * p.L;
    const int nb = (p.L + 1 + kCT - 1) / kCT;
    dim3 grid(nb * (nb + 1) / 2, p.ncg);
    auto k = p.real ? k_combine_bf16<true> : k_combine_bf16<false>;
    k<<<grid, 256, 0, s>>>((const float *)p.d_Q32, (float2 *)a, (float2 *)b, p.d_P32, p.d_M32, p.d_R32, p.L, K,
                           p.d_coff, p.B, p.real_transpose ? 2.f : 1.f);
    return cudaGetLastError();
}

cudaError_t launch_uncombine_bf16(const Plan &p, const void *a, const void *b, cudaStream_t s)
{
    const int K = p.real ? p.L * (p.L + 3) / 2 : p.L * p.L + 2 * p.L;
    const int ob_n = (p.L + 1 + kCT - 1) / kCT, lb_n = (p.L + 2 + kCT - 1) / kCT;
    // tiles (ob <= lb) of the row triangle; order blocks never exceed row blocks
    dim3 grid(lb_n * (lb_n + 1) / 2, p.ncg);
    (void)ob_n;
    auto k = p.real ? k_uncombine_bf16<true> : k_uncombine_bf16<false>;
    k<<<grid, 256, 0, s>>>((const float2 *)a, (const float2 *)b, (unsigned char *)p.d_gb, p.d_g_off, p.d_P32,
                           p.d_M32, p.d_R32, p.d_k1, p.L, K, p.gemm_n, p.d_coff, p.B,
                           p.real_transpose ? 0.5f : 1.f);
    return cudaGetLastError();
}

}  // namespace favest
