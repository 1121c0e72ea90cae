// Coefficient-side stages of the split-precision path (same formulas as combine.cu):
//   combine  : FP32 scalar sums Q (tensor-core GEMM output, rows l - mu, 8 columns per
//              field: component c, sign s of m, re/im) -> a_lm, b_lm (complex64), FP64 math
//   uncombine: a_lm, b_lm (complex64) -> scaled scalar coefficients g, written as three
//              bf16 pieces in the tensor-core B-operand layout (K-chunks of 32 rows by
//              N = 128 or 256 columns).
#include "favest_internal.h"

#include <cuda_bf16.h>

namespace favest {

namespace {


// grid (L+1, B): one CTA per (order mu, field); threads over degrees l = max(mu,1)..L.
// Q = [field][ntab rows][8]: the rows of order mu start at tab_off(L, mu), the
// n0 = ceil((L+2-mu)/2) rows l = mu, mu+2, .. first, then l = mu+1, mu+3, ..; a warp
// reads two contiguous runs of 32-byte records.  The coefficient stores of one CTA are
// 8-byte words 2l+1 apart; the CTAs of neighbouring orders fill the rest of each line.
__global__ void k_combine_bf16(const float *__restrict__ Q, float2 *__restrict__ a, float2 *__restrict__ bo,
                               const float *__restrict__ P, const float *__restrict__ M,
                               const float *__restrict__ R, int L, int K, const long long *__restrict__ coff)
{
    const int mu = blockIdx.x, bi = blockIdx.y;
    const size_t cb = coff ? (size_t)coff[bi] : (size_t)bi * K;
    const long long t0 = tab_off(L, mu);
    const float *qb = Q + ((size_t)bi * tab_off(L, L + 1) + t0) * 8;
    const int n0 = (L + 3 - mu) / 2;            // rows of even l - mu
    auto qrow = [&](int r) { return qb + (((r & 1) ? n0 : 0) + (r >> 1)) * 8; };
    for (int l = (mu > 1 ? mu : 1) + threadIdx.x; l <= L; l += blockDim.x) {
        const int r = l - mu;
        const float Pl = P[t0 + r], Ml = M[t0 + r], Rl = R[t0 + r];
        const float *q1 = qrow(r + 1);
        const float *q0 = qrow(r);
        const bool has_m = r > 0;
        const float *qm = qrow(has_m ? r - 1 : r);
        for (int s = 0; s < 2; ++s) {
            if (mu == 0 && s == 1) continue;
            const int m = s ? -mu : mu;
            const float sg = (s && (mu & 1)) ? -1.f : 1.f;
            const float Rm = Rl * (float)m;
            // th: cols s*2 + {0,1}; ph: 4 + s*2 + {0,1}
            const int ct = s * 2, cp = 4 + s * 2;
            const float t1x = q1[ct], t1y = q1[ct + 1], p1x = q1[cp], p1y = q1[cp + 1];
            const float t0x = q0[ct], t0y = q0[ct + 1], p0x = q0[cp], p0y = q0[cp + 1];
            const float tmx = has_m ? qm[ct] : 0.f, tmy = has_m ? qm[ct + 1] : 0.f;
            const float pmx = has_m ? qm[cp] : 0.f, pmy = has_m ? qm[cp + 1] : 0.f;
            const float ax = sg * fmaf(Pl, t1x, fmaf(-Ml, tmx, Rm * p0y));
            const float ay = sg * fmaf(Pl, t1y, fmaf(-Ml, tmy, -Rm * p0x));
            const float bx = sg * fmaf(Pl, p1x, fmaf(-Ml, pmx, -Rm * t0y));
            const float by = sg * fmaf(Pl, p1y, fmaf(-Ml, pmy, Rm * t0x));
            const size_t k = cb + l * l + l + m - 1;
            a[k] = make_float2(ax, ay);
            bo[k] = make_float2(bx, by);
        }
    }
}

__device__ __forceinline__ float2 cf(const float2 *__restrict__ c, int L, int l, int m, size_t cb)
{
    int am = m < 0 ? -m : m;
    if (l < 1 || l > L || am > l) return make_float2(0.f, 0.f);
    return c[cb + l * l + l + m - 1];
}

__device__ __forceinline__ void split3u(float f, unsigned short &h, unsigned short &m, unsigned short &l)
{
    __nv_bfloat16 bh = __float2bfloat16_rn(f);
    float r1 = f - __bfloat162float(bh);
    __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    float r2 = r1 - __bfloat162float(bm);
    __nv_bfloat16 bl = __float2bfloat16_rn(r2);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

// grid (L+1, B): threads over rows l' = mu..L+1.
// Order 0 is special: sin(theta) d_theta lambda_l^0 vanishes at the poles, so forming
// G(j, 0) as (sum_l lambda_l^0 g_l) / sin(theta_j) would amplify rounding errors near
// the poles by 1/sin(theta_1).  Instead d_theta lambda_l^0 = sqrt(l(l+1)) lambda_l^1 gives
//   G_th(j, 0) = sum_l a_l0 lambda_l^1(theta_j),  G_ph(j, 0) = sum_l b_l0 lambda_l^1(theta_j)
// with no division: order 0 is synthesised on the order-1 Legendre tiles (rows l = 1..L+1)
// and the inverse FFT stage skips the 1/sin(theta) factor for it.
__global__ void k_uncombine_bf16(const float2 *__restrict__ a, const float2 *__restrict__ b,
                                 unsigned char *__restrict__ gb, const long long *__restrict__ g_off,
                                 const float *__restrict__ P, const float *__restrict__ M,
                                 const float *__restrict__ R, const float *__restrict__ k1tab, int L, int K,
                                 int N, const long long *__restrict__ coff)
{
    const int mu = blockIdx.x, bi = blockIdx.y;
    const size_t cb = coff ? (size_t)coff[bi] : (size_t)bi * K;
    const long long t0 = tab_off(L, mu);
    const int nrow = L + 2 - (mu == 0 ? 1 : mu);
    const int nrow_p0 = (nrow + 1) / 2, nrow_p1 = nrow / 2;
    constexpr int KC = kGemmChunkK;
    const int nka0 = (nrow_p0 + KC - 1) / KC, nka1 = (nrow_p1 + KC - 1) / KC;
    const int fpt = N / 8;                        // fields per column tile
    const int nt = bi / fpt, bg = bi % fpt;
    const long long piece = (long long)KC * N * 2, chunk = 3 * piece;
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
        const int l = (mu == 0 ? 1 : mu) + r;
        float v[8];
        if (mu == 0) {
            // the order-1 tiles hold lambda_l^1 / kappa_l^(1)
            const float k1 = (l <= L) ? k1tab[l] : 0.f;
            const float2 a0 = cf(a, L, l, 0, cb), b0 = cf(b, L, l, 0, cb);
            v[0] = k1 * a0.x; v[1] = k1 * a0.y; v[2] = 0.f; v[3] = 0.f;
            v[4] = k1 * b0.x; v[5] = k1 * b0.y; v[6] = 0.f; v[7] = 0.f;
        } else
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            const int m = s ? -mu : mu;
            float gtx = 0.f, gty = 0.f, gpx = 0.f, gpy = 0.f;
            if (!(mu == 0 && s == 1)) {
                const float sg = (s && (mu & 1)) ? -1.f : 1.f;
                const float Pm = (r > 0) ? P[t0 + r - 1] : 0.f;
                const float Mp = (l + 1 <= L) ? M[t0 + r + 1] : 0.f;
                const float Rl = (l <= L) ? R[t0 + r] * (float)m : 0.f;
                float2 am1 = cf(a, L, l - 1, m, cb), ap1 = cf(a, L, l + 1, m, cb);
                float2 bm1 = cf(b, L, l - 1, m, cb), bp1 = cf(b, L, l + 1, m, cb);
                float2 a0 = cf(a, L, l, m, cb), b0 = cf(b, L, l, m, cb);
                gtx = sg * fmaf(Pm, am1.x, fmaf(-Mp, ap1.x, Rl * b0.y));
                gty = sg * fmaf(Pm, am1.y, fmaf(-Mp, ap1.y, -Rl * b0.x));
                gpx = sg * fmaf(Pm, bm1.x, fmaf(-Mp, bp1.x, -Rl * a0.y));
                gpy = sg * fmaf(Pm, bm1.y, fmaf(-Mp, bp1.y, Rl * a0.x));
            }
            v[0 * 4 + s * 2 + 0] = gtx;
            v[0 * 4 + s * 2 + 1] = gty;
            v[1 * 4 + s * 2 + 0] = gpx;
            v[1 * 4 + s * 2 + 1] = gpy;
        }
        const int p = r & 1, rp = r >> 1;
        const int nka = p ? nka1 : nka0;
        const int kc = rp / KC, rr = rp % KC;
        // chunk [K/8][N/8][8 k][8 n]: row group rr/8, column group = this field
        unsigned char *dst = gb + g_off[mu * 2 + p] + ((long long)nt * nka + kc) * chunk +
                             (long long)(rr / 8) * (fpt * 128) + bg * 128 + (rr % 8) * 16;
        unsigned w[3][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            unsigned short h0, m0, l0, h1, m1, l1;
            split3u(v[2 * i], h0, m0, l0);
            split3u(v[2 * i + 1], h1, m1, l1);
            w[0][i] = (unsigned)h0 | ((unsigned)h1 << 16);
            w[1][i] = (unsigned)m0 | ((unsigned)m1 << 16);
            w[2][i] = (unsigned)l0 | ((unsigned)l1 << 16);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
            *reinterpret_cast<uint4 *>(dst + q * piece) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
    }
}

}  // namespace

cudaError_t launch_combine_bf16(const Plan &p, void *a, void *b, cudaStream_t s)
{
    const int K = p.L * p.L + 2 * p.L;
    const int th = p.L >= 255 ? 256 : (p.L >= 63 ? 64 : 32);
    dim3 grid(p.L + 1, p.B);
    k_combine_bf16<<<grid, th, 0, s>>>((const float *)p.d_Q32, (float2 *)a, (float2 *)b, p.d_P32, p.d_M32,
                                       p.d_R32, p.L, K, p.d_coff);
    return cudaGetLastError();
}

cudaError_t launch_uncombine_bf16(const Plan &p, const void *a, const void *b, cudaStream_t s)
{
    const int K = p.L * p.L + 2 * p.L;
    dim3 grid(p.L + 1, p.B);
    const int th = p.L + 2 >= 256 ? 256 : 64;
    k_uncombine_bf16<<<grid, th, 0, s>>>((const float2 *)a, (const float2 *)b, (unsigned char *)p.d_gb,
                                         p.d_g_off, p.d_P32, p.d_M32, p.d_R32, p.d_k1, p.L, K, p.gemm_n, p.d_coff);
    return cudaGetLastError();
}

}  // namespace favest
