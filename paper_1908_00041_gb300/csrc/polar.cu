// Polar patch of the split-precision adjoint.
//
// The adjoint forms, per order mu and folded latitude j, the scalar sums
//   S_p(j) = sum_{l' = l - mu of parity p} g_l' lambda~_l'(theta_j),
//   g_l'   = P_{l'-1} a_{l'-1} - M_{l'+1} a_{l'+1} - i m R_l' b_l'        (theta part),
// and divides them by sin(theta_j).  Regrouping the sum by coefficient gives
//   S = sum_l a_l D_l - i m sum_l b_l Lambda_l,
//   D_l = P_l lambda~_{l+1} - M_l lambda~_{l-1} = sin(theta) d_theta lambda_l / sqrt(l(l+1)),
//   Lambda_l = R_l lambda~_l = lambda_l / sqrt(l(l+1)),
// (the identity sin(theta) d_theta lambda_l = l eps_{l+1} lambda_{l+1} - (l+1) eps_l lambda_{l-1}).
// Close to a pole D_l is O(sin(theta)) while its two parts are O(1): the tensor-core
// sum, which carries the parts separately at FP32-level precision, loses a factor of
// about 1/sin(theta_j) of its relative accuracy there, and the division by sin(theta_j)
// turns that into an absolute error of the field.  For the few rings with
// sin(theta_j) < kPolarSin this kernel recomputes S in the regrouped form, from D_l and
// Lambda_l evaluated in FP64 at plan time and stored in FP32, so nothing cancels.
// Orders mu >= pol_muc are left to the tensor-core sums: at these rings every
// lambda_l^mu with l <= L lies beyond its turning point (mu > 1.5 L sin(theta_j)) and is
// exponentially small, so their error is negligible.
//
// Only the theta/phi structure of the combine stage and the E/O parity split of the
// folded grid are used; the output goes to a buffer of its own, which the inverse DFT reads
// in place of the GEMM's sums for the patched (ring, order) pairs (so the patch does not
// wait for the GEMM),
//   polS[group][pol_jc][pol_muc][parity][8], columns c*4 + s*2 + (re, im): c = theta/phi,
//   s = 0: m = +mu, s = 1: m = -mu (with the factor (-1)^mu of lambda^{-mu}); for real
//   fields (REAL = true) slot s holds field 2q + s of the pair q at m = +mu, with the
//   half-spectrum coefficients (index l(l+1)/2 - 1 + mu of a field's K).
#include <cmath>
#include <vector>

#include "favest_internal.h"

namespace favest {

namespace {

constexpr double kPolarSin = 0.06;   // rings with sin(theta_j) below this are patched

double eps_pl(int l, int mu)
{
    const double num = (double)(l - mu) * (double)(l + mu);
    const double den = (double)(2 * l - 1) * (double)(2 * l + 1);
    return num > 0 ? std::sqrt(num / den) : 0.0;
}

constexpr int kPolarJ = 2;           // rings per warp
constexpr int kPolarPairs = 5;       // ring pairs (warps) per block
constexpr int kPolarChunk = 16;      // degrees per step; summed in plain FP32
constexpr int kPolarThreads = 32 * kPolarPairs;
constexpr int kPolarCoef = kPolarChunk * 4 * 32;                    // coefficient elements per step
constexpr int kPolarCoefBytes = kPolarCoef * 8;                     // 16 KB
constexpr int kPolarTabBytes = kPolarPairs * kPolarJ * kPolarChunk * 32 * 8;   // 80 KB
constexpr int kPolarSmem = 2 * (kPolarCoefBytes + kPolarTabBytes);             // double-buffered

// asynchronous copies global -> shared; src_bytes = 0 writes zeros without reading
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc, int src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }


// grid (pol_muc / 32, column groups, ceil(pol_jc / 10)), 160 threads, 112 KB of shared
// memory (two blocks per SM).  Lane = order mu within the tile; warp w takes the rings
// j0 = 2w, 2w + 1 of the block's 10 and sums over all degrees mu0..L in steps of 16.  Every step's operands are
// staged in shared memory by asynchronous copies issued one step ahead: the coefficients
// a, b at +-mu (once for all rings) and each warp's rows of the polar tables, so the sums
// read no global memory.  Per ring the thread keeps 2 banks x 8 columns: bank k collects,
// for even l, the D terms (k = 1) and Lambda terms (k = 0), for odd l the reverse, so that
// bank k holds output parity k ^ (mu & 1).  Terms are summed in FP32 over a step, step sums
// go into a Kahan-compensated running sum (a plain FP32 running sum over ~L terms would lose
// about sqrt(L) ulps).  Ring pairs whose turning-point bound lies below the tile keep the
// tensor-core values.  (The real transpose's factor ps, common to every term here since all
// orders are > 0, is applied to the final sums.)
template <bool REAL>
__global__ void __launch_bounds__(kPolarThreads, 2) k_polar_patch(
    const float2 *__restrict__ a, const float2 *__restrict__ b, const float2 *__restrict__ tab,
    const int *__restrict__ plim, float *__restrict__ polS, int L, int K, int jc, int muc,
    const long long *__restrict__ coff, int B, float ps)
{
    extern __shared__ float4 pol_sm[];
    typedef float2 CoefStep[kPolarChunk][4][32];                 // [degree][a+, a-, b+, b-][lane]
    typedef float2 TabStep[kPolarPairs][kPolarJ][kPolarChunk][32];   // [warp][ring][degree][lane]
    CoefStep *csb = reinterpret_cast<CoefStep *>(pol_sm);
    TabStep *tsb = reinterpret_cast<TabStep *>(reinterpret_cast<unsigned char *>(pol_sm) + 2 * kPolarCoefBytes);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int mu0 = blockIdx.x * 32;
    const int mu = mu0 + lane;
    const int f = blockIdx.y;
    const int jb = blockIdx.z * kPolarPairs * kPolarJ;
    const int je = jb + kPolarPairs * kPolarJ < jc ? jb + kPolarPairs * kPolarJ : jc;
    if (mu0 >= __ldg(plim + je - 1)) return;   // uniform: the last ring has the largest bound
    const int j0 = jb + warp * kPolarJ;
    const int nring = j0 < jc ? (jc - j0 < kPolarJ ? jc - j0 : kPolarJ) : 0;
    const bool wact = nring > 0 && mu0 < __ldg(plim + j0 + nring - 1);
    const bool active = mu >= 1 && mu <= L && mu < muc;
    const bool has1 = !REAL || 2 * f + 1 < B;       // the pair's second field exists
    // coefficient offsets: field f (complex), or the pair's fields 2f and 2f+1 (real)
    const size_t cb = REAL ? (coff ? (size_t)coff[2 * f] : (size_t)(2 * f) * K)
                           : (coff ? (size_t)coff[f] : (size_t)f * K);
    const size_t cb1 = (REAL && has1) ? (coff ? (size_t)coff[2 * f + 1] : (size_t)(2 * f + 1) * K) : cb;
    const int nstep = (L + 1 - mu0 + kPolarChunk - 1) / kPolarChunk;

    // one step's copies: coefficient element e = (degree e / 128, kind (e / 32) % 4, lane
    // e % 32), zero outside the coefficient triangle; the warp's table rows (ring, degree)
    // as 16 chunks of 16 bytes each (rows of degrees beyond L are left as they are: unused)
    auto load_step = [&](int st) {
        CoefStep &cs = csb[st & 1];
        for (int e = threadIdx.x; e < kPolarCoef; e += kPolarThreads) {
            const int i = e & 31, q = (e >> 5) & 3, d = e >> 7;
            const int m = mu0 + i, l = mu0 + st * kPolarChunk + d;
            const float2 *src = a;
            int nb = 0;
            if (m >= 1 && m < muc && l >= m && l <= L) {
                if (REAL) {
                    if (!(q & 1) || has1) {
                        src = ((q & 2) ? b : a) + ((q & 1) ? cb1 : cb) + (size_t)l * (l + 1) / 2 - 1 + m;
                        nb = 8;
                    }
                } else {
                    const size_t c0 = cb + (size_t)l * l + l - 1;
                    src = ((q & 2) ? b : a) + ((q & 1) ? c0 - m : c0 + m);
                    nb = 8;
                }
            }
            cp_async8(&cs[d][q][i], src, nb);
        }
        if (wact) {
            float2(*ts)[kPolarChunk][32] = tsb[st & 1][warp];
#pragma unroll
            for (int u = 0; u < kPolarJ * kPolarChunk / 2; ++u) {
                const int c = u * 32 + lane;                         // chunk: row c / 16, part c % 16
                const int r = c >> 4, part = c & 15, q = r / kPolarChunk, d = r % kPolarChunk;
                const int l = mu0 + st * kPolarChunk + d;
                if (q < nring && l <= L)
                    cp_async16(&ts[q][d][part * 2], tab + ((size_t)(j0 + q) * (L + 1) + l) * muc + mu0 + part * 2);
            }
        }
        cp_async_commit();
    };
    float sum[kPolarJ][2][8], cmp[kPolarJ][2][8];
#pragma unroll
    for (int q = 0; q < kPolarJ; ++q)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int c = 0; c < 8; ++c) sum[q][k][c] = cmp[q][k][c] = 0.f;
    const float w = (float)mu;

    load_step(0);
    for (int st = 0; st < nstep; ++st) {
        if (st + 1 < nstep) {
            load_step(st + 1);                       // in flight during this step's sums
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();                             // every thread's copies of step st landed
        const CoefStep &cs = csb[st & 1];
        const float2(*ts)[kPolarChunk][32] = tsb[st & 1][warp];
        const int lb = mu0 + st * kPolarChunk;       // even: mu0 and kPolarChunk are
        if (wact) {
            float acc[kPolarJ][2][8];
#pragma unroll
            for (int q = 0; q < kPolarJ; ++q)
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[q][k][c] = 0.f;
#pragma unroll
            for (int d = 0; d < kPolarChunk; ++d) {
                if (lb + d > L) break;
                const float2 ap = cs[d][0][lane], am = cs[d][1][lane];
                const float2 bp = cs[d][2][lane], bm = cs[d][3][lane];
                const int kd = (d & 1) ? 0 : 1, kl = (d & 1) ? 1 : 0;   // banks of the D and Lambda terms
#pragma unroll
                for (int q = 0; q < kPolarJ; ++q) {
                    if (q >= nring) break;
                    const float2 t = ts[q][d][lane];
                    const float D = t.x, wl = w * t.y;
                    const float wl1 = REAL ? wl : -wl;      // m of slot 1: +mu (real) or -mu
                    float *ad = acc[q][kd], *al = acc[q][kl];
                    ad[0] = fmaf(ap.x, D, ad[0]);
                    ad[1] = fmaf(ap.y, D, ad[1]);
                    ad[2] = fmaf(am.x, D, ad[2]);
                    ad[3] = fmaf(am.y, D, ad[3]);
                    ad[4] = fmaf(bp.x, D, ad[4]);
                    ad[5] = fmaf(bp.y, D, ad[5]);
                    ad[6] = fmaf(bm.x, D, ad[6]);
                    ad[7] = fmaf(bm.y, D, ad[7]);
                    // theta: -i m b Lambda ; phi: +i m a Lambda  (m = +mu for s = 0, -mu for s = 1)
                    al[0] = fmaf(wl, bp.y, al[0]);
                    al[1] = fmaf(-wl, bp.x, al[1]);
                    al[2] = fmaf(wl1, bm.y, al[2]);
                    al[3] = fmaf(-wl1, bm.x, al[3]);
                    al[4] = fmaf(-wl, ap.y, al[4]);
                    al[5] = fmaf(wl, ap.x, al[5]);
                    al[6] = fmaf(-wl1, am.y, al[6]);
                    al[7] = fmaf(wl1, am.x, al[7]);
                }
            }
#pragma unroll
            for (int q = 0; q < kPolarJ; ++q)
#pragma unroll
                for (int k = 0; k < 2; ++k)
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const float y = acc[q][k][c] - cmp[q][k][c];
                        const float t = sum[q][k][c] + y;
                        cmp[q][k][c] = (t - sum[q][k][c]) - y;
                        sum[q][k][c] = t;
                    }
        }
        __syncthreads();                             // before step st + 2 refills these buffers
    }
    if (!wact || !active) return;
#pragma unroll
    for (int q = 0; q < kPolarJ; ++q) {
        if (q >= nring) break;
        const int j = j0 + q;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            float v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                v[c] = sum[q][k][c] - cmp[q][k][c];
                if (REAL) v[c] *= ps;                // real transpose: every order here is > 0
            }
            const int par = k ^ (mu & 1);
            const float sg = (!REAL && (mu & 1)) ? -1.f : 1.f;     // columns of m = -mu
            float4 *dst = reinterpret_cast<float4 *>(polS + ((((size_t)f * jc + j) * muc + mu) * 2 + par) * 8);
            dst[0] = make_float4(v[0], v[1], sg * v[2], sg * v[3]);
            dst[1] = make_float4(v[4], v[5], sg * v[6], sg * v[7]);
        }
    }
}

}  // namespace

// Host: ring and order ranges, and the FP64 tables D_l, Lambda_l of every patched
// (ring, order) pair from the normalised three-term recurrence
//   lambda_mu^mu = (-1)^mu c_mu sin^mu(theta),
//   lambda_{l+1} = (cos(theta) lambda_l - eps_l lambda_{l-1}) / eps_{l+1},
// run on a mantissa with a separate binary exponent so that the polar starting values
// (far below the double range at high order) stay exact.
int build_polar_tables(Plan &p)
{
    const int L = p.L;
    int jc = 0;
    while (jc < p.J - (p.has_eq ? 1 : 0)) {
        const double x = p.h_x[jc];
        if (std::sqrt((1.0 - x) * (1.0 + x)) >= kPolarSin) break;
        ++jc;
    }
    int muc = (int)std::ceil(1.5 * (L + 1) * kPolarSin) + 16;
    muc = (muc + 31) / 32 * 32;
    const int mumax = (L + 1 + 31) / 32 * 32;
    if (muc > mumax) muc = mumax;
    p.pol_jc = jc;
    p.pol_muc = muc;
    if (jc == 0) return FAVEST_OK;

    std::vector<float2> tab((size_t)jc * (L + 1) * muc, make_float2(0.f, 0.f));
    std::vector<double> eps(L + 3), lam(L + 3);
    double cmu = 1.0 / std::sqrt(4.0 * 3.14159265358979323846);
    for (int mu = 1; mu < muc && mu <= L; ++mu) {
        cmu *= std::sqrt((2.0 * mu + 1.0) / (2.0 * mu));
        for (int l = mu; l <= L + 2; ++l) eps[l] = eps_pl(l, mu);
        for (int j = 0; j < jc; ++j) {
            const double x = p.h_x[j], s = std::sqrt((1.0 - x) * (1.0 + x));
            // start: (-1)^mu cmu s^mu as y * 2^e
            double y = (mu & 1) ? -cmu : cmu;
            int e = 0;
            for (int k = 0; k < mu; ++k) {
                int ex;
                y = std::frexp(y * s, &ex);
                e += ex;
            }
            double ym = 0.0;   // lambda_{l-1}
            lam[mu - 1] = 0.0;
            lam[mu] = std::ldexp(y, e);
            for (int l = mu; l <= L; ++l) {
                const double yn = (x * y - eps[l] * ym) / eps[l + 1];
                ym = y;
                y = yn;
                if (std::fabs(y) > 0x1p200) {
                    y *= 0x1p-200;
                    ym *= 0x1p-200;
                    e += 200;
                }
                lam[l + 1] = std::ldexp(y, e);
            }
            for (int l = mu; l <= L; ++l) {
                const double sl = 1.0 / std::sqrt((double)l * (l + 1.0));
                const double D = sl * (l * eps[l + 1] * lam[l + 1] - (l + 1.0) * eps[l] * lam[l - 1]);
                tab[((size_t)j * (L + 1) + l) * muc + mu] = make_float2((float)D, (float)(sl * lam[l]));
            }
        }
    }
    // per ring the first order whose tensor-core values it keeps (beyond its turning-point
    // bound); the inverse DFT takes the patched sums of ring j for the orders 1 <= mu < muc
    // whose tile of 32 starts below the bound of the last ring of j's warp pair (j | 1)
    std::vector<int> lim(jc);
    for (int j = 0; j < jc; ++j) {
        const double x = p.h_x[j];
        lim[j] = (int)std::ceil(1.5 * (L + 1) * std::sqrt((1.0 - x) * (1.0 + x))) + 16;
    }
    const size_t sbytes = (size_t)p.ncg * jc * muc * 16 * sizeof(float);
    if (plan_malloc((void **)&p.d_pol, tab.size() * sizeof(float2)) != cudaSuccess ||
        plan_malloc((void **)&p.d_pol_lim, lim.size() * sizeof(int)) != cudaSuccess ||
        plan_malloc((void **)&p.d_polS, sbytes) != cudaSuccess) {
        cudaGetLastError();
        return FAVEST_ENOMEM;
    }
    if (cudaMemcpy(p.d_pol_lim, lim.data(), lim.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p.d_polS, 0, sbytes) != cudaSuccess)
        return FAVEST_ECUDA;
    if (cudaStreamCreateWithFlags(&p.pol_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p.pol_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p.pol_join, cudaEventDisableTiming) != cudaSuccess)
        return FAVEST_ECUDA;
    if (cudaMemcpy(p.d_pol, tab.data(), tab.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess)
        return FAVEST_ECUDA;
    return FAVEST_OK;
}

cudaError_t launch_polar_patch(const Plan &p, const void *a, const void *b, cudaStream_t s)
{
    const int K = p.real ? p.L * (p.L + 3) / 2 : p.L * p.L + 2 * p.L;
    dim3 grid(p.pol_muc / 32, p.ncg, (p.pol_jc + kPolarPairs * kPolarJ - 1) / (kPolarPairs * kPolarJ));
    auto k = p.real ? k_polar_patch<true> : k_polar_patch<false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kPolarSmem);
    k<<<grid, kPolarThreads, kPolarSmem, s>>>((const float2 *)a, (const float2 *)b, p.d_pol, p.d_pol_lim, p.d_polS,
                                        p.L, K, p.pol_jc, p.pol_muc, p.d_coff, p.B, p.real_transpose ? 0.5f : 1.f);
    return cudaGetLastError();
}

}  // namespace favest
