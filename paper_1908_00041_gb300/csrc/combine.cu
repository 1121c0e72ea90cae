// O(L^2) coefficient-side stages.
//   combine   (forward): scalar sums Q_theta, Q_phi (degrees |m|..L+1) -> a_lm, b_lm
//   uncombine (adjoint): a_lm, b_lm -> scaled scalar coefficients g_theta, g_phi
// Both use the per-(l, mu) coefficients P, M, R (with the recurrence scaling kappa
// folded in), which make uncombine the exact transpose of combine:
//   a = P_l Qt(l+1) - M_l Qt(l-1) - i m R_l Qp(l)
//   b = i m R_l Qt(l) + P_l Qp(l+1) - M_l Qp(l-1)
//   gt(l') = P_{l'-1} a(l'-1) - M_{l'+1} a(l'+1) - i m R_{l'} b(l')
//   gp(l') = i m R_{l'} a(l') + P_{l'-1} b(l'-1) - M_{l'+1} b(l'+1)
// For m < 0 the Legendre stage uses lambda^{|m|}; lambda^{-mu} = (-1)^mu lambda^{mu}
// supplies the sign.
#include "favest_internal.h"
#include "fft_device.cuh"

namespace favest {

namespace {

template <typename TO>
__global__ void k_combine_fp64(const double2 *__restrict__ Q, TO *__restrict__ a, TO *__restrict__ b,
                               const double *__restrict__ P, const double *__restrict__ M,
                               const double *__restrict__ R, int L, int K, int ncol, int B,
                               const long long *__restrict__ coff)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * K) return;
    const int bi = (int)(t / K), k = (int)(t % K);
    int l = (int)sqrt((double)(k + 1));
    while (l * l + 2 * l < k + 1) ++l;
    while ((l - 1) * (l - 1) + 2 * (l - 1) >= k + 1) --l;
    const int m = k - l * l - l + 1;
    const int mu = m < 0 ? -m : m, s = m < 0;
    const double sg = (s && (mu & 1)) ? -1.0 : 1.0;
    const long long t0 = tab_off(L, mu);
    const long long row = t0 + (l - mu);
    const int cth = (bi * 2 + 0) * 2 + s, cph = (bi * 2 + 1) * 2 + s;
    const double Pl = P[row], Ml = M[row], Rl = R[row] * m;
    double2 qt1 = Q[(size_t)(row + 1) * ncol + cth], qp1 = Q[(size_t)(row + 1) * ncol + cph];
    double2 qt0 = Q[(size_t)row * ncol + cth], qp0 = Q[(size_t)row * ncol + cph];
    double2 qtm = make_double2(0.0, 0.0), qpm = make_double2(0.0, 0.0);
    if (l > mu) {
        qtm = Q[(size_t)(row - 1) * ncol + cth];
        qpm = Q[(size_t)(row - 1) * ncol + cph];
    }
    // -i m R Qp = (m R Qp.y, -m R Qp.x);  i m R Qt = (-m R Qt.y, m R Qt.x)
    double2 av = make_double2(sg * (Pl * qt1.x - Ml * qtm.x + Rl * qp0.y),
                              sg * (Pl * qt1.y - Ml * qtm.y - Rl * qp0.x));
    double2 bv = make_double2(sg * (-Rl * qt0.y + Pl * qp1.x - Ml * qpm.x),
                              sg * (Rl * qt0.x + Pl * qp1.y - Ml * qpm.y));
    const size_t cb = coff ? (size_t)coff[bi] : (size_t)bi * K;
    a[cb + k] = from_d2<TO>(av);
    b[cb + k] = from_d2<TO>(bv);
}

template <typename TI>
__device__ __forceinline__ double2 coef(const TI *__restrict__ c, int L, int l, int m, size_t cb)
{
    int am = m < 0 ? -m : m;
    if (l < 1 || l > L || am > l) return make_double2(0.0, 0.0);
    return to_d2(c[cb + l * l + l + m - 1]);
}

// grid.x = mu, grid.y = b*2 + s; threads stride over rows l' = mu..L+1
template <typename TI>
__global__ void k_uncombine_fp64(const TI *__restrict__ a, const TI *__restrict__ b,
                                 double2 *__restrict__ g, const double *__restrict__ P,
                                 const double *__restrict__ M, const double *__restrict__ R, int L,
                                 int K, int ncol, const long long *__restrict__ coff)
{
    const int mu = blockIdx.x;
    const int bi = blockIdx.y >> 1, s = blockIdx.y & 1;
    const int m = s ? -mu : mu;
    const double sg = (s && (mu & 1)) ? -1.0 : 1.0;
    const long long t0 = tab_off(L, mu);
    const int nrow = L + 2 - mu;
    const int cth = (bi * 2 + 0) * 2 + s, cph = (bi * 2 + 1) * 2 + s;
    const size_t cb = coff ? (size_t)coff[bi] : (size_t)bi * K;
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
        const int l = mu + r;
        double2 gt = make_double2(0.0, 0.0), gp = make_double2(0.0, 0.0);
        if (!(mu == 0 && s == 1)) {
            const double Pm = (r > 0) ? P[t0 + r - 1] : 0.0;
            const double Mp = (l + 1 <= L) ? M[t0 + r + 1] : 0.0;
            const double Rl = (l <= L) ? R[t0 + r] * m : 0.0;
            double2 am1 = coef(a, L, l - 1, m, cb), ap1 = coef(a, L, l + 1, m, cb);
            double2 bm1 = coef(b, L, l - 1, m, cb), bp1 = coef(b, L, l + 1, m, cb);
            double2 a0 = coef(a, L, l, m, cb), b0 = coef(b, L, l, m, cb);
            gt = make_double2(sg * (Pm * am1.x - Mp * ap1.x + Rl * b0.y),
                              sg * (Pm * am1.y - Mp * ap1.y - Rl * b0.x));
            gp = make_double2(sg * (-Rl * a0.y + Pm * bm1.x - Mp * bp1.x),
                              sg * (Rl * a0.x + Pm * bm1.y - Mp * bp1.y));
        }
        g[(size_t)(t0 + r) * ncol + cth] = gt;
        g[(size_t)(t0 + r) * ncol + cph] = gp;
    }
}

// Real fields: half-spectrum coefficients (m >= 0, index l(l+1)/2 - 1 + m of a field's
// KR = L(L+3)/2); field bf = 2q + f uses the columns (q*2 + c)*2 + f at m = +mu.
template <typename TO>
__global__ void k_combine_fp64_real(const double2 *__restrict__ Q, TO *__restrict__ a, TO *__restrict__ b,
                                    const double *__restrict__ P, const double *__restrict__ M,
                                    const double *__restrict__ R, int L, int KR, int ncol, int B, double ps,
                                    const long long *__restrict__ coff)
{
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * KR) return;
    const int bf = (int)(t / KR), k = (int)(t % KR);
    // k = l(l+1)/2 - 1 + m with 0 <= m <= l
    int l = (int)((sqrt(8.0 * (k + 1) + 1.0) - 1.0) / 2.0);
    while ((l + 1) * (l + 2) / 2 - 1 <= k) ++l;
    while (l * (l + 1) / 2 - 1 > k) --l;
    const int mu = k - (l * (l + 1) / 2 - 1);
    const long long row = tab_off(L, mu) + (l - mu);
    const int q = bf >> 1, f = bf & 1;
    const int cth = (q * 2 + 0) * 2 + f, cph = (q * 2 + 1) * 2 + f;
    const double Pl = P[row], Ml = M[row], Rl = R[row] * mu;
    double2 qt1 = Q[(size_t)(row + 1) * ncol + cth], qp1 = Q[(size_t)(row + 1) * ncol + cph];
    double2 qt0 = Q[(size_t)row * ncol + cth], qp0 = Q[(size_t)row * ncol + cph];
    double2 qtm = make_double2(0.0, 0.0), qpm = make_double2(0.0, 0.0);
    if (l > mu) {
        qtm = Q[(size_t)(row - 1) * ncol + cth];
        qpm = Q[(size_t)(row - 1) * ncol + cph];
    }
    double2 av = make_double2(Pl * qt1.x - Ml * qtm.x + Rl * qp0.y, Pl * qt1.y - Ml * qtm.y - Rl * qp0.x);
    double2 bv = make_double2(-Rl * qt0.y + Pl * qp1.x - Ml * qpm.x, Rl * qt0.x + Pl * qp1.y - Ml * qpm.y);
    const double sc = mu > 0 ? ps : 1.0;   // real transpose: orders m > 0 doubled
    const size_t cb = coff ? (size_t)coff[bf] : (size_t)bf * KR;
    a[cb + k] = from_d2<TO>(make_double2(sc * av.x, sc * av.y));
    b[cb + k] = from_d2<TO>(make_double2(sc * bv.x, sc * bv.y));
}

template <typename TI>
__device__ __forceinline__ double2 coef_half(const TI *__restrict__ c, int L, int l, int mu, size_t cb)
{
    if (l < 1 || l > L || mu > l) return make_double2(0.0, 0.0);
    return to_d2(c[cb + l * (l + 1) / 2 - 1 + mu]);
}

// grid.x = mu, grid.y = real field; threads stride over rows l' = mu..L+1
template <typename TI>
__global__ void k_uncombine_fp64_real(const TI *__restrict__ a, const TI *__restrict__ b, double2 *__restrict__ g,
                                      const double *__restrict__ P, const double *__restrict__ M,
                                      const double *__restrict__ R, int L, int KR, int ncol, double ps,
                                      const long long *__restrict__ coff)
{
    const int mu = blockIdx.x, bf = blockIdx.y;
    const long long t0 = tab_off(L, mu);
    const int nrow = L + 2 - mu;
    const int q = bf >> 1, f = bf & 1;
    const int cth = (q * 2 + 0) * 2 + f, cph = (q * 2 + 1) * 2 + f;
    const size_t cb = coff ? (size_t)coff[bf] : (size_t)bf * KR;
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) {
        const int l = mu + r;
        const double Pm = (r > 0) ? P[t0 + r - 1] : 0.0;
        const double Mp = (l + 1 <= L) ? M[t0 + r + 1] : 0.0;
        const double Rl = (l <= L) ? R[t0 + r] * mu : 0.0;
        double2 am1 = coef_half(a, L, l - 1, mu, cb), ap1 = coef_half(a, L, l + 1, mu, cb);
        double2 bm1 = coef_half(b, L, l - 1, mu, cb), bp1 = coef_half(b, L, l + 1, mu, cb);
        double2 a0 = coef_half(a, L, l, mu, cb), b0 = coef_half(b, L, l, mu, cb);
        const double sc = mu > 0 ? ps : 1.0;   // real transpose: orders m > 0 halved
        g[(size_t)(t0 + r) * ncol + cth] = make_double2(sc * (Pm * am1.x - Mp * ap1.x + Rl * b0.y),
                                                        sc * (Pm * am1.y - Mp * ap1.y - Rl * b0.x));
        g[(size_t)(t0 + r) * ncol + cph] = make_double2(sc * (-Rl * a0.y + Pm * bm1.x - Mp * bp1.x),
                                                        sc * (Rl * a0.x + Pm * bm1.y - Mp * bp1.y));
    }
}

}  // namespace

cudaError_t launch_combine_fp64(const Plan &p, void *a, void *b, cudaStream_t s)
{
    if (p.real) {
        const int KR = p.L * (p.L + 3) / 2;
        const long long n = (long long)p.B * KR;
        const unsigned grid = (unsigned)((n + 255) / 256);
        if (p.io == FAVEST_IO_R64)
            k_combine_fp64_real<double2><<<grid, 256, 0, s>>>((const double2 *)p.d_Q, (double2 *)a, (double2 *)b,
                                                             p.d_P, p.d_M, p.d_R, p.L, KR, p.ncol, p.B,
                                                             p.real_transpose ? 2.0 : 1.0, p.d_coff);
        else
            k_combine_fp64_real<float2><<<grid, 256, 0, s>>>((const double2 *)p.d_Q, (float2 *)a, (float2 *)b,
                                                            p.d_P, p.d_M, p.d_R, p.L, KR, p.ncol, p.B,
                                                            p.real_transpose ? 2.0 : 1.0, p.d_coff);
        return cudaGetLastError();
    }
    const int K = p.L * p.L + 2 * p.L;
    long long n = (long long)p.B * K;
    int th = 256;
    long long grid = (n + th - 1) / th;
    if (p.io == FAVEST_IO_C128)
        k_combine_fp64<double2><<<(unsigned)grid, th, 0, s>>>((const double2 *)p.d_Q, (double2 *)a,
                                                              (double2 *)b, p.d_P, p.d_M, p.d_R, p.L, K,
                                                              p.ncol, p.B, p.d_coff);
    else
        k_combine_fp64<float2><<<(unsigned)grid, th, 0, s>>>((const double2 *)p.d_Q, (float2 *)a,
                                                             (float2 *)b, p.d_P, p.d_M, p.d_R, p.L, K,
                                                             p.ncol, p.B, p.d_coff);
    return cudaGetLastError();
}

cudaError_t launch_uncombine_fp64(const Plan &p, const void *a, const void *b, cudaStream_t s)
{
    if (p.real) {
        const int KR = p.L * (p.L + 3) / 2;
        dim3 grid(p.L + 1, p.B);
        const int th = p.L + 2 >= 256 ? 256 : 64;
        if (p.io == FAVEST_IO_R64)
            k_uncombine_fp64_real<double2><<<grid, th, 0, s>>>((const double2 *)a, (const double2 *)b,
                                                               (double2 *)p.d_Q, p.d_P, p.d_M, p.d_R, p.L, KR,
                                                               p.ncol, p.real_transpose ? 0.5 : 1.0, p.d_coff);
        else
            k_uncombine_fp64_real<float2><<<grid, th, 0, s>>>((const float2 *)a, (const float2 *)b,
                                                              (double2 *)p.d_Q, p.d_P, p.d_M, p.d_R, p.L, KR,
                                                              p.ncol, p.real_transpose ? 0.5 : 1.0, p.d_coff);
        return cudaGetLastError();
    }
    const int K = p.L * p.L + 2 * p.L;
    dim3 grid(p.L + 1, p.B * 2);
    int th = p.L + 2 >= 256 ? 256 : 64;
    if (p.io == FAVEST_IO_C128)
        k_uncombine_fp64<double2><<<grid, th, 0, s>>>((const double2 *)a, (const double2 *)b,
                                                      (double2 *)p.d_Q, p.d_P, p.d_M, p.d_R, p.L, K,
                                                      p.ncol, p.d_coff);
    else
        k_uncombine_fp64<float2><<<grid, th, 0, s>>>((const float2 *)a, (const float2 *)b,
                                                     (double2 *)p.d_Q, p.d_P, p.d_M, p.d_R, p.L, K,
                                                     p.ncol, p.d_coff);
    return cudaGetLastError();
}

}  // namespace favest
