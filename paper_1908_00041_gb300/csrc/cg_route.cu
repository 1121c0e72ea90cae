// The paper's Clebsch-Gordan route on the FP64 path (Sec. 4, Thm. 1 and Thm. 2): vector
// transforms of fields given by their Cartesian components T^(1), T^(2), T^(3), through
// scalar spherical harmonic transforms of degree L+1.
//
// The scalar transforms run on the FP64 kernels in scalar mode: scalar field s = 3f + c
// (component c of vector field f) occupies the column pair (s, sign of m) of the sums
//   Q[row (l, mu)][2 s + (m < 0)] = sum_j y_l^mu(theta_j) w_j F_s(j, m),   l = mu..L+1,
// with the plain point weights w_j and the scaled recurrence values y = lambda / kappa, so
//   F_lm(T^(c)) = kappa_l^mu Q[.][2 s] (m >= 0),  (-1)^mu kappa_l^mu Q[.][2 s + 1] (m < 0)
// (lambda_l^{-mu} = (-1)^mu lambda_l^mu).  The synthesis reads the same layout.
//
// Forward (Thm. 1, eq. almblmviaFlm).  Every xi/mu factor of the theorem at its shifted
// index is a product of c_l, d_l (eq. cl,dl,betal) and a Clebsch-Gordan value of the
// OUTPUT index (l, m) (eq. Blm1/Blm2), e.g. xi^(1)_{l-1,m-1} = c_l C^{l,m}_{l-1,m-1,1,1}:
//   a_lm = 1/sqrt2 [ c_l C0 Fm(l-1, m-1) + d_l C1 Fm(l+1, m-1) + c_l C4 Fp(l-1, m+1)
//                  + d_l C5 Fp(l+1, m+1) ] + c_l C2 F3(l-1, m) + d_l C3 F3(l+1, m),
//   b_lm = -i/sqrt2 [ C6 Fm(l, m-1) + C7 Fp(l, m+1) ] - i C8 F3(l, m),
// with Fm = -F(T1) + i F(T2), Fp = F(T1) + i F(T2), F3 = F(T3), Ck = C_k(l, m) below, and
// F(l', m') = 0 unless |m'| <= l' <= L+1.
//
// Adjoint (Thm. 2, eq. SLvecviascal).  Since S_K is linear and zero-padding a sequence
// beyond degree K leaves S_K unchanged, the three syntheses of each component are one
// synthesis of degree L+1 of the summed coefficients
//   g1 = -(nu1 + nu2 + eta1)/sqrt2,  g2 = -(nu3 + nu4 - eta2)/sqrt2,  g3 = nu5 + nu6 + eta3
// (eqs. nulm1, nulm2, etalm), with a, b read as zero outside 1 <= l <= L, |m| <= l and
// every nu evaluated for all |m| <= l (the reading of their garbled support conditions).
#include <cmath>

#include "favest_internal.h"

namespace favest {

namespace {

// The nine Clebsch-Gordan closed forms of eq. ninecoeff for the coupled state (l, m):
//   0: C^{l,m}_{l-1,m-1,1,1}  1: C^{l,m}_{l+1,m-1,1,1}  2: C^{l,m}_{l-1,m,1,0}
//   3: C^{l,m}_{l+1,m,1,0}    4: C^{l,m}_{l-1,m+1,1,-1} 5: C^{l,m}_{l+1,m+1,1,-1}
//   6: C^{l,m}_{l,m-1,1,1}    7: C^{l,m}_{l,m+1,1,-1}   8: C^{l,m}_{l,m,1,0}
// Callers use a value only where its uncoupled state (l', m') exists, with l >= 1.
__device__ double clebsch(int k, int l, int m)
{
    const double L = l, M = m;
    double num, den, sg = 1.0;
    switch (k) {
    case 0: num = (L + M) * (L + M - 1.0); den = (2.0 * L) * (2.0 * L - 1.0); break;
    case 1: num = (L - M + 1.0) * (L - M + 2.0); den = (2.0 * L + 2.0) * (2.0 * L + 3.0); break;
    case 2: num = (L + M) * (L - M); den = L * (2.0 * L - 1.0); break;
    case 3: num = (L - M + 1.0) * (L + M + 1.0); den = (2.0 * L + 3.0) * (L + 1.0); sg = -1.0; break;
    case 4: num = (L - M) * (L - M - 1.0); den = (2.0 * L) * (2.0 * L - 1.0); break;
    case 5: num = (L + M + 1.0) * (L + M + 2.0); den = (2.0 * L + 3.0) * (2.0 * L + 2.0); break;
    case 6: num = (L + M) * (L - M + 1.0); den = L * (2.0 * L + 2.0); sg = -1.0; break;
    case 7: num = (L + M + 1.0) * (L - M); den = L * (2.0 * L + 2.0); break;
    default: return M / sqrt(L * (L + 1.0));
    }
    return num > 0.0 ? sg * sqrt(num / den) : 0.0;
}

__device__ __forceinline__ double cl_of(int l) { return sqrt((l + 1.0) / (2.0 * l + 1.0)); }
__device__ __forceinline__ double dl_of(int l) { return sqrt(l / (2.0 * l + 1.0)); }

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }   // i a

// FwdSHT F_{l,m} of scalar field s from the scaled sums; 0 outside |m| <= l <= L+1
__device__ __forceinline__ double2 fsht(const double2 *__restrict__ Q, const double *__restrict__ kap, int L,
                                        int ncol, int s, int l, int m)
{
    const int mu = m < 0 ? -m : m;
    if (l < 0 || l > L + 1 || mu > l) return make_double2(0.0, 0.0);
    const long long row = tab_off(L, mu) + (l - mu);
    const double k = kap[row] * ((m < 0 && (mu & 1)) ? -1.0 : 1.0);
    return cscale(k, Q[row * ncol + 2 * s + (m < 0)]);
}

// one thread per (field, coefficient (l, m), l = 1..L)
__global__ void k_cg_combine(const double2 *__restrict__ Q, const double *__restrict__ kap, double2 *__restrict__ a,
                             double2 *__restrict__ b, int L, int K, int ncol, int B)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * K) return;
    const int f = (int)(t / K), k = (int)(t % K);
    int l = (int)sqrt((double)(k + 1));
    while (l * l + 2 * l < k + 1) ++l;
    while ((l - 1) * (l - 1) + 2 * (l - 1) >= k + 1) --l;
    const int m = k - l * l - l + 1;
    const int s1 = 3 * f, s2 = s1 + 1, s3 = s1 + 2;
    auto Fm = [&](int ll, int mm) {          // -F(T1) + i F(T2)
        const double2 x = fsht(Q, kap, L, ncol, s1, ll, mm), y = fsht(Q, kap, L, ncol, s2, ll, mm);
        return make_double2(-x.x - y.y, -x.y + y.x);
    };
    auto Fp = [&](int ll, int mm) {          // F(T1) + i F(T2)
        const double2 x = fsht(Q, kap, L, ncol, s1, ll, mm), y = fsht(Q, kap, L, ncol, s2, ll, mm);
        return make_double2(x.x - y.y, x.y + y.x);
    };
    const double cl = cl_of(l), dl = dl_of(l), r2 = 0.70710678118654752440;
    double2 sum = cscale(cl * clebsch(0, l, m), Fm(l - 1, m - 1));
    sum = cadd(sum, cscale(dl * clebsch(1, l, m), Fm(l + 1, m - 1)));
    sum = cadd(sum, cscale(cl * clebsch(4, l, m), Fp(l - 1, m + 1)));
    sum = cadd(sum, cscale(dl * clebsch(5, l, m), Fp(l + 1, m + 1)));
    double2 av = cscale(r2, sum);
    av = cadd(av, cscale(cl * clebsch(2, l, m), fsht(Q, kap, L, ncol, s3, l - 1, m)));
    av = cadd(av, cscale(dl * clebsch(3, l, m), fsht(Q, kap, L, ncol, s3, l + 1, m)));
    double2 t2 = cscale(clebsch(6, l, m), Fm(l, m - 1));
    t2 = cadd(t2, cscale(clebsch(7, l, m), Fp(l, m + 1)));
    // b = -i/sqrt2 t2 - i C8 F3
    const double2 bv = cadd(cscale(-r2, cmuli(t2)), cscale(-clebsch(8, l, m), cmuli(fsht(Q, kap, L, ncol, s3, l, m))));
    a[(size_t)f * K + k] = av;
    b[(size_t)f * K + k] = bv;
}

__device__ __forceinline__ double2 coef(const double2 *__restrict__ c, int L, int K, int f, int l, int m)
{
    if (l < 1 || l > L || m < -l || m > l) return make_double2(0.0, 0.0);
    return c[(size_t)f * K + l * l + l + m - 1];
}

// one thread per (field, scalar coefficient (l, m), l = 0..L+1)
__global__ void k_cg_uncombine(const double2 *__restrict__ a, const double2 *__restrict__ b,
                               const double *__restrict__ kap, double2 *__restrict__ Q, int L, int K, int ncol, int B)
{
    const int n = (L + 2) * (L + 2);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)B * n) return;
    const int f = (int)(t / n), idx = (int)(t % n);
    int l = (int)sqrt((double)idx);
    while (l * l > idx) --l;
    while ((l + 1) * (l + 1) <= idx) ++l;
    const int m = idx - l * l - l;
    const double2 z = make_double2(0.0, 0.0);
    // a and b terms where the coefficient exists (the CG value of its coupled state)
    const double2 ap1p = coef(a, L, K, f, l + 1, m + 1), ap1m = coef(a, L, K, f, l + 1, m - 1);
    const double2 am1p = coef(a, L, K, f, l - 1, m + 1), am1m = coef(a, L, K, f, l - 1, m - 1);
    const double2 ap10 = coef(a, L, K, f, l + 1, m), am10 = coef(a, L, K, f, l - 1, m);
    const double2 bp = coef(b, L, K, f, l, m + 1), bm = coef(b, L, K, f, l, m - 1), b0 = coef(b, L, K, f, l, m);
    const double c1 = cl_of(l + 1), d1 = l >= 2 ? dl_of(l - 1) : 0.0;
    const double2 u1 = (l + 1 <= L && m + 1 <= l + 1) ? cscale(clebsch(0, l + 1, m + 1), ap1p) : z;
    const double2 v1 = (l + 1 <= L && m - 1 >= -(l + 1)) ? cscale(clebsch(4, l + 1, m - 1), ap1m) : z;
    const double2 u2 = (l >= 2 && m + 1 <= l - 1) ? cscale(clebsch(1, l - 1, m + 1), am1p) : z;
    const double2 v2 = (l >= 2 && m - 1 >= -(l - 1)) ? cscale(clebsch(5, l - 1, m - 1), am1m) : z;
    const double2 w5 = (l + 1 <= L) ? cscale(c1 * clebsch(2, l + 1, m), ap10) : z;
    const double2 w6 = (l >= 2 && m >= -(l - 1) && m <= l - 1) ? cscale(d1 * clebsch(3, l - 1, m), am10) : z;
    const double2 e6 = (l >= 1 && m + 1 <= l) ? cscale(clebsch(6, l, m + 1), bp) : z;
    const double2 e7 = (l >= 1 && m - 1 >= -l) ? cscale(clebsch(7, l, m - 1), bm) : z;
    const double2 e8 = (l >= 1) ? cscale(clebsch(8, l, m), b0) : z;
    // nu1 = c (u1 - v1), nu2 = d (u2 - v2), nu3 = i c (u1 + v1), nu4 = i d (u2 + v2)
    const double2 nu1 = cscale(c1, make_double2(u1.x - v1.x, u1.y - v1.y));
    const double2 nu2 = cscale(d1, make_double2(u2.x - v2.x, u2.y - v2.y));
    const double2 nu3 = cmuli(cscale(c1, cadd(u1, v1)));
    const double2 nu4 = cmuli(cscale(d1, cadd(u2, v2)));
    // eta1 = i (e6 - e7), eta2 = e6 + e7, eta3 = i e8
    const double2 eta1 = cmuli(make_double2(e6.x - e7.x, e6.y - e7.y));
    const double2 eta2 = cadd(e6, e7);
    const double2 eta3 = cmuli(e8);
    const double r2 = 0.70710678118654752440;
    const double2 g1 = cscale(-r2, cadd(cadd(nu1, nu2), eta1));
    const double2 g2 = cscale(-r2, make_double2(nu3.x + nu4.x - eta2.x, nu3.y + nu4.y - eta2.y));
    const double2 g3 = cadd(cadd(w5, w6), eta3);
    const int mu = m < 0 ? -m : m;
    const long long row = tab_off(L, mu) + (l - mu);
    const double kk = kap[row] * ((m < 0 && (mu & 1)) ? -1.0 : 1.0);
    const double2 g[3] = {g1, g2, g3};
#pragma unroll
    for (int c = 0; c < 3; ++c) Q[row * ncol + 2 * (3 * f + c) + (m < 0)] = cscale(kk, g[c]);
}

// ---------------------------------------------------------------------------------------
// Stability ratios of the forward route (Sec. 5.5, eq. r_stable).  Thm. 1 writes
// Y^div_lm(x)^* as six terms xi_q Y*_{l',m'}(x) u_q and Y^curl_lm(x)^* as three terms, with the
// constant vectors u_- = (-1, i, 0)/sqrt2 (orders m-1), u_+ = (1, i, 0)/sqrt2 (orders m+1) and
// e_3 (order m).  All terms of one sum carry the same phase e^{-i m phi} (e^{-i(m-/+1) phi} of
// the scalar harmonic times the e^{+/-i phi} that u_-/+ contributes to e_theta and e_phi), so the
// sizes depend on theta alone and are taken at phi = 0, where Y_{l',m'} = lambda_{l'}^{m'} is
// real (lambda^{-mu} = (-1)^mu lambda^mu, one sign per order).  With
//   A = xi1 lambda_{l-1}^{m-1} + xi2 lambda_{l+1}^{m-1},  C = xi3 lambda_{l-1}^{m+1} + xi4 lambda_{l+1}^{m+1},
//   E = xi5 lambda_{l-1}^m + xi6 lambda_{l+1}^m,
// the T^(1), T^(2), T^(3) weights are (C - A)/sqrt2, i (A + C)/sqrt2, E, so
//   |Y^div_lm|^2 = A^2 + C^2 + E^2,    Vhat = sqrt2 (sum of the six |xi_q lambda_q|),
// and with P = mu1 lambda_l^{m-1}, Q = mu3 lambda_l^{m+1}, R = mu2 lambda_l^m
//   |Y^curl_lm|^2 = P^2 + Q^2 + R^2,   Vtilde = sqrt2 (|P| + |Q| + |R|).
// rho = size / V (a point where V = 0 has no ratio).  Both ratios are invariant under a
// common scale of the three orders' lambda columns, which the kernel exploits below.
//
// One thread per (point, order mu): the orders b, b+1, b+2 with b = max(mu-1, 0) cover
// m = +mu (orders mu-1, mu, mu+1), m = -mu (the same three, mirrored) and, for mu = 0, m = 0
// (orders 1, 0, 1).  The three columns run the normalised three-term recurrence in lockstep
// over the degree n = b..L+1 from starts lambda_o^o / sin(theta)^b = c_o sin^(o-b) (the
// common factor sin^b removed so nothing underflows near the poles); whenever the newest
// values pass 2^400 all columns are scaled by 2^-400 together.  After degree n the window
// holds degrees n-2, n-1, n and the thread forms the ratios of l = n-1.  The extremes over
// the points are reduced per warp and merged with 64-bit atomics on the bit patterns, which
// order like the values for non-negative doubles.

constexpr int kStabThreads = 256;

__device__ __forceinline__ double sel3(int j, double a0, double a1, double a2)
{
    return j == 0 ? a0 : (j == 1 ? a1 : a2);
}

__device__ __forceinline__ void warp_maxmin(double &mx, double &mn)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    }
}

__global__ void k_stability_init(double *ext, int K)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    ext[i] = 0.0;
    ext[K + i] = __longlong_as_double(0x7ff0000000000000LL);
    ext[2 * K + i] = 0.0;
    ext[3 * K + i] = __longlong_as_double(0x7ff0000000000000LL);
}

// ext: [4][K] = max rho_hat, min rho_hat, max rho_tilde, min rho_tilde per coefficient
__global__ void __launch_bounds__(kStabThreads) k_stability(const double *__restrict__ z, int npts, int L, int K,
                                                           double *ext)
{
    const int k = blockIdx.x * kStabThreads + threadIdx.x;
    const bool live = k < npts;                      // dead lanes follow the loop (warp shuffles)
    const double x = live ? z[k] : 0.0;
    const double s = sqrt((1.0 - x) * (1.0 + x));
    const int mu = blockIdx.y, b = mu > 0 ? mu - 1 : 0;
    const double r2 = 1.4142135623730951;

    // c_o = |lambda_o^o| / sin^o = sqrt((2o+1)/(4 pi) (2o-1)!!/(2o)!!)
    double cb = 0.28209479177387814;                 // 1/sqrt(4 pi)
    for (int o = 1; o <= b; ++o) cb *= sqrt((2.0 * o + 1.0) / (2.0 * o));
    const double start[3] = {cb, cb * sqrt((2.0 * b + 3.0) / (2.0 * b + 2.0)) * s,
                             cb * sqrt((2.0 * b + 3.0) / (2.0 * b + 2.0)) * sqrt((2.0 * b + 5.0) / (2.0 * b + 4.0)) * s * s};
    double w0[3] = {0.0, 0.0, 0.0}, w1[3] = {0.0, 0.0, 0.0}, w2[3] = {0.0, 0.0, 0.0};   // degrees n-2, n-1, n
    double eprev[3] = {0.0, 0.0, 0.0};               // eps_{n-1}^o of the previous step
    for (int n = b; n <= L + 1; ++n) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int o = b + j;
            w0[j] = w1[j];
            w1[j] = w2[j];
            double v = 0.0;
            if (n == o) {
                v = start[j];
            } else if (n == o + 1) {
                v = sqrt(2.0 * o + 3.0) * x * w1[j];
                eprev[j] = 1.0 / sqrt(2.0 * o + 3.0);                        // eps_{o+1}^o
            } else if (n > o + 1) {
                const double e = sqrt(((double)n * n - (double)o * o) / (4.0 * n * n - 1.0));   // eps_n^o
                v = (x * w1[j] - eprev[j] * w0[j]) / e;
                eprev[j] = e;
            }
            w2[j] = v;
        }
        const int l = n - 1;
        if (l >= 1 && l >= mu && l <= L) {
            const double cl = cl_of(l), dl = dl_of(l);
            for (int sg = 0; sg < (mu > 0 ? 2 : 1); ++sg) {
                const int m = sg ? -mu : mu;
                // columns of the orders |m-1|, |m|, |m+1|
                const int jm = mu == 0 ? 1 : (sg ? 2 : 0), j0 = mu == 0 ? 0 : 1, jp = mu == 0 ? 1 : (sg ? 0 : 2);
                const double t1 = cl * clebsch(0, l, m) * sel3(jm, w0[0], w0[1], w0[2]);
                const double t2 = dl * clebsch(1, l, m) * sel3(jm, w2[0], w2[1], w2[2]);
                const double t3 = cl * clebsch(4, l, m) * sel3(jp, w0[0], w0[1], w0[2]);
                const double t4 = dl * clebsch(5, l, m) * sel3(jp, w2[0], w2[1], w2[2]);
                const double t5 = cl * clebsch(2, l, m) * sel3(j0, w0[0], w0[1], w0[2]);
                const double t6 = dl * clebsch(3, l, m) * sel3(j0, w2[0], w2[1], w2[2]);
                const double A = t1 + t2, C = t3 + t4, E = t5 + t6;
                const double vh = r2 * (fabs(t1) + fabs(t2) + fabs(t3) + fabs(t4) + fabs(t5) + fabs(t6));
                const double P = clebsch(6, l, m) * sel3(jm, w1[0], w1[1], w1[2]);
                const double Q = clebsch(7, l, m) * sel3(jp, w1[0], w1[1], w1[2]);
                const double R = clebsch(8, l, m) * sel3(j0, w1[0], w1[1], w1[2]);
                const double vt = r2 * (fabs(P) + fabs(Q) + fabs(R));
                const double inf = __longlong_as_double(0x7ff0000000000000LL);
                double hmx = 0.0, hmn = inf, tmx = 0.0, tmn = inf;
                if (live && vh > 0.0) hmx = hmn = sqrt(A * A + C * C + E * E) / vh;
                if (live && vt > 0.0) tmx = tmn = sqrt(P * P + Q * Q + R * R) / vt;
                warp_maxmin(hmx, hmn);
                warp_maxmin(tmx, tmn);
                if ((threadIdx.x & 31) == 0) {
                    unsigned long long *e = reinterpret_cast<unsigned long long *>(ext);
                    const int i = l * l + l + m - 1;
                    atomicMax(e + i, (unsigned long long)__double_as_longlong(hmx));
                    atomicMin(e + K + i, (unsigned long long)__double_as_longlong(hmn));
                    atomicMax(e + 2 * K + i, (unsigned long long)__double_as_longlong(tmx));
                    atomicMin(e + 3 * K + i, (unsigned long long)__double_as_longlong(tmn));
                }
            }
        }
        if (n >= b + 2) {
            double big = 0.0;
#pragma unroll
            for (int j = 0; j < 3; ++j) big = fmax(big, fmax(fabs(w1[j]), fabs(w2[j])));
            if (big > 0x1p400) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    w1[j] *= 0x1p-400;
                    w2[j] *= 0x1p-400;
                }
            }
        }
    }
}

// r[4] = r_hat, kappa_hat, r_tilde, kappa_tilde over l <= L, 1 <= |m| <= l; one block
__global__ void __launch_bounds__(kStabThreads) k_stability_reduce(const double *__restrict__ ext, int K, double *r)
{
    const double inf = __longlong_as_double(0x7ff0000000000000LL);
    double hmx = 0.0, hmn = inf, tmx = 0.0, tmn = inf;
    for (int i = threadIdx.x; i < K; i += kStabThreads) {
        int l = (int)sqrt((double)(i + 1));
        while (l * l + 2 * l < i + 1) ++l;
        while ((l - 1) * (l - 1) + 2 * (l - 1) >= i + 1) --l;
        if (i - l * l - l + 1 == 0) continue;        // m = 0 is outside eq. r_stable
        hmx = fmax(hmx, ext[i]);
        hmn = fmin(hmn, ext[K + i]);
        tmx = fmax(tmx, ext[2 * K + i]);
        tmn = fmin(tmn, ext[3 * K + i]);
    }
    warp_maxmin(hmx, hmn);
    warp_maxmin(tmx, tmn);
    __shared__ double sh[4][kStabThreads / 32];
    const int wid = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[0][wid] = hmx;
        sh[1][wid] = hmn;
        sh[2][wid] = tmx;
        sh[3][wid] = tmn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kStabThreads / 32; ++w) {
            hmx = fmax(hmx, sh[0][w]);
            hmn = fmin(hmn, sh[1][w]);
            tmx = fmax(tmx, sh[2][w]);
            tmn = fmin(tmn, sh[3][w]);
        }
        r[0] = hmx;
        r[1] = 1.0 / hmn;
        r[2] = tmx;
        r[3] = 1.0 / tmn;
    }
}

// ---------------------------------------------------------------------------------------
// Real fields on the Clebsch-Gordan route.  Real vector fields A = field 2q and B = field
// 2q+1 are transformed as the complex field z = A + i B.  The transforms are linear and
// the coefficients of a real field are Hermitian, alpha_{l,-m} = (-1)^m conj(alpha_lm)
// (the header's real-field relation), so those of z, c = alpha + i beta, separate as
//   alpha_lm = (c_lm + (-1)^m conj c_{l,-m}) / 2,  beta_lm = (c_lm - (-1)^m conj c_{l,-m}) / (2i),
// and conversely c_lm = alpha_lm + i beta_lm, c_{l,-m} = (-1)^m (conj alpha_lm + i conj beta_lm)
// for m >= 0; the synthesis of c is A + i B.  Half spectra: index l(l+1)/2 - 1 + m, m >= 0.

// one thread per (pair q, component plane element): z = A + i B (B = 0 past the last field)
__global__ void k_cg_pack_fields(const double *__restrict__ Tr, double2 *__restrict__ Tc, long long plane, int nreal,
                                 int npair)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)npair * 3 * plane) return;
    const int q = (int)(t / (3 * plane));
    const long long r = t - (long long)q * 3 * plane;          // component * plane + point
    const double A = Tr[(long long)(2 * q) * 3 * plane + r];
    const double B = 2 * q + 1 < nreal ? Tr[(long long)(2 * q + 1) * 3 * plane + r] : 0.0;
    Tc[t] = make_double2(A, B);
}

__global__ void k_cg_unpack_fields(const double2 *__restrict__ Tc, double *__restrict__ Tr, long long plane, int nreal,
                                   int npair)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)npair * 3 * plane) return;
    const int q = (int)(t / (3 * plane));
    const long long r = t - (long long)q * 3 * plane;
    const double2 z = Tc[t];
    Tr[(long long)(2 * q) * 3 * plane + r] = z.x;
    if (2 * q + 1 < nreal) Tr[(long long)(2 * q + 1) * 3 * plane + r] = z.y;
}

__device__ __forceinline__ void half_lm(int h, int &l, int &m)
{
    l = (int)((sqrt(8.0 * (h + 1) + 1.0) - 1.0) * 0.5);
    while (l * (l + 1) / 2 - 1 > h) --l;
    while ((l + 1) * (l + 2) / 2 - 1 <= h) ++l;
    m = h - (l * (l + 1) / 2 - 1);
}

// one thread per (pair q, half-spectrum index (l, m >= 0)), both families
__global__ void k_cg_unpack_coefs(const double2 *__restrict__ ac, const double2 *__restrict__ bc,
                                  double2 *__restrict__ ah, double2 *__restrict__ bh, int L, int nreal, int npair)
{
    const int K = L * L + 2 * L, H = L * (L + 3) / 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)npair * H) return;
    const int q = (int)(t / H), h = (int)(t % H);
    int l, m;
    half_lm(h, l, m);
    const double sg = (m & 1) ? -1.0 : 1.0;
    const long long ip = (long long)q * K + l * l + l + m - 1, im = (long long)q * K + l * l + l - m - 1;
    const double2 *src[2] = {ac, bc};
    double2 *dst[2] = {ah, bh};
#pragma unroll
    for (int fam = 0; fam < 2; ++fam) {
        const double2 cp = src[fam][ip], cm = src[fam][im];
        const double2 w = make_double2(sg * cm.x, -sg * cm.y);      // (-1)^m conj c_{l,-m}
        dst[fam][(long long)(2 * q) * H + h] = make_double2(0.5 * (cp.x + w.x), 0.5 * (cp.y + w.y));
        // (c - w) / (2i) = -i (c - w) / 2
        if (2 * q + 1 < nreal)
            dst[fam][(long long)(2 * q + 1) * H + h] = make_double2(0.5 * (cp.y - w.y), -0.5 * (cp.x - w.x));
    }
}

__global__ void k_cg_pack_coefs(const double2 *__restrict__ ah, const double2 *__restrict__ bh,
                                double2 *__restrict__ ac, double2 *__restrict__ bc, int L, int nreal, int npair)
{
    const int K = L * L + 2 * L, H = L * (L + 3) / 2;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)npair * H) return;
    const int q = (int)(t / H), h = (int)(t % H);
    int l, m;
    half_lm(h, l, m);
    const double sg = (m & 1) ? -1.0 : 1.0;
    const long long ip = (long long)q * K + l * l + l + m - 1, im = (long long)q * K + l * l + l - m - 1;
    const double2 *src[2] = {ah, bh};
    double2 *dst[2] = {ac, bc};
#pragma unroll
    for (int fam = 0; fam < 2; ++fam) {
        const double2 al = src[fam][(long long)(2 * q) * H + h];
        const double2 be = 2 * q + 1 < nreal ? src[fam][(long long)(2 * q + 1) * H + h] : make_double2(0.0, 0.0);
        dst[fam][ip] = make_double2(al.x - be.y, al.y + be.x);                  // alpha + i beta
        if (m > 0)                                                            // (-1)^m (conj alpha + i conj beta)
            dst[fam][im] = make_double2(sg * (al.x + be.y), sg * (be.x - al.y));
    }
}

}  // namespace

cudaError_t launch_cg_combine(const Plan &p, void *a, void *b, cudaStream_t s)
{
    const int K = p.L * p.L + 2 * p.L;
    const long long n = (long long)p.B * K;
    k_cg_combine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2 *)p.d_Q, p.d_kap, (double2 *)a,
                                                           (double2 *)b, p.L, K, p.ncol, p.B);
    return cudaGetLastError();
}

cudaError_t launch_cg_uncombine(const Plan &p, const void *a, const void *b, cudaStream_t s)
{
    const int K = p.L * p.L + 2 * p.L;
    const long long n = (long long)p.B * (p.L + 2) * (p.L + 2);
    k_cg_uncombine<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2 *)a, (const double2 *)b, p.d_kap,
                                                             (double2 *)p.d_Q, p.L, K, p.ncol, p.B);
    return cudaGetLastError();
}

cudaError_t launch_cg_pack_fields(const Plan &p, const void *Tr, cudaStream_t s)
{
    const long long plane = (long long)p.nlat * p.nphi, n = (long long)p.B * 3 * plane;
    k_cg_pack_fields<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double *)Tr, (double2 *)p.d_cgT, plane,
                                                               p.cg_real, p.B);
    return cudaGetLastError();
}

cudaError_t launch_cg_unpack_fields(const Plan &p, void *Tr, cudaStream_t s)
{
    const long long plane = (long long)p.nlat * p.nphi, n = (long long)p.B * 3 * plane;
    k_cg_unpack_fields<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2 *)p.d_cgT, (double *)Tr, plane,
                                                                 p.cg_real, p.B);
    return cudaGetLastError();
}

cudaError_t launch_cg_pack_coefs(const Plan &p, const void *a, const void *b, cudaStream_t s)
{
    const long long n = (long long)p.B * (p.L * (p.L + 3) / 2);
    k_cg_pack_coefs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2 *)a, (const double2 *)b,
                                                              (double2 *)p.d_cga, (double2 *)p.d_cgb, p.L, p.cg_real,
                                                              p.B);
    return cudaGetLastError();
}

cudaError_t launch_cg_unpack_coefs(const Plan &p, void *a, void *b, cudaStream_t s)
{
    const long long n = (long long)p.B * (p.L * (p.L + 3) / 2);
    k_cg_unpack_coefs<<<(unsigned)((n + 255) / 256), 256, 0, s>>>((const double2 *)p.d_cga, (const double2 *)p.d_cgb,
                                                                (double2 *)a, (double2 *)b, p.L, p.cg_real, p.B);
    return cudaGetLastError();
}

}  // namespace favest

extern "C" int favest_cg_stability(int L, int npts, const double *cos_theta, double *per_coef, double *ratios,
                                   void *stream)
{
    using namespace favest;
    if (L < 1 || L > 1023 || npts < 1 || npts > (1 << 28) || !cos_theta || !ratios) return FAVEST_EINVAL;
    for (int k = 0; k < npts; ++k)
        if (!(fabs(cos_theta[k]) < 1.0)) return FAVEST_EINVAL;    // also rejects NaN
    const int K = L * L + 2 * L;
    const size_t nz = (size_t)npts, bytes = (nz + 4 * (size_t)K + 4) * sizeof(double);
    double *d = nullptr;
    if (plan_malloc((void **)&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        return FAVEST_ENOMEM;
    }
    double *dz = d, *dext = d + nz, *dr = dext + 4 * (size_t)K;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t err = cudaMemcpyAsync(dz, cos_theta, nz * sizeof(double), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) {
        k_stability_init<<<(K + kStabThreads - 1) / kStabThreads, kStabThreads, 0, s>>>(dext, K);
        k_stability<<<dim3((unsigned)((npts + kStabThreads - 1) / kStabThreads), (unsigned)(L + 1)), kStabThreads, 0,
                      s>>>(dz, npts, L, K, dext);
        k_stability_reduce<<<1, kStabThreads, 0, s>>>(dext, K, dr);
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpyAsync(ratios, dr, 4 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess && per_coef)
        err = cudaMemcpyAsync(per_coef, dext, 4 * (size_t)K * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    cudaFree(d);
    return err == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
}
