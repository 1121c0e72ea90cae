// C ABI of the favest library: plan construction (host FP64 tables), argument
// validation and launch sequencing.  See include/favest.h for the contract.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <atomic>
#include <cstring>
#include <string>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "favest_internal.h"

using namespace favest;


namespace {

const char *kErrStr[] = {
    "success",
    "invalid argument",
    "out of memory",
    "CUDA runtime error",
    "unsupported request",
    "device-side wait timed out",
    "device-side error",
    "index table bounds check failed",
};

// ---------------------------------------------------------------------------
// Gauss-Legendre rule: Newton's method on P_n from Tricomi's asymptotic initial
// guess; P_n and P_n' by the three-term recurrence and (1-x^2) P_n' = n (P_{n-1} - x P_n).
// ---------------------------------------------------------------------------
void legendre_pn(int n, double x, double &pn, double &dpn)
{
    double pm1 = 1.0, p = x;
    if (n == 0) { pn = 1.0; dpn = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        double pp1 = ((2 * k + 1) * x * p - k * pm1) / (k + 1);
        pm1 = p;
        p = pp1;
    }
    pn = p;
    dpn = n * (pm1 - x * p) / ((1.0 - x) * (1.0 + x));
}

int gl_rule(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        // Tricomi: x_i ~ (1 - (n-1)/(8 n^3)) cos(pi (4i + 3) / (4n + 2))
        double t = pi * (4.0 * i + 3.0) / (4.0 * n + 2.0);
        double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(t);
        double pn = 0, dpn = 1;
        for (int it = 0; it < 60; ++it) {
            legendre_pn(n, z, pn, dpn);
            double dz = pn / dpn;
            z -= dz;
            if (std::fabs(dz) <= 4e-17 * std::fabs(z) + 1e-300) break;
        }
        legendre_pn(n, z, pn, dpn);
        double wt = 2.0 / ((1.0 - z) * (1.0 + z) * dpn * dpn);
        x[i] = z;
        w[i] = wt;
        x[n - 1 - i] = -z;
        w[n - 1 - i] = wt;
    }
    if (n & 1) x[n / 2] = 0.0;
    return FAVEST_OK;
}

double eps_lm(int l, int mu)
{
    double num = (double)(l - mu) * (double)(l + mu);
    double den = (double)(2 * l - 1) * (double)(2 * l + 1);
    return num > 0 ? std::sqrt(num / den) : 0.0;
}

int factorize(int n, int *rad)
{
    int k = 0;
    while (n % 4 == 0 && k < kMaxRadixStages) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < kMaxRadixStages) { rad[k++] = 2; n /= 2; }
    for (int f = 3; n > 1 && k < kMaxRadixStages; f += 2)
        while (n % f == 0 && k < kMaxRadixStages) { rad[k++] = f; n /= f; }
    return n == 1 ? k : -1;
}

template <typename T>
cudaError_t dalloc(T **p, size_t count)
{
    *p = nullptr;
    if (count == 0) return cudaSuccess;
    return plan_malloc((void **)p, count * sizeof(T));
}

template <typename T>
cudaError_t upload(T **p, const std::vector<T> &h)
{
    cudaError_t e = dalloc(p, h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_plan(Plan &p)
{
    void *ptrs[] = {p.d_x, p.d_sin, p.d_omega, p.d_omega_unit, p.d_cmu, p.d_A, p.d_P, p.d_M, p.d_R,
                    p.d_status, p.d_F, p.d_Q, p.d_G, p.fft.tw64, p.fft.tw32, p.d_lam, p.d_Fb, p.d_gb,
                    p.d_jcmin, p.d_omega32, p.d_omega_unit32, p.d_isc32, p.d_kap,
                    p.d_Q32, p.d_S32, p.d_lam_rb, p.d_g_off, p.d_items_f, p.d_items_a,
                    p.d_P32, p.d_M32, p.d_R32, p.d_k1, p.d_perm, p.d_pol, p.d_wring, p.d_ggroups,
                    p.fft.blue_chirp, p.fft.blue_spec, p.fft.blue_tw, p.d_cgT, p.d_cga, p.d_cgb, p.d_Adf, p.d_xdf,
                    p.d_pol_lim, p.d_polS};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (p.pol_fork) cudaEventDestroy(p.pol_fork);
    if (p.pol_join) cudaEventDestroy(p.pol_join);
    if (p.pol_stream) cudaStreamDestroy(p.pol_stream);
    std::free(p.h_x);
    std::free(p.h_w);
}

// In-place radix-2 FFT of M = 2^lg points, FP64, exp(-2 pi i / M) (host; natural order).
void host_fft_pow2(std::vector<double2> &v, int lg)
{
    const int M = 1 << lg;
    for (int i = 1, j = 0; i < M; ++i) {              // bit reversal
        int bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(v[i], v[j]);
    }
    for (int len = 2; len <= M; len <<= 1) {
        for (int i = 0; i < M; i += len) {
            for (int k = 0; k < len / 2; ++k) {
                const long double ang = -2.0L * 3.141592653589793238462643383279502884L * k / len;
                const double c = (double)cosl(ang), sn = (double)sinl(ang);
                const double2 a = v[i + k], b = v[i + k + len / 2];
                const double2 t = make_double2(b.x * c - b.y * sn, b.x * sn + b.y * c);
                v[i + k] = make_double2(a.x + t.x, a.y + t.y);
                v[i + k + len / 2] = make_double2(a.x - t.x, a.y - t.y);
            }
        }
    }
}

// Tables of the FP32 DFT's Bluestein stages, one per prime radix R >= 17 (the radices the
// in-register butterflies do not cover): chirp c_t = exp(-i pi t^2 / R) from the exactly
// reduced t^2 mod 2R, the spectrum of its conjugate zero-padded to M = 2^lg >= 2R - 1 (FP64,
// scaled by 1/M; natural order for the radix-16 engine, M <= 4096, bit-reversed for the radix-2
// passes used at M = 8192), and the M-point twiddles.  P butterflies of a stage run per round
// in a scratch of up to 32 KB (at least one butterfly), which with the DFT buffer of 4 rings
// must fit one CTA's shared memory.
int build_bluestein(Plan &p)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<float2> chirp, spec, twm;
    size_t scratch = 0;
    for (int st = 0; st < p.fft.nstages; ++st) {
        const int R = p.fft.radix[st];
        p.fft.blue_lg[st] = 0;
        if (R < 17) continue;
        int lg = 1;
        while ((1 << lg) < 2 * R - 1) ++lg;
        if (lg < 5) lg = 5;
        if (lg > 13) return FAVEST_EUNSUPPORTED;
        const int M = 1 << lg;
        const size_t pts = lg <= 12 ? (size_t)M + M / 16 : (size_t)M;   // padded for the engine
        const int nbf4 = 4 * (p.nphi / R);
        int P = (int)(32768 / (8 * pts));
        if (P < 1) P = 1;
        if (P > nbf4) P = nbf4;
        scratch = std::max(scratch, (size_t)8 * pts * P);
        p.fft.blue_lg[st] = lg;
        p.fft.blue_P[st] = P;
        p.fft.blue_off[st] = (int)chirp.size();
        p.fft.blue_moff[st] = (int)spec.size();
        std::vector<double2> b(M, make_double2(0.0, 0.0));
        for (int t = 0; t < R; ++t) {
            const long long q = ((long long)t * t) % (2LL * R);
            const long double ang = -pi * (long double)q / (long double)R;
            const double c = (double)cosl(ang), sn = (double)sinl(ang);
            chirp.push_back(make_float2((float)c, (float)sn));
            b[t] = make_double2(c, -sn);                          // conj(c_t)
            if (t > 0) b[M - t] = make_double2(c, -sn);
        }
        host_fft_pow2(b, lg);
        for (int i = 0; i < M; ++i) {
            int r = i;
            if (lg > 12) {
                r = 0;
                for (int k = 0; k < lg; ++k) r |= ((i >> k) & 1) << (lg - 1 - k);
            }
            spec.push_back(make_float2((float)(b[r].x / M), (float)(b[r].y / M)));
        }
        for (int k = 0; k < M; ++k) {
            const long double ang = -2.0L * pi * k / M;
            twm.push_back(make_float2((float)cosl(ang), (float)sinl(ang)));
        }
    }
    if (chirp.empty()) return FAVEST_OK;
    const size_t ring_bytes = (size_t)32 * p.nphi;
    if (ring_bytes + std::max(scratch, (size_t)24576) > 227 * 1024) return FAVEST_EUNSUPPORTED;
    cudaError_t e;
    if ((e = upload(&p.fft.blue_chirp, chirp)) || (e = upload(&p.fft.blue_spec, spec)) ||
        (e = upload(&p.fft.blue_tw, twm)))
        return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    p.fft.blue_scratch = scratch;
    return FAVEST_OK;
}

std::atomic<long long> g_alloc_calls{0};
std::atomic<long long> g_alloc_fail_at{-1};

int build_tables(Plan &p)
{
    const int L = p.L;
    const int J = p.J;
    cudaError_t e;
    std::vector<double> x(J), s(J), om(J), omu(J);
    for (int j = 0; j < J; ++j) {
        double xj = p.h_x[j];
        double sj = std::sqrt((1.0 - xj) * (1.0 + xj));
        x[j] = xj;
        s[j] = sj;
        om[j] = p.h_w[j] * (2.0 * 3.14159265358979323846 / p.nphi) / sj;
        omu[j] = 1.0 / sj;
    }
    std::vector<double> wring(p.nlat);
    for (int j = 0; j < p.nlat; ++j) wring[j] = p.h_w[j] * (2.0 * 3.14159265358979323846 / p.nphi);
    if ((e = upload(&p.d_x, x)) || (e = upload(&p.d_sin, s)) || (e = upload(&p.d_omega, om)) ||
        (e = upload(&p.d_omega_unit, omu)) || (e = upload(&p.d_wring, wring)))
        return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;

    std::vector<double> cmu(L + 2);
    cmu[0] = 1.0 / std::sqrt(4.0 * 3.14159265358979323846);
    for (int mu = 1; mu <= L + 1; ++mu) cmu[mu] = cmu[mu - 1] * std::sqrt((2.0 * mu + 1.0) / (2.0 * mu));

    // orders 0..L (0..L+1 for the degree-(L+1) scalar transforms of the CG route)
    const int mumax = L + (p.nscal > 0 ? 1 : 0);
    const long long ntab = tab_off(L, mumax + 1);
    p.ntab = ntab;
    std::vector<double> A(ntab), P(ntab), M(ntab), R(ntab), kap(L + 3), K(ntab);
    for (int mu = 0; mu <= mumax; ++mu) {
        const long long t0 = tab_off(L, mu);
        // kappa_l = lambda_l / y_l with kappa_mu = kappa_{mu+1} = 1
        kap[mu] = 1.0;
        if (mu + 1 <= L + 2) kap[mu + 1] = 1.0;
        for (int l = mu + 2; l <= L + 2; ++l) kap[l] = kap[l - 2] * eps_lm(l - 1, mu) / eps_lm(l, mu);
        for (int l = mu; l <= L + 1; ++l) {
            const long long t = t0 + (l - mu);
            double a = 0.0;
            if (l == mu + 1) a = std::sqrt(2.0 * mu + 3.0);
            else if (l >= mu + 2) a = kap[l - 1] / (eps_lm(l - 1, mu) * kap[l - 2]);
            A[t] = a;
            const double sl = l >= 1 ? 1.0 / std::sqrt((double)l * (l + 1.0)) : 0.0;
            P[t] = sl * l * eps_lm(l + 1, mu) * kap[l + 1];
            M[t] = (l > mu) ? sl * (l + 1.0) * eps_lm(l, mu) * kap[l - 1] : 0.0;
            R[t] = sl * kap[l];
            K[t] = kap[l];
        }
    }
    if ((e = upload(&p.d_cmu, cmu)) || (e = upload(&p.d_A, A)) || (e = upload(&p.d_P, P)) ||
        (e = upload(&p.d_M, M)) || (e = upload(&p.d_R, R)))
        return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    if (p.nscal > 0 && (e = upload(&p.d_kap, K))) return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    if (p.precision == FAVEST_BF16X6) {
        std::vector<float> P32(ntab), M32(ntab), R32(ntab), k1(L + 1, 0.f);
        for (long long t = 0; t < ntab; ++t) {
            P32[t] = (float)P[t];
            M32[t] = (float)M[t];
            R32[t] = (float)R[t];
        }
        for (int l = 1; l <= L; ++l) k1[l] = (float)(R[tab_off(L, 1) + (l - 1)] * std::sqrt((double)l * (l + 1.0)));
        std::vector<float> om32(J), omu32(J);
        std::vector<float2> isc(2 * J);
        for (int j = 0; j < J; ++j) {
            om32[j] = (float)om[j];
            omu32[j] = (float)omu[j];
            isc[j] = make_float2((float)(1.0 / s[j]), 1.0f);
            isc[J + j] = make_float2((float)(wring[j] / s[j]), (float)wring[j]);
        }
        // the generator's double-float operands: hi = the nearest float, lo = the nearest float
        // to the remainder (together about 48 bits of the FP64 value)
        std::vector<float2> Adf(ntab), xdf(J);
        for (long long t = 0; t < ntab; ++t) {
            const float h = (float)A[t];
            Adf[t] = make_float2(h, (float)(A[t] - (double)h));
        }
        for (int j = 0; j < J; ++j) {
            const float h = (float)x[j];
            xdf[j] = make_float2(h, (float)(x[j] - (double)h));
        }
        if ((e = upload(&p.d_Adf, Adf)) || (e = upload(&p.d_xdf, xdf)))
            return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
        if ((e = upload(&p.d_P32, P32)) || (e = upload(&p.d_M32, M32)) || (e = upload(&p.d_R32, R32)) ||
            (e = upload(&p.d_k1, k1)) || (e = upload(&p.d_omega32, om32)) ||
            (e = upload(&p.d_omega_unit32, omu32)) || (e = upload(&p.d_isc32, isc)))
            return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    }

    // FFT twiddles exp(-2 pi i k / n), angles reduced exactly
    const int n = p.nphi;
    p.fft.n = n;
    p.fft.nstages = factorize(n, p.fft.radix);
    if (p.fft.nstages < 0) return FAVEST_EUNSUPPORTED;
    if (p.precision == FAVEST_BF16X6) {
        const int st = build_bluestein(p);
        if (st != FAVEST_OK) return st;
    }
    std::vector<double2> tw(n);
    std::vector<float2> tw32(n);
    for (int k = 0; k < n; ++k) {
        long double ang = 2.0L * 3.141592653589793238462643383279502884L * (long double)k / (long double)n;
        double cr = (double)cosl(ang), ci = -(double)sinl(ang);
        tw[k] = make_double2(cr, ci);
        tw32[k] = make_float2((float)cr, (float)ci);
    }
    // Power-of-two lengths (the split path's radix-16 engine) append the twiddles of its two
    // radix-16 stages in [q][k] order, q < 16: at block length n, w^(q k) for k < n/16, at
    // n/16, w^(16 q k) for k < n/256; a warp's threads (consecutive k) then read consecutive
    // entries instead of entries q apart.  Values are those of tw32, copied.
    if (p.precision == FAVEST_BF16X6 && n >= 64 && n <= 4096 && (n & (n - 1)) == 0) {
        const int hA = n / 16, hB = n / 256;
        tw32.resize((size_t)n + 16 * hA + 16 * hB);
        for (int q = 0; q < 16; ++q) {
            for (int k = 0; k < hA; ++k) tw32[(size_t)n + q * hA + k] = tw32[q * k];
            for (int k = 0; k < hB; ++k) tw32[(size_t)n + 16 * hA + q * hB + k] = tw32[16 * q * k];
        }
    }
    // Other lengths of the split path: the same [q][k] order per mixed-radix stage (radices
    // 2, 4 and the odd primes up to 13; Bluestein stages keep reading the plain table).
    if (p.precision == FAVEST_BF16X6 && !(n >= 64 && n <= 4096 && (n & (n - 1)) == 0)) {
        int Nb = n;
        for (int st = 0; st < p.fft.nstages; ++st) {
            const int R = p.fft.radix[st], h = Nb / R, ts = n / Nb;
            p.fft.tw_off[st] = -1;
            if (R <= 13 && !p.fft.blue_lg[st]) {
                p.fft.tw_off[st] = (int)tw32.size();
                for (int q = 0; q < R; ++q)
                    for (int k = 0; k < h; ++k) {
                        const float2 w = tw32[(size_t)q * k * ts];   // q k ts < R h ts = n
                        tw32.push_back(w);
                    }
            }
            Nb = h;
        }
    }
    if ((e = upload(&p.fft.tw64, tw)) || (e = upload(&p.fft.tw32, tw32)))
        return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    // in-place decimation-in-frequency FFT leaves frequency m at position pos(m):
    //   pos(m; n, r0 r1 ..) = (m mod r0) * (n / r0) + pos(m div r0; n / r0, r1 ..)
    // The split path transforms power-of-two lengths 2^6..2^11 with its own radix-16
    // engine (natural order in and out); other lengths use the mixed-radix list and perm.
    p.fft_log2n = 0;
    if (p.precision == FAVEST_BF16X6 && n >= 64 && n <= 4096 && (n & (n - 1)) == 0)
        while ((1 << p.fft_log2n) < n) ++p.fft_log2n;
    std::vector<int> perm(n);
    for (int m = 0; m < n; ++m) {
        int pos = 0, len = n, mm = m;
        for (int st = 0; st < p.fft.nstages; ++st) {
            const int r = p.fft.radix[st];
            len /= r;
            pos += (mm % r) * len;
            mm /= r;
        }
        perm[m] = pos;
    }
    if ((e = upload(&p.d_perm, perm)))
        return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    return FAVEST_OK;
}

// Tensor map of the forward B operand Fb[j/8][field][j%8][mu][parity][8] (FP32 records of
// 64 bytes): a box {8, 1, 8, N/8, 4} at (x0 = parity*8, mu, 0, (N/8)*field_tile, 4*K_chunk)
// lands in shared memory as [K/8][N/8][8 j][8 n] floats, the element order of the MN-major
// core-matrix layout that the GEMM's converter warps then write as three bf16 pieces.
int make_fb_tensor_map(Plan &p)
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return FAVEST_EUNSUPPORTED;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t L1 = (cuuint64_t)(p.L + 1);
    cuuint64_t dims[5] = {16, L1, 8, (cuuint64_t)p.nf, (cuuint64_t)(p.JP / 8)};
    cuuint64_t strides[4] = {64, 64 * L1, 512 * L1, 512 * L1 * (cuuint64_t)p.nf};
    cuuint32_t box[5] = {8, 1, 8, (cuuint32_t)(p.gemm_n / 8), (cuuint32_t)(kGemmChunkK / 8)};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = encode(&p.tmap_fb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, p.d_Fb, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FAVEST_OK : FAVEST_EUNSUPPORTED;
}

// Tensor map of the adjoint GEMM output S32[group][JP/4][L+1][parity][4][8] (fp32) as the
// inverse DFT reads it: dimensions (32 floats of a latitude group, parity, mu, latitude
// group, column group); a box {8, 2, kInvChunk, 1, 1} at (8 (j % 4), 0, mu0, j / 4, group)
// lands in shared memory as [order][parity][8 floats]: the sum records of latitude j for
// kInvChunk consecutive orders (orders beyond L are filled with zeros).
int make_s32_tensor_map(Plan &p)
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return FAVEST_EUNSUPPORTED;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t L1 = (cuuint64_t)(p.L + 1), G = (cuuint64_t)(p.JP / 4);
    cuuint64_t dims[5] = {32, 2, L1, G, (cuuint64_t)p.nf};
    cuuint64_t strides[4] = {128, 256, 256 * L1, 256 * L1 * G};
    cuuint32_t box[5] = {8, 2, (cuuint32_t)kInvChunk, 1, 1};
    cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    CUresult r = encode(&p.tmap_s32, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, p.d_S32, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FAVEST_OK : FAVEST_EUNSUPPORTED;
}

// A GEMM operand buffer as seen by the TMA: a 2-D array of 512-byte rows (256 bf16 each),
// loaded in boxes of box_rows whole rows (one operand chunk).
// Tensor map of the Legendre operand [piece][row block][JP latitudes][8 rows] (bf16) as
// (256 = 32 latitudes x 8 rows, latitude block, row block, piece): a box {256, yb, zb, 3}
// lands in shared memory as [piece][zb row blocks][32 yb latitudes][8 rows], each piece a
// core-matrix layout of the MMA (8 consecutive latitudes x 8 rows per 128-byte matrix).
// Boxes past the last row block read zeros.
int make_lam_tensor_map(Plan &p, int yb, int zb, CUtensorMap *out)
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return FAVEST_EUNSUPPORTED;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    const cuuint64_t JP = (cuuint64_t)p.JP, RB = (cuuint64_t)p.lam_rb_total;
    cuuint64_t dims[4] = {256, JP / 32, RB, 3};
    cuuint64_t strides[3] = {512, JP * 16, RB * JP * 16};
    cuuint32_t box[4] = {256, (cuuint32_t)yb, (cuuint32_t)zb, 3};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, p.d_lam, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FAVEST_OK : FAVEST_EUNSUPPORTED;
}

int make_row_tensor_map(void *base, size_t bytes, int box_rows, CUtensorMap *out)
{
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return FAVEST_EUNSUPPORTED;
    auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    if (bytes % 512 || bytes / 512 > 0x7fffffffULL || box_rows < 1 || box_rows > 256) return FAVEST_EINVAL;
    cuuint64_t dims[2] = {256, (cuuint64_t)(bytes / 512)};
    cuuint64_t strides[1] = {512};
    cuuint32_t box[2] = {256, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FAVEST_OK : FAVEST_EUNSUPPORTED;
}

// Turning-point bounds of the split path.  Below its turning point (sin theta <
// mu / (l + 1/2)) lambda_l^mu(theta) decays exponentially towards the pole, and far below
// it the values are smaller than any FP32 rounding of the sums they enter.  For every
// order mu and folded latitude j this returns the first degree l >= mu at which
// |lambda_l^mu(theta_j)| (orthonormal) reaches kTurnEps, or L + 2 if no l <= L + 1 does.
// The values are run on a mantissa with a separate (logarithmic) exponent, so that the
// polar starting values far below the double range are handled exactly.  Every
// (l, mu, j) left out by the generator and the GEMM item ranges lies below this bound,
// i.e. is smaller than kTurnEps in magnitude.
constexpr double kTurnEps = 1e-13;

std::vector<int> turning_bounds(const Plan &p)
{
    const int L = p.L, J = p.J;
    std::vector<int> lf((size_t)(L + 1) * J, L + 2);
    const double leps = std::log(kTurnEps);
    const double lbig = std::log(0x1p200);
    double lcmu = 0.5 * std::log(1.0 / (4.0 * 3.14159265358979323846));   // log c_mu
    std::vector<double> eps(L + 3);
    for (int mu = 0; mu <= L; ++mu) {
        if (mu > 0) lcmu += 0.5 * std::log((2.0 * mu + 1.0) / (2.0 * mu));
        for (int l = mu; l <= L + 2; ++l) eps[l] = eps_lm(l, mu);
        for (int j = 0; j < J; ++j) {
            const double x = p.h_x[j], sn = std::sqrt((1.0 - x) * (1.0 + x));
            // lambda_l = y * exp(e), starting from lambda_mu^mu = (-1)^mu c_mu sin^mu (sign dropped)
            double y = 1.0, ym = 0.0, e = lcmu + mu * std::log(sn);
            double thr = std::exp(leps - e);       // |y| >= thr  <=>  |lambda| >= kTurnEps
            int l = mu;
            while (l <= L + 1 && !(std::fabs(y) >= thr)) {
                const double yn = (x * y - eps[l] * ym) / eps[l + 1];
                ym = y;
                y = yn;
                ++l;
                if (std::fabs(y) > 0x1p200) {
                    y *= 0x1p-200;
                    ym *= 0x1p-200;
                    e += lbig;
                    thr = std::exp(leps - e);
                }
            }
            lf[(size_t)mu * J + j] = l;
        }
    }
    return lf;
}

// Split-precision path: operand tile offsets, GEMM work items, buffers.
//   Lam (A operands): contiguous 24 KB chunks (three 8 KB bf16 pieces of 128 x 32), bulk copies
//   Fb  (forward B):  [JP/8][nf][8][L+1][2][3][8] bf16, gathered by a 5-D TMA box
//   g   (adjoint B):  contiguous chunks of three 32 x N bf16 pieces (N = gemm_n)
//   Q32 (forward out): [nf][ntab][8] fp32: field, then for each order mu (from row
//                      tab_off(L, mu)) its rows l = mu, mu+2, .. followed by l = mu+1, ..
//   S32 (adjoint out): [nf][JP/4][L+1][2][4][8] fp32: field, latitude group of 4, mu,
//                      parity, latitude within the group
// The GEMM epilogue stores 128-byte groups of 4 rows (one per 4 lanes of a warp); the
// inverse FFT of latitude j reads the 32-byte record of j, and the blocks of the 4
// latitudes of a group, adjacent in launch order, share each 128-byte line.
// Host-side layout of the split path: everything alloc_workspace_bf16 derives from (L,
// batch, io, latitudes) before it touches the device, so that check_layout_bf16 and
// favest_debug_check_layout can examine it without a GPU.
struct SplitLayout {
    std::vector<int> rb;                          // per (mu, parity): first row block of Lam
    std::vector<long long> off_g;                 // per (mu, parity): coefficient operand offset (bytes)
    std::vector<int> jcmin;                       // per mu: first generated latitude chunk
    std::vector<TcItem> itf, ita;                 // GEMM items, launch order
    long long CHB = 0;                            // bytes per B chunk (adjoint)
    long long rb_total = 0;                       // row blocks of Lam in all
    size_t lam_bytes = 0, fb_bytes = 0, g_bytes = 0, q_bytes = 0, s_bytes = 0;
};

int layout_bf16(Plan &p, SplitLayout &Y)
{
    const int L = p.L;
    const int KC = kGemmChunkK;
    p.gemm_n = (p.force_gemm_n == 256 || 8 * p.ncg > 128) ? 256 : 128;
    const long long CHB = 3LL * KC * p.gemm_n * 2;   // bytes per B chunk (3 pieces of KC x N)
    Y.CHB = CHB;
    p.JP = (p.J + 127) / 128 * 128;
    p.ncolr = (8 * p.ncg + p.gemm_n - 1) / p.gemm_n * p.gemm_n;
    p.n_tiles = p.ncolr / p.gemm_n;
    p.nf = p.ncolr / 8;
    p.nk_f = p.JP / KC;
    const int fpt = p.gemm_n / 8;                  // column groups per column tile
    const long long L1 = L + 1;
    std::vector<int> &rb = Y.rb;
    std::vector<long long> &off_g = Y.off_g;
    rb.assign(2 * (L + 1), 0);
    off_g.assign(2 * (L + 1), 0);
    const int J = p.J;
    const std::vector<int> lf = turning_bounds(p);
    // generator: first latitude per order, rounded down to a K-chunk of 32
    std::vector<int> &jcmin = Y.jcmin;
    jcmin.assign(L + 1, 0);
    p.gen_values = 0;
    for (int mu = 0; mu <= L; ++mu) {
        int jmin = J;
        for (int j = 0; j < J; ++j)
            if (lf[(size_t)mu * J + j] <= L + 1) { jmin = j; break; }
        const int jc = jmin / KC * KC, jlast = (J - 1) / KC * KC;
        jcmin[mu] = jc < jlast ? jc : jlast;
        p.gen_values += (double)(L + 2 - mu) * (J - jcmin[mu]);
    }
    p.gemm_pairs_f = p.gemm_pairs_a = 0;
    long long nrb = 0, gsz = 0;
    std::vector<TcItem> &itf = Y.itf, &ita = Y.ita;
    itf.clear();
    ita.clear();
    auto nrow_p = [&](int mu, int par) { const int n = L + 2 - mu; return par ? n / 2 : (n + 1) / 2; };
    // pass 1: operand storage offsets per (mu, parity)
    for (int mu = 0; mu <= L; ++mu) {
        for (int par = 0; par < 2; ++par) {
            const int np = nrow_p(mu, par);
            // the adjoint of order 0 runs on the order-1 Legendre functions (see uncombine)
            const int npa = nrow_p(mu == 0 ? 1 : mu, par);
            const int idx = mu * 2 + par;
            rb[idx] = (int)nrb;
            off_g[idx] = gsz;
            nrb += (np + 7) / 8;                 // row blocks of 8 rows of this parity
            gsz += (long long)p.n_tiles * ((npa + KC - 1) / KC) * CHB;
        }
    }
    // pass 2: GEMM work items
    for (int mu = 0; mu <= L; ++mu) {
        for (int par = 0; par < 2; ++par) {
            const int idx = mu * 2 + par;
            const int np = nrow_p(mu, par);
            const int mt = (np + 127) / 128;
            for (int m = 0; m < mt; ++m) {
                // first latitude chunk holding a value above the bound for a row of the tile
                const int rhi = (128 * m + 127 < np - 1) ? 128 * m + 127 : np - 1;
                const int lhi = mu + par + 2 * rhi;
                int kc0 = p.nk_f - 1;
                for (int c = 0; c < p.nk_f - 1 && kc0 == p.nk_f - 1; ++c)
                    for (int j = c * KC; j < (c + 1) * KC && j < J; ++j)
                        if (lf[(size_t)mu * J + j] <= lhi) { kc0 = c; break; }
                const int trows = np - 128 * m < 128 ? np - 128 * m : 128;
                p.gemm_pairs_f += (double)trows * (J - kc0 * KC > 0 ? J - kc0 * KC : 0);
                for (int nt = 0; nt < p.n_tiles; ++nt) {
                    TcItem I{};
                    // A: latitude block kc0 + c (32 latitudes), row blocks 16 m .. 16 m + 15
                    I.ay = kc0;
                    I.ady = 1;
                    I.az = rb[idx] + 16 * m;
                    I.adz = 0;
                    I.b_box = 1;
                    I.bx = par * 8;
                    I.by = fpt * nt;
                    I.bw = mu;
                    I.bk = kc0;
                    // rows of (mu, par) are consecutive in Q32 (see the layout note above)
                    const long long qrow = tab_off(L, mu) + (par ? nrow_p(mu, 0) : 0) + 128LL * m;
                    I.out_off = ((long long)fpt * nt * p.ntab + qrow) * 8;
                    I.out_ld = 32;
                    I.col_gs = p.ntab * 8;
                    I.nk = p.nk_f - kc0;
                    I.rows = trows;
                    I.group = 0;
                    itf.push_back(I);
                }
            }
            const int amu = mu == 0 ? 1 : mu;
            const int npa = nrow_p(amu, par);
            const int nka = (npa + KC - 1) / KC;
            for (int t = 0; t < p.JP / 128; ++t) {
                // first row chunk (rows l = amu + par + 2 r) reaching the tile's lowest bound
                int lmin = L + 2;
                for (int j = 128 * t; j < 128 * t + 128 && j < J; ++j) {
                    const int v = lf[(size_t)amu * J + j];
                    lmin = v < lmin ? v : lmin;
                }
                int kc0 = nka - 1;
                for (int c = 0; c < nka - 1; ++c)
                    if (amu + par + 2 * (KC * c + KC - 1) >= lmin) { kc0 = c; break; }
                const int tl = J - 128 * t < 128 ? J - 128 * t : 128;
                p.gemm_pairs_a += (double)(tl > 0 ? tl : 0) * (npa - KC * kc0);
                for (int nt = 0; nt < p.n_tiles; ++nt) {
                    TcItem I{};
                    // A: latitude blocks 4 t .. 4 t + 3 (128 latitudes), row blocks of chunk
                    // kc0 + c: 4 (kc0 + c) .. + 3 of (amu, par)
                    I.ay = 4 * t;
                    I.ady = 0;
                    I.az = rb[amu * 2 + par] + 4 * kc0;
                    I.adz = 4;
                    I.b_off = off_g[idx] + ((long long)nt * nka + kc0) * CHB;
                    I.b_stride = (int)CHB;
                    I.out_off = ((((long long)fpt * nt * (p.JP / 4) + 32LL * t) * L1 + mu) * 2 + par) * 32;
                    I.out_ld = L1 * 2 * 32;
                    I.col_gs = (long long)(p.JP / 4) * L1 * 2 * 32;
                    I.nk = nka - kc0;
                    I.rows = 128;
                    I.group = 1;
                    ita.push_back(I);
                }
            }
        }
    }
    // The GEMMs' CTAs take the listed items in order as they free up (see legendre_tc.cu),
    // so the order decides which items run together.  Forward: (order,
    // parity, row tile), so that the row tiles of one order, which read the same B operand,
    // run at the same time on neighbouring CTAs and share it through L2.  Adjoint: the
    // latitude tiles of one (order, parity), which read the same coefficient operand over
    // different K depths (turning-point skip), kept together, the groups in decreasing order
    // of their deepest tile.
    {
        const size_t per = (size_t)(p.JP / 128) * p.n_tiles;   // items of one (order, parity)
        const size_t ng = ita.size() / per;
        std::vector<int> gmax(ng), gi(ng);
        for (size_t g = 0; g < ng; ++g) {
            int m = 0;
            for (size_t u = 0; u < per; ++u) m = std::max(m, ita[g * per + u].nk);
            gmax[g] = m;
            gi[g] = (int)g;
        }
        std::stable_sort(gi.begin(), gi.end(), [&](int a, int b) { return gmax[a] > gmax[b]; });
        std::vector<TcItem> grouped;
        grouped.reserve(ita.size());
        for (int g : gi)
            for (size_t u = 0; u < per; ++u) grouped.push_back(ita[g * per + u]);
        ita.swap(grouped);
    }
    p.n_items_f = (int)itf.size();
    p.n_items_a = (int)ita.size();
    Y.rb_total = nrb;
    Y.lam_bytes = (size_t)3 * nrb * p.JP * 16;
    Y.fb_bytes = (size_t)p.JP * p.nf * L1 * 64;
    Y.g_bytes = (size_t)gsz;
    Y.q_bytes = (size_t)p.nf * p.ntab * 8 * sizeof(float);
    Y.s_bytes = (size_t)p.nf * (p.JP / 4) * L1 * 2 * 32 * sizeof(float);
    return FAVEST_OK;
}

// Bounds of every index the split path's kernels take from the layout: each GEMM item's
// operand chunks (byte ranges of the A and B buffers, 512-byte row alignment of the TMA
// row boxes; the forward B operand's 5-D box coordinates against the tensor map's extents),
// its output rows and column groups against the output buffer and against the rows of its
// own order, and the per-order operand regions (in range, in order, not overlapping).
// FAVEST_EINTERNAL with a description in msg (when given) on the first violation.
int check_layout_bf16(const Plan &p, const SplitLayout &Y, char *msg, size_t msg_len)
{
    auto fail = [&](const char *what, long long a, long long b, long long c) {
        if (msg && msg_len) std::snprintf(msg, msg_len, "%s (%lld, %lld, %lld)", what, a, b, c);
        return FAVEST_EINTERNAL;
    };
    const int L = p.L, N = p.gemm_n, KC = kGemmChunkK;
    const long long L1 = L + 1;
    auto nrow_p = [&](int mu, int par) { const int n = L + 2 - mu; return par ? n / 2 : (n + 1) / 2; };
    if (p.JP % 128 || p.JP < p.J || p.nf * 8 != p.ncolr || p.n_tiles * N != p.ncolr || p.nf < p.ncg)
        return fail("grid or column padding", p.JP, p.nf, p.ncolr);
    if ((int)Y.rb.size() != 2 * L1 || (int)Y.off_g.size() != 2 * L1 || (int)Y.jcmin.size() != L1)
        return fail("table sizes", (long long)Y.rb.size(), (long long)Y.jcmin.size(), L1);
    if (Y.lam_bytes != (size_t)3 * Y.rb_total * p.JP * 16) return fail("Legendre buffer size", Y.rb_total, p.JP, 0);
    // per-(mu, parity) regions: Legendre row blocks and coefficient operand, in order, inside
    // their buffers
    for (int idx = 0; idx < 2 * L1; ++idx) {
        const int mu = idx / 2, par = idx % 2;
        const int np = nrow_p(mu, par), npa = nrow_p(mu == 0 ? 1 : mu, par);
        const long long er = (long long)Y.rb[idx] + (np + 7) / 8;
        const long long eg = Y.off_g[idx] + (long long)p.n_tiles * ((npa + KC - 1) / KC) * Y.CHB;
        const long long nr_ = idx + 1 < 2 * L1 ? Y.rb[idx + 1] : Y.rb_total;
        const long long ng_ = idx + 1 < 2 * L1 ? Y.off_g[idx + 1] : (long long)Y.g_bytes;
        if (Y.rb[idx] < 0 || er > nr_) return fail("Legendre row blocks", mu, par, er);
        if (Y.off_g[idx] < 0 || eg > ng_) return fail("coefficient operand region", mu, par, eg);
        if (Y.off_g[idx] % 512) return fail("operand region alignment", mu, par, Y.off_g[idx]);
    }
    for (int mu = 0; mu <= L; ++mu)
        if (Y.jcmin[mu] < 0 || Y.jcmin[mu] % KC || Y.jcmin[mu] >= p.J) return fail("generator start", mu, Y.jcmin[mu], p.J);
    const long long qf = (long long)(Y.q_bytes / sizeof(float)), sf = (long long)(Y.s_bytes / sizeof(float));
    // the epilogue writes row r < rows, column group g < N/8 at out_off + (r/4) out_ld +
    // (r%4) 8 + g col_gs (8 floats): the last row and group bound it from above
    auto out_span = [&](const TcItem &I, long long &lo, long long &hi) {
        const int r = I.rows - 1;
        lo = I.out_off;
        hi = I.out_off + (long long)(r / 4) * I.out_ld + (r % 4) * 8 + 7 + (long long)(N / 8 - 1) * I.col_gs;
    };
    for (size_t i = 0; i < Y.itf.size(); ++i) {
        const TcItem &I = Y.itf[i];
        if (I.nk < 1 || I.rows < 1 || I.rows > 128 || I.group != 0 || !I.b_box) return fail("forward item shape", (long long)i, I.nk, I.rows);
        // 5-D box {8, 1, 8, N/8, 4} at (bx, bw, 0, by, 4 (bk + c)) in dims {16, L+1, 8, nf, JP/8}
        if ((I.bx != 0 && I.bx != 8) || I.bw < 0 || I.bw > L || I.by < 0 || I.by + N / 8 > p.nf || I.bk < 0 ||
            (long long)(KC / 8) * (I.bk + I.nk) > p.JP / 8)
            return fail("forward item B box", (long long)i, I.bw, I.bk + I.nk);
        // A: latitude blocks ay .. ay + nk - 1 (of JP / 32), row blocks az .. az + 15: the
        // tile's first row block and its valid rows lie in the row blocks of its own
        // (order, parity) (rows beyond them are read but their outputs are not written)
        {
            const int mu = I.bw, par = I.bx / 8, idx = mu * 2 + par;
            const long long r0 = Y.rb[idx], r1 = r0 + (nrow_p(mu, par) + 7) / 8;
            if (I.ady != 1 || I.adz != 0 || I.ay < 0 || (long long)I.ay + I.nk > p.JP / 32 || I.az < r0 ||
                (long long)I.az + (I.rows + 7) / 8 > r1)
                return fail("forward item A box", (long long)i, I.ay, I.az);
        }
        long long lo, hi;
        out_span(I, lo, hi);
        if (lo < 0 || hi >= qf) return fail("forward item output", (long long)i, lo, hi);
        // rows of the item's own order and parity: Q32 rows tab_off(L, mu) .. tab_off(L, mu+1)
        const long long qrow = (I.out_off / 8) % p.ntab;
        const int mu = I.bw;
        if (qrow < tab_off(L, mu) || qrow + I.rows > tab_off(L, mu + 1)) return fail("forward item rows", (long long)i, mu, qrow);
    }
    for (size_t i = 0; i < Y.ita.size(); ++i) {
        const TcItem &I = Y.ita[i];
        if (I.nk < 1 || I.rows != 128 || I.group != 1 || I.b_box) return fail("adjoint item shape", (long long)i, I.nk, I.rows);
        // A: latitude blocks ay .. ay + 3, row blocks az + 4 c .. + 3: the chunks start in the
        // row blocks of the item's own (order, parity) (order 1 for order 0) and run past
        // them by less than one chunk (those rows meet zero coefficient rows)
        {
            const long long q = I.out_off / 32;
            const int par = (int)(q % 2), mu = (int)((q / 2) % L1), amu = mu == 0 ? 1 : mu;
            const long long r0 = Y.rb[amu * 2 + par], nb = (nrow_p(amu, par) + 7) / 8;
            if (I.ady != 0 || I.adz != 4 || I.ay < 0 || I.ay % 4 || (long long)I.ay + 4 > p.JP / 32 || I.az < r0 ||
                (I.az - r0) % 4 || (long long)I.az + 4LL * I.nk > r0 + (nb + 3) / 4 * 4)
                return fail("adjoint item A box", (long long)i, I.ay, I.az);
        }
        if (I.b_off < 0 || I.b_off % 512 || I.b_stride % 512 || I.b_off + (long long)(I.nk - 1) * I.b_stride + Y.CHB > (long long)Y.g_bytes)
            return fail("adjoint item B chunks", (long long)i, I.b_off, I.nk);
        long long lo, hi;
        out_span(I, lo, hi);
        if (lo < 0 || hi >= sf) return fail("adjoint item output", (long long)i, lo, hi);
    }
    return FAVEST_OK;
}

int alloc_workspace_bf16(Plan &p)
{
    SplitLayout Y;
    int st = layout_bf16(p, Y);
    if (st == FAVEST_OK) st = check_layout_bf16(p, Y, nullptr, 0);
    if (st != FAVEST_OK) return st;
    const int L = p.L;
    const long long CHB = Y.CHB;
    const std::vector<long long> &off_g = Y.off_g;
    const std::vector<int> &jcmin = Y.jcmin;
    const std::vector<TcItem> &itf = Y.itf, &ita = Y.ita;
    const size_t lam_bytes = Y.lam_bytes, fb_bytes = Y.fb_bytes, q_bytes = Y.q_bytes, s_bytes = Y.s_bytes;
    const long long gsz = (long long)Y.g_bytes;
    p.lam_rb_total = Y.rb_total;
    if (plan_malloc(&p.d_lam, lam_bytes) != cudaSuccess ||
        plan_malloc(&p.d_Fb, fb_bytes) != cudaSuccess ||
        plan_malloc(&p.d_gb, (size_t)gsz) != cudaSuccess || plan_malloc((void **)&p.d_Q32, q_bytes) != cudaSuccess ||
        plan_malloc((void **)&p.d_S32, s_bytes) != cudaSuccess ||
        plan_malloc((void **)&p.d_status, kStatusWords * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return FAVEST_ENOMEM;
    }
    // padded operand positions (latitudes >= J, fields >= B, rows beyond each order's
    // range) and the latitudes below each order's turning bound must hold zeros; they
    // are never written afterwards
    if (cudaMemset(p.d_lam, 0, lam_bytes) != cudaSuccess ||
        cudaMemset(p.d_Fb, 0, fb_bytes) != cudaSuccess ||
        cudaMemset(p.d_gb, 0, (size_t)gsz) != cudaSuccess ||
        cudaMemset(p.d_status, 0, kStatusWords * sizeof(int)) != cudaSuccess)
        return FAVEST_ECUDA;
    cudaError_t e;
    if ((e = upload(&p.d_lam_rb, Y.rb)) || (e = upload(&p.d_g_off, off_g)) || (e = upload(&p.d_items_f, itf)) || (e = upload(&p.d_items_a, ita)) ||
        (e = upload(&p.d_jcmin, jcmin)))
        return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    p.ws_bytes = lam_bytes + fb_bytes + (size_t)gsz + q_bytes + s_bytes;
    const int pst = build_polar_tables(p);
    if (pst != FAVEST_OK) return pst;
    p.ws_bytes += (size_t)p.pol_jc * (L + 1) * p.pol_muc * sizeof(float2);
    st = make_lam_tensor_map(p, 1, 16, &p.tmap_lam_f);         // forward: 32 latitudes x 16 row blocks
    if (st == FAVEST_OK) st = make_lam_tensor_map(p, 4, 4, &p.tmap_lam_a);   // adjoint: 128 x 4
    if (st == FAVEST_OK) st = make_fb_tensor_map(p);
    if (st == FAVEST_OK) st = make_s32_tensor_map(p);
    if (st == FAVEST_OK) st = make_row_tensor_map(p.d_gb, (size_t)gsz, (int)(CHB / 512), &p.tmap_gb);
    if (st != FAVEST_OK) return st;
    std::vector<GemmGroup> gg(2);
    gg[0].tmap_a = p.tmap_lam_f;
    gg[0].tmap_b = p.tmap_fb;
    gg[0].out = p.d_Q32;
    gg[1].tmap_a = p.tmap_lam_a;
    gg[1].tmap_b = p.tmap_gb;
    gg[1].out = p.d_S32;
    if ((e = upload(&p.d_ggroups, gg))) return e == cudaErrorMemoryAllocation ? FAVEST_ENOMEM : FAVEST_ECUDA;
    p.h_items_f = itf;
    p.h_items_a = ita;
    return FAVEST_OK;
}

int alloc_workspace(Plan &p)
{
    const int nmu = p.L + 1 + (p.nscal > 0 ? 1 : 0);
    // scattered points: only the sums Q (the point kernels replace the grid stages)
    size_t fbytes = p.scattered ? 0 : (size_t)nmu * p.ncol * p.nlat * sizeof(double2);
    size_t qbytes = (size_t)p.ntab * p.ncol * sizeof(double2);
    // inverse DFT rows: 2 per group of 4 columns, or 2 per real field (2 fields per group)
    size_t gbytes = p.scattered ? 0 : (size_t)(p.real ? p.ncol : p.ncol / 2) * p.nlat * p.nphi * sizeof(double2);
    if ((fbytes && plan_malloc(&p.d_F, fbytes) != cudaSuccess) || plan_malloc(&p.d_Q, qbytes) != cudaSuccess ||
        (gbytes && plan_malloc(&p.d_G, gbytes) != cudaSuccess) ||
        plan_malloc((void **)&p.d_status, kStatusWords * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return FAVEST_ENOMEM;
    }
    cudaMemset(p.d_status, 0, kStatusWords * sizeof(int));
    // the padding columns (an odd count of scalar or real fields) read as zero
    if ((p.nscal > 0 || p.real) &&
        (cudaMemset(p.d_Q, 0, qbytes) != cudaSuccess || (fbytes && cudaMemset(p.d_F, 0, fbytes) != cudaSuccess)))
        return FAVEST_ECUDA;
    p.ws_bytes = fbytes + qbytes + gbytes;
    return FAVEST_OK;
}

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

int check_device(const Plan &p)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FAVEST_ECUDA;
    return dev == p.device ? FAVEST_OK : FAVEST_EINVAL;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA; }

const char *kKernelNames[KID_COUNT] = {
    "fft_fwd", "legendre_analysis", "combine", "uncombine", "legendre_synthesis", "fft_inv",
    "gen_lambda_fwd", "tc_gemm_fwd", "gen_lambda_adj", "tc_gemm_adj", "polar_patch", "cg_combine", "cg_uncombine",
    "gen_lambda_both", "cg_pack", "cg_unpack",
};

cudaEvent_t take_event(Plan &p)
{
    cudaEvent_t e = nullptr;
    if (!p.event_pool.empty()) {
        e = p.event_pool.back();
        p.event_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

// Launch `fn` on stream s, bracketed by events when profiling is enabled.
template <typename Fn>
cudaError_t timed(Plan &p, int kid, cudaStream_t s, Fn fn)
{
    if (!p.profiling) return fn();
    cudaEvent_t e0 = take_event(p), e1 = take_event(p);
    if (e0) cudaEventRecord(e0, s);
    cudaError_t err = fn();
    if (e1) cudaEventRecord(e1, s);
    if (e0 && e1) p.recs.push_back({kid, e0, e1});
    else {
        if (e0) p.event_pool.push_back(e0);
        if (e1) p.event_pool.push_back(e1);
    }
    return err;
}

void release_events(Plan &p)
{
    for (auto &r : p.recs) {
        cudaEventDestroy(r.e0);
        cudaEventDestroy(r.e1);
    }
    p.recs.clear();
    for (auto e : p.event_pool) cudaEventDestroy(e);
    p.event_pool.clear();
}

}  // namespace

extern "C" {

const char *favest_strerror(int status)
{
    int i = -status;
    if (i < 0 || i >= (int)(sizeof(kErrStr) / sizeof(kErrStr[0]))) return "unknown status";
    return kErrStr[i];
}

int favest_debug_fail_alloc(long long k)
{
    if (k < -1) return FAVEST_EINVAL;
    g_alloc_fail_at.store(-1);
    g_alloc_calls.store(0);
    g_alloc_fail_at.store(k);
    return FAVEST_OK;
}

long long favest_debug_alloc_count(void) { return g_alloc_calls.load(); }

int favest_gl_grid(int nlat, double *x, double *w)
{
    if (nlat < 1 || !x || !w) return FAVEST_EINVAL;
    return gl_rule(nlat, x, w);
}

}  // extern "C"

namespace favest {

cudaError_t plan_malloc(void **p, size_t bytes)
{
    const long long k = g_alloc_calls.fetch_add(1);
    if (k == g_alloc_fail_at.load()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

// Argument checks and the host-side fields of a plan (grid sizes, column layout,
// latitudes and weights in h_x / h_w, which the caller frees with std::free on failure
// paths that do not go through free_plan); no CUDA call.
int plan_init_host(Plan &p, int L, int batch, int precision, int io_type, const double *cos_theta,
                   const double *w_lat, int force_gemm_n, int cg_route)
{
    if (L < 1 || L > 4095 || batch < 1 || batch > 4096) return FAVEST_EINVAL;
    if (L > 2559) return FAVEST_EUNSUPPORTED;   // J <= 1280 latitudes per CTA in the FP64 kernels
    if (precision != FAVEST_FP64 && precision != FAVEST_BF16X6) return FAVEST_EINVAL;
    if (io_type != FAVEST_IO_C128 && io_type != FAVEST_IO_C64 && io_type != FAVEST_IO_R32 && io_type != FAVEST_IO_R64)
        return FAVEST_EINVAL;
    if ((cos_theta == nullptr) != (w_lat == nullptr)) return FAVEST_EINVAL;
    const int nlat = L + 1;
    if (cos_theta) {
        for (int j = 0; j < nlat; ++j) {
            double xj = cos_theta[j], xm = cos_theta[nlat - 1 - j];
            if (!(xj > -1.0 && xj < 1.0) || !(w_lat[j] > 0.0)) return FAVEST_EINVAL;
            if (std::fabs(xj + xm) > 1e-14 || std::fabs(w_lat[j] - w_lat[nlat - 1 - j]) > 1e-14)
                return FAVEST_EINVAL;
            if (j > 0 && !(cos_theta[j] < cos_theta[j - 1])) return FAVEST_EINVAL;
        }
    }
    if (precision == FAVEST_BF16X6 && (io_type == FAVEST_IO_C128 || io_type == FAVEST_IO_R64)) return FAVEST_EUNSUPPORTED;
    const bool real_io = io_type == FAVEST_IO_R32 || io_type == FAVEST_IO_R64;
    if (real_io && cg_route) return FAVEST_EINVAL;
    p.force_gemm_n = force_gemm_n;
    p.L = L;
    p.B = batch;
    p.precision = precision;
    p.io = io_type;
    p.real = real_io ? 1 : 0;
    p.ncg = p.real ? (batch + 1) / 2 : batch;
    p.nlat = nlat;
    p.nphi = 2 * (L + 1);
    p.J = (nlat + 1) / 2;
    // untuned generator shape: two latitude chains per thread only where the grid stays
    // large (L = 1023: 0.94 against 0.91 ms; L = 511: 0.26 against 0.21 ms with one chain)
    p.gen_nj = p.J >= 384 ? 2 : 1;
    p.has_eq = nlat & 1;
    p.ncol = 4 * batch;
    if (p.real) p.ncol = 4 * ((batch + 1) / 2);   // a pair of real fields per group of 4 columns
    if (cg_route) {
        // 3 scalar fields per vector field, 2 per group of 4 columns (sign of m, re/im)
        p.nscal = 3 * batch;
        p.ncol = 4 * ((p.nscal + 1) / 2);
        p.scattered = cg_route == 2;
    }
    p.ct = (p.ncol % 8 == 0) ? 8 : 4;
    p.ng = p.ncol / p.ct;
    if (p.J > 1280) return FAVEST_EUNSUPPORTED;
    p.h_x = (double *)std::malloc(sizeof(double) * nlat);
    p.h_w = (double *)std::malloc(sizeof(double) * nlat);
    if (!p.h_x || !p.h_w) return FAVEST_ENOMEM;
    if (cos_theta) {
        std::memcpy(p.h_x, cos_theta, sizeof(double) * nlat);
        std::memcpy(p.h_w, w_lat, sizeof(double) * nlat);
    } else {
        gl_rule(nlat, p.h_x, p.h_w);
    }
    return FAVEST_OK;
}

int plan_create_internal(int L, int batch, int precision, int io_type, const double *cos_theta,
                         const double *w_lat, int force_gemm_n, favest_plan *out, int cg_route)
{
    if (!out) return FAVEST_EINVAL;
    *out = nullptr;
    favest_plan_s *h = new (std::nothrow) favest_plan_s();
    if (!h) return FAVEST_ENOMEM;
    Plan &p = h->p;
    int st = plan_init_host(p, L, batch, precision, io_type, cos_theta, w_lat, force_gemm_n, cg_route);
    if (st != FAVEST_OK) {
        std::free(p.h_x);
        std::free(p.h_w);
        p.h_x = p.h_w = nullptr;
        delete h;
        return st;
    }
    if (cudaGetDevice(&p.device) != cudaSuccess) { free_plan(p); delete h; return FAVEST_ECUDA; }
    cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, p.device);
    if (precision == FAVEST_BF16X6) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, p.device);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, p.device);
        if (major != 10 || minor != 3) { free_plan(p); delete h; return FAVEST_EUNSUPPORTED; }
    }
    st = build_tables(p);
    if (st == FAVEST_OK) st = (precision == FAVEST_BF16X6) ? alloc_workspace_bf16(p) : alloc_workspace(p);
    if (st != FAVEST_OK) {
        cudaGetLastError();
        free_plan(p);
        delete h;
        return st;
    }
    if (cudaDeviceSynchronize() != cudaSuccess) { free_plan(p); delete h; return FAVEST_ECUDA; }
    *out = h;
    return FAVEST_OK;
}

}  // namespace favest

extern "C" {

int favest_debug_check_layout(int L, int batch, int precision, int io_type, int gemm_n, int poison, char *msg,
                              int msg_len)
{
    if (msg && msg_len > 0) msg[0] = 0;
    if (gemm_n != 0 && gemm_n != 256) return FAVEST_EINVAL;
    if (poison < 0 || poison > 3) return FAVEST_EINVAL;
    if (msg_len < 0 || (msg_len > 0 && !msg)) return FAVEST_EINVAL;
    Plan p;
    int st = plan_init_host(p, L, batch, precision, io_type, nullptr, nullptr, gemm_n, 0);
    if (st == FAVEST_OK && precision == FAVEST_BF16X6) {
        p.ntab = tab_off(L, L + 1);   // orders 0..L, as build_tables sets it
        SplitLayout Y;
        st = layout_bf16(p, Y);
        if (st == FAVEST_OK && poison == 1 && !Y.itf.empty()) Y.itf[0].bw = L + 1;      // order out of range
        if (st == FAVEST_OK && poison == 2 && !Y.ita.empty()) Y.ita.back().nk += 1;    // one chunk too many
        if (st == FAVEST_OK && poison == 3 && L >= 2) Y.rb[2] = Y.rb[1];               // overlapping regions
        if (st == FAVEST_OK) st = check_layout_bf16(p, Y, msg, msg_len > 0 ? (size_t)msg_len : 0);
    }
    std::free(p.h_x);
    std::free(p.h_w);
    p.h_x = p.h_w = nullptr;
    return st;
}

int favest_plan_create(int L, int batch, int precision, int io_type, const double *cos_theta,
                       const double *w_lat, favest_plan *out)
{
    return favest::plan_create_internal(L, batch, precision, io_type, cos_theta, w_lat, 0, out);
}

int favest_fwd(favest_plan plan, const void *Tth, const void *Tph, void *a, void *b, void *stream)
{
    return favest_fwd_ex(plan, Tth, Tph, a, b, 0, stream);
}

int favest_cg_plan_create(int L, int batch, const double *cos_theta, const double *w_lat, favest_plan *out)
{
    if (batch > 4096 / 3 + 1) return FAVEST_EINVAL;
    return favest::plan_create_internal(L, batch, FAVEST_FP64, FAVEST_IO_C128, cos_theta, w_lat, 0, out, 1);
}

int favest_cg_plan_create_ex(int L, int batch, int io_type, const double *cos_theta, const double *w_lat,
                             favest_plan *out)
{
    if (io_type == FAVEST_IO_C128) return favest_cg_plan_create(L, batch, cos_theta, w_lat, out);
    if (!out) return FAVEST_EINVAL;
    *out = nullptr;
    if (io_type != FAVEST_IO_R64 || batch < 1 || batch > 2 * (4096 / 3 + 1)) return FAVEST_EINVAL;
    // real fields 2q, 2q+1 as the complex field q of a complex plan
    favest_plan h = nullptr;
    int st = favest::plan_create_internal(L, (batch + 1) / 2, FAVEST_FP64, FAVEST_IO_C128, cos_theta, w_lat, 0, &h, 1);
    if (st != FAVEST_OK) return st;
    favest::Plan &p = h->p;
    p.cg_real = batch;
    const size_t K = (size_t)L * L + 2 * (size_t)L;
    const size_t tb = (size_t)p.B * 3 * p.nlat * p.nphi * sizeof(double2), cb = (size_t)p.B * K * sizeof(double2);
    if (favest::plan_malloc(&p.d_cgT, tb) != cudaSuccess || favest::plan_malloc(&p.d_cga, cb) != cudaSuccess ||
        favest::plan_malloc(&p.d_cgb, cb) != cudaSuccess) {
        cudaGetLastError();
        favest_plan_destroy(h);
        return FAVEST_ENOMEM;
    }
    p.ws_bytes += tb + 2 * cb;
    *out = h;
    return FAVEST_OK;
}

int favest_adj(favest_plan plan, const void *a, const void *b, void *Tth, void *Tph, void *stream)
{
    return favest_adj_ex(plan, a, b, Tth, Tph, 0, stream);
}

namespace {

// Restores a plan field when the call returns.
struct FlagScope {
    int &ref, saved;
    FlagScope(int &r, int v) : ref(r), saved(r) { ref = v; }
    ~FlagScope() { ref = saved; }
};

// Generator launch of a split-precision call that needs the Legendre operand in layout
// `mine` (kGenFwd or kGenAdj).  Without FAVEST_FLAG_SHARE_LAMBDA: generate that layout.
// With it: if the previous call on the plan generated both layouts for this one, use them
// (no launch); otherwise generate both and leave the other layout to the next call.  Any
// call ends an earlier pairing, so an operand is used by at most the call right after the
// one that generated it.
cudaError_t legendre_operand(Plan &p, int mine, bool share, cudaStream_t s)
{
    const int pending = p.lam_pending;
    p.lam_pending = 0;
    if (share && pending == mine) return cudaSuccess;
    if (share) {
        cudaError_t e = timed(p, KID_GEN_BOTH, s, [&] { return launch_gen_lambda(p, kGenBoth, s); });
        if (e == cudaSuccess) p.lam_pending = kGenBoth & ~mine;
        return e;
    }
    return timed(p, mine == kGenFwd ? KID_GEN_FWD : KID_GEN_ADJ, s, [&] { return launch_gen_lambda(p, mine, s); });
}

}  // namespace

int favest_fwd_ex(favest_plan plan, const void *Tth, const void *Tph, void *a, void *b, int flags, void *stream)
{
    if (!plan || !Tth || !Tph || !a || !b) return FAVEST_EINVAL;
    if (flags & ~(FAVEST_FLAG_UNIT_WEIGHTS | FAVEST_FLAG_REAL_TRANSPOSE | FAVEST_FLAG_SHARE_LAMBDA))
        return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (p.nscal > 0) return FAVEST_EINVAL;     // Clebsch-Gordan plans take favest_fwd_cart
    if ((flags & FAVEST_FLAG_REAL_TRANSPOSE) && !p.real) return FAVEST_EINVAL;
    FlagScope unit(p.unit_weights, p.unit_weights | ((flags & FAVEST_FLAG_UNIT_WEIGHTS) ? 1 : 0));
    FlagScope rtr(p.real_transpose, (flags & FAVEST_FLAG_REAL_TRANSPOSE) ? 1 : 0);
    size_t el = (p.io == FAVEST_IO_C128 || p.precision == FAVEST_BF16X6 || p.real) ? 16 : 8;
    if (!aligned(Tth, el) || !aligned(Tph, el) || !aligned(a, el) || !aligned(b, el)) return FAVEST_EINVAL;
    int st = check_device(p);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (p.precision == FAVEST_BF16X6) {
        e = timed(p, KID_FFT_FWD, s, [&] { return launch_fft_fwd_bf16(p, Tth, Tph, s); });
        if (e == cudaSuccess) e = legendre_operand(p, kGenFwd, (flags & FAVEST_FLAG_SHARE_LAMBDA) != 0, s);
        if (e == cudaSuccess) e = timed(p, KID_GEMM_FWD, s, [&] { return launch_tc_gemm(p, true, s); });
        if (e == cudaSuccess) e = timed(p, KID_COMBINE, s, [&] { return launch_combine_bf16(p, a, b, s); });
        return cuda_status(e);
    }
    e = timed(p, KID_FFT_FWD, s, [&] { return launch_fft_fwd_fp64(p, Tth, Tph, s); });
    if (e == cudaSuccess) e = timed(p, KID_ANALYSIS, s, [&] { return launch_analysis_fp64(p, s); });
    if (e == cudaSuccess) e = timed(p, KID_COMBINE, s, [&] { return launch_combine_fp64(p, a, b, s); });
    return cuda_status(e);
}

int favest_adj_ex(favest_plan plan, const void *a, const void *b, void *Tth, void *Tph, int flags, void *stream)
{
    if (!plan || !Tth || !Tph || !a || !b) return FAVEST_EINVAL;
    if (flags & ~(FAVEST_FLAG_WEIGHTED | FAVEST_FLAG_REAL_TRANSPOSE | FAVEST_FLAG_SHARE_LAMBDA)) return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (p.nscal > 0) return FAVEST_EINVAL;
    if ((flags & FAVEST_FLAG_REAL_TRANSPOSE) && !p.real) return FAVEST_EINVAL;
    FlagScope weighted(p.adj_weighted, (flags & FAVEST_FLAG_WEIGHTED) ? 1 : 0);
    FlagScope rtr(p.real_transpose, (flags & FAVEST_FLAG_REAL_TRANSPOSE) ? 1 : 0);
    size_t el = (p.io == FAVEST_IO_C128 || p.precision == FAVEST_BF16X6 || p.real) ? 16 : 8;
    if (!aligned(Tth, el) || !aligned(Tph, el) || !aligned(a, el) || !aligned(b, el)) return FAVEST_EINVAL;
    int st = check_device(p);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e;
    if (p.precision == FAVEST_BF16X6) {
        // the polar patch reads only the coefficients and its tables and writes a buffer of
        // its own: it runs on the plan's side stream next to the uncombine, generator and
        // GEMM, forked from and joined back into the caller's stream (graph capture follows)
        e = cudaSuccess;
        if (p.pol_jc > 0) {
            e = cudaEventRecord(p.pol_fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(p.pol_stream, p.pol_fork, 0);
            if (e == cudaSuccess)
                e = timed(p, KID_POLAR, p.pol_stream, [&] { return launch_polar_patch(p, a, b, p.pol_stream); });
            if (e == cudaSuccess) e = cudaEventRecord(p.pol_join, p.pol_stream);
        }
        if (e == cudaSuccess) e = timed(p, KID_UNCOMBINE, s, [&] { return launch_uncombine_bf16(p, a, b, s); });
        if (e == cudaSuccess) e = legendre_operand(p, kGenAdj, (flags & FAVEST_FLAG_SHARE_LAMBDA) != 0, s);
        if (e == cudaSuccess) e = timed(p, KID_GEMM_ADJ, s, [&] { return launch_tc_gemm(p, false, s); });
        if (e == cudaSuccess && p.pol_jc > 0) e = cudaStreamWaitEvent(s, p.pol_join, 0);
        if (e == cudaSuccess) e = timed(p, KID_FFT_INV, s, [&] { return launch_fft_inv_bf16(p, Tth, Tph, s); });
        return cuda_status(e);
    }
    e = timed(p, KID_UNCOMBINE, s, [&] { return launch_uncombine_fp64(p, a, b, s); });
    if (e == cudaSuccess) e = timed(p, KID_SYNTHESIS, s, [&] { return launch_synthesis_fp64(p, s); });
    if (e == cudaSuccess) e = timed(p, KID_FFT_INV, s, [&] { return launch_fft_inv_fp64(p, Tth, Tph, s); });
    return cuda_status(e);
}

int favest_fwd_cart(favest_plan plan, const void *T, void *a, void *b, void *stream)
{
    if (!plan || !T || !a || !b) return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (p.nscal == 0) return FAVEST_EINVAL;
    if (!aligned(T, 16) || !aligned(a, 16) || !aligned(b, 16)) return FAVEST_EINVAL;
    int st = check_device(p);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // real fields: packed in pairs into the plan's complex fields, coefficients split after
    const void *Tc = T;
    void *ac = a, *bc = b;
    if (p.cg_real) {
        e = timed(p, KID_CG_PACK, s, [&] { return launch_cg_pack_fields(p, T, s); });
        Tc = p.d_cgT;
        ac = p.d_cga;
        bc = p.d_cgb;
    }
    // three scalar FwdSHTs of degree L+1 (DFT, analysis with the point weights), Thm. 1
    if (e == cudaSuccess) e = timed(p, KID_FFT_FWD, s, [&] { return launch_fft_fwd_fp64(p, Tc, Tc, s); });
    if (e == cudaSuccess) e = timed(p, KID_ANALYSIS, s, [&] { return launch_analysis_fp64(p, s); });
    if (e == cudaSuccess) e = timed(p, KID_CG_COMBINE, s, [&] { return launch_cg_combine(p, ac, bc, s); });
    if (e == cudaSuccess && p.cg_real) e = timed(p, KID_CG_UNPACK, s, [&] { return launch_cg_unpack_coefs(p, a, b, s); });
    return cuda_status(e);
}

int favest_adj_cart(favest_plan plan, const void *a, const void *b, void *T, void *stream)
{
    if (!plan || !T || !a || !b) return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (p.nscal == 0) return FAVEST_EINVAL;
    if (!aligned(T, 16) || !aligned(a, 16) || !aligned(b, 16)) return FAVEST_EINVAL;
    int st = check_device(p);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    const void *ac = a, *bc = b;
    void *Tc = T;
    if (p.cg_real) {
        e = timed(p, KID_CG_PACK, s, [&] { return launch_cg_pack_coefs(p, a, b, s); });
        ac = p.d_cga;
        bc = p.d_cgb;
        Tc = p.d_cgT;
    }
    // Thm. 2: summed nu/eta coefficients, three scalar syntheses of degree L+1
    if (e == cudaSuccess) e = timed(p, KID_CG_UNCOMBINE, s, [&] { return launch_cg_uncombine(p, ac, bc, s); });
    if (e == cudaSuccess) e = timed(p, KID_SYNTHESIS, s, [&] { return launch_synthesis_fp64(p, s); });
    if (e == cudaSuccess) e = timed(p, KID_FFT_INV, s, [&] { return launch_fft_inv_fp64(p, Tc, Tc, s); });
    if (e == cudaSuccess && p.cg_real) e = timed(p, KID_CG_UNPACK, s, [&] { return launch_cg_unpack_fields(p, T, s); });
    return cuda_status(e);
}

int favest_set_weights_unit(favest_plan plan, int flag)
{
    if (!plan || (flag != 0 && flag != 1)) return FAVEST_EINVAL;
    plan->p.unit_weights = flag;
    return FAVEST_OK;
}

int favest_plan_L(favest_plan plan) { return plan ? plan->p.L : FAVEST_EINVAL; }
int favest_plan_batch(favest_plan plan) { return plan ? (plan->p.cg_real ? plan->p.cg_real : plan->p.B) : FAVEST_EINVAL; }
int favest_plan_precision(favest_plan plan) { return plan ? plan->p.precision : FAVEST_EINVAL; }
size_t favest_plan_workspace_bytes(favest_plan plan) { return plan ? plan->p.ws_bytes : 0; }

int favest_launches_per_call(favest_plan plan, int adjoint)
{
    if (!plan) return FAVEST_EINVAL;
    if (plan->p.precision != FAVEST_BF16X6) return 3;
    return (adjoint && plan->p.pol_jc > 0) ? 5 : 4;
}

int favest_status(favest_plan plan, void *stream)
{
    if (!plan) return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return FAVEST_ECUDA;
    int v = 0;
    if (cudaMemcpy(&v, p.d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return FAVEST_ECUDA;
    if (v != 0) cudaMemset(p.d_status, 0, sizeof(int));
    return v;
}

int favest_profile_enable(favest_plan plan, int enable)
{
    if (!plan || (enable != 0 && enable != 1)) return FAVEST_EINVAL;
    plan->p.profiling = enable;
    return FAVEST_OK;
}

int favest_profile_read(favest_plan plan, int max_kernels, char *names, double *ms, long long *launches)
{
    if (!plan || max_kernels < 0 || (max_kernels > 0 && (!names || !ms || !launches))) return FAVEST_EINVAL;
    Plan &p = plan->p;
    double tot[KID_COUNT] = {0};
    long long cnt[KID_COUNT] = {0};
    int status = FAVEST_OK;
    for (auto &r : p.recs) {
        float t = 0.f;
        if (cudaEventSynchronize(r.e1) != cudaSuccess || cudaEventElapsedTime(&t, r.e0, r.e1) != cudaSuccess)
            status = FAVEST_ECUDA;
        tot[r.kernel] += t;
        cnt[r.kernel] += 1;
        p.event_pool.push_back(r.e0);
        p.event_pool.push_back(r.e1);
    }
    p.recs.clear();
    if (status != FAVEST_OK) return status;
    int k = 0;
    for (int i = 0; i < KID_COUNT && k < max_kernels; ++i) {
        if (!cnt[i]) continue;
        std::snprintf(names + 32 * k, 32, "%s", kKernelNames[i]);
        ms[k] = tot[i];
        launches[k] = cnt[i];
        ++k;
    }
    return k;
}

int favest_selftest_wait_timeout(favest_plan plan, unsigned poll_limit, double *elapsed_ms)
{
    if (!plan || poll_limit == 0) return FAVEST_EINVAL;
    Plan &p = plan->p;
    if (p.precision != FAVEST_BF16X6) return FAVEST_EUNSUPPORTED;
    int st = check_device(p);
    if (st) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return FAVEST_ECUDA;
    cudaEventRecord(e0, 0);
    cudaError_t e = launch_gemm_selftest(p, poll_limit, 0);
    cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return FAVEST_ECUDA;
    if (elapsed_ms) *elapsed_ms = ms;
    return favest_status(plan, nullptr);   // reads and clears the status word
}

int favest_kernel_work(favest_plan plan, const char *kernel, double *bytes, double *flops, int *pipe)
{
    if (!plan || !kernel || !bytes || !flops || !pipe) return FAVEST_EINVAL;
    const Plan &p = plan->p;
    const double L = p.L, B = p.B, J = p.J, L1 = p.L + 1, K = (double)p.L * p.L + 2.0 * p.L;
    const double nlat = p.nlat, nphi = p.nphi;
    // recurrence steps: rows l = mu..L+1 of every order, at every folded latitude
    double rows = 0;
    for (int mu = 0; mu <= p.L + (p.nscal > 0 ? 1 : 0); ++mu) rows += p.L + 2 - mu;
    const double steps = rows * J;
    const std::string k(kernel);
    *bytes = 0;
    *flops = 0;
    *pipe = 0;
    if (p.precision == FAVEST_BF16X6) {
        // G column groups of 8 (a complex field, or a pair of real fields); real fields
        // are 4-byte values and keep KR = L(L+3)/2 coefficients per family
        const double G = p.ncg;
        const double grid = 2.0 * B * nlat * nphi * (p.real ? 4.0 : 8.0);
        const double coef = 2.0 * B * (p.real ? (double)p.L * (p.L + 3) / 2.0 : K) * 8.0;
        const double kc = p.real ? (double)p.L * (p.L + 3) / 2.0 : K;
        const double fftf = 2.0 * G * nlat * 5.0 * nphi * std::log2(nphi);
        // generator and GEMMs: the values and (row, latitude) pairs above the turning
        // bound, i.e. the work these kernels are given (the rest is below 1e-13)
        const double gv = p.gen_values, pf = p.gemm_pairs_f, pa = p.gemm_pairs_a;
        if (k == "fft_fwd") { *bytes = grid + J * G * L1 * 64.0; *flops = fftf; }
        else if (k == "fft_inv") { *bytes = J * G * L1 * 64.0 + grid; *flops = fftf; }
        // the generator runs its recurrence in double-float FP32 arithmetic and is bound by
        // its writes (6 bytes per value, in the one layout both directions read)
        else if (k == "gen_lambda_fwd" || k == "gen_lambda_adj" || k == "gen_lambda_both") {
            *bytes = gv * 6.0;          // one layout serves both directions
            *flops = gv * 4.0;
        }
        else if (k == "tc_gemm_fwd") { *bytes = pf * 6.0 + J * G * L1 * 64.0 + rows * G * 32.0; *flops = 12.0 * pf * 8.0 * G; }
        else if (k == "tc_gemm_adj") { *bytes = pa * 6.0 + rows * G * 48.0 + J * G * L1 * 64.0; *flops = 12.0 * pa * 8.0 * G; }
        else if (k == "combine") { *bytes = rows * G * 32.0 + coef; *flops = 16.0 * B * kc; }
        else if (k == "uncombine") { *bytes = coef + rows * G * 48.0; *flops = 24.0 * B * kc; }
        else if (k == "polar_patch") {
            const double jc = p.pol_jc, mc = p.pol_muc;
            *bytes = jc * L1 * mc * 8.0 + 2.0 * B * L * (p.real ? 1.0 : 2.0) * mc * 8.0 + jc * G * mc * 64.0;
            *flops = jc * mc * L * G * 32.0;
            *pipe = 3;
        } else return FAVEST_EINVAL;
        return FAVEST_OK;
    }
    // field and coefficient element bytes
    const double io = p.io == FAVEST_IO_C128 ? 16.0 : (p.io == FAVEST_IO_R32 ? 4.0 : 8.0);
    const double cio = (p.io == FAVEST_IO_C128 || p.io == FAVEST_IO_R64) ? 16.0 : 8.0;
    const double kc = p.real ? (double)p.L * (p.L + 3) / 2.0 : K;
    // component planes: 2 per field, or the 3 Cartesian scalar fields of the CG route
    const double planes = p.nscal > 0 ? (double)p.nscal : 2.0 * B;
    const double grid = planes * nlat * nphi * io;
    const double nmu = p.L + 1 + (p.nscal > 0 ? 1 : 0);
    const double fbuf = nmu * p.ncol * nlat * 16.0, qbuf = (double)p.ntab * p.ncol * 16.0;
    const double gbuf = p.ncol / 2.0 * nlat * nphi * 16.0;
    // per step: 2 recurrence instructions + 2 FMAs (re, im) per column
    const double leg = steps * (4.0 + 4.0 * p.ncol);
    const double fftf = (p.real ? B : planes) * nlat * 5.0 * nphi * std::log2(nphi);
    if (k == "fft_fwd") { *bytes = grid + fbuf; *flops = fftf; }
    else if (k == "fft_inv") { *bytes = gbuf + grid; *flops = fftf; }
    else if (k == "legendre_analysis") { *bytes = fbuf + qbuf; *flops = leg; *pipe = 1; }
    else if (k == "legendre_synthesis") { *bytes = qbuf + gbuf; *flops = leg; *pipe = 1; }
    else if (k == "combine") { *bytes = qbuf + 2.0 * B * kc * cio; *flops = 16.0 * B * kc; }
    else if (k == "uncombine") { *bytes = 2.0 * B * kc * cio + qbuf; *flops = 24.0 * B * kc; }
    else if (k == "cg_combine") { *bytes = qbuf + 2.0 * B * K * cio; *flops = 120.0 * B * K; }
    else if (k == "cg_uncombine") { *bytes = 2.0 * B * K * cio + qbuf; *flops = 120.0 * B * (L + 2) * (L + 2); }
    else return FAVEST_EINVAL;
    return FAVEST_OK;
}

void favest_plan_destroy(favest_plan plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    release_events(plan->p);
    free_plan(plan->p);
    delete plan;
}

}  // extern "C"
