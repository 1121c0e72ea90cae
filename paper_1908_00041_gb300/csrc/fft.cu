// Longitude DFT stage: one complex DFT of length nphi = 2(L+1) per latitude ring,
// component and field, done in shared memory by a mixed-radix Stockham FFT
// (radices 4, 2, then odd primes; an odd prime p uses a direct p-point DFT).
// Twiddles are FP64 values of exp(-2 pi i k / n) formed on the host from exactly
// reduced angles.
#include "favest_internal.h"
#include "fft_device.cuh"

namespace favest {

namespace {

// Forward: read ring (b, c, j) of T (io type TI), FFT in FP64, scatter bins m = -L..L
// into Fraw[mu][col][j], col = (b*2 + c)*2 + (m < 0).
// Scalar mode (nscal > 0, the Clebsch-Gordan route): ring (s = b*2 + c, j) is plane s of
// Tth (planes of nlat*nphi elements back to back), rings s >= nscal are zero, and the
// bins run to m = +-(L+1): both take the Nyquist bin n/2, which is order L+1 of the
// degree-(L+1) scalar transforms on this grid.
template <typename TI>
__global__ void __launch_bounds__(256) k_fft_fwd_fp64(
    const TI *__restrict__ Tth, const TI *__restrict__ Tph, double2 *__restrict__ Fraw,
    RadixPlanArg rp, const double2 *__restrict__ tw, int L, int nlat, int ncol, const long long *__restrict__ toff,
    int nscal)
{
    extern __shared__ double2 sm_fft[];
    const int n = rp.n;
    const int ring = blockIdx.x;               // ((b*2 + c) * nlat + j)
    const int j = ring % nlat;
    const int bc = ring / nlat;
    const int c = bc & 1, b = bc >> 1;
    double2 *buf0 = sm_fft, *buf1 = sm_fft + n;
    if (nscal > 0) {
        const bool live = bc < nscal;
        const TI *src = Tth + ((size_t)bc * nlat + j) * n;
        for (int k = threadIdx.x; k < n; k += blockDim.x) buf0[k] = live ? to_d2(src[k]) : make_double2(0.0, 0.0);
    } else {
        const size_t fb = toff ? (size_t)toff[b] : (size_t)b * nlat * n;   // field b's plane
        const TI *src = (c == 0 ? Tth : Tph) + fb + (size_t)j * n;
        for (int k = threadIdx.x; k < n; k += blockDim.x) buf0[k] = to_d2(src[k]);
    }
    __syncthreads();
    const double2 *out = stockham<false>(buf0, buf1, tw, rp);
    const int mmax = nscal > 0 ? L + 1 : L;
    for (int m = -mmax + (int)threadIdx.x; m <= mmax; m += blockDim.x) {
        int bin = m < 0 ? m + n : m;
        double2 v = out[bin];
        int mu = m < 0 ? -m : m;
        int col0 = (b * 2 + c) * 2;
        size_t base = (size_t)mu * ncol;
        if (m <= 0) Fraw[(base + col0 + 1) * nlat + j] = v;
        if (m >= 0) Fraw[(base + col0 + 0) * nlat + j] = v;
    }
}

// Inverse: read spectrum row G[b][c][j][bin] (Nyquist bin L+1 taken as zero), inverse
// FFT (no 1/n), scale by wring[j] when given (the weighted adjoint W A c), write ring
// to T (io type TO).  Scalar mode (nscal > 0): ring s goes to plane s of Tth (s < nscal)
// and the Nyquist bin, written by the synthesis for order L+1, is kept.
template <typename TO>
__global__ void __launch_bounds__(256) k_fft_inv_fp64(
    const double2 *__restrict__ G, TO *__restrict__ Tth, TO *__restrict__ Tph,
    RadixPlanArg rp, const double2 *__restrict__ tw, const double *__restrict__ wring, int L, int nlat,
    const long long *__restrict__ toff, int nscal)
{
    extern __shared__ double2 sm_fft[];
    const int n = rp.n;
    const int ring = blockIdx.x;
    const int j = ring % nlat;
    const int bc = ring / nlat;
    const int c = bc & 1, b = bc >> 1;
    if (nscal > 0 && bc >= nscal) return;      // uniform over the CTA
    const double2 *src = G + (size_t)ring * n;
    double2 *buf0 = sm_fft, *buf1 = sm_fft + n;
    for (int k = threadIdx.x; k < n; k += blockDim.x)
        buf0[k] = (k == L + 1 && nscal == 0) ? make_double2(0.0, 0.0) : src[k];
    __syncthreads();
    const double2 *out = stockham<true>(buf0, buf1, tw, rp);
    const size_t fb = nscal > 0 ? (size_t)bc * nlat * n : toff ? (size_t)toff[b] : (size_t)b * nlat * n;
    TO *dst = (nscal > 0 || c == 0 ? Tth : Tph) + fb + (size_t)j * n;
    if (wring) {
        const double w = wring[j];
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double2 v = out[k];
            dst[k] = from_d2<TO>(make_double2(w * v.x, w * v.y));
        }
    } else {
        for (int k = threadIdx.x; k < n; k += blockDim.x) dst[k] = from_d2<TO>(out[k]);
    }
}

// Real fields.  Ring (field b, j) carries z = T_th + i T_ph (both real), whose spectrum Z
// gives both component spectra: F_th(m) = (Z(m) + conj Z(-m)) / 2, F_ph(m) = (Z(m) -
// conj Z(-m)) / (2i), kept for m = 0..L (F(-m) = conj F(m)).  The fields 2q and 2q+1 share
// the column group of 4 of pair q: col = (q*2 + c)*2 + (b % 2).
template <typename TR>
__global__ void __launch_bounds__(256) k_rfft_fwd_fp64(
    const TR *__restrict__ Tth, const TR *__restrict__ Tph, double2 *__restrict__ Fraw, RadixPlanArg rp,
    const double2 *__restrict__ tw, int L, int nlat, int ncol, const long long *__restrict__ toff)
{
    extern __shared__ double2 sm_fft[];
    const int n = rp.n;
    const int ring = blockIdx.x;               // b * nlat + j
    const int j = ring % nlat, b = ring / nlat;
    const size_t fb = (toff ? (size_t)toff[b] : (size_t)b * nlat * n) + (size_t)j * n;
    const TR *st = Tth + fb, *sp = Tph + fb;
    double2 *buf0 = sm_fft, *buf1 = sm_fft + n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) buf0[k] = make_double2((double)st[k], (double)sp[k]);
    __syncthreads();
    const double2 *out = stockham<false>(buf0, buf1, tw, rp);
    const int q = b >> 1, f = b & 1;
    for (int m = threadIdx.x; m <= L; m += blockDim.x) {
        const double2 z = out[m], zc = out[m == 0 ? 0 : n - m];
        const double2 fth = make_double2(0.5 * (z.x + zc.x), 0.5 * (z.y - zc.y));
        const double2 fph = make_double2(0.5 * (z.y + zc.y), 0.5 * (zc.x - z.x));
        const size_t base = (size_t)m * ncol;
        Fraw[(base + (q * 2 + 0) * 2 + f) * nlat + j] = fth;
        Fraw[(base + (q * 2 + 1) * 2 + f) * nlat + j] = fph;
    }
}

// Real fields, inverse: the synthesis leaves G_c(j, m), m = 0..L, in row b*2 + c; the
// spectrum of z = T_th + i T_ph is Z(m) = G_th(m) + i G_ph(m), Z(-m) = conj G_th(m) +
// i conj G_ph(m) (m >= 1), Z(0) = Re G_th(0) + i Re G_ph(0), and the Nyquist bin 0.
template <typename TR>
__global__ void __launch_bounds__(256) k_rfft_inv_fp64(
    const double2 *__restrict__ G, TR *__restrict__ Tth, TR *__restrict__ Tph, RadixPlanArg rp,
    const double2 *__restrict__ tw, const double *__restrict__ wring, int L, int nlat,
    const long long *__restrict__ toff)
{
    extern __shared__ double2 sm_fft[];
    const int n = rp.n;
    const int ring = blockIdx.x;               // b * nlat + j
    const int j = ring % nlat, b = ring / nlat;
    const double2 *gt = G + ((size_t)(b * 2 + 0) * nlat + j) * n;
    const double2 *gp = G + ((size_t)(b * 2 + 1) * nlat + j) * n;
    double2 *buf0 = sm_fft, *buf1 = sm_fft + n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double2 v = make_double2(0.0, 0.0);
        if (k == 0) {
            v = make_double2(gt[0].x, gp[0].x);
        } else if (k <= L) {
            const double2 a = gt[k], c = gp[k];
            v = make_double2(a.x - c.y, a.y + c.x);
        } else if (k > L + 1) {
            const double2 a = gt[n - k], c = gp[n - k];
            v = make_double2(a.x + c.y, c.x - a.y);
        }
        buf0[k] = v;
    }
    __syncthreads();
    const double2 *out = stockham<true>(buf0, buf1, tw, rp);
    const double w = wring ? wring[j] : 1.0;
    const size_t fb = (toff ? (size_t)toff[b] : (size_t)b * nlat * n) + (size_t)j * n;
    TR *dt = Tth + fb, *dp = Tph + fb;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        dt[k] = (TR)(w * out[k].x);
        dp[k] = (TR)(w * out[k].y);
    }
}

int fft_threads(int n) { return n >= 512 ? 256 : (n >= 128 ? 128 : 64); }

}  // namespace

cudaError_t launch_fft_fwd_fp64(const Plan &p, const void *Tth, const void *Tph, cudaStream_t s)
{
    RadixPlanArg rp = make_radix_arg(p.fft);
    if (p.real) {
        const size_t smem = 2 * (size_t)p.nphi * sizeof(double2);
        const int th = fft_threads(p.nphi);
        if (p.io == FAVEST_IO_R64) {
            auto k = k_rfft_fwd_fp64<double>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<p.B * p.nlat, th, smem, s>>>((const double *)Tth, (const double *)Tph, (double2 *)p.d_F, rp,
                                             p.fft.tw64, p.L, p.nlat, p.ncol, p.d_toff);
        } else {
            auto k = k_rfft_fwd_fp64<float>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<p.B * p.nlat, th, smem, s>>>((const float *)Tth, (const float *)Tph, (double2 *)p.d_F, rp,
                                             p.fft.tw64, p.L, p.nlat, p.ncol, p.d_toff);
        }
        return cudaGetLastError();
    }
    int grid = p.ncol / 4 * 2 * p.nlat;        // rings: 2 per group of 4 columns (b, c)
    size_t smem = 2 * (size_t)p.nphi * sizeof(double2);
    int th = fft_threads(p.nphi);
    if (p.io == FAVEST_IO_C128) {
        auto k = k_fft_fwd_fp64<double2>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, th, smem, s>>>((const double2 *)Tth, (const double2 *)Tph, (double2 *)p.d_F,
                                 rp, p.fft.tw64, p.L, p.nlat, p.ncol, p.d_toff, p.nscal);
    } else {
        auto k = k_fft_fwd_fp64<float2>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, th, smem, s>>>((const float2 *)Tth, (const float2 *)Tph, (double2 *)p.d_F,
                                 rp, p.fft.tw64, p.L, p.nlat, p.ncol, p.d_toff, p.nscal);
    }
    return cudaGetLastError();
}

cudaError_t launch_fft_inv_fp64(const Plan &p, void *Tth, void *Tph, cudaStream_t s)
{
    RadixPlanArg rp = make_radix_arg(p.fft);
    if (p.real) {
        const size_t smem = 2 * (size_t)p.nphi * sizeof(double2);
        const int th = fft_threads(p.nphi);
        const double *wr = p.adj_weighted ? p.d_wring : nullptr;
        if (p.io == FAVEST_IO_R64) {
            auto k = k_rfft_inv_fp64<double>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<p.B * p.nlat, th, smem, s>>>((const double2 *)p.d_G, (double *)Tth, (double *)Tph, rp, p.fft.tw64,
                                             wr, p.L, p.nlat, p.d_toff);
        } else {
            auto k = k_rfft_inv_fp64<float>;
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k<<<p.B * p.nlat, th, smem, s>>>((const double2 *)p.d_G, (float *)Tth, (float *)Tph, rp, p.fft.tw64,
                                             wr, p.L, p.nlat, p.d_toff);
        }
        return cudaGetLastError();
    }
    int grid = p.ncol / 4 * 2 * p.nlat;
    size_t smem = 2 * (size_t)p.nphi * sizeof(double2);
    int th = fft_threads(p.nphi);
    if (p.io == FAVEST_IO_C128) {
        auto k = k_fft_inv_fp64<double2>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, th, smem, s>>>((const double2 *)p.d_G, (double2 *)Tth, (double2 *)Tph, rp,
                                 p.fft.tw64, p.adj_weighted ? p.d_wring : nullptr, p.L, p.nlat, p.d_toff,
                                 p.nscal);
    } else {
        auto k = k_fft_inv_fp64<float2>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<grid, th, smem, s>>>((const double2 *)p.d_G, (float2 *)Tth, (float2 *)Tph, rp,
                                 p.fft.tw64, p.adj_weighted ? p.d_wring : nullptr, p.L, p.nlat, p.d_toff,
                                 p.nscal);
    }
    return cudaGetLastError();
}

}  // namespace favest
