// FP64 Legendre stage: the scaled FP64 recurrence fused with the quadrature-weighted
// contraction (forward) or with the coefficient sum (adjoint), one CTA per
// (order mu, column group).  Equatorial symmetry lambda_l^m(-x) = (-1)^{l+m} lambda_l^m(x)
// folds each latitude pair (j, nlat-1-j) into one recurrence.
#include "favest_internal.h"
#include "recurrence.cuh"

namespace favest {

namespace {

// Eight warps per CTA: the FP64 units sit in the SM's four sub-partitions, so fewer than
// four resident warps cannot keep the FP64 pipe full.  The synthesis takes ceil(J / 64)
// warps on small grids, two latitudes per thread: warps without latitudes would still issue
// their FP64 instructions into the same pipe.
constexpr int kAnaThreads = 256;
constexpr int kAnaJpt = 2;        // latitudes per recurrence thread up to J = 512 (L <= 1023)
constexpr int kBigJpt = 5;        // beyond: J <= 1280 (L <= 2559)
constexpr int kWin = 4;           // rows per renormalisation window of the synthesis (even)

// Forward Legendre stage.  Fraw: [mu][ncol][nlat] raw longitude spectra; Q: [tab][ncol].
// The reduction over latitudes is what makes this stage costly if every thread keeps the
// partial sums of its own latitudes: a warp reduction per window of rows then costs every
// lane V*31/32 additions for V values (about 30% of the FP64 instructions at 4 columns; that
// form ran at 0.62 of the FP64 rate at L = 1023).  Here the recurrence threads (two
// latitudes each) write a window of R rows of values y_l(x_j) to
// shared memory, and the contraction threads then each own one output (row, column) and a
// strided subset of the latitudes, so the only reduction left is over the TPO threads of an
// output (TPO - 1 adds per window and output).  Windows are double-buffered: one barrier per
// window separates the recurrence of window k+1 from the contraction of window k.
template <int CT, int R, int JPT>
__global__ void __launch_bounds__(kAnaThreads) k_analysis_fp64_t(
    const double2 *__restrict__ Fraw, double2 *__restrict__ Q, const double *__restrict__ xj,
    const double *__restrict__ sj, const double *__restrict__ omega, const double *__restrict__ cmu,
    const double *__restrict__ Atab, int L, int nlat, int J, int has_eq, int ncol, int ng)
{
    constexpr int NOUT = R * CT, TPO = kAnaThreads / NOUT;
    static_assert(kAnaThreads % NOUT == 0 && TPO >= 1 && TPO <= 32 && (TPO & (TPO - 1)) == 0, "output mapping");
    // a warp's lanes then share one window row, so the shuffles below run warp-uniformly
    static_assert(R <= 8 && 8 % R == 0, "window rows");
    extern __shared__ double sm_ana[];
    const int mu = blockIdx.x / ng, g = blockIdx.x % ng;
    const int nrow = L + 2 - mu;
    const long long t0 = tab_off(L, mu);
    double2 *Fs = reinterpret_cast<double2 *>(sm_ana);          // [2][CT][J]
    double *Y = sm_ana + 2 * 2 * CT * J;                        // [2][R][J]
    double *As = Y + 2 * R * J;                                 // [nrow]

    for (int idx = threadIdx.x; idx < CT * J; idx += blockDim.x) {
        int ct = idx / J, j = idx % J;
        const double2 *src = Fraw + ((size_t)mu * ncol + g * CT + ct) * nlat;
        double2 f1 = src[j];
        double w = omega[j];
        double2 fp, fm;
        if (has_eq && j == J - 1) {
            fp = make_double2(w * f1.x, w * f1.y);
            fm = make_double2(0.0, 0.0);
        } else {
            double2 f2 = src[nlat - 1 - j];
            fp = make_double2(w * (f1.x + f2.x), w * (f1.y + f2.y));
            fm = make_double2(w * (f1.x - f2.x), w * (f1.y - f2.y));
        }
        Fs[(0 * CT + ct) * J + j] = fp;
        Fs[(1 * CT + ct) * J + j] = fm;
    }
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) As[r] = Atab[t0 + r];
    __syncthreads();

    // recurrence role: latitudes threadIdx.x + i * kAnaThreads
    double x[JPT], y1[JPT], y2[JPT];
    int c[JPT];
    const double cm = cmu[mu];
#pragma unroll
    for (int i = 0; i < JPT; ++i) {
        int j = threadIdx.x + i * kAnaThreads;
        x[i] = 0.0; y1[i] = 0.0; y2[i] = 0.0; c[i] = 1 << 20;
        if (j < J) {
            x[i] = xj[j];
            sectoral_start(cm, sj[j], mu, y1[i], c[i]);
        }
    }
    // contraction role: output (row w of the window, column ct), latitudes jsub + k TPO
    const int out = threadIdx.x / TPO, jsub = threadIdx.x % TPO;
    const int wo = out / CT, cto = out % CT;

    for (int r0 = 0, buf = 0; r0 < nrow; r0 += R, buf ^= 1) {
        double *Yb = Y + buf * R * J;
#pragma unroll
        for (int w = 0; w < R; ++w) {
            const int r = r0 + w;
            if (r < nrow) {
                const double a = As[r];
#pragma unroll
                for (int i = 0; i < JPT; ++i) {
                    const int j = threadIdx.x + i * kAnaThreads;
                    if (j < J) {
                        double yl = y1[i];
                        if (r > 0) {
                            yl = fma(a * x[i], y1[i], -y2[i]);
                            y2[i] = y1[i];
                            y1[i] = yl;
                        }
                        Yb[w * J + j] = (c[i] == 0) ? yl : 0.0;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < JPT; ++i) renorm(y1[i], y2[i], c[i]);
        __syncthreads();
        const int r = r0 + wo;
        if (r < nrow) {                        // uniform over the TPO lanes of an output
            const double *yr = Yb + wo * J;
            const double2 *fr = Fs + ((r & 1) * CT + cto) * J;   // parity of l + mu = parity of r
            double ax = 0.0, ay = 0.0, bx = 0.0, by = 0.0;
            int j = jsub;
            for (; j + TPO < J; j += 2 * TPO) {
                const double ya = yr[j], yb = yr[j + TPO];
                const double2 fa = fr[j], fb = fr[j + TPO];
                ax = fma(ya, fa.x, ax);
                ay = fma(ya, fa.y, ay);
                bx = fma(yb, fb.x, bx);
                by = fma(yb, fb.y, by);
            }
            if (j < J) {
                const double ya = yr[j];
                const double2 fa = fr[j];
                ax = fma(ya, fa.x, ax);
                ay = fma(ya, fa.y, ay);
            }
            ax += bx;
            ay += by;
#pragma unroll
            for (int o = TPO / 2; o >= 1; o >>= 1) {
                ax += __shfl_xor_sync(0xffffffffu, ax, o, TPO);
                ay += __shfl_xor_sync(0xffffffffu, ay, o, TPO);
            }
            if (jsub == 0) Q[(size_t)(t0 + r) * ncol + g * CT + cto] = make_double2(ax, ay);
        }
    }
}

constexpr int kSynThreads = 256;

// Adjoint Legendre stage.  gtab: [tab][ncol] scaled coefficients; G: [B][2][nlat][nphi].
// Vector mode divides the sums by sin(theta_j).  Scalar mode (the Clebsch-Gordan route)
// does not, and order L+1 exists there: its orders +-(L+1) share the Nyquist bin, so the
// two sign columns are added into it.  Real fields (real != 0): column (q*2 + c)*2 + f is
// component c of field 2q + f at m = +mu, written to row (2q + f)*2 + c at bin mu.
template <int CT, int JPT>
__global__ void __launch_bounds__(kSynThreads) k_synthesis_fp64(
    const double2 *__restrict__ gtab, double2 *__restrict__ G, const double *__restrict__ xj,
    const double *__restrict__ sj, const double *__restrict__ cmu, const double *__restrict__ Atab,
    int L, int nlat, int nphi, int J, int has_eq, int ncol, int ng, int scalar, int real)
{
    extern __shared__ double sm_syn[];
    const int mu = blockIdx.x / ng, g = blockIdx.x % ng;
    const int nrow = L + 2 - mu;
    const long long t0 = tab_off(L, mu);
    double2 *gs = reinterpret_cast<double2 *>(sm_syn);   // [nrow][CT]
    double *As = sm_syn + 2 * CT * nrow;                 // [nrow]
    for (int idx = threadIdx.x; idx < nrow * CT; idx += blockDim.x) {
        int r = idx / CT, ct = idx % CT;
        gs[idx] = gtab[(size_t)(t0 + r) * ncol + g * CT + ct];
    }
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) As[r] = Atab[t0 + r];
    __syncthreads();

    double x[JPT], y1[JPT], y2[JPT];
    int c[JPT];
    double2 accE[JPT][CT], accO[JPT][CT];
    const double cm = cmu[mu];
#pragma unroll
    for (int i = 0; i < JPT; ++i) {
        int j = threadIdx.x + i * blockDim.x;
        x[i] = 0.0; y1[i] = 0.0; y2[i] = 0.0; c[i] = 1 << 20;
        if (j < J) {
            x[i] = xj[j];
            sectoral_start(cm, sj[j], mu, y1[i], c[i]);
        }
#pragma unroll
        for (int ct = 0; ct < CT; ++ct) {
            accE[i][ct] = make_double2(0.0, 0.0);
            accO[i][ct] = make_double2(0.0, 0.0);
        }
    }
    for (int r0 = 0; r0 < nrow; r0 += kWin) {
#pragma unroll
        for (int w = 0; w < kWin; ++w) {
            const int r = r0 + w;
            if (r < nrow) {
                const double a = As[r];
#pragma unroll
                for (int i = 0; i < JPT; ++i) {
                    double yl = y1[i];
                    if (r > 0) {
                        yl = fma(a * x[i], y1[i], -y2[i]);
                        y2[i] = y1[i];
                        y1[i] = yl;
                    }
                    const double yv = (c[i] == 0) ? yl : 0.0;
#pragma unroll
                    for (int ct = 0; ct < CT; ++ct) {
                        double2 gv = gs[r * CT + ct];
                        if (w & 1) {
                            accO[i][ct].x = fma(yv, gv.x, accO[i][ct].x);
                            accO[i][ct].y = fma(yv, gv.y, accO[i][ct].y);
                        } else {
                            accE[i][ct].x = fma(yv, gv.x, accE[i][ct].x);
                            accE[i][ct].y = fma(yv, gv.y, accE[i][ct].y);
                        }
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < JPT; ++i) renorm(y1[i], y2[i], c[i]);
    }
#pragma unroll
    for (int i = 0; i < JPT; ++i) {
        const int j = threadIdx.x + i * blockDim.x;
        if (j >= J) continue;
        const double is = scalar ? 1.0 : 1.0 / sj[j];
        const bool eq = has_eq && j == J - 1;
        const bool nyq = mu == L + 1;                 // scalar mode only
#pragma unroll
        for (int ct = 0; ct < CT; ++ct) {
            const int col = g * CT + ct;
            const int s = col & 1;
            const int bc = real ? ((col >> 2) * 2 + s) * 2 + ((col >> 1) & 1) : col >> 1;   // output row
            if (!real && (mu == 0 || nyq) && s == 1) continue;
            const int bin = (s && !real) ? nphi - mu : mu;
            double2 e = accE[i][ct], o = accO[i][ct];
            if (nyq && ct + 1 < CT) {                 // add the m = -(L+1) column (ct + 1)
                e.x += accE[i][ct + 1].x;
                e.y += accE[i][ct + 1].y;
                o.x += accO[i][ct + 1].x;
                o.y += accO[i][ct + 1].y;
            }
            G[((size_t)bc * nlat + j) * nphi + bin] = make_double2((e.x + o.x) * is, (e.y + o.y) * is);
            if (!eq)
                G[((size_t)bc * nlat + (nlat - 1 - j)) * nphi + bin] =
                    make_double2((e.x - o.x) * is, (e.y - o.y) * is);
        }
    }
}

}  // namespace

// Threads per CTA of the FP64 Legendre kernels: the warps that J latitudes fill at two per
// thread, raised (up to one latitude per thread) while the grid would leave fewer than about
// 24 warps per SM to hide the FP64 latency (min_warps_grid = 24 x SMs / CTAs; 0: none).
int fp64_threads(int J, int maxthreads, int min_warps_grid)
{
    int w = (J + 63) / 64;
    const int wmax = (J + 31) / 32;
    if (w < min_warps_grid) w = min_warps_grid < wmax ? min_warps_grid : wmax;
    if (w < 1) w = 1;
    return w * 32 < maxthreads ? w * 32 : maxthreads;
}

template <int CT, int R, int JPT>
cudaError_t launch_analysis_t(const Plan &p, cudaStream_t s, const double *omega)
{
    const int ngt = p.ncol / CT;
    const int grid = (p.L + 1 + (p.nscal > 0 ? 1 : 0)) * ngt;
    const int nrowmax = p.L + 2;
    const size_t smem = (size_t)(4 * CT * p.J + 2 * R * p.J + ((nrowmax + 1) & ~1)) * sizeof(double);
    auto k = k_analysis_fp64_t<CT, R, JPT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, kAnaThreads, smem, s>>>((const double2 *)p.d_F, (double2 *)p.d_Q, p.d_x, p.d_sin, omega, p.d_cmu,
                                      p.d_A, p.L, p.nlat, p.J, p.has_eq, p.ncol, ngt);
    return cudaGetLastError();
}

// Shared memory of one analysis CTA (bytes) and the largest a CTA may take on sm_100-class
// parts.
size_t analysis_smem(int CT, int R, int J, int L) { return (size_t)(4 * CT * J + 2 * R * J + L + 3) * 8; }
constexpr size_t kMaxSmem = 227 * 1024;

cudaError_t launch_analysis_fp64(const Plan &p, cudaStream_t s)
{
    if (p.J > kAnaThreads * kBigJpt) return cudaErrorInvalidValue;
    // orders 0..L, and L+1 for the scalar transforms of degree L+1 (Clebsch-Gordan route).
    // Windows of 8 rows and 8 columns per CTA where the columns allow, else 4 (measured on
    // GB300: L = 1023, 32 fields 214 -> 134 ms; L = 511, one field 1.34 -> 1.10 ms against the
    // per-thread reduction form).  Beyond 512 latitudes the staged spectra and windows must
    // still fit one CTA's shared memory: 4 columns with 2-row windows, else 2 columns with
    // 4-row windows (J <= 1280).
    const double *omega = p.nscal > 0 ? p.d_wring : p.unit_weights ? p.d_omega_unit : p.d_omega;
    if (p.J <= kAnaThreads * kAnaJpt)
        return p.ncol % 8 == 0 ? launch_analysis_t<8, 8, kAnaJpt>(p, s, omega)
                               : launch_analysis_t<4, 8, kAnaJpt>(p, s, omega);
    if (analysis_smem(4, 2, p.J, p.L) <= kMaxSmem) return launch_analysis_t<4, 2, kBigJpt>(p, s, omega);
    return launch_analysis_t<2, 4, kBigJpt>(p, s, omega);
}

template <int CT, int JPT>
cudaError_t launch_synthesis_t(const Plan &p, cudaStream_t s)
{
    const int nt = fp64_threads(p.J, kSynThreads, 0);
    const int ngt = p.ncol / CT;
    const int grid = (p.L + 1 + (p.nscal > 0 ? 1 : 0)) * ngt;
    const int nrowmax = p.L + 2;
    const size_t smem = (size_t)(2 * CT * nrowmax + nrowmax) * sizeof(double);
    auto k = k_synthesis_fp64<CT, JPT>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<grid, nt, smem, s>>>((const double2 *)p.d_Q, (double2 *)p.d_G, p.d_x, p.d_sin, p.d_cmu, p.d_A, p.L,
                             p.nlat, p.nphi, p.J, p.has_eq, p.ncol, ngt, p.nscal > 0, p.real);
    return cudaGetLastError();
}

cudaError_t launch_synthesis_fp64(const Plan &p, cudaStream_t s)
{
    if (p.J > kSynThreads * kBigJpt) return cudaErrorInvalidValue;
    // beyond 512 latitudes: five per thread and two columns per CTA (the accumulators of
    // JPT latitudes x CT columns live in registers)
    if (p.J > kSynThreads * kAnaJpt) return launch_synthesis_t<2, kBigJpt>(p, s);
    return p.ct == 8 ? launch_synthesis_t<8, kAnaJpt>(p, s) : launch_synthesis_t<4, kAnaJpt>(p, s);
}

}  // namespace favest
