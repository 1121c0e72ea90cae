// favest_fwd_fp64_noalloc: the FP64 forward transform without any device allocation.
//
// Some callers cannot allocate device memory at the point where they need a
// transform: code running inside a CUDA graph capture that must not allocate,
// real-time loops that cannot afford allocation latency or failure, plug-ins handed a
// context whose memory is already fully reserved by a pool they do not own.  For them
// this entry point keeps all of its scratch (Gauss-Legendre grid, recurrence and
// combine tables, twiddles, longitude spectra, scalar sums) in one file-scope device
// array of kScratchBytes, created when the library is loaded and held by every GPU that
// loads the library until the process exits.  The caller passes only inputs, outputs
// and a stream.
//
// Set-up: the first call in a CUDA context (with that context's device current) looks
// up the array's device address with cudaGetSymbolAddress and caches it with the
// context's unique id; a later call in another context of the same device (after
// cudaDeviceReset, or under a new primary context) looks it up again.  Make the first
// call in a context outside any stream capture.  Every call rebuilds the constant tables
// in the array, so no state has to survive between calls, and calls that overlap on the
// GPU (different streams, or different host threads) race on the shared array.
//
// The kernels of this path have no device-side waits and record no status: a call
// reports launch failures through its return code only.
#include <cmath>
#include <mutex>

#include "favest_internal.h"

namespace {

constexpr size_t kScratchBytes = 32u << 20;   // 32 MB
constexpr int kMaxDevices = 64;
constexpr int kMaxBatch = 4096;

static __device__ __align__(256) unsigned char g_favest_scratch[kScratchBytes];

std::mutex g_mu;
struct ScratchAddr {
    unsigned long long ctx_id = 0;   // 0: not looked up yet (context ids start at 1)
    void *ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

using PfnCtxGetCurrent = CUresult (*)(CUcontext *);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long *);

// Unique id of the calling thread's current context (driver entry points reached
// through the runtime, so the library does not link the driver library); 0 on failure.
unsigned long long current_ctx_id()
{
    static PfnCtxGetCurrent get_current = nullptr;
    static PfnCtxGetId get_id = nullptr;
    if (!get_current || !get_id) {
        void *f1 = nullptr, *f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || !f1 ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess || !f2)
            return 0;
        get_current = reinterpret_cast<PfnCtxGetCurrent>(f1);
        get_id = reinterpret_cast<PfnCtxGetId>(f2);
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// ---- device-side constant tables (same formulas as the plan builder) ----
__device__ double eps_d(int l, int mu)
{
    double num = (double)(l - mu) * (double)(l + mu);
    double den = (double)(2 * l - 1) * (double)(2 * l + 1);
    return num > 0 ? sqrt(num / den) : 0.0;
}

// Gauss-Legendre nodes (descending) and weights; one thread per node pair.
__global__ void k_na_gl(int n, int J, int nphi, double *x, double *s, double *om, double *omu)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (n + 1) / 2) return;
    const double pi = 3.14159265358979323846;
    double t = pi * (4.0 * i + 3.0) / (4.0 * n + 2.0);
    double z = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(t);
    double pn = 0, dpn = 1;
    for (int it = 0; it < 60; ++it) {
        double pm1 = 1.0, p = z;
        for (int k = 1; k < n; ++k) {
            double pp1 = ((2 * k + 1) * z * p - k * pm1) / (k + 1);
            pm1 = p;
            p = pp1;
        }
        pn = (n == 0) ? 1.0 : p;
        dpn = n * (pm1 - z * p) / ((1.0 - z) * (1.0 + z));
        double dz = pn / dpn;
        z -= dz;
        if (fabs(dz) <= 4e-17 * fabs(z) + 1e-300) break;
    }
    {
        double pm1 = 1.0, p = z;
        for (int k = 1; k < n; ++k) {
            double pp1 = ((2 * k + 1) * z * p - k * pm1) / (k + 1);
            pm1 = p;
            p = pp1;
        }
        dpn = n * (pm1 - z * p) / ((1.0 - z) * (1.0 + z));
    }
    if ((n & 1) && i == n / 2) z = 0.0;
    const double w = 2.0 / ((1.0 - z) * (1.0 + z) * dpn * dpn);
    if (i < J) {
        const double sj = sqrt((1.0 - z) * (1.0 + z));
        x[i] = z;
        s[i] = sj;
        om[i] = w * (2.0 * pi / nphi) / sj;
        omu[i] = 1.0 / sj;
    }
}

// cmu, and per order mu the recurrence multipliers A and combine coefficients P, M, R.
__global__ void k_na_tables(int L, double *cmu, double *A, double *P, double *M, double *R, double *kapbuf)
{
    const int mu = blockIdx.x * blockDim.x + threadIdx.x;
    if (mu > L) return;
    double c = 1.0 / sqrt(4.0 * 3.14159265358979323846);
    for (int k = 1; k <= mu; ++k) c *= sqrt((2.0 * k + 1.0) / (2.0 * k));
    cmu[mu] = c;
    double *kap = kapbuf + (size_t)mu * (L + 3);
    kap[mu] = 1.0;
    kap[mu + 1] = 1.0;
    for (int l = mu + 2; l <= L + 2; ++l) kap[l] = kap[l - 2] * eps_d(l - 1, mu) / eps_d(l, mu);
    const long long t0 = favest::tab_off(L, mu);
    for (int l = mu; l <= L + 1; ++l) {
        const long long t = t0 + (l - mu);
        double a = 0.0;
        if (l == mu + 1) a = sqrt(2.0 * mu + 3.0);
        else if (l >= mu + 2) a = kap[l - 1] / (eps_d(l - 1, mu) * kap[l - 2]);
        A[t] = a;
        const double sl = l >= 1 ? 1.0 / sqrt((double)l * (l + 1.0)) : 0.0;
        P[t] = sl * l * eps_d(l + 1, mu) * kap[l + 1];
        M[t] = (l > mu) ? sl * (l + 1.0) * eps_d(l, mu) * kap[l - 1] : 0.0;
        R[t] = sl * kap[l];
    }
}

__global__ void k_na_twiddles(int n, double2 *tw)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    double sv, cv;
    sincospi(2.0 * (double)k / (double)n, &sv, &cv);
    tw[k] = make_double2(cv, -sv);
}

int factorize_na(int n, int *rad)
{
    int k = 0;
    while (n % 4 == 0 && k < favest::kMaxRadixStages) { rad[k++] = 4; n /= 4; }
    while (n % 2 == 0 && k < favest::kMaxRadixStages) { rad[k++] = 2; n /= 2; }
    for (int f = 3; n > 1 && k < favest::kMaxRadixStages; f += 2)
        while (n % f == 0 && k < favest::kMaxRadixStages) { rad[k++] = f; n /= f; }
    return n == 1 ? k : -1;
}

}  // namespace

extern "C" size_t favest_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" int favest_fwd_fp64_noalloc(int L, int batch, const void *Tth, const void *Tph, void *a, void *b,
                                       void *stream)
{
    using namespace favest;
    if (L < 1 || L > 1023 || batch < 1 || batch > kMaxBatch || !Tth || !Tph || !a || !b) return FAVEST_EINVAL;
    if (((uintptr_t)Tth | (uintptr_t)Tph | (uintptr_t)a | (uintptr_t)b) % 16) return FAVEST_EINVAL;
    // the longitude spectra alone take 64 batch (L+1)^2 bytes: refuse early, before any
    // layout arithmetic (all sizes below are size_t products of values this bounds)
    if ((size_t)batch > kScratchBytes / (64 * (size_t)(L + 1) * (size_t)(L + 1))) return FAVEST_EINVAL;
    const int nlat = L + 1, nphi = 2 * (L + 1), J = (nlat + 1) / 2, ncol = 4 * batch;
    const long long ntab = tab_off(L, L + 1);
    // scratch layout
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t o_x = take((size_t)J * 8), o_s = take((size_t)J * 8), o_om = take((size_t)J * 8),
                 o_omu = take((size_t)J * 8);
    const size_t o_cmu = take((size_t)(L + 1) * 8);
    const size_t o_A = take((size_t)ntab * 8), o_P = take((size_t)ntab * 8), o_M = take((size_t)ntab * 8),
                 o_R = take((size_t)ntab * 8);
    const size_t o_kap = take((size_t)(L + 1) * (L + 3) * 8);
    const size_t o_tw = take((size_t)nphi * 16);
    const size_t o_F = take((size_t)(L + 1) * (size_t)ncol * nlat * 16);
    const size_t o_Q = take((size_t)ntab * (size_t)ncol * 16);
    if (off > kScratchBytes) return FAVEST_EINVAL;   // (L, batch) needs more than 32 MB of scratch

    // An error left unread by an earlier runtime call on this thread would be returned by
    // the launch checks below as if it were this call's: refuse without launching and
    // leave it for its owner to read.
    if (cudaPeekAtLastError() != cudaSuccess) return FAVEST_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return FAVEST_ECUDA;
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const unsigned long long ctx = current_ctx_id();
        if (ctx == 0) return FAVEST_ECUDA;
        if (g_scratch[dev].ctx_id != ctx) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_favest_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();   // the lookup's own error
                return FAVEST_ECUDA;
            }
            g_scratch[dev].ptr = ptr;
            g_scratch[dev].ctx_id = ctx;
        }
        base = (unsigned char *)g_scratch[dev].ptr;
    }
    cudaStream_t s = (cudaStream_t)stream;

    Plan p;   // host-side description only; every device pointer points into the scratch array
    p.L = L;
    p.B = batch;
    p.precision = FAVEST_FP64;
    p.io = FAVEST_IO_C128;
    p.nlat = nlat;
    p.nphi = nphi;
    p.J = J;
    p.has_eq = nlat & 1;
    p.ncol = ncol;
    p.ct = (batch % 2 == 0) ? 8 : 4;
    p.ng = p.ncol / p.ct;
    p.unit_weights = 0;
    p.device = dev;
    cudaDeviceGetAttribute(&p.num_sms, cudaDevAttrMultiProcessorCount, dev);
    p.ntab = ntab;
    p.d_x = (double *)(base + o_x);
    p.d_sin = (double *)(base + o_s);
    p.d_omega = (double *)(base + o_om);
    p.d_omega_unit = (double *)(base + o_omu);
    p.d_cmu = (double *)(base + o_cmu);
    p.d_A = (double *)(base + o_A);
    p.d_P = (double *)(base + o_P);
    p.d_M = (double *)(base + o_M);
    p.d_R = (double *)(base + o_R);
    p.d_F = base + o_F;
    p.d_Q = base + o_Q;
    p.d_status = nullptr;   // the FP64 kernels record no device-side status
    p.fft.n = nphi;
    p.fft.nstages = factorize_na(nphi, p.fft.radix);
    p.fft.tw64 = (double2 *)(base + o_tw);
    if (p.fft.nstages < 0) return FAVEST_EUNSUPPORTED;

    // tables (rebuilt on every call: the array keeps whatever the previous call left)
    k_na_gl<<<(nlat / 2 + 1 + 127) / 128, 128, 0, s>>>(nlat, J, nphi, p.d_x, p.d_sin, p.d_omega, p.d_omega_unit);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_na_tables<<<(L + 1 + 63) / 64, 64, 0, s>>>(L, p.d_cmu, p.d_A, p.d_P, p.d_M, p.d_R,
                                                    (double *)(base + o_kap));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_na_twiddles<<<(nphi + 255) / 256, 256, 0, s>>>(nphi, p.fft.tw64);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_fft_fwd_fp64(p, Tth, Tph, s);
    if (e == cudaSuccess) e = launch_analysis_fp64(p, s);
    if (e == cudaSuccess) e = launch_combine_fp64(p, a, b, s);
    return e == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
}
