// Vector spherical harmonic transforms at arbitrary points (the paper's interface
// FaVeST_fwd(T, L, X, w) / FaVeST_adj(a, b, X), Sec. 4.4): FP64, fields given by their
// Cartesian components T = T^(1) e_x + T^(2) e_y + T^(3) e_z at npts points x_k of the unit
// sphere with weights w_k.
//
// The route is the paper's own (Thm. 1, Thm. 2): the vector transforms are fixed O(L^2)
// combinations of scalar spherical harmonic transforms of degree L+1 of the three Cartesian
// components, and those combinations (k_cg_combine / k_cg_uncombine of the Clebsch-Gordan
// plan, eqs. ninecoeff, nulm1, nulm2, etalm) do not depend on the point set.  What changes
// with scattered points is the scalar stage: with no tensor-product structure there is no
// longitude FFT and no equatorial fold, so each scalar sum runs over the points directly,
//   forward:  Q[row(l, mu)][2 s + (m < 0)] = sum_k y_l^mu(x_k) w_k T^(s)_k e^{-i m phi_k},  m = +-mu,
//   adjoint:  T^(s)_k = sum_mu e^{+i mu phi_k} S_k[2 s] + e^{-i mu phi_k} S_k[2 s + 1],
//             S_k[col] = sum_l y_l^mu(x_k) g[row(l, mu)][col],
// for every order mu = 0..L+1 and degree l = mu..L+1 (the scalar transforms reach degree
// L+1), y = lambda / kappa the library's scaled FP64 recurrence.  No division by sin(theta)
// occurs, so points at or near the poles need no special treatment.  The cost is that of the
// definition, O(npts L^2) FP64 work: the paper obtains these scalar sums with the NFFT-based
// NFSFT instead, which this library does not build.
//
// Forward kernel: a CTA takes one (order, column group, point chunk); its threads run the
// recurrences of two points each over all rows, reduce each 4-row window over the CTA (warp
// transpose reduction, then across warps through shared memory) and keep the running sums
// of the chunk in shared memory.  Chunks are summed by a second kernel in a fixed order, so
// results do not depend on scheduling.
// Adjoint kernel: a CTA takes a tile of points, one column group and a strided subset of the
// orders; each order's coefficients are staged in shared memory and every thread sums them
// against its points' recurrence values.  Order subsets are summed by a second kernel.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "favest_internal.h"
#include "recurrence.cuh"

namespace favest {

namespace {

constexpr int kScThreads = 256;
constexpr int kScPpt = 2;            // points per thread
constexpr int kScWin = 4;            // rows per reduction window
constexpr int kScCT = 4;             // columns per CTA: two scalar fields, both signs of m

// Column col of a group holds scalar field sc = col / 2 at m = +mu (col even) or -mu.
// Scalar field sc = 3 f + c is component c of vector field f.
__device__ __forceinline__ bool scalar_of(int col, int nscal, int &f, int &c, int &neg)
{
    const int sc = col >> 1;
    neg = col & 1;
    f = sc / 3;
    c = sc - 3 * f;
    return sc < nscal;
}

__global__ void __launch_bounds__(kScThreads) k_sc_analysis(
    const double2 *__restrict__ T, double2 *__restrict__ out, const double *__restrict__ px,
    const double *__restrict__ ps, const double *__restrict__ pphi, const double *__restrict__ pw,
    const double *__restrict__ cmu, const double *__restrict__ Atab, int L, int npts, int nscal, int ncol, int ng,
    int chunk, long long ntab)
{
    constexpr int CT = kScCT, V = kScWin * CT * 2, nwarps = kScThreads / 32;
    extern __shared__ double sm_sc[];
    const int mu = blockIdx.x / ng, g = blockIdx.x % ng;
    const int nrow = L + 2 - mu;
    const long long t0 = tab_off(L, mu);
    double2 *acc = reinterpret_cast<double2 *>(sm_sc);          // [nrow][CT]
    double *As = sm_sc + 2 * CT * nrow;                          // [nrow]
    double *red = As + ((nrow + 1) & ~1);                        // [nwarps][V]
    for (int i = threadIdx.x; i < nrow * CT; i += blockDim.x) acc[i] = make_double2(0.0, 0.0);
    for (int r = threadIdx.x; r < nrow; r += blockDim.x) As[r] = Atab[t0 + r];
    __syncthreads();
    const int k0 = blockIdx.y * chunk;
    const int k1 = min(npts, k0 + chunk);
    const double cm = cmu[mu];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int tile = k0; tile < k1; tile += kScThreads * kScPpt) {
        double x[kScPpt], y1[kScPpt], y2[kScPpt];
        int c[kScPpt];
        double2 F[kScPpt][CT];
#pragma unroll
        for (int i = 0; i < kScPpt; ++i) {
            const int k = tile + threadIdx.x + i * kScThreads;
            x[i] = 0.0; y1[i] = 0.0; y2[i] = 0.0; c[i] = 1 << 20;   // inactive points stay silent
#pragma unroll
            for (int ct = 0; ct < CT; ++ct) F[i][ct] = make_double2(0.0, 0.0);
            if (k < k1) {
                x[i] = px[k];
                sectoral_start(cm, ps[k], mu, y1[i], c[i]);
                double sn, cs;
                sincos((double)mu * pphi[k], &sn, &cs);
                const double w = pw[k];
#pragma unroll
                for (int ct = 0; ct < CT; ++ct) {
                    int f, cc, neg;
                    if (scalar_of(g * CT + ct, nscal, f, cc, neg)) {
                        const double2 t = T[((size_t)f * npts + k) * 3 + cc];
                        // w T e^{-i m phi}, m = +mu (neg = 0) or -mu
                        const double si = neg ? sn : -sn;
                        F[i][ct] = make_double2(w * (t.x * cs - t.y * si), w * (t.x * si + t.y * cs));
                    }
                }
            }
        }
        for (int r0 = 0; r0 < nrow; r0 += kScWin) {
            double v[V];
#pragma unroll
            for (int q = 0; q < V; ++q) v[q] = 0.0;
#pragma unroll
            for (int w = 0; w < kScWin; ++w) {
                const int r = r0 + w;
                if (r < nrow) {
                    const double a = As[r];
#pragma unroll
                    for (int i = 0; i < kScPpt; ++i) {
                        double yl = y1[i];
                        if (r > 0) {
                            yl = fma(a * x[i], y1[i], -y2[i]);
                            y2[i] = y1[i];
                            y1[i] = yl;
                        }
                        const double yv = (c[i] == 0) ? yl : 0.0;
#pragma unroll
                        for (int ct = 0; ct < CT; ++ct) {
                            v[(w * CT + ct) * 2 + 0] = fma(yv, F[i][ct].x, v[(w * CT + ct) * 2 + 0]);
                            v[(w * CT + ct) * 2 + 1] = fma(yv, F[i][ct].y, v[(w * CT + ct) * 2 + 1]);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < kScPpt; ++i) renorm(y1[i], y2[i], c[i]);
            warp_transpose_reduce<V>(v);
            constexpr int per = V / 32;
#pragma unroll
            for (int q = 0; q < per; ++q) red[warp * V + lane * per + q] = v[q];
            __syncthreads();
            if (threadIdx.x < V) {
                const int vi = threadIdx.x;
                double tot = 0.0;
                for (int wq = 0; wq < nwarps; ++wq) tot += red[wq * V + vi];
                const int w = vi / (CT * 2), ct = (vi / 2) % CT, im = vi & 1;
                const int r = r0 + w;
                if (r < nrow) {
                    double *d = reinterpret_cast<double *>(&acc[r * CT + ct]);
                    d[im] += tot;
                }
            }
            __syncthreads();
        }
    }
    double2 *dst = out + (size_t)blockIdx.y * ntab * ncol;
    for (int i = threadIdx.x; i < nrow * CT; i += blockDim.x) {
        const int r = i / CT, ct = i % CT;
        dst[(size_t)(t0 + r) * ncol + g * CT + ct] = acc[i];
    }
}

// Q[i] = sum over parts of part[p][i] (fixed order), i < n
__global__ void k_sc_sum_parts(const double2 *__restrict__ part, double2 *__restrict__ Q, long long n, int nparts)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 s = part[i];
    for (int p = 1; p < nparts; ++p) {
        const double2 v = part[(size_t)p * n + i];
        s.x += v.x;
        s.y += v.y;
    }
    Q[i] = s;
}

__global__ void __launch_bounds__(kScThreads) k_sc_synthesis(
    const double2 *__restrict__ Q, double2 *__restrict__ out, const double *__restrict__ px,
    const double *__restrict__ ps, const double *__restrict__ pphi, const double *__restrict__ cmu,
    const double *__restrict__ Atab, int L, int npts, int nscal, int ncol, int nsplit)
{
    constexpr int CT = kScCT, NS = CT / 2;
    extern __shared__ double sm_sy[];
    const int g = blockIdx.y, z = blockIdx.z;
    double2 *gs = reinterpret_cast<double2 *>(sm_sy);    // [L+2][CT]
    double *As = sm_sy + 2 * CT * (L + 2);                 // [L+2]
    double x[kScPpt], s[kScPpt], phi[kScPpt];
    bool act[kScPpt];
    double2 acc[kScPpt][NS];
#pragma unroll
    for (int i = 0; i < kScPpt; ++i) {
        const int k = blockIdx.x * kScThreads * kScPpt + threadIdx.x + i * kScThreads;
        act[i] = k < npts;
        x[i] = act[i] ? px[k] : 0.0;
        s[i] = act[i] ? ps[k] : 0.0;
        phi[i] = act[i] ? pphi[k] : 0.0;
#pragma unroll
        for (int q = 0; q < NS; ++q) acc[i][q] = make_double2(0.0, 0.0);
    }
    for (int mu = z; mu <= L + 1; mu += nsplit) {
        const int nrow = L + 2 - mu;
        const long long t0 = tab_off(L, mu);
        __syncthreads();                                   // previous order's reads done
        for (int i = threadIdx.x; i < nrow * CT; i += blockDim.x) {
            const int r = i / CT, ct = i % CT;
            gs[i] = Q[(size_t)(t0 + r) * ncol + g * CT + ct];
        }
        for (int r = threadIdx.x; r < nrow; r += blockDim.x) As[r] = Atab[t0 + r];
        __syncthreads();
        const double cm = cmu[mu];
        double y1[kScPpt], y2[kScPpt];
        int c[kScPpt];
        double2 S[kScPpt][CT];
#pragma unroll
        for (int i = 0; i < kScPpt; ++i) {
            y1[i] = 0.0; y2[i] = 0.0; c[i] = 1 << 20;
            if (act[i]) sectoral_start(cm, s[i], mu, y1[i], c[i]);
#pragma unroll
            for (int ct = 0; ct < CT; ++ct) S[i][ct] = make_double2(0.0, 0.0);
        }
        for (int r0 = 0; r0 < nrow; r0 += kScWin) {
#pragma unroll
            for (int w = 0; w < kScWin; ++w) {
                const int r = r0 + w;
                if (r < nrow) {
                    const double a = As[r];
#pragma unroll
                    for (int i = 0; i < kScPpt; ++i) {
                        double yl = y1[i];
                        if (r > 0) {
                            yl = fma(a * x[i], y1[i], -y2[i]);
                            y2[i] = y1[i];
                            y1[i] = yl;
                        }
                        const double yv = (c[i] == 0) ? yl : 0.0;
#pragma unroll
                        for (int ct = 0; ct < CT; ++ct) {
                            const double2 gv = gs[r * CT + ct];
                            S[i][ct].x = fma(yv, gv.x, S[i][ct].x);
                            S[i][ct].y = fma(yv, gv.y, S[i][ct].y);
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < kScPpt; ++i) renorm(y1[i], y2[i], c[i]);
        }
#pragma unroll
        for (int i = 0; i < kScPpt; ++i) {
            double sn, cs;
            sincos((double)mu * phi[i], &sn, &cs);
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                // e^{+i mu phi} S[2q] + e^{-i mu phi} S[2q+1] (order 0 has the m >= 0 column only)
                const double2 p = S[i][2 * q], m = S[i][2 * q + 1];
                acc[i][q].x += p.x * cs - p.y * sn;
                acc[i][q].y += p.x * sn + p.y * cs;
                if (mu > 0) {
                    acc[i][q].x += m.x * cs + m.y * sn;
                    acc[i][q].y += m.y * cs - m.x * sn;
                }
            }
        }
    }
    // out: [nsplit][nscal][npts] partial syntheses (nsplit == 1: the caller's [B][npts][3])
#pragma unroll
    for (int i = 0; i < kScPpt; ++i) {
        const int k = blockIdx.x * kScThreads * kScPpt + threadIdx.x + i * kScThreads;
        if (!act[i]) continue;
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            const int sc = g * NS + q;
            if (sc >= nscal) continue;
            const int f = sc / 3, cc = sc - 3 * f;
            out[(size_t)z * nscal * npts + ((size_t)f * npts + k) * 3 + cc] = acc[i][q];
        }
    }
}

}  // namespace

}  // namespace favest

struct favest_scatter_s {
    favest_plan cg = nullptr;        // Clebsch-Gordan plan (tables, sums Q, combine kernels)
    int L = 0, B = 0, npts = 0;
    int nchunk = 1, chunk = 0;       // forward point chunks
    int nsplit = 1;                  // adjoint order subsets
    double *d_px = nullptr, *d_ps = nullptr, *d_phi = nullptr, *d_w = nullptr;
    double2 *d_part = nullptr;       // forward chunk sums or adjoint partial fields
};

namespace {

void scatter_free(favest_scatter_s *h)
{
    void *ptrs[] = {h->d_px, h->d_ps, h->d_phi, h->d_w, h->d_part};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (h->cg) favest_plan_destroy(h->cg);
    delete h;
}

}  // namespace

extern "C" {

int favest_scatter_create(int L, int batch, int npts, const double *X, const double *w, favest_scatter *out)
{
    using namespace favest;
    if (!out) return FAVEST_EINVAL;
    *out = nullptr;
    // L <= 2047: one order's staged coefficients (and sums) fit a CTA's shared memory
    if (L < 1 || L > 2047 || batch < 1 || batch > 1366 || npts < 1 || npts > (1 << 26) || !X) return FAVEST_EINVAL;
    std::vector<double> hx(npts), hs(npts), hphi(npts), hw(npts);
    for (int k = 0; k < npts; ++k) {
        const double a = X[3 * k], b = X[3 * k + 1], z = X[3 * k + 2];
        const double r = std::sqrt(a * a + b * b + z * z);
        if (!std::isfinite(r) || std::fabs(r - 1.0) > 1e-10) return FAVEST_EINVAL;
        const double wk = w ? w[k] : 1.0;
        if (!std::isfinite(wk)) return FAVEST_EINVAL;
        hx[k] = z / r;
        hs[k] = std::sqrt(a * a + b * b) / r;
        hphi[k] = std::atan2(b, a);
        hw[k] = wk;
    }
    favest_scatter_s *h = new (std::nothrow) favest_scatter_s();
    if (!h) return FAVEST_ENOMEM;
    h->L = L;
    h->B = batch;
    h->npts = npts;
    int st = plan_create_internal(L, batch, FAVEST_FP64, FAVEST_IO_C128, nullptr, nullptr, 0, &h->cg, 2);
    if (st != FAVEST_OK) {
        h->cg = nullptr;
        scatter_free(h);
        return st;
    }
    const Plan &p = h->cg->p;
    // forward: enough (order, group, chunk) CTAs for about four per SM, chunks of at least
    // one tile of points; adjoint: enough (point tile, group, order subset) CTAs likewise
    const long long want = 4LL * p.num_sms;
    const int ng4 = p.ncol / kScCT;                 // column groups of the scattered kernels
    const long long per = (long long)(L + 2) * ng4;
    const int tile = kScThreads * kScPpt;
    const int ntiles = (npts + tile - 1) / tile;
    long long nc = (want + per - 1) / per;
    if (nc > ntiles) nc = ntiles;
    if (nc < 1) nc = 1;
    h->chunk = ((ntiles + (int)nc - 1) / (int)nc) * tile;
    h->nchunk = (npts + h->chunk - 1) / h->chunk;
    long long ns = (want + (long long)ntiles * ng4 - 1) / ((long long)ntiles * ng4);
    if (ns > L + 2) ns = L + 2;
    if (ns > 16) ns = 16;
    if (ns < 1) ns = 1;
    h->nsplit = (int)ns;
    const size_t fwd_part = h->nchunk > 1 ? (size_t)h->nchunk * p.ntab * p.ncol : 0;
    const size_t adj_part = h->nsplit > 1 ? (size_t)h->nsplit * p.nscal * npts : 0;
    const size_t npart = fwd_part > adj_part ? fwd_part : adj_part;
    auto up = [&](double **d, const std::vector<double> &v) {
        if (plan_malloc((void **)d, v.size() * sizeof(double)) != cudaSuccess) return FAVEST_ENOMEM;
        return cudaMemcpy(*d, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess
                   ? FAVEST_OK
                   : FAVEST_ECUDA;
    };
    if ((st = up(&h->d_px, hx)) || (st = up(&h->d_ps, hs)) || (st = up(&h->d_phi, hphi)) || (st = up(&h->d_w, hw))) {
        cudaGetLastError();
        scatter_free(h);
        return st;
    }
    if (npart && plan_malloc((void **)&h->d_part, npart * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        scatter_free(h);
        return FAVEST_ENOMEM;
    }
    *out = h;
    return FAVEST_OK;
}

int favest_scatter_fwd(favest_scatter plan, const void *T, void *a, void *b, void *stream)
{
    using namespace favest;
    if (!plan || !T || !a || !b) return FAVEST_EINVAL;
    if (((uintptr_t)T | (uintptr_t)a | (uintptr_t)b) % 16) return FAVEST_EINVAL;
    Plan &p = plan->cg->p;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FAVEST_ECUDA;
    if (dev != p.device) return FAVEST_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const int CT = kScCT, nwarps = kScThreads / 32, V = kScWin * CT * 2;
    const int nrowmax = p.L + 2;
    const size_t smem = (size_t)(2 * CT * nrowmax + ((nrowmax + 1) & ~1) + nwarps * V) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_sc_analysis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return FAVEST_ECUDA;
    double2 *dst = plan->nchunk > 1 ? plan->d_part : (double2 *)p.d_Q;
    const int ng4 = p.ncol / CT;
    dim3 grid((p.L + 2) * ng4, plan->nchunk);
    k_sc_analysis<<<grid, kScThreads, smem, s>>>((const double2 *)T, dst, plan->d_px, plan->d_ps, plan->d_phi,
                                                 plan->d_w, p.d_cmu, p.d_A, p.L, plan->npts, p.nscal, p.ncol, ng4,
                                                 plan->chunk, p.ntab);
    e = cudaGetLastError();
    if (e == cudaSuccess && plan->nchunk > 1) {
        const long long n = p.ntab * p.ncol;
        k_sc_sum_parts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(plan->d_part, (double2 *)p.d_Q, n, plan->nchunk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_cg_combine(p, a, b, s);
    return e == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
}

int favest_scatter_adj(favest_scatter plan, const void *a, const void *b, void *T, void *stream)
{
    using namespace favest;
    if (!plan || !T || !a || !b) return FAVEST_EINVAL;
    if (((uintptr_t)T | (uintptr_t)a | (uintptr_t)b) % 16) return FAVEST_EINVAL;
    Plan &p = plan->cg->p;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return FAVEST_ECUDA;
    if (dev != p.device) return FAVEST_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = launch_cg_uncombine(p, a, b, s);
    if (e != cudaSuccess) return FAVEST_ECUDA;
    const int CT = kScCT;
    const size_t smem = (size_t)(2 * CT * (p.L + 2) + (p.L + 2)) * sizeof(double);
    e = cudaFuncSetAttribute(k_sc_synthesis, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return FAVEST_ECUDA;
    const int tile = kScThreads * kScPpt;
    dim3 grid((plan->npts + tile - 1) / tile, p.ncol / CT, plan->nsplit);
    double2 *dst = plan->nsplit > 1 ? plan->d_part : (double2 *)T;
    k_sc_synthesis<<<grid, kScThreads, smem, s>>>((const double2 *)p.d_Q, dst, plan->d_px, plan->d_ps, plan->d_phi,
                                                  p.d_cmu, p.d_A, p.L, plan->npts, p.nscal, p.ncol, plan->nsplit);
    e = cudaGetLastError();
    if (e == cudaSuccess && plan->nsplit > 1) {
        const long long n = (long long)p.nscal * plan->npts;
        k_sc_sum_parts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(plan->d_part, (double2 *)T, n, plan->nsplit);
        e = cudaGetLastError();
    }
    return e == cudaSuccess ? FAVEST_OK : FAVEST_ECUDA;
}

int favest_scatter_npts(favest_scatter plan) { return plan ? plan->npts : FAVEST_EINVAL; }

void favest_scatter_destroy(favest_scatter plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    scatter_free(plan);
}

}  // extern "C"
