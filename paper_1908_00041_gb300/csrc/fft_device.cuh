// Shared-memory Stockham FFT (device helpers).
#pragma once
#include <cuda_runtime.h>

#include "favest_internal.h"

namespace favest {

struct RadixPlanArg {
    int n;
    int nstages;
    int radix[kMaxRadixStages];
    int blue_lg[kMaxRadixStages], blue_P[kMaxRadixStages];   // see FftPlan
    int blue_off[kMaxRadixStages], blue_moff[kMaxRadixStages];
    int tw_off[kMaxRadixStages];                               // see FftPlan
    const float2 *blue_chirp, *blue_spec, *blue_tw;
};

inline RadixPlanArg make_radix_arg(const FftPlan &f)
{
    RadixPlanArg r;
    r.n = f.n;
    r.nstages = f.nstages;
    for (int i = 0; i < kMaxRadixStages; ++i) r.radix[i] = i < f.nstages ? f.radix[i] : 1;
    for (int i = 0; i < kMaxRadixStages; ++i) {
        r.blue_lg[i] = f.blue_lg[i];
        r.blue_P[i] = f.blue_P[i];
        r.blue_off[i] = f.blue_off[i];
        r.blue_moff[i] = f.blue_moff[i];
        r.tw_off[i] = f.tw_off[i];
    }
    r.blue_chirp = f.blue_chirp;
    r.blue_spec = f.blue_spec;
    r.blue_tw = f.blue_tw;
    return r;
}

__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(float2 v) { return make_double2(v.x, v.y); }
template <typename T> __device__ __forceinline__ T from_d2(double2 v);
template <> __device__ __forceinline__ double2 from_d2<double2>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 from_d2<float2>(double2 v)
{
    return make_float2((float)v.x, (float)v.y);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// twiddle w^q for w = exp(-+2 pi i / n), q reduced mod n by the caller
template <bool INV>
__device__ __forceinline__ double2 twid(const double2 *__restrict__ tw, int q)
{
    double2 t = __ldg(tw + q);
    return INV ? make_double2(t.x, -t.y) : t;
}

// One Stockham pass of radix R over n points: y[(i/Ns)*Ns*R + i%Ns + q*Ns] =
//   sum_r x[i + r n/R] w^{(i%Ns) r n/(Ns R)} w_R^{q r}
// Radices 2 and 4: one thread per butterfly.  Other (odd prime) radices: one thread per
// output (butterfly i, q); its twiddle exponent r ((i%Ns) n/(Ns R) + q n/R) mod n advances
// by one addition per term (the step is below n), summed over r in order.
template <bool INV>
__device__ __forceinline__ void stockham_pass(const double2 *__restrict__ x, double2 *__restrict__ y,
                                              const double2 *__restrict__ tw, int n, int R, int Ns)
{
    const int nb = n / R;
    const int tstep = n / (Ns * R);
    if (R != 2 && R != 4) {
        const int rstep = n / R;
        for (int t = threadIdx.x; t < nb * R; t += blockDim.x) {
            const int i = t % nb, q = t / nb;
            const int k = i % Ns;
            const int d = k * tstep + q * rstep;       // < n / R + (R - 1) n / R = n
            double2 acc = make_double2(0.0, 0.0);
            int tq = 0;
            for (int r = 0; r < R; ++r) {
                acc = cadd(acc, cmul(x[i + r * nb], twid<INV>(tw, tq)));
                tq += d;
                if (tq >= n) tq -= n;
            }
            y[(i / Ns) * Ns * R + k + q * Ns] = acc;
        }
        return;
    }
    for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const int k = i % Ns;
        const int obase = (i / Ns) * Ns * R + k;
        if (R == 2) {
            double2 v0 = x[i], v1 = cmul(x[i + nb], twid<INV>(tw, k * tstep));
            y[obase] = cadd(v0, v1);
            y[obase + Ns] = csub(v0, v1);
        } else if (R == 4) {
            double2 v0 = x[i];
            double2 v1 = cmul(x[i + nb], twid<INV>(tw, k * tstep));
            double2 v2 = cmul(x[i + 2 * nb], twid<INV>(tw, 2 * k * tstep));
            double2 v3 = cmul(x[i + 3 * nb], twid<INV>(tw, 3 * k * tstep));
            double2 s02 = cadd(v0, v2), d02 = csub(v0, v2);
            double2 s13 = cadd(v1, v3), d13 = csub(v1, v3);
            // forward: -i * d13 ; inverse: +i * d13
            double2 rot = INV ? make_double2(-d13.y, d13.x) : make_double2(d13.y, -d13.x);
            y[obase] = cadd(s02, s13);
            y[obase + Ns] = cadd(d02, rot);
            y[obase + 2 * Ns] = csub(s02, s13);
            y[obase + 3 * Ns] = csub(d02, rot);
        }
    }
}

// Full transform; returns the buffer holding the result (buf0 or buf1).
template <bool INV>
__device__ const double2 *stockham(double2 *buf0, double2 *buf1, const double2 *__restrict__ tw,
                                   const RadixPlanArg &rp)
{
    double2 *x = buf0, *y = buf1;
    int Ns = 1;
    for (int s = 0; s < rp.nstages; ++s) {
        const int R = rp.radix[s];
        stockham_pass<INV>(x, y, tw, rp.n, R, Ns);
        __syncthreads();
        Ns *= R;
        double2 *t = x; x = y; y = t;
    }
    return x;
}

}  // namespace favest
