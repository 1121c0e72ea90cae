// FP64 scaled three-term recurrence for normalised associated Legendre functions
// (device helpers shared by the FP64 and tensor-core Legendre kernels).
//
// For order mu >= 0 the library runs
//     y_mu     = lambda_mu^mu(theta) * 2^(600 c)          (sectoral start, scaled)
//     y_{mu+1} = A_{mu+1} x y_mu
//     y_l      = A_l x y_{l-1} - y_{l-2},   l >= mu+2,   x = cos(theta)
// where y_l = lambda_l^mu / kappa_l (kappa folded into the combine coefficients).
// c >= 0 counts factors 2^600 by which the running values are scaled up while the
// true values lie below the double range (near the poles at high order); while c > 0
// the true value is below 2^-300 and contributes nothing at FP64 resolution, so it is
// emitted as zero.  Renormalisation checks use integer operations on the exponent
// bits, so they cost no FP64 pipe slots.
#pragma once
#include <cuda_runtime.h>

namespace favest {

constexpr int kScaleBits = 600;       // one scale step = 2^600
constexpr int kStartFloor = -200;     // start values are lifted to >= 2^-200
constexpr int kRenormAt = 300;        // scaled values >= 2^300 are stepped down

// f (> 0, normal) -> f in [0.5, 1), e += exponent
__device__ __forceinline__ void frexp_acc(double &f, int &e)
{
    int hi = __double2hiint(f);
    int lo = __double2loint(f);
    int k = ((unsigned)hi >> 20 & 0x7ff) - 1022;
    hi = (hi & 0x800fffff) | (1022 << 20);
    f = __hiloint2double(hi, lo);
    e += k;
}

// lambda_mu^mu(theta) = (-1)^mu cmu sin(theta)^mu as (y, c): true = y * 2^(-600 c)
__device__ __forceinline__ void sectoral_start(double cmu, double s, int mu, double &y, int &c)
{
    double f = 1.0, base = s;
    int e = 0, eb = 0;
    frexp_acc(base, eb);
    int n = mu;
    while (n) {
        if (n & 1) {
            f *= base;
            e += eb;
            frexp_acc(f, e);
        }
        n >>= 1;
        if (n) {
            base *= base;
            eb *= 2;
            frexp_acc(base, eb);
        }
    }
    double v = (mu & 1) ? -cmu * f : cmu * f;
    int cc = 0;
    if (e < kStartFloor) cc = (kStartFloor - e + kScaleBits - 1) / kScaleBits;
    y = ldexp(v, e + kScaleBits * cc);
    c = cc;
}

// Step a scaled pair down by 2^600 when the newest value reached 2^300.
__device__ __forceinline__ void renorm(double &y1, double &y2, int &c)
{
    if (c > 0) {
        int ex = ((unsigned)__double2hiint(y1) >> 20) & 0x7ff;
        if (ex >= 1023 + kRenormAt) {
            y1 *= 0x1p-600;
            y2 *= 0x1p-600;
            c -= 1;
        }
    }
}

// ---------------------------------------------------------------------------------------
// The same recurrence in double-float arithmetic (value = h + l, two FP32 numbers, about
// 44 significant bits) for the split path's generator, whose output keeps 24 bits: the
// FP32 pipe issues 64 times the FP64 one on this GPU.  The products and sums are the
// error-free transformations of Dekker (product through an FMA) and Knuth (two-sum), with
// _rn intrinsics so that no multiply-add is contracted behind their backs.
//   y_l = (A_l x) y_{l-1} - y_{l-2} with A_l and x given as double-float pairs.
// FP32 has an 8-bit exponent, so the scaling runs in steps of 2^100: values are lifted to at
// least 2^-60 at the start and stepped down by 2^-100 when they reach 2^40 (checked every 16
// rows, over which they grow by less than 3^16 < 2^26); while c > 0 the true value is below
// 2^-60 and is emitted as zero.
struct Df {
    float h, l;
};

// One step y = (a x) y1 - y2.  The two products are kept as unnormalised pairs (p, e), the
// high product plus the FMA-exact low part of its leading term and the cross terms (the
// low x low terms, relative size 2^-48, are dropped); only the difference is renormalised,
// by Knuth's two-sum of the high parts and a fast two-sum at the end.  19 FP32 operations.
__device__ __forceinline__ Df df_step(Df a, Df x, Df y1, Df y2)
{
    const float p = __fmul_rn(a.h, x.h);
    float e = __fmaf_rn(a.h, x.h, -p);                 // exact low part of a.h x.h
    e = __fmaf_rn(a.h, x.l, e);
    e = __fmaf_rn(a.l, x.h, e);
    const float P = __fmul_rn(p, y1.h);
    float E = __fmaf_rn(p, y1.h, -P);                  // exact low part of p y1.h
    E = __fmaf_rn(p, y1.l, E);
    E = __fmaf_rn(e, y1.h, E);
    const float s = __fsub_rn(P, y2.h);
    const float bb = __fsub_rn(s, P);                  // two-sum of P and -y2.h
    float t = __fadd_rn(__fsub_rn(P, __fsub_rn(s, bb)), __fsub_rn(-y2.h, bb));
    t = __fadd_rn(t, __fsub_rn(E, y2.l));
    const float r = __fadd_rn(s, t);
    return Df{r, __fsub_rn(t, __fsub_rn(r, s))};
}

constexpr int kDfScaleBits = 100;     // one scale step = 2^100
constexpr int kDfStartFloor = -60;    // start values are lifted to >= 2^-60
constexpr int kDfRenormAt = 40;       // scaled values >= 2^40 are stepped down

// lambda_mu^mu(theta) = (-1)^mu cmu sin(theta)^mu as a double-float (y, c): true = y 2^(-100 c)
__device__ __forceinline__ void sectoral_start_df(double cmu, double s, int mu, Df &y, int &c)
{
    double f = 1.0, base = s;
    int e = 0, eb = 0;
    frexp_acc(base, eb);
    int n = mu;
    while (n) {
        if (n & 1) {
            f *= base;
            e += eb;
            frexp_acc(f, e);
        }
        n >>= 1;
        if (n) {
            base *= base;
            eb *= 2;
            frexp_acc(base, eb);
        }
    }
    const double v = (mu & 1) ? -cmu * f : cmu * f;
    int cc = 0;
    if (e < kDfStartFloor) cc = (kDfStartFloor - e + kDfScaleBits - 1) / kDfScaleBits;
    const double d = ldexp(v, e + kDfScaleBits * cc);
    const float h = (float)d;
    y = Df{h, (float)(d - (double)h)};
    c = cc;
}

// Step a scaled pair down by 2^100 when the newest value reached 2^40.
__device__ __forceinline__ void renorm_df(Df &y1, Df &y2, int &c)
{
    if (c > 0) {
        const int ex = (__float_as_int(y1.h) >> 23) & 0xff;
        if (ex >= 127 + kDfRenormAt) {
            y1 = Df{y1.h * 0x1p-100f, y1.l * 0x1p-100f};
            y2 = Df{y2.h * 0x1p-100f, y2.l * 0x1p-100f};
            c -= 1;
        }
    }
}

// Sum V values (V a multiple of 32) over the 32 lanes of a warp: afterwards lane l holds in
// v[0 .. V/32) the warp totals of the values with indices l*V/32 .. l*V/32 + V/32 - 1.
// Each level halves the values a lane keeps and exchanges the other half with the lane o
// apart, so the warp adds V*31/32 pairs instead of V*31 for a plain butterfly per value.
template <int V>
__device__ __forceinline__ void warp_transpose_reduce(double (&v)[V])
{
#pragma unroll
    for (int lev = 0; lev < 5; ++lev) {
        const int o = 16 >> lev;
        const int h = V >> (lev + 1);
        const bool up = (threadIdx.x & o) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            double send = up ? v[i] : v[i + h];
            double keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

}  // namespace favest
