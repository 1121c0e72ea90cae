// Longitude DFT stage of the split-precision path (FP32 arithmetic, FP64-derived
// twiddles rounded to FP32).  One CTA per (field b, folded latitude j) handles the four
// rings theta/phi x (j, nlat-1-j):
//   forward: T -> FFT -> weighted equatorial fold F+- = omega_j (F_j +- F_j') -> three
//            bf16 pieces written straight into the tensor-core B-operand layout.
//   inverse: gathers the even/odd Legendre sums E, O of every order, forms
//            G_j = (E + O) / sin(theta_j), G_j' = (E - O) / sin(theta_j), inverse FFT.
#include "favest_internal.h"
#include "fft_device.cuh"

#include <cuda_bf16.h>

namespace favest {

namespace {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 caddf(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csubf(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <bool INV>
__device__ __forceinline__ float2 twf(const float2 *__restrict__ tw, int q)
{
    float2 t = __ldg(tw + q);
    return INV ? make_float2(t.x, -t.y) : t;
}

// one Stockham pass of radix R over `nr` rings of n points stored back to back
template <bool INV>
__device__ __forceinline__ void pass_f32(const float2 *__restrict__ x, float2 *__restrict__ y,
                                         const float2 *__restrict__ tw, int n, int R, int Ns, int nr)
{
    const int nb = n / R;
    const int tstep = n / (Ns * R);
    for (int t = threadIdx.x; t < nb * nr; t += blockDim.x) {
        const int ring = t / nb, i = t % nb;
        const float2 *xr = x + ring * n;
        float2 *yr = y + ring * n;
        const int k = i % Ns;
        const int obase = (i / Ns) * Ns * R + k;
        if (R == 2) {
            float2 v0 = xr[i], v1 = cmulf(xr[i + nb], twf<INV>(tw, k * tstep));
            yr[obase] = caddf(v0, v1);
            yr[obase + Ns] = csubf(v0, v1);
        } else if (R == 4) {
            float2 v0 = xr[i];
            float2 v1 = cmulf(xr[i + nb], twf<INV>(tw, k * tstep));
            float2 v2 = cmulf(xr[i + 2 * nb], twf<INV>(tw, 2 * k * tstep));
            float2 v3 = cmulf(xr[i + 3 * nb], twf<INV>(tw, 3 * k * tstep));
            float2 s02 = caddf(v0, v2), d02 = csubf(v0, v2);
            float2 s13 = caddf(v1, v3), d13 = csubf(v1, v3);
            float2 rot = INV ? make_float2(-d13.y, d13.x) : make_float2(d13.y, -d13.x);
            yr[obase] = caddf(s02, s13);
            yr[obase + Ns] = caddf(d02, rot);
            yr[obase + 2 * Ns] = csubf(s02, s13);
            yr[obase + 3 * Ns] = csubf(d02, rot);
        } else {
            const int rstep = n / R;
            for (int q = 0; q < R; ++q) {
                float2 acc = make_float2(0.f, 0.f);
                for (int r = 0; r < R; ++r) {
                    int t1 = (int)(((long long)k * r * tstep) % n);
                    int tq = t1 + ((q * r) % R) * rstep;
                    if (tq >= n) tq -= n;
                    acc = caddf(acc, cmulf(xr[i + r * nb], twf<INV>(tw, tq)));
                }
                yr[obase + q * Ns] = acc;
            }
        }
    }
}

template <bool INV>
__device__ float2 *stockham_f32(float2 *b0, float2 *b1, const float2 *__restrict__ tw, const RadixPlanArg &rp,
                                int nr)
{
    float2 *x = b0, *y = b1;
    int Ns = 1;
    for (int s = 0; s < rp.nstages; ++s) {
        pass_f32<INV>(x, y, tw, rp.n, rp.radix[s], Ns, nr);
        __syncthreads();
        Ns *= rp.radix[s];
        float2 *t = x; x = y; y = t;
    }
    return x;
}

__device__ __forceinline__ void split3f(float f, unsigned short &h, unsigned short &m, unsigned short &l)
{
    __nv_bfloat16 bh = __float2bfloat16_rn(f);
    float r1 = f - __bfloat162float(bh);
    __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    float r2 = r1 - __bfloat162float(bm);
    __nv_bfloat16 bl = __float2bfloat16_rn(r2);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

// write 8 floats (one core-matrix row) as three bf16 pieces
__device__ __forceinline__ void store_row3(unsigned char *dst, const float (&v)[8], int piece_bytes)
{
    unsigned w[3][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        unsigned short h0, m0, l0, h1, m1, l1;
        split3f(v[2 * i], h0, m0, l0);
        split3f(v[2 * i + 1], h1, m1, l1);
        w[0][i] = (unsigned)h0 | ((unsigned)h1 << 16);
        w[1][i] = (unsigned)m0 | ((unsigned)m1 << 16);
        w[2][i] = (unsigned)l0 | ((unsigned)l1 << 16);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        *reinterpret_cast<uint4 *>(dst + q * piece_bytes) = make_uint4(w[q][0], w[q][1], w[q][2], w[q][3]);
}

constexpr int kChunkBytes = 3 * 16384;

// grid: B * J CTAs (field-major); shared: 2 * 4 * n float2
__global__ void __launch_bounds__(256) k_fft_fwd_bf16(
    const float2 *__restrict__ Tth, const float2 *__restrict__ Tph, unsigned char *__restrict__ Fb,
    RadixPlanArg rp, const float2 *__restrict__ tw, const double *__restrict__ omega, int L, int nlat, int J,
    int has_eq, int n_tiles, int nk_f)
{
    extern __shared__ float2 sm_f[];
    const int n = rp.n;
    const int b = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;    // rings: (th, j), (ph, j), (th, j'), (ph, j')
    float2 *buf0 = sm_f, *buf1 = sm_f + 4 * n;
    const int jm = nlat - 1 - j;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const int ring = idx / n, k = idx % n;
        const float2 *src = (ring & 1) ? Tph : Tth;
        const int jj = (ring < 2) ? j : jm;
        buf0[idx] = src[((size_t)b * nlat + jj) * n + k];
    }
    __syncthreads();
    const float2 *F = stockham_f32<false>(buf0, buf1, tw, rp, nr);
    const float w = (float)omega[j];
    const int nt = b / 16, bg = b % 16, kc = j / 64, jj = j % 64;
    for (int mu = threadIdx.x; mu <= L; mu += blockDim.x) {
        float vp[8], vm[8];
        // n % 8 = c*4 + s*2 + im ; s = 0: +mu (bin mu), s = 1: -mu (bin n - mu, or 0 at mu = 0)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const int bin = (s == 0 || mu == 0) ? mu : n - mu;
                float2 a = F[c * n + bin];
                float2 z = eq ? make_float2(0.f, 0.f) : F[(2 + c) * n + bin];
                const int base = c * 4 + s * 2;
                vp[base] = w * (a.x + z.x);
                vp[base + 1] = w * (a.y + z.y);
                vm[base] = eq ? 0.f : w * (a.x - z.x);
                vm[base + 1] = eq ? 0.f : w * (a.y - z.y);
            }
        }
        const size_t row_off = (size_t)(jj / 8) * 2048 + bg * 128 + (jj % 8) * 16;
        unsigned char *dp = Fb + (((size_t)(mu * 2 + 0) * n_tiles + nt) * nk_f + kc) * kChunkBytes + row_off;
        unsigned char *dm = Fb + (((size_t)(mu * 2 + 1) * n_tiles + nt) * nk_f + kc) * kChunkBytes + row_off;
        store_row3(dp, vp, 16384);
        store_row3(dm, vm, 16384);
    }
}

// grid: B * J; S32 = [mu][p][JP][ncolr] fp32; shared 2 * 4 * n float2
__global__ void __launch_bounds__(256) k_fft_inv_bf16(
    const float *__restrict__ S32, float2 *__restrict__ Tth, float2 *__restrict__ Tph, RadixPlanArg rp,
    const float2 *__restrict__ tw, const double *__restrict__ sj, int L, int nlat, int J, int JP, int has_eq,
    int ncolr)
{
    extern __shared__ float2 sm_i[];
    const int n = rp.n;
    const int b = blockIdx.x / J, j = blockIdx.x % J;
    const bool eq = has_eq && j == J - 1;
    const int nr = eq ? 2 : 4;
    float2 *buf0 = sm_i, *buf1 = sm_i + 4 * n;
    const float is = (float)(1.0 / sj[j]);
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) buf0[idx] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int mu = threadIdx.x; mu <= L; mu += blockDim.x) {
        // order 0 arrives already divided by sin(theta) (synthesised on lambda^1)
        const float sc = mu == 0 ? 1.0f : is;
        const float4 *e = reinterpret_cast<const float4 *>(S32 + (((size_t)mu * 2 + 0) * JP + j) * ncolr + 8 * b);
        const float4 *o = reinterpret_cast<const float4 *>(S32 + (((size_t)mu * 2 + 1) * JP + j) * ncolr + 8 * b);
        float4 e0 = e[0], e1 = e[1], o0 = o[0], o1 = o[1];
        float ev[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
        float ov[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
#pragma unroll
        for (int c = 0; c < 2; ++c) {
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                if (mu == 0 && s == 1) continue;
                const int bin = s ? n - mu : mu;
                const int k = c * 4 + s * 2;
                buf0[c * n + bin] = make_float2((ev[k] + ov[k]) * sc, (ev[k + 1] + ov[k + 1]) * sc);
                if (!eq) buf0[(2 + c) * n + bin] = make_float2((ev[k] - ov[k]) * sc, (ev[k + 1] - ov[k + 1]) * sc);
            }
        }
    }
    __syncthreads();
    const float2 *T = stockham_f32<true>(buf0, buf1, tw, rp, nr);
    const int jm = nlat - 1 - j;
    for (int idx = threadIdx.x; idx < nr * n; idx += blockDim.x) {
        const int ring = idx / n, k = idx % n;
        float2 *dst = (ring & 1) ? Tph : Tth;
        const int jj = (ring < 2) ? j : jm;
        dst[((size_t)b * nlat + jj) * n + k] = T[idx];
    }
}

}  // namespace

cudaError_t launch_fft_fwd_bf16(const Plan &p, const void *Tth, const void *Tph, cudaStream_t s)
{
    RadixPlanArg rp = make_radix_arg(p.fft);
    const size_t smem = 2 * 4 * (size_t)p.nphi * sizeof(float2);
    auto k = k_fft_fwd_bf16;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<p.B * p.J, 256, smem, s>>>((const float2 *)Tth, (const float2 *)Tph, (unsigned char *)p.d_Fb, rp,
                                   p.fft.tw32, p.unit_weights ? p.d_omega_unit : p.d_omega, p.L, p.nlat, p.J,
                                   p.has_eq, p.n_tiles, p.nk_f);
    return cudaGetLastError();
}

cudaError_t launch_fft_inv_bf16(const Plan &p, void *Tth, void *Tph, cudaStream_t s)
{
    RadixPlanArg rp = make_radix_arg(p.fft);
    const size_t smem = 2 * 4 * (size_t)p.nphi * sizeof(float2);
    auto k = k_fft_inv_bf16;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<p.B * p.J, 256, smem, s>>>((const float *)p.d_S32, (float2 *)Tth, (float2 *)Tph, rp, p.fft.tw32,
                                   p.d_sin, p.L, p.nlat, p.J, p.JP, p.has_eq, p.ncolr);
    return cudaGetLastError();
}

}  // namespace favest
