// Internal declarations of the favest CUDA library (not part of the C ABI).
//
// Transform structure (both precisions).  For every order mu = |m| the vector
// transform reduces to two scalar Legendre transforms of degree L+1 plus an O(L)
// combine per order, because
//     sin(theta) d_theta lambda_l^m = l eps_{l+1}^m lambda_{l+1}^m - (l+1) eps_l^m lambda_{l-1}^m
// (eps_l^m = sqrt((l^2-m^2)/(4l^2-1))).  This is the theta/phi-component analogue of
// the paper's Thm. 1 and Thm. 2 (vector transform = combination of scalar transforms
// of degrees L-1..L+1); the paper reaches it through Cartesian components and
// Clebsch-Gordan coefficients.
//
// Forward, per field and component c in {theta, phi}:
//   F_c(j, m)  = sum_k T_c(j, k) e^{-i m phi_k}                       (longitude FFT)
//   Q_c(l, m)  = sum_j lambda_l^m(theta_j) omega_j F_c(j, m),  l = |m|..L+1
//                omega_j = W_j (2 pi / nphi) / sin(theta_j)         (Legendre stage)
//   a_lm = P_l Q_th(l+1) - M_l Q_th(l-1) - i m R_l Q_ph(l)
//   b_lm = i m R_l Q_th(l) + P_l Q_ph(l+1) - M_l Q_ph(l-1)           (combine)
// Adjoint: the exact transpose (uncombine -> Legendre synthesis -> 1/sin -> inverse FFT).
//
// The recurrence runs on rescaled values y_l = lambda_l / kappa_l chosen so that
//   y_l = A_l x y_{l-1} - y_{l-2}   (two FP64 instructions per value);
// kappa is folded into the per-(l, mu) combine coefficients P, M, R.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>
#include <vector>

#include "../../include/favest.h"

namespace favest {

constexpr int kMaxRadixStages = 24;

struct FftPlan {
    int n = 0;
    int nstages = 0;
    int radix[kMaxRadixStages];
    double2 *tw64 = nullptr;   // device, e^{-2 pi i k / n}, k = 0..n-1
    float2 *tw32 = nullptr;    // device, same rounded to float; powers of two 64..4096 append
                               // the radix-16 stage tables ([q][k], 17 n / 16 entries)
    // FP32 DFT stages of prime radices R >= 17 (above the in-register forms) run Bluestein's
    // chirp transform, a cyclic convolution of power-of-two length M = 2^blue_lg >= 2R - 1;
    // per stage st (blue_lg[st] = 0: not such a stage):
    int blue_lg[kMaxRadixStages] = {0};
    int blue_P[kMaxRadixStages] = {0};     // butterflies per round
    int blue_off[kMaxRadixStages] = {0};   // stage's offset into the chirp table (points)
    int blue_moff[kMaxRadixStages] = {0};  // stage's offset into the spectrum / twiddle tables
    size_t blue_scratch = 0;               // bytes of shared-memory scratch the largest stage needs
    // split path, lengths other than powers of two: offset (complexes, into tw32) of stage st's
    // twiddles in [q][k] order, entry q h + k = w_n^(q k n / Nb) for q < R, k < h = Nb / R
    // (-1: a Bluestein stage, which reads the plain table)
    int tw_off[kMaxRadixStages] = {0};
    float2 *blue_chirp = nullptr;   // [R] per stage: exp(-i pi t^2 / R), t^2 reduced mod 2R exactly
    float2 *blue_spec = nullptr;    // [M] per stage: DFT_M of the conjugate chirp / M (natural
                                    //     order; bit-reversed for M = 8192)
    float2 *blue_tw = nullptr;      // [M] per stage: exp(-2 pi i k / M)
};

constexpr int kGemmChunkK = 32;   // K depth of one tensor-core operand chunk
// Device status words of a plan or ragged batch: [0] the status (0 or a FAVEST_E* code),
// [1..2] the forward GEMM's item scheduler, [3..4] the adjoint's (next item, CTAs done;
// zero between launches: the last CTA of a launch resets them).
constexpr int kStatusWords = 5;
inline int *gemm_sched(int *status, bool fwd) { return status + (fwd ? 1 : 3); }
constexpr int kInvChunk = 256;    // orders per TMA box of the inverse DFT's sum records (16 KB)

// One tensor-core GEMM work item: out[rows][N] = sum over nk K-chunks of A_c * B_c, each
// chunk three bf16 pieces.  A (the Legendre operand, one layout for both directions) is
// read through a 4-D tensor map (256 bf16 = 32 latitudes x 8 rows, latitude block of 32,
// row block of 8, piece): chunk c is the box at (0, ay + c ady, az + c adz, 0), 32 x 128
// (forward: one latitude block, 16 row blocks) or 128 x 32 (adjoint: 4 latitude blocks,
// 4 row blocks).  B: chunk c starts b_off + c * b_stride bytes into the B buffer (a
// multiple of 512: the TMA addresses the buffer as rows of 512 bytes) (b_box = 0), or
// (b_box = 1) is the forward operand's 5-D box at (bx, bw, 0, by, 4 * (bk + c)) (FP32
// records; the forward GEMM splits them into the bf16 pieces).  Output row r (< rows) of
// field column group g (8 floats) is written at
//   out + out_off + (r / 4) * out_ld + (r % 4) * 8 + g * col_gs.
struct TcItem {
    long long b_off;
    long long out_off;  // floats
    long long out_ld;   // floats between groups of 4 rows
    long long col_gs;   // floats between field column groups
    int nk;             // K-chunks
    int rows;           // valid output rows (<= 128)
    int ay, ady;        // A box: latitude block of chunk 0, step per chunk
    int az, adz;        // A box: row block of chunk 0, step per chunk
    int b_stride;       // bytes between consecutive B chunks
    int b_box;          // 1: B through the 5-D tensor map
    int bx, by, bw;     // 5-D box coordinates: x of the parity's 8 floats, first field, order
    int bk;             // 5-D box: first K-chunk (chunks below it are skipped)
    int group;          // index into the launch's GemmGroup array
};

// Operand tensor maps and output buffer shared by the items of one group (one plan and
// one direction); a launch may serve the items of several groups (ragged batches).
struct GemmGroup {             // aligned as CUtensorMap requires
    CUtensorMap tmap_a, tmap_b;
    float *out;
};

struct Plan {
    int L = 0, B = 0, precision = 0, io = 0;
    // real fields (FAVEST_IO_R32): orders m >= 0 only; the tensor-core stages see one
    // column group of 8 per PAIR of fields (columns c*4 + f*2 + re/im, f = field in the
    // pair) where complex fields take one group each (columns c*4 + s*2 + re/im, s = sign
    // of m)
    int real = 0;
    int ncg = 0;              // column groups: B (complex) or ceil(B / 2) (real)
    // Clebsch-Gordan route (FP64 plans from favest_cg_plan_create): the columns carry
    // nscal = 3B scalar fields (the Cartesian components of the B vector fields), the
    // scalar transforms run to degree L+1 (orders 0..L+1) with the plain quadrature
    // weights, and d_kap holds kappa_l^mu for every table row; 0 for the other plans
    int nscal = 0;
    double *d_kap = nullptr;
    // scalar sums at arbitrary points (favest_scatter_create): a Clebsch-Gordan plan whose
    // sums Q are formed by the point kernels, so no grid workspace is allocated
    int scattered = 0;
    // real-field Clebsch-Gordan plans: real vector fields 2q and 2q+1 travel as the complex
    // field q = T_2q + i T_2q+1 of this (complex, B = ceil(cg_real / 2)) plan; d_cgT holds the
    // packed fields [B][3][nlat][nphi] and d_cga, d_cgb their full coefficient sets [B][L^2+2L]
    // (complex double)
    int cg_real = 0;              // number of real fields (0: a complex plan)
    void *d_cgT = nullptr, *d_cga = nullptr, *d_cgb = nullptr;
    int nlat = 0, nphi = 0, J = 0, has_eq = 0;
    int ncol = 0;             // complex columns per order: 4 per field (c, sign of m)
    int ct = 0, ng = 0;       // FP64 column group width and count
    int unit_weights = 0;
    int adj_weighted = 0;         // set for the duration of a weighted adjoint call
    int real_transpose = 0;       // set for the duration of a FAVEST_FLAG_REAL_TRANSPOSE call
    int device = 0;
    int num_sms = 0;
    long long ntab = 0;       // sum_mu (L + 2 - mu): rows of every per-(l, mu) table

    // host copies
    double *h_x = nullptr, *h_w = nullptr;

    // device constant tables
    double *d_x = nullptr;        // [J] cos(theta_j), northern half (+ equator)
    double *d_sin = nullptr;      // [J] sin(theta_j)
    double *d_omega = nullptr;    // [J] quadrature weight / sin(theta_j)
    double *d_omega_unit = nullptr;  // [J] 1 / sin(theta_j)
    double *d_wring = nullptr;    // [nlat] point weights W_j * 2 pi / nphi
    // ragged batches: element offsets of field b's grid (per component plane) and of its
    // coefficients in the caller's buffers; null = dense [batch][...] layout
    const long long *d_toff = nullptr, *d_coff = nullptr;
    double *d_cmu = nullptr;      // [L+1] sectoral normalisation sqrt((2mu+1)!!/(4pi (2mu)!!))
    double *d_A = nullptr;        // [ntab] recurrence multipliers A_l^mu
    double *d_P = nullptr;        // [ntab] combine coefficient P_l^mu
    double *d_M = nullptr;        // [ntab] combine coefficient M_l^mu
    double *d_R = nullptr;        // [ntab] combine coefficient R_l^mu
    int *d_status = nullptr;      // device status words (kStatusWords)

    // split-precision (BF16X6) path
    int JP = 0;               // folded latitudes padded to a multiple of 128
    int gemm_n = 128;         // GEMM tile width: 256 columns (32 groups) or 128 (16 groups)
    int ncolr = 0;            // columns per order: 8 per column group, padded to gemm_n
    int n_tiles = 0;          // ncolr / gemm_n
    int nk_f = 0;             // forward K-chunks: JP / kGemmChunkK
    int n_items_f = 0, n_items_a = 0;
    // Legendre operand (bf16 x 3), one layout that both directions' GEMMs read:
    // [piece][row block][JP latitudes][8 rows] (16-byte units of 8 consecutive rows of one
    // parity at one latitude), the row blocks of (mu, parity) from lam_rb[mu*2+p] on
    // (lam_rb_total in all).  Zeroed at plan creation; the generator never writes the
    // latitudes below an order's turning bound (jc_min), which therefore stay zero.
    void *d_lam = nullptr;
    int *d_lam_rb = nullptr;
    long long lam_rb_total = 0;
    int *d_jcmin = nullptr;       // [L+1] first latitude (multiple of 32) generated per order
    double gen_values = 0;        // recurrence values generated per direction
    // Legendre operand shared by a pair of calls (FAVEST_FLAG_SHARE_LAMBDA): kGenFwd when
    // the last call generated both layouts and the next forward call may use the forward
    // one without generating it, kGenAdj likewise for the next adjoint call, 0 otherwise
    int lam_pending = 0;
    double gemm_pairs_f = 0, gemm_pairs_a = 0;   // (row, latitude) pairs the GEMMs contract
    void *d_Fb = nullptr;         // forward B operand (FP32 records, split into bf16 x 3 by the GEMM)
    void *d_gb = nullptr;         // adjoint B operand (bf16 x 3)
    float *d_Q32 = nullptr;       // forward GEMM output [group][l][mu][8]
    float *d_S32 = nullptr;       // adjoint GEMM output [group][JP/4][mu][parity][4][8]
    int nf = 0;                   // column groups padded to a multiple of gemm_n / 8 (ncolr / 8)
    // The Legendre operand as the GEMMs' TMA sees it: one 4-D map per direction (the same
    // tensor, a 32 x 128 or 128 x 32 box); adjoint B: a 2-D array of 512-byte rows (every
    // chunk starts on a row and spans whole rows); forward B: 5-D map of Fb.
    CUtensorMap tmap_lam_f, tmap_lam_a, tmap_fb, tmap_gb;
    // the inverse DFT's view of S32: (32 floats, parity, mu, latitude group, column group),
    // boxes of 8 floats x 2 parities x kInvChunk orders
    CUtensorMap tmap_s32;
    GemmGroup *d_ggroups = nullptr;   // [2]: forward (Lam, Fb, Q32), adjoint (Lam, g, S32)
    std::vector<TcItem> h_items_f, h_items_a;   // host copies (merged by ragged batches)
    int gen_lt = 128, gen_mb = 1;  // generator shape: latitudes per block, orders per thread
    int gen_nj = 2;                // latitude chains per generator thread (1 or 2)
    int force_gemm_n = 0;          // 256: use 256-column GEMM tiles whatever the batch
    long long *d_g_off = nullptr;  // [mu*2+p] coefficient operand offsets
    float *d_P32 = nullptr, *d_M32 = nullptr, *d_R32 = nullptr;   // FP32 copies of P, M, R
    float *d_k1 = nullptr;        // [L+1] kappa of order 1 (order-0 adjoint on order-1 tiles)
    float2 *d_Adf = nullptr;      // [ntab] A_l^mu as double-float pairs (hi, lo) for the generator
    float2 *d_xdf = nullptr;      // [J] cos(theta_j) as double-float pairs
    // FP32 copies of the per-latitude factors the DFT stages apply ([J] each):
    float *d_omega32 = nullptr, *d_omega_unit32 = nullptr;   // omega_j, 1 / sin(theta_j)
    float2 *d_isc32 = nullptr;    // [2][J] (1/sin, 1) and (w_j/sin, w_j): inverse DFT scales
    int *d_perm = nullptr;        // [nphi] digit-reversal positions of the in-place FFT
    int fft_log2n = 0;            // log2(nphi) when nphi = 2^6..2^11 (power-of-two engine), else 0
    // polar patch of the split adjoint: rings j < pol_jc, orders 1 <= mu < pol_muc
    int pol_jc = 0, pol_muc = 0;
    float2 *d_pol = nullptr;      // [pol_jc][L+1][pol_muc] (D_l, Lambda_l) in fp32
    int *d_pol_lim = nullptr;     // [pol_jc] first order beyond ring j's turning bound (+16)
    float *d_polS = nullptr;      // [ncg][pol_jc][pol_muc][2][8] patched even/odd sums
    // the patch runs on a stream of its own next to the adjoint's other stages
    cudaStream_t pol_stream = nullptr;
    cudaEvent_t pol_fork = nullptr, pol_join = nullptr;
    TcItem *d_items_f = nullptr, *d_items_a = nullptr;

    // workspace
    void *d_F = nullptr;          // forward: raw longitude spectra [mu][col][nlat]
    void *d_Q = nullptr;          // scalar coefficients Q or g: [tab row][col]
    void *d_G = nullptr;          // adjoint: spectra rows [B][2][nlat][nphi]
    size_t ws_bytes = 0;

    FftPlan fft;

    // profiling: event pairs recorded around each launch while enabled
    int profiling = 0;
    struct Rec { int kernel; cudaEvent_t e0, e1; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> event_pool;
};

enum KernelId {
    KID_FFT_FWD = 0, KID_ANALYSIS, KID_COMBINE, KID_UNCOMBINE, KID_SYNTHESIS, KID_FFT_INV,
    KID_GEN_FWD, KID_GEMM_FWD, KID_GEN_ADJ, KID_GEMM_ADJ, KID_POLAR, KID_CG_COMBINE, KID_CG_UNCOMBINE,
    KID_GEN_BOTH, KID_CG_PACK, KID_CG_UNPACK, KID_COUNT
};

__host__ __device__ inline long long tab_off(int L, int mu) {
    return (long long)mu * (L + 2) - (long long)mu * (mu - 1) / 2;
}

// launchers (return cudaError_t of the launch)
cudaError_t launch_fft_fwd_fp64(const Plan &p, const void *Tth, const void *Tph, cudaStream_t s);
cudaError_t launch_fft_inv_fp64(const Plan &p, void *Tth, void *Tph, cudaStream_t s);
cudaError_t launch_analysis_fp64(const Plan &p, cudaStream_t s);
cudaError_t launch_synthesis_fp64(const Plan &p, cudaStream_t s);
cudaError_t launch_combine_fp64(const Plan &p, void *a, void *b, cudaStream_t s);
cudaError_t launch_uncombine_fp64(const Plan &p, const void *a, const void *b, cudaStream_t s);

cudaError_t launch_fft_fwd_bf16(const Plan &p, const void *Tth, const void *Tph, cudaStream_t s);
cudaError_t launch_fft_inv_bf16(const Plan &p, void *Tth, void *Tph, cudaStream_t s);
// Legendre operand layouts a generator launch writes (bit mask)
constexpr int kGenFwd = 1, kGenAdj = 2, kGenBoth = 3;
cudaError_t launch_gen_lambda(const Plan &p, int layouts, cudaStream_t s);
cudaError_t launch_gen_lambda_shape(const Plan &p, int layouts, int lt, int mb, int nj, cudaStream_t s);
// failure-path self-test: one GEMM item with no operand loads and the given wait bound
cudaError_t launch_gemm_selftest(const Plan &p, uint32_t poll_limit, cudaStream_t s);
// one persistent GEMM launch over an explicit item list (items[i].group indexes groups)
cudaError_t launch_tc_gemm_items(int gemm_n, const GemmGroup *groups, const TcItem *items, int nitems,
                                 int a_mn_major, int *status, int num_sms, cudaStream_t s);
cudaError_t launch_tc_gemm(const Plan &p, bool fwd, cudaStream_t s);
cudaError_t launch_combine_bf16(const Plan &p, void *a, void *b, cudaStream_t s);
cudaError_t launch_uncombine_bf16(const Plan &p, const void *a, const void *b, cudaStream_t s);
cudaError_t launch_polar_patch(const Plan &p, const void *a, const void *b, cudaStream_t s);
// Clebsch-Gordan route (FP64): scalar sums -> a, b (Thm. 1); a, b -> scalar coefficients (Thm. 2)
cudaError_t launch_cg_combine(const Plan &p, void *a, void *b, cudaStream_t s);
cudaError_t launch_cg_uncombine(const Plan &p, const void *a, const void *b, cudaStream_t s);
cudaError_t launch_cg_pack_fields(const Plan &p, const void *Tr, cudaStream_t s);
cudaError_t launch_cg_unpack_fields(const Plan &p, void *Tr, cudaStream_t s);
cudaError_t launch_cg_pack_coefs(const Plan &p, const void *a, const void *b, cudaStream_t s);
cudaError_t launch_cg_unpack_coefs(const Plan &p, void *a, void *b, cudaStream_t s);
int build_polar_tables(Plan &p);   // host: chooses pol_jc, pol_muc and uploads d_pol

// Every device allocation a plan (or batch, or scattered-point plan) makes goes through
// plan_malloc: it counts the calls and fails the one favest_debug_fail_alloc chose, so that
// tests can drive each allocation's error path without exhausting the device.
cudaError_t plan_malloc(void **p, size_t bytes);

int plan_create_internal(int L, int batch, int precision, int io_type, const double *cos_theta,
                         const double *w_lat, int force_gemm_n, favest_plan *out, int cg_route = 0);

}  // namespace favest

struct favest_plan_s {
    favest::Plan p;
};
