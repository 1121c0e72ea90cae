/*
 * favest.h -- C ABI of the GB300 (sm_103a) vector spherical harmonic transform
 * library: forward and adjoint transforms (FwdVSHT / AdjVSHT) of tangent fields on
 * a Gauss-Legendre tensor grid, after Le Gia, Li and Wang, "FaVeST -- Fast Vector
 * Spherical Harmonic Transforms" (arXiv 1908.00041).
 *
 * Definitions (paper Sec. 3 and Sec. 4):
 *   Y^div_lm  = grad* Y_lm / sqrt(l(l+1))          (B-family of eqs. Blm1, vsh)
 *   Y^curl_lm = x cross grad* Y_lm / sqrt(l(l+1))  (D-family of eqs. Blm2, vsh)
 *   FwdVSHT (Def. FwdVSHT, eq. fwdvsht2):
 *       a_lm = sum_k w_k Y^div_lm(x_k)^* T_k,   b_lm = sum_k w_k Y^curl_lm(x_k)^* T_k
 *   AdjVSHT (Def. AdjVSHT, eq. SLvec):
 *       S_L(a, b; x) = sum_{l=1}^{L} sum_{m=-l}^{l} a_lm Y^div_lm(x) + b_lm Y^curl_lm(x)
 * where the family names follow the paper's equations literally: Y^div (the paper's
 * "divergence-free" family) is the surface gradient family and Y^curl the surface
 * curl family.  Y_lm uses the Condon-Shortley phase and Y_{l,-m} = (-1)^m conj(Y_lm).
 *
 * Grid (Sec. 5.1, Gauss-Legendre tensor product rule): nlat = L+1 latitudes with
 * nodes x_j = cos(theta_j) in descending order (theta ascending) and latitude weights
 * W_j (sum 2); nphi = 2(L+1) longitudes phi_k = 2 pi k / nphi.  The quadrature weight
 * of point (j, k) is W_j * 2 pi / nphi.  This rule integrates every product of two
 * degree-L vector harmonics exactly, so favest_fwd(favest_adj(a, b)) == (a, b).
 *
 * Data layouts (all device memory unless stated):
 *   tangent field, per component (T_theta and T_phi are separate planes):
 *       [batch][nlat][nphi] complex, row-major; T = T_theta e_theta + T_phi e_phi
 *   coefficients a, b: [batch][L^2 + 2L] complex, l-major: index l^2 + l + m - 1
 *       for l = 1..L, m = -l..l  (paper Sec. 4.4, FaVeST_fwd output order).
 *   complex = interleaved (re, im); element type set by the plan's io type:
 *       FAVEST_IO_C128 = double, FAVEST_IO_C64 = float.
 *
 * Real fields (FAVEST_IO_R32 / FAVEST_IO_R64; the paper's fields are real, T_k in R^3,
 * Sec. 3): both components are real planes [batch][nlat][nphi] of float / double, and since then
 * a_{l,-m} = (-1)^m conj(a_lm) (likewise b), only orders m >= 0 are stored:
 *       a, b: [batch][L(L+3)/2] complex float / double, l-major: index l(l+1)/2 - 1 + m
 *       for l = 1..L, m = 0..l.
 * The forward transform of a real field returns exactly these entries of the complex
 * transform (a_l0 and b_l0 are real).  The adjoint evaluates the real field
 * Re S_L(a~, b~) of the Hermitian extension a~_{l,-m} = (-1)^m conj(a_lm) (m >= 1),
 * i.e. S_L of the extension with the imaginary parts of a_l0, b_l0 ignored; for
 * coefficients of a real field that is S_L itself.
 *
 * Ownership: the caller owns every data buffer and stream.  A plan owns its constant
 * tables and its device workspace; both are freed by favest_plan_destroy.
 *
 * Errors: every call returns a status code and never aborts the process.  Argument
 * errors are detected on the host before anything is launched.  Transform calls are
 * asynchronous on the given stream (a cudaStream_t passed as void*, NULL = legacy
 * default stream); a device-side failure is recorded in the plan's status word and
 * reported by favest_status.  Calls on one plan must not overlap in time (the plan's
 * workspace is shared by its calls).
 */
#ifndef FAVEST_H
#define FAVEST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct favest_plan_s *favest_plan;

enum favest_status_code {
    FAVEST_OK = 0,
    FAVEST_EINVAL = -1,        /* bad argument (size, pointer, alignment, grid)   */
    FAVEST_ENOMEM = -2,        /* device or host allocation failed                */
    FAVEST_ECUDA = -3,         /* a CUDA runtime call failed                      */
    FAVEST_EUNSUPPORTED = -4,  /* valid request this library or device cannot serve */
    FAVEST_ETIMEOUT = -5,      /* a bounded device-side wait gave up              */
    FAVEST_EDEVICE = -6,       /* a kernel recorded an internal error             */
    FAVEST_EINTERNAL = -7      /* a plan's own index tables failed their bounds check
                                  (see favest_debug_check_layout)                   */
};

/* Arithmetic of the Legendre contraction.  The recurrence, its underflow scaling,
 * the normalisation constants and the quadrature weights are FP64 in every mode (the
 * split-precision generator runs the recurrence in double-float arithmetic, pairs of FP32
 * numbers of about 44 significant bits, seeded from FP64 values). */
enum favest_precision {
    FAVEST_FP64 = 0,    /* FP64 everywhere (FFT, recurrence, contraction)                */
    FAVEST_BF16X6 = 1   /* FP32 FFT; double-float recurrence; Legendre contraction on tcgen05
                           tensor cores: both operands split into three bf16 pieces
                           (24 significant bits, full FP32 exponent range), the 6 piece
                           products of weight >= 2^-16 formed, the leading product
                           accumulated over K blocks of 32 and summed in FP32 with
                           round-to-nearest; complex64 fields and coefficients only     */
};

enum favest_io_type {
    FAVEST_IO_C128 = 0,  /* complex double */
    FAVEST_IO_C64 = 1,   /* complex float  */
    FAVEST_IO_R32 = 2,   /* real fields (float), half-spectrum complex float coefficients */
    FAVEST_IO_R64 = 3    /* real fields (double), half-spectrum complex double coefficients */
};

/*
 * Gauss-Legendre rule on [-1, 1] (host).  x[nlat] receives the nodes in descending
 * order, w[nlat] the weights (sum 2).  Returns FAVEST_EINVAL if nlat < 1 or a
 * pointer is NULL.
 */
int favest_gl_grid(int nlat, double *x, double *w);

/*
 * Create a plan for degree L and a batch of `batch` fields (1 <= batch <= 4096) on the
 * current CUDA device.  1 <= L <= 2559 (up to 1280 latitude pairs); L = 2560..4095 returns
 * FAVEST_EUNSUPPORTED, L < 1, L > 4095 or a batch outside 1..4096 FAVEST_EINVAL.  FAVEST_BF16X6
 * requires io_type FAVEST_IO_C64 or FAVEST_IO_R32 (FAVEST_EUNSUPPORTED otherwise) and
 * a device with tcgen05 tensor cores (sm_100 family; its FP32 longitude DFT takes any
 * nphi = 2(L+1), prime factors from 17 up through Bluestein stages); FAVEST_IO_R64 requires
 * FAVEST_FP64 (FAVEST_EUNSUPPORTED
 * otherwise), FAVEST_IO_R32 works with both precisions.  Real-field plans take 16-byte
 * aligned pointers.
 *   cos_theta, w_lat: optional host arrays of nlat = L+1 latitude nodes (descending)
 *       and latitude weights; NULL selects the built-in Gauss-Legendre rule.  When
 *       given, the nodes must lie strictly inside (-1, 1) and both arrays must be
 *       symmetric about the equator (x_{n-1-j} = -x_j, w_{n-1-j} = w_j to 1e-14);
 *       otherwise FAVEST_EINVAL.
 *   precision: enum favest_precision; io_type: enum favest_io_type.
 * Allocates the plan's constant tables and workspace on the device (FAVEST_ENOMEM on
 * failure).  *out receives the plan (NULL on failure).
 */
int favest_plan_create(int L, int batch, int precision, int io_type,
                       const double *cos_theta, const double *w_lat, favest_plan *out);

/*
 * FwdVSHT (Def. FwdVSHT, eq. fwdvsht2) of `batch` fields.
 *   Tth, Tph: device, [batch][nlat][nphi] complex (plan io type), read only.
 *   a, b:     device, [batch][L^2+2L] complex (plan io type), written.
 *   (FAVEST_IO_R32: real float fields and [batch][L(L+3)/2] coefficients, m >= 0.)
 * Pointers must be aligned to the complex element size (to 16 bytes for
 * FAVEST_BF16X6 plans).  Asynchronous on `stream`.
 */
int favest_fwd(favest_plan plan, const void *Tth, const void *Tph, void *a, void *b,
               void *stream);

/*
 * AdjVSHT (Def. AdjVSHT, eq. SLvec) of `batch` coefficient sets, evaluated on the
 * plan's grid.
 *   a, b:     device, [batch][L^2+2L] complex, read only.
 *   Tth, Tph: device, [batch][nlat][nphi] complex, written (the Nyquist longitude
 *             bin m = L+1 carries no coefficient and is zero).
 *   (FAVEST_IO_R32: [batch][L(L+3)/2] coefficients, m >= 0, and real float fields;
 *   see the real-field note at the top of this file.)
 */
int favest_adj(favest_plan plan, const void *a, const void *b, void *Tth, void *Tph,
               void *stream);

/*
 * The paper's Clebsch-Gordan route (Sec. 4, Thm. 1, Thm. 2, Algs. 1-2), FP64: the same
 * transforms for fields given by Cartesian components, T = T^(1) e_x + T^(2) e_y + T^(3) e_z
 * (as FaVeST_fwd(T, L, X, w) takes them, Sec. 4.4), computed through scalar spherical
 * harmonic transforms of degree L+1 of the three components on the plan's grid:
 *   forward (Thm. 1): a_lm, b_lm as fixed combinations, with the Clebsch-Gordan values of
 *     eq. ninecoeff and c_l, d_l of eq. cl,dl,betal, of the FwdSHTs (eq. Flm) of T^(1),
 *     T^(2), T^(3) at degrees l-1, l, l+1 and orders m-1, m, m+1;
 *   adjoint (Thm. 2): the nu/eta coefficient sets (eqs. nulm1, nulm2, etalm; a, b read as
 *     zero outside 1 <= l <= L, |m| <= l) summed per component into one scalar synthesis
 *     of degree L+1 each (the AdjSHTs S_{L-1}, S_L, S_{L+1} of the theorem are linear).
 * Both are identities for any point set; on the Gauss-Legendre grid they equal favest_fwd
 * and favest_adj of the theta/phi components to rounding (tested).
 *
 * favest_cg_plan_create: an FP64 plan for `batch` such fields (1 <= batch <= 1366),
 *   arguments and errors as favest_plan_create.  The plan serves only the two calls below;
 *   favest_fwd/favest_adj on it return FAVEST_EINVAL, and these calls on other plans too.
 * favest_fwd_cart: T device [batch][3][nlat][nphi] complex double (component planes x, y,
 *   z of each field), read only; a, b device [batch][L^2+2L] complex double, written.
 * favest_adj_cart: a, b read; T written in the same layout.
 * Pointers 16-byte aligned; asynchronous on `stream`.
 */
int favest_cg_plan_create(int L, int batch, const double *cos_theta, const double *w_lat,
                          favest_plan *out);
/*
 * favest_cg_plan_create_ex: as favest_cg_plan_create for io_type FAVEST_IO_C128; with
 *   FAVEST_IO_R64 a plan for `batch` REAL fields (1 <= batch <= 2732; the paper's fields,
 *   Sec. 3): favest_fwd_cart then takes T device [batch][3][nlat][nphi] double and writes
 *   half-spectrum a, b device [batch][L(L+3)/2] complex double (m >= 0, the real-field
 *   layout at the top of this file), favest_adj_cart the reverse.  Fields 2q and 2q+1 are
 *   transformed together as the complex field T_2q + i T_2q+1 (the transforms are linear
 *   and a real field's coefficients satisfy a_{l,-m} = (-1)^m conj(a_lm)), through pack
 *   and unpack kernels around the complex route and a workspace of ceil(batch/2) complex
 *   fields and coefficient sets.  Other io types: FAVEST_EINVAL.
 */
int favest_cg_plan_create_ex(int L, int batch, int io_type, const double *cos_theta, const double *w_lat,
                             favest_plan *out);
int favest_fwd_cart(favest_plan plan, const void *T, void *a, void *b, void *stream);
int favest_adj_cart(favest_plan plan, const void *a, const void *b, void *T, void *stream);

/*
 * Transforms at arbitrary points, the paper's interface FaVeST_fwd(T, L, X, w) and
 * FaVeST_adj(a, b, X) (Sec. 4.4; point sets of Sec. 5.1 such as spherical designs), FP64:
 *   forward (Def. FwdVSHT, eq. fwdvsht2): a_lm = sum_k w_k Y^div_lm(x_k)^* T_k,
 *                                         b_lm = sum_k w_k Y^curl_lm(x_k)^* T_k;
 *   adjoint (Def. AdjVSHT, eq. SLvec):    T_k = S_L(a, b; x_k),
 * for fields given by their Cartesian components at npts points x_k.  Both run the paper's
 * route (Thm. 1, Thm. 2): scalar spherical harmonic transforms of degree L+1 of the three
 * Cartesian components, here summed directly over the points (O(npts L^2) FP64 work; the
 * paper uses NFFT-based fast transforms instead), combined with the Clebsch-Gordan values of
 * eq. ninecoeff exactly as favest_fwd_cart / favest_adj_cart do.  No quadrature exactness is
 * assumed: favest_scatter_fwd is the weighted sum itself, whatever the points and weights.
 *
 * favest_scatter_create: L = 1..2047, batch = 1..1366 fields, npts = 1..2^26 points.
 *   X: host [npts][3], the points as unit vectors (|x_k| = 1 to 1e-10, FAVEST_EINVAL
 *      otherwise; they are normalised); points at or near the poles are allowed.
 *   w: host [npts] point weights, or NULL for unit weights (then the forward is A^H, the
 *      exact adjoint of favest_scatter_adj).
 *   Copies the points to device memory the plan owns (with its tables and workspace:
 *   O(L^2 batch + npts) doubles).  *out receives the plan (NULL on failure).
 * favest_scatter_fwd: T device [batch][npts][3] complex double (x, y, z components of each
 *   point), read only; a, b device [batch][L^2+2L] complex double, written (l-major).
 * favest_scatter_adj: a, b read; T written in the same layout (the tangent field S_L(a, b)
 *   at the points, so T_k . x_k = 0 to rounding).
 * Pointers 16-byte aligned; asynchronous on `stream`; calls on one plan must not overlap.
 * Errors as for the grid transforms.  favest_scatter_npts returns the point count.
 */
typedef struct favest_scatter_s *favest_scatter;
int favest_scatter_create(int L, int batch, int npts, const double *X, const double *w, favest_scatter *out);
int favest_scatter_fwd(favest_scatter plan, const void *T, void *a, void *b, void *stream);
int favest_scatter_adj(favest_scatter plan, const void *a, const void *b, void *T, void *stream);
int favest_scatter_npts(favest_scatter plan);
void favest_scatter_destroy(favest_scatter plan);

/*
 * Stability ratios of the forward Clebsch-Gordan route (Sec. 5.5, eq. r_stable).  Thm. 1
 * writes Y^div_lm(x)^* as six terms xi_q Y*_{l',m'}(x) u_q and Y^curl_lm(x)^* as three terms
 * mu_q Y*_{l,m'}(x) u_q (u_q unit vectors).  Per point x_k and coefficient (l, m):
 *   rho_hat   = |Y^div_lm(x_k)|  / Vhat,    Vhat   = sqrt2 sum_q |xi_q| |Y_{l',m'}(x_k)|,
 *   rho_tilde = |Y^curl_lm(x_k)| / Vtilde,  Vtilde = sqrt2 sum_q |mu_q| |Y_{l,m'}(x_k)|,
 * i.e. the printed ratio of the size of the sum to the sum of the sizes of its terms
 * (|xi| taken since Clebsch-Gordan values can be negative; a point where V = 0 has no
 * ratio and is skipped).  Both depend on the colatitude only.
 *   L: 1..1023.  npts: 1..2^28.
 *   cos_theta: host [npts], cos(theta_k) of the points, each strictly inside (-1, 1).
 *   per_coef: host [4][L^2+2L] or NULL; receives per coefficient (l-major order) the
 *     maximum and minimum over the points of rho_hat, then of rho_tilde (0 and +inf for a
 *     coefficient no point gives a ratio).
 *   ratios: host [4]: r_hat = max rho_hat, kappa_hat = max 1/rho_hat, r_tilde, kappa_tilde,
 *     over l <= L, 1 <= |m| <= l (the range of eq. r_stable) and the points.  The printed
 *     ratio is at most 1/sqrt2 (triangle inequality); kappa is the condition number of the
 *     route's sums in the sense of Higham's summation analysis, which Sec. 5.5 cites.
 * Copies the points to a device buffer of the library's own (freed before returning),
 * runs on `stream` and synchronises it; FAVEST_EINVAL for bad arguments, FAVEST_ENOMEM
 * if the buffer cannot be allocated, FAVEST_ECUDA if a copy or launch fails.
 */
int favest_cg_stability(int L, int npts, const double *cos_theta, double *per_coef, double *ratios,
                        void *stream);

/*
 * Weighting of the forward transform.  flag = 0 (default): the quadrature weights of
 * eq. fwdvsht2.  flag = 1: unit weights, i.e. favest_fwd computes A^H T, the exact
 * adjoint of favest_adj (used by reverse-mode differentiation of AdjVSHT).
 */
int favest_set_weights_unit(favest_plan plan, int flag);

/*
 * The two transforms with per-call options (the operators reverse-mode
 * differentiation needs; with flags = 0 they are favest_fwd and favest_adj).  Writing
 * A for AdjVSHT (coefficients -> grid) and W for the diagonal of point weights
 * W_j * 2 pi / nphi, FwdVSHT is A^H W, so
 *   d/dT of FwdVSHT  is  (A^H W)^H = W A:  favest_adj_ex with FAVEST_FLAG_WEIGHTED,
 *                        which multiplies the synthesised field by W in the inverse
 *                        longitude DFT stage;
 *   d/dc of AdjVSHT  is  A^H:              favest_fwd_ex with FAVEST_FLAG_UNIT_WEIGHTS.
 * Real-field plans (FAVEST_IO_R32/R64) map real fields to half spectra, and their
 * transposes for the real inner products (Re sum conj(u) v on coefficients) add a factor
 * per order, which FAVEST_FLAG_REAL_TRANSPOSE applies:
 *   favest_adj_ex: orders m > 0 of a, b enter with weight 1/2, so that with
 *     FAVEST_FLAG_WEIGHTED the call computes W Re sum_{m >= 0} (a_lm Y^div + b_lm Y^curl),
 *     the transpose of the real FwdVSHT;
 *   favest_fwd_ex: orders m > 0 of the result are doubled, so that with
 *     FAVEST_FLAG_UNIT_WEIGHTS the call is the transpose of the real AdjVSHT.
 * The factors 1/2 and 2 are exact.  On complex plans the flag is FAVEST_EINVAL.
 *
 * FAVEST_FLAG_SHARE_LAMBDA (both calls; split-precision plans, ignored by FP64 plans): an
 * adjoint and a forward transform on the same plan and degree contract the same Legendre
 * values lambda_l^m(theta_j) (Sec. 3, definition of Y_lm), which the split path
 * regenerates by its recurrence in every call.  With this flag on two consecutive
 * calls of opposite direction (adjoint then forward, or forward then adjoint), the first
 * call's recurrence pass writes the values in the layouts of both directions and the second
 * call uses them without a generator launch (one launch fewer, see
 * favest_launches_per_call).  A flagged call that does not directly follow such a first
 * call (no call on the plan in between) generates both layouts itself.  Results are bitwise
 * identical with and without the flag.  The second call must be ordered after the first on
 * the device (same stream, or synchronised), as every call on one plan must be.
 *
 * Any other flag bit is FAVEST_EINVAL.  Calls on one plan must not overlap in time on
 * the host (the flags live in the plan for the duration of the call).
 */
enum { FAVEST_FLAG_UNIT_WEIGHTS = 1, FAVEST_FLAG_WEIGHTED = 2, FAVEST_FLAG_REAL_TRANSPOSE = 4,
       FAVEST_FLAG_SHARE_LAMBDA = 8 };
int favest_fwd_ex(favest_plan plan, const void *Tth, const void *Tph, void *a, void *b, int flags,
                  void *stream);
int favest_adj_ex(favest_plan plan, const void *a, const void *b, void *Tth, void *Tph, int flags,
                  void *stream);

/* Plan properties (host). */
int favest_plan_L(favest_plan plan);
int favest_plan_batch(favest_plan plan);
int favest_plan_precision(favest_plan plan);
size_t favest_plan_workspace_bytes(favest_plan plan);

/*
 * Synchronise `stream` and return the plan's device status word (FAVEST_OK, or the
 * first device-side error recorded since the last call); clears the word.
 */
int favest_status(favest_plan plan, void *stream);

/* Release the plan and everything it owns.  NULL is ignored. */
void favest_plan_destroy(favest_plan plan);

/* Static description of a status code. */
const char *favest_strerror(int status);

/* Number of kernels each transform call launches without FAVEST_FLAG_SHARE_LAMBDA (for
 * launch accounting); the second call of a pair sharing the Legendre operand launches one
 * fewer. */
int favest_launches_per_call(favest_plan plan, int adjoint);

/*
 * Autotuner of the split-precision path's recurrence generator.  The generator
 * runs 128 threads per block as (128 / lt) orders x lt latitudes (lt = 32, 64, 128),
 * each block covering mb order groups in turn (mb = 1, 2, 4), each thread running the
 * recurrences of 1 or 2 latitudes (lt apart) side by side.  favest_plan_tune times the
 * candidate shapes for this plan's degree on `stream` (synchronising it, a few
 * milliseconds) and keeps the fastest; favest_plan_gen_shape reports (lt, mb) of the
 * shape in use.  Plans start with (128, 1), with 2 latitudes per thread from 384 folded
 * latitudes (L >= 766) up and 1 below.  The generated
 * values do not depend on the shape.  FP64 plans have nothing to tune (returns FAVEST_OK).
 */
int favest_plan_tune(favest_plan plan, void *stream);
int favest_plan_gen_shape(favest_plan plan, int *lt, int *mb);
/* Latitude recurrences per generator thread of the shape in use (1 or 2); FAVEST_EINVAL for
 * a null plan. */
int favest_plan_gen_chains(favest_plan plan);

/*
 * Apply a generator shape without timing (e.g. one a previous favest_plan_tune chose for the
 * same degree, batch, precision and GPU, kept in a cache): lt latitudes per block, mb order
 * groups per block, nj latitude chains per thread.  Accepted shapes are exactly those the
 * tuner times: (lt, mb, nj) with nj in {1, 2} and (lt, mb) in {(128, 1), (64, 1), (32, 1),
 * (128, 2), (64, 2), (32, 2), (32, 4)}; anything else, or a NULL plan, returns FAVEST_EINVAL.
 * On an FP64 plan (no generator) a valid shape is accepted and ignored.  Host-only; affects
 * the plan's later calls, never its results (every shape computes identical values).
 */
int favest_plan_set_gen_shape(favest_plan plan, int lt, int mb, int nj);

/*
 * Ragged batches: nfields fields of individual degrees L[i] (host array), each on its
 * own (L[i]+1) x 2(L[i]+1) Gauss-Legendre grid.  The caller's buffers hold the fields
 * packed: component plane of field i at element offset field_off[i] of Tth and of Tph
 * (elements of the io type, starting on 16 bytes), its coefficients (L[i]^2 + 2 L[i] of each family)
 * at element offset coef_off[i] of a and of b; null offset arrays mean packed in field
 * order (each plane rounded up to 16 bytes).  favest_batch_field_elems / favest_batch_coef_elems give the buffer lengths.
 *
 * Fields are grouped by degree.  In the split-precision form the tensor-core Legendre
 * stage of all groups is one persistent kernel launch over a merged work queue of
 * (degree group, order, parity, row or latitude tile) items; the longitude DFTs, combine
 * and generator stages run once per degree group.  Flags:
 *   FAVEST_BATCH_AUTOTUNE  tune each group's generator shape at creation (favest_plan_tune)
 *   FAVEST_BATCH_GRAPH     replay each direction as a CUDA graph: the first call with a
 *                          given set of buffers runs directly, the second captures the
 *                          launch sequence, later ones launch the captured graph
 * Errors as for the single-field calls; favest_batch_status reads and clears the device
 * status words of all groups.  Calls on one batch must not overlap on the host.
 * Real fields (FAVEST_IO_R32, FAVEST_IO_R64): real planes and half-spectrum coefficient
 * sets (L(L+3)/2 per family); field offsets must then be multiples of 16 bytes.
 */
typedef struct favest_batch_s *favest_batch;
enum { FAVEST_BATCH_AUTOTUNE = 1, FAVEST_BATCH_GRAPH = 2 };
int favest_batch_create(int nfields, const int *L, const long long *field_off, const long long *coef_off,
                        int precision, int io_type, int flags, favest_batch *out);
int favest_fwd_batched(favest_batch batch, const void *Tth, const void *Tph, void *a, void *b, void *stream);
int favest_adj_batched(favest_batch batch, const void *a, const void *b, void *Tth, void *Tph, void *stream);
int favest_batch_ngroups(favest_batch batch);
int favest_batch_group(favest_batch batch, int g, int *L, int *nfields, int *gen_lt, int *gen_mb);
long long favest_batch_field_elems(favest_batch batch);
long long favest_batch_coef_elems(favest_batch batch);
int favest_batch_status(favest_batch batch, void *stream);
void favest_batch_destroy(favest_batch batch);

/*
 * Per-kernel timing (a profiling aid).  While enabled (enable = 1), every transform
 * call records a CUDA event pair around each kernel it launches, on the call's
 * stream.  favest_profile_read synchronises those events and returns, for up to
 * max_kernels distinct kernels, the name (NUL-terminated, at most 31 characters, in
 * names[k*32]), the accumulated milliseconds ms[k] and the launch count launches[k];
 * it then clears the records.  Returns the number of kernels written (>= 0) or a
 * negative status.  Leave timing disabled while capturing a CUDA graph.
 */
int favest_profile_enable(favest_plan plan, int enable);
int favest_profile_read(favest_plan plan, int max_kernels, char *names, double *ms,
                        long long *launches);

/*
 * Failure-path self-test (no counterpart in the paper).  Launches the split-precision
 * tensor-core GEMM of this plan on one work item with its operand loads switched off and
 * every device-side wait bounded by poll_limit mbarrier polls, on the legacy stream, and
 * synchronises.  The waits cannot complete, so the kernel must give up, record
 * FAVEST_ETIMEOUT in the plan's status word, release its tensor memory and return; the
 * call returns that status (read and cleared as favest_status does) and, if elapsed_ms
 * is not null, the kernel's duration.  The context stays usable.  FAVEST_EUNSUPPORTED for
 * FP64 plans.
 */
int favest_selftest_wait_timeout(favest_plan plan, unsigned poll_limit, double *elapsed_ms);

/*
 * Allocation-failure test hook (no counterpart in the paper).  Every device allocation that
 * plan, batch and scattered-point creation make is counted; favest_debug_fail_alloc(k)
 * resets the count and makes the k-th allocation from now (k = 0 the first) fail as if the
 * device were out of memory, or disarms the hook (k = -1).  A creation call that meets the
 * failure returns FAVEST_ENOMEM after releasing everything it had allocated.
 * favest_debug_alloc_count() returns the allocations counted since the last
 * favest_debug_fail_alloc call.  FAVEST_EINVAL for k < -1.  Process-wide; not for use while
 * other threads create plans.
 */
int favest_debug_fail_alloc(long long k);
long long favest_debug_alloc_count(void);

/*
 * Bounds check of a plan's index tables without creating the plan (no counterpart in the
 * paper; no CUDA call, so it runs on a host without a GPU).  Builds the host-side tables
 * that favest_plan_create builds for (L, batch, precision, io_type) on the Gauss-Legendre
 * grid -- for FAVEST_BF16X6 the tensor-core GEMM work items of both directions, the
 * per-(order, parity) operand regions and the forward operand's TMA box coordinates, with
 * gemm_n = 0 (the plan's own tile width) or 256 (the width ragged batches use) -- and
 * checks every index the kernels take from them against the buffer it addresses: the
 * Legendre operand's boxes (row and latitude blocks) against the rows of the item's own
 * order and the tensor's extents, the other operands' chunk ranges, 512-byte row
 * alignment and box coordinates, output rows and column groups against the output buffer
 * and the rows of the item's own order, regions in order and disjoint.  FP64 plans have no such tables and
 * return FAVEST_OK once their arguments pass.  Returns FAVEST_OK; the argument errors of
 * favest_plan_create (FAVEST_EINVAL, FAVEST_EUNSUPPORTED) and FAVEST_EINVAL for another
 * gemm_n or msg_len < 0; or FAVEST_EINTERNAL with a description of the first violation
 * written to msg (NUL-terminated, at most msg_len bytes; msg may be null when msg_len is
 * 0).  favest_plan_create runs the same check and fails with FAVEST_EINTERNAL likewise.
 * poison (tests of the check itself; 0 in normal use) corrupts the check's own copy of the
 * tables first: 1 moves the first forward item to order L + 1, 2 gives the last adjoint
 * item one K-chunk too many, 3 makes the Legendre row blocks of the first two (order,
 * parity) regions overlap; other values give FAVEST_EINVAL.
 */
int favest_debug_check_layout(int L, int batch, int precision, int io_type, int gemm_n, int poison, char *msg,
                              int msg_len);

/*
 * Algorithmic work of one launch of a kernel of this plan, by the name that
 * favest_profile_read reports: *bytes = the minimum DRAM traffic (every operand read
 * once, every result written once, no re-reads, no padding), *flops = arithmetic
 * (an FMA counted as 2; for a recurrence every multiply-add of the exact recurrence
 * counts as 2), *pipe = the unit that bounds it in this design
 * (0 = HBM, 1 = FP64 pipe, 2 = tensor pipe, 3 = FP32 pipe).  Host-only, no GPU work.
 * Returns FAVEST_OK, or FAVEST_EINVAL for an unknown name.
 */
int favest_kernel_work(favest_plan plan, const char *kernel, double *bytes, double *flops, int *pipe);

/*
 * Measure the current device's FP64 and FP32 fused multiply-add throughput
 * (TFLOP/s, an FMA counted as 2 flops) with short register-resident FMA streams,
 * ~20 ms.  Used as the roofline denominator of the FP64-pipe-bound kernels.
 */
int favest_probe_peaks(double *fp64_tflops, double *fp32_tflops);

/*
 * FwdVSHT in FP64 without allocating device memory (this entry point has no
 * counterpart in the paper; it serves callers that cannot call cudaMalloc where they
 * need the transform -- inside a stream capture that must not allocate, in real-time
 * loops that cannot risk allocation latency or failure, or in plug-ins whose device
 * memory is reserved by someone else's pool).
 *
 * Computes exactly what favest_fwd computes for an FP64 plan with the built-in
 * Gauss-Legendre grid and FAVEST_IO_C128 data: Tth, Tph device [batch][L+1][2(L+1)]
 * complex double in, a, b device [batch][L^2+2L] complex double out (16-byte
 * aligned), asynchronously on `stream`.
 *
 * Scratch: a single file-scope device array of favest_noalloc_scratch_bytes() = 32 MB,
 * held by every GPU that loads the library until the process exits.  A request whose
 * scratch (grid and recurrence tables, spectra, scalar sums; about
 * 96 (L+1)^2 batch + 24 (L+1)^2 bytes) exceeds it (L = 511 fits for batch 1 only;
 * L = 511 with batch 2, or L = 1023, does not), L > 1023 or batch > 4096 returns
 * FAVEST_EINVAL before anything is launched.  No cudaMalloc, cudaFree or other
 * allocating call is made.  The first call in a CUDA context looks up the array's
 * device address (cudaGetSymbolAddress) with that context current, and looks it up
 * again in a new context of the same device (e.g. after cudaDeviceReset); make the
 * first call in each context before any stream capture.  Every call rewrites the tables
 * it needs, but all calls share the one array: calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Errors: FAVEST_EINVAL as above or for NULL or misaligned pointers; FAVEST_ECUDA if a
 * launch fails, or if the CUDA runtime already holds an unread error from an earlier
 * call on this host thread when the call starts (nothing is launched then, and that
 * error is left for its owner to read with cudaGetLastError).  The kernels of this path
 * record no device-side status (favest_status has no plan to read here).
 */
int favest_fwd_fp64_noalloc(int L, int batch, const void *Tth, const void *Tph, void *a, void *b,
                            void *stream);
size_t favest_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* FAVEST_H */
