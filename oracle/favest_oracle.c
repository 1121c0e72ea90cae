/*
 * CPU oracle for the forward and adjoint vector spherical harmonic transforms
 * (FwdVSHT / AdjVSHT) of FaVeST (Le Gia, Li, Wang; arXiv 1908.00041).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain FP64 statement of what
 * the transforms compute.  It shares no code with the CUDA library: only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark load it.
 *
 * Forms provided (each cites the passage it restates):
 *   O1 "literal"   : Cartesian vector spherical harmonics built exactly as the
 *                    paper defines them (Sec. 3: eqs. Blm1, Blm2, vsh2 with the nine
 *                    Clebsch-Gordan closed forms of eq. ninecoeff), then the direct
 *                    weighted sums of Def. FwdVSHT (eq. fwdvsht2) and the partial sum
 *                    of Def. AdjVSHT (eq. SLvec).
 *   O3 "separable" : the same sums on a Gauss-Legendre tensor grid, regrouped into
 *                    an exact per-ring DFT followed by the Legendre sum, using the
 *                    theta/phi closed forms Y^div = grad Y / sqrt(l(l+1)) and
 *                    Y^curl = x cross grad Y / sqrt(l(l+1)) (pinned against O1 by the
 *                    tests).
 * Normalised associated Legendre values use Fukushima's extended-exponent
 * "X-number" arithmetic (J. Geodesy 86, 2012) so that no value underflows at any
 * degree; this is deliberately a different scaling scheme from the GPU path.
 *
 * Readings of the paper adopted here:
 *   - negative orders: Y_{l,-m} = (-1)^m conj(Y_{l,m})  (the conjugate is missing
 *     from the printed definition in Sec. 3);
 *   - P_l^m carries the Condon-Shortley phase (-1)^m (the only choice for which
 *     the Clebsch-Gordan combination of eq. vsh is tangent);
 *   - the Nyquist longitude bin m = n_phi/2 is not a coefficient.
 *
 * Complex arrays are interleaved (re, im) doubles.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

/* ------------------------------------------------------------------------- */
/* Gauss-Legendre rule (Sec. 5.1, "Gauss-Legendre tensor product rule")      */
/* Nodes x_j = cos(theta_j) in descending order (theta ascending), weights    */
/* sum to 2.  Newton iteration on P_n with the three-term recurrence.         */
/* ------------------------------------------------------------------------- */
int orc_gl(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {   /* recompute the derivative at the converged node */
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1; p1 = p2;
            }
            double pn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
        }
        double wt = 2.0 / ((1.0 - z * z) * dp * dp);
        x[i] = z;          w[i] = wt;
        x[n - 1 - i] = -z; w[n - 1 - i] = wt;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* X-numbers: value = f * BIG^e with BIG = 2^960 (Fukushima 2012).           */
/* ------------------------------------------------------------------------- */
#define XBIG   0x1p960
#define XBIGI  0x1p-960
#define XBIGS  0x1p480
#define XBIGSI 0x1p-480

typedef struct { double f; int e; } xnum;

static void xnorm(xnum *x)
{
    if (x->f == 0.0) { x->e = 0; return; }
    double a = fabs(x->f);
    if (a >= XBIGS) { x->f *= XBIGI; x->e += 1; }
    else if (a < XBIGSI) { x->f *= XBIG; x->e -= 1; }
}

static double x2f(xnum x)
{
    if (x.e == 0) return x.f;
    if (x.e < 0) return (x.e == -1) ? x.f * XBIGI : 0.0;
    return x.f * XBIG;   /* never happens for normalised Legendre values */
}

/* f*x + g*y for X-numbers x, y and ordinary doubles f, g */
static xnum xlsum2(double f, xnum x, double g, xnum y)
{
    xnum z;
    if (x.f == 0.0) { z.f = g * y.f; z.e = y.e; xnorm(&z); return z; }
    if (y.f == 0.0) { z.f = f * x.f; z.e = x.e; xnorm(&z); return z; }
    int d = x.e - y.e;
    if (d == 0)       { z.f = f * x.f + g * y.f;          z.e = x.e; }
    else if (d == 1)  { z.f = f * x.f + g * y.f * XBIGI;  z.e = x.e; }
    else if (d == -1) { z.f = g * y.f + f * x.f * XBIGI;  z.e = y.e; }
    else if (d > 1)   { z.f = f * x.f;                    z.e = x.e; }
    else              { z.f = g * y.f;                    z.e = y.e; }
    xnorm(&z);
    return z;
}

/* eps_l^m = sqrt((l^2 - m^2) / (4 l^2 - 1)) */
static double eps_lm(int l, int m)
{
    double v = ((double)l * l - (double)m * m) / (4.0 * l * l - 1.0);
    return v > 0.0 ? sqrt(v) : 0.0;
}

/*
 * lambda_l^m(theta) for l = m..lmax at one point, m >= 0:
 *   lambda_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m(cos theta)
 * (the theta factor of Y_lm in Sec. 3), with the Condon-Shortley phase.
 * out[l - m] receives lambda_l^m.  Textbook recurrences:
 *   lambda_0^0 = 1/sqrt(4 pi),  lambda_m^m = -sqrt((2m+1)/(2m)) sin(theta) lambda_{m-1}^{m-1},
 *   lambda_{m+1}^m = sqrt(2m+3) cos(theta) lambda_m^m,
 *   eps_l^m lambda_l^m = cos(theta) lambda_{l-1}^m - eps_{l-1}^m lambda_{l-2}^m.
 */
void orc_lambda_col(int m, int lmax, double cost, double sint, double *out)
{
    if (lmax < m) return;
    xnum pmm = { 1.0 / sqrt(4.0 * M_PI), 0 };
    for (int k = 1; k <= m; ++k) {
        pmm.f *= -sqrt((2.0 * k + 1.0) / (2.0 * k)) * sint;
        xnorm(&pmm);
    }
    out[0] = x2f(pmm);
    if (lmax == m) return;
    xnum zero = { 0.0, 0 };
    xnum p1 = xlsum2(sqrt(2.0 * m + 3.0) * cost, pmm, 0.0, zero);
    out[1] = x2f(p1);
    xnum p0 = pmm;
    for (int l = m + 2; l <= lmax; ++l) {
        double el = eps_lm(l, m), el1 = eps_lm(l - 1, m);
        xnum p2 = xlsum2(cost / el, p1, -el1 / el, p0);
        out[l - m] = x2f(p2);
        p0 = p1; p1 = p2;
    }
}

/* Index of (l, m) in a scalar table with l = 0..lmax, m = -l..l: l^2 + l + m */
static inline int sidx(int l, int m) { return l * l + l + m; }

/*
 * Scalar spherical harmonics Y_lm(theta, phi), l = 0..lmax, |m| <= l, at one
 * point (Sec. 3).  y[sidx(l,m)] complex.  e^{i m phi} is taken from (cm, sm)
 * arrays holding cos(m phi), sin(m phi) for m = 0..lmax.
 */
static void sh_table(int lmax, double cost, double sint, const double *cm,
                     const double *sm, cplx *y, double *col)
{
    for (int m = 0; m <= lmax; ++m) {
        orc_lambda_col(m, lmax, cost, sint, col);
        cplx e = cm[m] + I * sm[m];
        double sg = (m & 1) ? -1.0 : 1.0;
        for (int l = m; l <= lmax; ++l) {
            cplx v = col[l - m] * e;
            y[sidx(l, m)] = v;
            if (m > 0) y[sidx(l, -m)] = sg * conj(v);
        }
    }
}

void orc_sh_point(int lmax, double theta, double phi, double *yout)
{
    double *cm = malloc(sizeof(double) * (lmax + 1)), *sm = malloc(sizeof(double) * (lmax + 1));
    double *col = malloc(sizeof(double) * (lmax + 2));
    for (int m = 0; m <= lmax; ++m) { cm[m] = cos(m * phi); sm[m] = sin(m * phi); }
    sh_table(lmax, cos(theta), sin(theta), cm, sm, (cplx *)yout, col);
    free(cm); free(sm); free(col);
}

/* ------------------------------------------------------------------------- */
/* O1: literal vector spherical harmonics (Sec. 3, Definition of VSH)         */
/* ------------------------------------------------------------------------- */

/* c_l, d_l of eq. cl,dl,betal */
static double c_l(int l) { return sqrt((l + 1.0) / (2.0 * l + 1.0)); }
static double d_l(int l) { return sqrt((double)l / (2.0 * l + 1.0)); }

static double sqrt0(double v) { return v > 0.0 ? sqrt(v) : 0.0; }

/*
 * The nine Clebsch-Gordan values of eq. ninecoeff, C^{l,m}_{j1,m1,1,q}.
 * cg[0] = C^{l,m}_{l-1,m-1,1,1}   cg[1] = C^{l,m}_{l+1,m-1,1,1}
 * cg[2] = C^{l,m}_{l-1,m,1,0}     cg[3] = C^{l,m}_{l+1,m,1,0}
 * cg[4] = C^{l,m}_{l-1,m+1,1,-1}  cg[5] = C^{l,m}_{l+1,m+1,1,-1}
 * cg[6] = C^{l,m}_{l,m-1,1,1}     cg[7] = C^{l,m}_{l,m+1,1,-1}
 * cg[8] = C^{l,m}_{l,m,1,0}
 */
void orc_cg9(int l, int m, double *cg)
{
    double L = l, M = m;
    cg[0] = sqrt0((L + M) * (L + M - 1.0) / ((2.0 * L) * (2.0 * L - 1.0)));
    cg[1] = sqrt0((L - M + 1.0) * (L - M + 2.0) / ((2.0 * L + 2.0) * (2.0 * L + 3.0)));
    cg[2] = sqrt0((L + M) * (L - M) / (L * (2.0 * L - 1.0)));
    cg[3] = -sqrt0((L - M + 1.0) * (L + M + 1.0) / ((2.0 * L + 3.0) * (L + 1.0)));
    cg[4] = sqrt0((L - M) * (L - M - 1.0) / ((2.0 * L) * (2.0 * L - 1.0)));
    cg[5] = sqrt0((L + M + 1.0) * (L + M + 2.0) / ((2.0 * L + 3.0) * (2.0 * L + 2.0)));
    cg[6] = -sqrt0((L + M) * (L - M + 1.0) / (L * (2.0 * L + 2.0)));
    cg[7] = sqrt0((L + M + 1.0) * (L - M) / (L * (2.0 * L + 2.0)));
    cg[8] = M / sqrt(L * (L + 1.0));
}

/* Y_{l',m'} from the table, 0 outside 0 <= |m'| <= l' <= lmax (reading of eqs. Blm1/Blm2) */
static inline cplx ysafe(const cplx *y, int lmax, int l, int m)
{
    if (l < 0 || l > lmax || m < -l || m > l) return 0.0;
    return y[sidx(l, m)];
}

/* Index of (l, m), l = 1..L, |m| <= l, in a coefficient sequence: l^2 + l + m - 1 */
static inline int cidx(int l, int m) { return l * l + l + m - 1; }

/*
 * Cartesian Y^div_lm and Y^curl_lm for l = 1..L at one point from a scalar table
 * y (lmax >= L+1): eq. Blm1 (B_q), eq. Blm2 (D_q), eq. vsh2.
 * ydiv[3*cidx(l,m) + i], i = 0,1,2 (x, y, z components).
 */
static void vsh_from_table(int L, const cplx *y, cplx *ydiv, cplx *ycurl)
{
    const int lmax = L + 1;
    const double r2 = 1.0 / sqrt(2.0);
    for (int l = 1; l <= L; ++l) {
        double cl = c_l(l), dl = d_l(l);
        for (int m = -l; m <= l; ++m) {
            double cg[9];
            orc_cg9(l, m, cg);
            cplx Bp = cl * cg[0] * ysafe(y, lmax, l - 1, m - 1) + dl * cg[1] * ysafe(y, lmax, l + 1, m - 1);
            cplx B0 = cl * cg[2] * ysafe(y, lmax, l - 1, m) + dl * cg[3] * ysafe(y, lmax, l + 1, m);
            cplx Bm = cl * cg[4] * ysafe(y, lmax, l - 1, m + 1) + dl * cg[5] * ysafe(y, lmax, l + 1, m + 1);
            cplx Dp = I * cg[6] * ysafe(y, lmax, l, m - 1);
            cplx D0 = I * cg[8] * ysafe(y, lmax, l, m);
            cplx Dm = I * cg[7] * ysafe(y, lmax, l, m + 1);
            int k = cidx(l, m);
            ydiv[3 * k + 0] = -r2 * (Bp - Bm);
            ydiv[3 * k + 1] = -r2 * I * (Bp + Bm);
            ydiv[3 * k + 2] = B0;
            ycurl[3 * k + 0] = -r2 * (Dp - Dm);
            ycurl[3 * k + 1] = -r2 * I * (Dp + Dm);
            ycurl[3 * k + 2] = D0;
        }
    }
}

/* Y^div, Y^curl (Cartesian) for all l = 1..L at (theta, phi).  Outputs K*3 complex. */
void orc_vsh_point(int L, double theta, double phi, double *ydiv, double *ycurl)
{
    int lmax = L + 1;
    cplx *y = malloc(sizeof(cplx) * (lmax + 1) * (lmax + 1));
    double *cm = malloc(sizeof(double) * (lmax + 1)), *sm = malloc(sizeof(double) * (lmax + 1));
    double *col = malloc(sizeof(double) * (lmax + 2));
    for (int m = 0; m <= lmax; ++m) { cm[m] = cos(m * phi); sm[m] = sin(m * phi); }
    sh_table(lmax, cos(theta), sin(theta), cm, sm, y, col);
    vsh_from_table(L, y, (cplx *)ydiv, (cplx *)ycurl);
    free(y); free(cm); free(sm); free(col);
}

/*
 * O1 FwdVSHT at arbitrary points (Def. FwdVSHT, eq. fwdvsht2):
 *   a_lm = sum_k w_k Y^div_lm(x_k)^* T_k,   b_lm = sum_k w_k Y^curl_lm(x_k)^* T_k,
 * where ^* is the conjugate transpose.  T: npts x 3 complex (Cartesian).
 * a, b: K = L^2 + 2L complex each.
 */
void orc_fwd_literal(int L, int npts, const double *theta, const double *phi,
                     const double *w, const double *Tc, double *aout, double *bout)
{
    const int K = L * L + 2 * L, lmax = L + 1;
    const cplx *T = (const cplx *)Tc;
    cplx *a = (cplx *)aout, *b = (cplx *)bout;
    for (int k = 0; k < K; ++k) { a[k] = 0.0; b[k] = 0.0; }
    cplx *y = malloc(sizeof(cplx) * (lmax + 1) * (lmax + 1));
    cplx *yd = malloc(sizeof(cplx) * 3 * K), *yc = malloc(sizeof(cplx) * 3 * K);
    double *cm = malloc(sizeof(double) * (lmax + 1)), *sm = malloc(sizeof(double) * (lmax + 1));
    double *col = malloc(sizeof(double) * (lmax + 2));
    for (int p = 0; p < npts; ++p) {
        for (int m = 0; m <= lmax; ++m) { cm[m] = cos(m * phi[p]); sm[m] = sin(m * phi[p]); }
        sh_table(lmax, cos(theta[p]), sin(theta[p]), cm, sm, y, col);
        vsh_from_table(L, y, yd, yc);
        const cplx *t = T + 3 * p;
        for (int k = 0; k < K; ++k) {
            cplx sa = 0.0, sb = 0.0;
            for (int i = 0; i < 3; ++i) {
                sa += conj(yd[3 * k + i]) * t[i];
                sb += conj(yc[3 * k + i]) * t[i];
            }
            a[k] += w[p] * sa;
            b[k] += w[p] * sb;
        }
    }
    free(y); free(yd); free(yc); free(cm); free(sm); free(col);
}

/*
 * O1 AdjVSHT at arbitrary points (Def. AdjVSHT, eq. SLvec):
 *   S_L(a, b; x) = sum_{l=1}^{L} sum_{m=-l}^{l} (a_lm Y^div_lm(x) + b_lm Y^curl_lm(x)).
 * Output T: npts x 3 complex (Cartesian).
 */
void orc_adj_literal(int L, const double *ain, const double *bin, int npts,
                     const double *theta, const double *phi, double *Tout)
{
    const int K = L * L + 2 * L, lmax = L + 1;
    const cplx *a = (const cplx *)ain, *b = (const cplx *)bin;
    cplx *T = (cplx *)Tout;
    cplx *y = malloc(sizeof(cplx) * (lmax + 1) * (lmax + 1));
    cplx *yd = malloc(sizeof(cplx) * 3 * K), *yc = malloc(sizeof(cplx) * 3 * K);
    double *cm = malloc(sizeof(double) * (lmax + 1)), *sm = malloc(sizeof(double) * (lmax + 1));
    double *col = malloc(sizeof(double) * (lmax + 2));
    for (int p = 0; p < npts; ++p) {
        for (int m = 0; m <= lmax; ++m) { cm[m] = cos(m * phi[p]); sm[m] = sin(m * phi[p]); }
        sh_table(lmax, cos(theta[p]), sin(theta[p]), cm, sm, y, col);
        vsh_from_table(L, y, yd, yc);
        cplx s[3] = { 0.0, 0.0, 0.0 };
        for (int k = 0; k < K; ++k)
            for (int i = 0; i < 3; ++i) s[i] += a[k] * yd[3 * k + i] + b[k] * yc[3 * k + i];
        for (int i = 0; i < 3; ++i) T[3 * p + i] = s[i];
    }
    free(y); free(yd); free(yc); free(cm); free(sm); free(col);
}

/* ------------------------------------------------------------------------- */
/* Grid helpers                                                              */
/* ------------------------------------------------------------------------- */

/* exp(i 2 pi q / n) for integer q, reduced exactly modulo n before the angle is formed */
static inline cplx unit_root(long long q, int n)
{
    long long r = q % n;
    if (r < 0) r += n;
    double ang = 2.0 * M_PI * (double)r / (double)n;
    return cos(ang) + I * sin(ang);
}

/*
 * O1 on a latitude-longitude grid, one coefficient at a time (for sampled checks
 * at any size).  Grid: nlat nodes x[j] = cos(theta_j), latitude weights W[j],
 * nphi equispaced longitudes phi_k = 2 pi k / nphi; point weight W_j * 2 pi / nphi.
 * Tth, Tph: nlat x nphi complex (spherical components of T).  For each requested
 * (l, m) the literal sum over all nlat*nphi points is evaluated; the six scalar
 * Legendre columns it needs are computed once per latitude.
 */
void orc_fwd_literal_grid_coefs(int L, int nlat, int nphi, const double *x, const double *W,
                                const double *Tthc, const double *Tphc, int ncoef,
                                const int *ells, const int *ms, double *aout, double *bout)
{
    const cplx *Tth = (const cplx *)Tthc, *Tph = (const cplx *)Tphc;
    cplx *a = (cplx *)aout, *b = (cplx *)bout;
    const double r2 = 1.0 / sqrt(2.0), dphi = 2.0 * M_PI / nphi;
    #pragma omp parallel for schedule(dynamic) if (ncoef > 1)
    for (int c = 0; c < ncoef; ++c) {
        double *colp = malloc(sizeof(double) * (L + 4));
        int l = ells[c], m = ms[c];
        double cl = c_l(l), dl = d_l(l), cg[9];
        orc_cg9(l, m, cg);
        cplx sa = 0.0, sb = 0.0;
        for (int j = 0; j < nlat; ++j) {
            double ct = x[j], st = sqrt((1.0 - x[j]) * (1.0 + x[j]));
            /* lam[dl][dm] = lambda_{l+dl}^{m+dm}(theta_j) for dl, dm in {-1,0,1} (signed orders) */
            double lam[3][3];
            for (int dm = -1; dm <= 1; ++dm) {
                int mm = m + dm, am = abs(mm);
                for (int d = -1; d <= 1; ++d) lam[d + 1][dm + 1] = 0.0;
                if (am > l + 1) continue;
                orc_lambda_col(am, l + 1, ct, st, colp);
                double sg = (mm < 0 && (am & 1)) ? -1.0 : 1.0;
                for (int d = -1; d <= 1; ++d) {
                    int ll = l + d;
                    if (ll >= am) lam[d + 1][dm + 1] = sg * colp[ll - am];
                }
            }
            double wj = W[j] * dphi;
            for (int k = 0; k < nphi; ++k) {
                /* Y_{l',m'}(x_jk) = lambda_{l'}^{m'} e^{i m' phi_k} */
                cplx e[3];
                for (int dm = -1; dm <= 1; ++dm) e[dm + 1] = unit_root((long long)(m + dm) * k, nphi);
                cplx Bp = cl * cg[0] * lam[0][0] * e[0] + dl * cg[1] * lam[2][0] * e[0];
                cplx B0 = cl * cg[2] * lam[0][1] * e[1] + dl * cg[3] * lam[2][1] * e[1];
                cplx Bm = cl * cg[4] * lam[0][2] * e[2] + dl * cg[5] * lam[2][2] * e[2];
                cplx Dp = I * cg[6] * lam[1][0] * e[0];
                cplx D0 = I * cg[8] * lam[1][1] * e[1];
                cplx Dm = I * cg[7] * lam[1][2] * e[2];
                cplx yd[3] = { -r2 * (Bp - Bm), -r2 * I * (Bp + Bm), B0 };
                cplx yc[3] = { -r2 * (Dp - Dm), -r2 * I * (Dp + Dm), D0 };
                /* T_k in Cartesian: T_theta e_theta + T_phi e_phi */
                cplx e1 = unit_root(k, nphi);
                double cp = creal(e1), sp = cimag(e1);
                cplx tt = Tth[(size_t)j * nphi + k], tp = Tph[(size_t)j * nphi + k];
                cplx t[3] = { tt * ct * cp - tp * sp, tt * ct * sp + tp * cp, -tt * st };
                for (int i = 0; i < 3; ++i) {
                    sa += wj * conj(yd[i]) * t[i];
                    sb += wj * conj(yc[i]) * t[i];
                }
            }
        }
        a[c] = sa; b[c] = sb;
        free(colp);
    }
}

/*
 * O1 AdjVSHT at selected grid points (j, k): the literal partial sum of eq. SLvec
 * evaluated in Cartesian form and projected on e_theta, e_phi.  Also returns the
 * normal component x . S_L (should vanish: tangency, Sec. 3).
 */
void orc_adj_literal_grid_points(int L, int nlat, int nphi, const double *x,
                                 const double *ain, const double *bin, int npts,
                                 const int *js, const int *ks, double *Tthout,
                                 double *Tphout, double *normal_out)
{
    const int K = L * L + 2 * L, lmax = L + 1;
    const cplx *a = (const cplx *)ain, *b = (const cplx *)bin;
    cplx *Tth = (cplx *)Tthout, *Tph = (cplx *)Tphout, *nrm = (cplx *)normal_out;
    #pragma omp parallel for schedule(dynamic) if (npts > 1)
    for (int p = 0; p < npts; ++p) {
        cplx *y = malloc(sizeof(cplx) * (lmax + 1) * (lmax + 1));
        cplx *yd = malloc(sizeof(cplx) * 3 * K), *yc = malloc(sizeof(cplx) * 3 * K);
        double *cm = malloc(sizeof(double) * (lmax + 1)), *sm = malloc(sizeof(double) * (lmax + 1));
        double *col = malloc(sizeof(double) * (lmax + 2));
        int j = js[p], k = ks[p];
        double ct = x[j], st = sqrt((1.0 - x[j]) * (1.0 + x[j]));
        for (int m = 0; m <= lmax; ++m) {
            cplx e = unit_root((long long)m * k, nphi);
            cm[m] = creal(e); sm[m] = cimag(e);
        }
        sh_table(lmax, ct, st, cm, sm, y, col);
        vsh_from_table(L, y, yd, yc);
        cplx s[3] = { 0.0, 0.0, 0.0 };
        for (int q = 0; q < K; ++q)
            for (int i = 0; i < 3; ++i) s[i] += a[q] * yd[3 * q + i] + b[q] * yc[3 * q + i];
        cplx e1 = unit_root(k, nphi);
        double cp = creal(e1), sp = cimag(e1);
        Tth[p] = s[0] * ct * cp + s[1] * ct * sp - s[2] * st;
        Tph[p] = -s[0] * sp + s[1] * cp;
        if (nrm) nrm[p] = s[0] * st * cp + s[1] * st * sp + s[2] * ct;
        free(y); free(yd); free(yc); free(cm); free(sm); free(col);
    }
}

/* ------------------------------------------------------------------------- */
/* O3: separable form on the grid (same sums, regrouped)                      */
/*   Y^div_lm  = s_l e^{i m phi} ( dtheta(lambda) e_theta + i m lambda / sin(theta) e_phi )   */
/*   Y^curl_lm = s_l e^{i m phi} ( -i m lambda / sin(theta) e_theta + dtheta(lambda) e_phi )  */
/*   s_l = 1/sqrt(l(l+1)),  sin(theta) dtheta(lambda_l) = l cos(theta) lambda_l -            */
/*                                               (2l+1) eps_l^m lambda_{l-1}                */
/* ------------------------------------------------------------------------- */

/* lam[l], dlam[l] = lambda_l^m, dtheta lambda_l^m for l = |m|..L (signed order m) */
static void lam_dlam(int L, int m, double ct, double st, double *lam, double *dlam)
{
    int am = abs(m);
    double sg = (m < 0 && (am & 1)) ? -1.0 : 1.0;
    orc_lambda_col(am, L, ct, st, lam + am);
    for (int l = am; l <= L; ++l) lam[l] *= sg;
    for (int l = am; l <= L; ++l) {
        double prev = (l > am) ? lam[l - 1] : 0.0;
        dlam[l] = (l * ct * lam[l] - (2.0 * l + 1.0) * eps_lm(l, am) * prev) / st;
    }
}

/*
 * Full FwdVSHT on the grid, O(L^3): exact direct DFT per ring (no FFT), then the
 * Legendre sums.  Tth, Tph: nlat x nphi complex.  a, b: K complex.
 * Requires nphi >= 2L+1 (all |m| <= L resolved) and nodes strictly inside (0, pi).
 */
void orc_fwd_sep_orders(int L, int nlat, int nphi, const double *x, const double *W,
                        const double *Tthc, const double *Tphc, double *aout, double *bout,
                        int mstart, int mstep)
{
    const cplx *Tth = (const cplx *)Tthc, *Tph = (const cplx *)Tphc;
    cplx *a = (cplx *)aout, *b = (cplx *)bout;
    const double dphi = 2.0 * M_PI / nphi;
    #pragma omp parallel for schedule(dynamic)
    for (int mi = mstart; mi < 2 * L + 1; mi += mstep) {
        int m = mi - L;
        double *lam = malloc(sizeof(double) * (L + 2)), *dlam = malloc(sizeof(double) * (L + 2));
        cplx *Fth = malloc(sizeof(cplx) * nlat), *Fph = malloc(sizeof(cplx) * nlat);
        for (int j = 0; j < nlat; ++j) {
            cplx s1 = 0.0, s2 = 0.0;
            for (int k = 0; k < nphi; ++k) {
                cplx e = unit_root(-(long long)m * k, nphi);
                s1 += Tth[(size_t)j * nphi + k] * e;
                s2 += Tph[(size_t)j * nphi + k] * e;
            }
            Fth[j] = s1; Fph[j] = s2;
        }
        int l0 = abs(m) > 1 ? abs(m) : 1;
        cplx *sa = calloc(L + 1, sizeof(cplx)), *sb = calloc(L + 1, sizeof(cplx));
        for (int j = 0; j < nlat; ++j) {
            double ct = x[j], st = sqrt((1.0 - x[j]) * (1.0 + x[j]));
            lam_dlam(L, m, ct, st, lam, dlam);
            double wj = W[j] * dphi;
            for (int l = l0; l <= L; ++l) {
                double mls = m * lam[l] / st;
                sa[l] += wj * (dlam[l] * Fth[j] - I * mls * Fph[j]);
                sb[l] += wj * (I * mls * Fth[j] + dlam[l] * Fph[j]);
            }
        }
        for (int l = l0; l <= L; ++l) {
            double s = 1.0 / sqrt(l * (l + 1.0));
            a[cidx(l, m)] = s * sa[l];
            b[cidx(l, m)] = s * sb[l];
        }
        free(sa); free(sb); free(lam); free(dlam); free(Fth); free(Fph);
    }
}

void orc_fwd_sep(int L, int nlat, int nphi, const double *x, const double *W,
                 const double *Tthc, const double *Tphc, double *aout, double *bout)
{
    orc_fwd_sep_orders(L, nlat, nphi, x, W, Tthc, Tphc, aout, bout, 0, 1);
}

/* AdjVSHT on the grid restricted to the orders m = mstart - L, mstart - L + mstep, ...
 * (all orders for mstart = 0, mstep = 1), O(L^3): Legendre sums per (ring, m), then
 * an exact direct inverse DFT per ring over those orders.  Output Tth, Tph: nlat x
 * nphi complex. */
void orc_adj_sep_orders(int L, int nlat, int nphi, const double *x, const double *ain,
                        const double *bin, double *Tthout, double *Tphout, int mstart, int mstep)
{
    const cplx *a = (const cplx *)ain, *b = (const cplx *)bin;
    cplx *Tth = (cplx *)Tthout, *Tph = (cplx *)Tphout;
    const int nm = 2 * L + 1;
    cplx *Gth = calloc((size_t)nlat * nm, sizeof(cplx)), *Gph = calloc((size_t)nlat * nm, sizeof(cplx));
    #pragma omp parallel for schedule(dynamic)
    for (int mi = mstart; mi < nm; mi += mstep) {
        int m = mi - L;
        double *lam = malloc(sizeof(double) * (L + 2)), *dlam = malloc(sizeof(double) * (L + 2));
        int l0 = abs(m) > 1 ? abs(m) : 1;
        for (int j = 0; j < nlat; ++j) {
            double ct = x[j], st = sqrt((1.0 - x[j]) * (1.0 + x[j]));
            lam_dlam(L, m, ct, st, lam, dlam);
            cplx g1 = 0.0, g2 = 0.0;
            for (int l = l0; l <= L; ++l) {
                double s = 1.0 / sqrt(l * (l + 1.0));
                double mls = m * lam[l] / st;
                cplx al = a[cidx(l, m)], bl = b[cidx(l, m)];
                g1 += s * (al * dlam[l] - I * mls * bl);
                g2 += s * (I * mls * al + bl * dlam[l]);
            }
            Gth[(size_t)j * nm + mi] = g1;
            Gph[(size_t)j * nm + mi] = g2;
        }
        free(lam); free(dlam);
    }
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < nlat; ++j) {
        for (int k = 0; k < nphi; ++k) {
            cplx s1 = 0.0, s2 = 0.0;
            for (int mi = mstart; mi < nm; mi += mstep) {
                cplx e = unit_root((long long)(mi - L) * k, nphi);
                s1 += Gth[(size_t)j * nm + mi] * e;
                s2 += Gph[(size_t)j * nm + mi] * e;
            }
            Tth[(size_t)j * nphi + k] = s1;
            Tph[(size_t)j * nphi + k] = s2;
        }
    }
    free(Gth); free(Gph);
}

void orc_adj_sep(int L, int nlat, int nphi, const double *x, const double *ain,
                 const double *bin, double *Tthout, double *Tphout)
{
    orc_adj_sep_orders(L, nlat, nphi, x, ain, bin, Tthout, Tphout, 0, 1);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
