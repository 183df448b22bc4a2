/*
 * Oracle for the spin-weighted (polarisation) transforms: the extension that
 * Szydlarski et al., arXiv:1106.0159, name as future work (Section 6), built
 * on the scalar problem statement of Section 2.
 *
 * TEST INFRASTRUCTURE ONLY, like sht_oracle.c: a plain, slow CPU statement
 * of what the spin-2 transforms compute.  The library never loads it and
 * shares no code with it.  Arithmetic is long double throughout.
 *
 * Definitions (the paper has none; these are the standard ones, stated in
 * the normalisation of the scalar oracle, i.e. without a Condon-Shortley
 * factor):
 *
 *   sY_lm(theta, phi) = slambda_lm(theta) exp(i m phi), with
 *   slambda_lm(theta) = sqrt((l+m)! (l-m)! (2l+1) / (4 pi (l+s)! (l-s)!))
 *                       sum_r C(l-s, r) C(l+s, r+s-m) (-1)^(l-r-s)
 *                             sin(theta/2)^(2l-2r-s+m) cos(theta/2)^(2r+s-m)
 *   (Goldberg et al. 1967 without their (-1)^m; for s = 0 this is the scalar
 *   lambda_lm of eqs. assLegRec-pm1m).  Here it is evaluated by the
 *   three-term recurrence in l of the Wigner d-functions, l >= l0 = max(m, |s|):
 *     slambda_{l+1} = A_l [ (x + m s / (l (l+1))) slambda_l - B_l slambda_{l-1} ],
 *     A_l = sqrt((2l+3)/(2l+1)) (l+1)(2l+1) / sqrt(((l+1)^2 - m^2)((l+1)^2 - s^2)),
 *     B_l = sqrt((2l+1)/(2l-1)) sqrt((l^2 - m^2)(l^2 - s^2)) / (l (2l+1)),
 *   started from the single surviving term of the sum at l = l0 (formed in
 *   log space from lgamma and carried with an explicit binary exponent).
 *   tests/test_oracle_spin.py pins it to the explicit sum evaluated in
 *   50-digit arithmetic, to closed forms, to the spin sum rule and to the
 *   scalar oracle at s = 0.
 *
 *   Polarisation maps Q, U and coefficients E_lm, B_lm (m >= 0 stored; a
 *   real field has E_{l,-m} = (-1)^m conj(E_lm), the same for B):
 *     Q + iU = sum_{l >= 2} sum_{|m| <= l} 2a_lm 2Y_lm,   2a_lm = -(E_lm + i B_lm),
 *     Q - iU = sum 2a'_lm (-2)Y_lm,                      2a'_lm = -(E_lm - i B_lm),
 *   and the analysis with conj(Y) and the ring weights w_r, as in the scalar
 *   eq. map2almDef:
 *     2a_lm = sum w (Q + iU) conj(2Y_lm),  2a'_lm = sum w (Q - iU) conj((-2)Y_lm),
 *     E = -(2a + 2a')/2,  B = i (2a - 2a')/2.
 *   Separable form (the analogue of eqs. DeltaDef / almdef), with
 *   W_lm = (2lambda_lm + (-2)lambda_lm)/2, X_lm = (2lambda_lm - (-2)lambda_lm)/2:
 *     Delta^Q_m = -sum_l (E_lm W_lm + i B_lm X_lm),  Delta^U_m = -sum_l (B_lm W_lm - i E_lm X_lm),
 *     Q = Delta^Q_0 + 2 Re sum_{m>0} Delta^Q_m exp(i m phi)  (and U likewise),
 *     E_lm = -sum_r (W_lm Dq_m(r) + i X_lm Du_m(r)),  B_lm = sum_r (i X_lm Dq_m(r) - W_lm Du_m(r)),
 *   with Dq, Du the weighted ring sums of eq. almfftdef applied to Q and U.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef long double real;

static const real SPI_L = 3.14159265358979323846264338327950288L;

static real lfact(int n) { return lgammal((real)n + 1.0L); }

static real log_binom(int n, int k) { return lfact(n) - lfact(k) - lfact(n - k); }

static long s_alm_index(int lmax, int l, int m) { return (long)m * (2L * lmax + 3L - m) / 2L + (l - m); }

/*
 * slambda_lm(theta) for l = m..lmax into out[0 .. lmax-m] (zero for l < max(m, |s|) and for
 * values below the long double range).  0 <= theta <= pi.
 */
static void spin_lambda_column(real theta, int lmax, int m, int s, real *out)
{
    const int n = lmax - m + 1;
    if (n <= 0) return;
    for (int i = 0; i < n; ++i) out[i] = 0.0L;
    const int as = s < 0 ? -s : s;
    const int l0 = m > as ? m : as;
    if (l0 > lmax) return;
    /* the one term of the sum that survives at l = l0 */
    const int r0 = (m - s) > 0 ? (m - s) : 0;
    const int ksin = 2 * l0 - 2 * r0 - s + m, kcos = 2 * r0 + s - m;
    const real sh = sinl(0.5L * theta), chh = cosl(0.5L * theta);
    if ((ksin > 0 && sh == 0.0L) || (kcos > 0 && chh == 0.0L)) return; /* the whole column vanishes */
    real lg = 0.5L * (lfact(l0 + m) + lfact(l0 - m) + logl(2.0L * l0 + 1.0L) - logl(4.0L * SPI_L) - lfact(l0 + s) -
                      lfact(l0 - s)) +
              log_binom(l0 - s, r0) + log_binom(l0 + s, r0 + s - m);
    if (ksin > 0) lg += (real)ksin * logl(sh);
    if (kcos > 0) lg += (real)kcos * logl(chh);
    const real sign = ((l0 - r0 - s) & 1) ? -1.0L : 1.0L;
    const real l2 = lg / logl(2.0L);
    long e = (long)floorl(l2);
    real p1 = sign * exp2l(l2 - (real)e), p2 = 0.0L; /* slambda_l, slambda_{l-1}, scaled by 2^-e */
    out[l0 - m] = ldexpl(p1, (int)(e < -40000 ? -40000 : e));
    const real x = cosl(theta), M = (real)m, S = (real)s;
    for (int l = l0; l < lmax; ++l) {
        const real L = (real)l, L1 = L + 1.0L;
        const real A = sqrtl((2.0L * L + 3.0L) / (2.0L * L + 1.0L)) * L1 * (2.0L * L + 1.0L) /
                       sqrtl((L1 * L1 - M * M) * (L1 * L1 - S * S));
        real B = 0.0L, g = 0.0L;
        if (l > 0) {
            B = sqrtl((2.0L * L + 1.0L) / (2.0L * L - 1.0L)) * sqrtl((L * L - M * M) * (L * L - S * S)) /
                (L * (2.0L * L + 1.0L));
            g = M * S / (L * L1);
        }
        const real p = A * ((x + g) * p1 - B * p2);
        p2 = p1;
        p1 = p;
        if (fabsl(p1) > 0x1p+256L || fabsl(p2) > 0x1p+256L) {
            p1 = ldexpl(p1, -256);
            p2 = ldexpl(p2, -256);
            e += 256;
        }
        out[l + 1 - m] = ldexpl(p1, (int)(e < -40000 ? -40000 : e));
    }
}

static int64_t s_ring_offset(const int64_t *nphi, int r)
{
    int64_t o = 0;
    for (int i = 0; i < r; ++i) o += nphi[i];
    return o;
}

/* ------------------------------------------------------------------ exported */

/* slambda_lm(theta), l = m..lmax, rounded to double (s any integer, m >= 0). */
void oracle_spin_lambda(double theta, int lmax, int m, int s, double *out)
{
    const int n = lmax - m + 1;
    if (n <= 0) return;
    real *col = (real *)malloc(sizeof(real) * (size_t)n);
    spin_lambda_column((real)theta, lmax, m, s, col);
    for (int i = 0; i < n; ++i) out[i] = (double)col[i];
    free(col);
}

/*
 * Separable spin-2 synthesis, Legendre part: Delta^Q_m(r), Delta^U_m(r) for the selected rings,
 * dq/du[(k (mmax+1) + m) 2 + {0,1}] for ring rings[k]; E and B are complex, m-major triangle.
 */
void oracle_spin_delta_synth(int nrings, const double *theta, int lmax, int mmax, const double *E, const double *B,
                             int nsel, const int *rings, double *dq, double *du)
{
    (void)nrings;
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nsel; ++k) {
        real *cp = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        real *cm = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        const real th = (real)theta[rings[k]];
        for (int m = 0; m <= mmax; ++m) {
            spin_lambda_column(th, lmax, m, 2, cp);
            spin_lambda_column(th, lmax, m, -2, cm);
            real qr = 0, qi = 0, ur = 0, ui = 0;
            for (int l = (m > 2 ? m : 2); l <= lmax; ++l) {
                const long i = s_alm_index(lmax, l, m);
                const real W = 0.5L * (cp[l - m] + cm[l - m]), X = 0.5L * (cp[l - m] - cm[l - m]);
                const real er = (real)E[2 * i], ei = m > 0 ? (real)E[2 * i + 1] : 0.0L;
                const real br = (real)B[2 * i], bi = m > 0 ? (real)B[2 * i + 1] : 0.0L;
                /* -(E W + i B X) and -(B W - i E X) */
                qr -= er * W - bi * X;
                qi -= ei * W + br * X;
                ur -= br * W + ei * X;
                ui -= bi * W - er * X;
            }
            const long o = ((long)k * (mmax + 1) + m) * 2;
            dq[o] = (double)qr;
            dq[o + 1] = (double)qi;
            du[o] = (double)ur;
            du[o + 1] = (double)ui;
        }
        free(cp);
        free(cm);
    }
}

/*
 * Separable spin-2 analysis, Legendre part: E_lm, B_lm for l = m..lmax (zero below l = 2) of the
 * selected m from the weighted ring sums dq, du ([k][nrings] complex, k over ms).  Output for
 * ms[k] is the (lmax - m + 1) complex values of E (then B), concatenated in the order of ms.
 */
void oracle_spin_legendre_anal(int nrings, const double *theta, int lmax, int nm, const int *ms, const double *dq,
                               const double *du, double *E, double *B)
{
    long *start = (long *)malloc(sizeof(long) * (size_t)(nm + 1));
    start[0] = 0;
    for (int k = 0; k < nm; ++k) start[k + 1] = start[k] + (lmax - ms[k] + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nm; ++k) {
        const int m = ms[k];
        const int n = lmax - m + 1;
        real *cp = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        real *cm = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        real *acc = (real *)calloc((size_t)n * 4, sizeof(real));
        for (int r = 0; r < nrings; ++r) {
            spin_lambda_column((real)theta[r], lmax, m, 2, cp);
            spin_lambda_column((real)theta[r], lmax, m, -2, cm);
            const long o = ((long)k * nrings + r) * 2;
            const real qr = (real)dq[o], qi = (real)dq[o + 1], ur = (real)du[o], ui = (real)du[o + 1];
            for (int j = 0; j < n; ++j) {
                const real W = 0.5L * (cp[j] + cm[j]), X = 0.5L * (cp[j] - cm[j]);
                /* E = -(W Dq + i X Du),  B = i X Dq - W Du */
                acc[4 * j + 0] -= W * qr - X * ui;
                acc[4 * j + 1] -= W * qi + X * ur;
                acc[4 * j + 2] += -X * qi - W * ur;
                acc[4 * j + 3] += X * qr - W * ui;
            }
        }
        for (int j = 0; j < n; ++j) {
            const long o = (start[k] + j) * 2;
            E[o] = (double)acc[4 * j + 0];
            E[o + 1] = m == 0 ? 0.0 : (double)acc[4 * j + 1];
            B[o] = (double)acc[4 * j + 2];
            B[o + 1] = m == 0 ? 0.0 : (double)acc[4 * j + 3];
        }
        free(cp);
        free(cm);
        free(acc);
    }
    free(start);
}

/*
 * Pixel-by-pixel spin-2 synthesis from the definition: Q + iU = sum_{l, |m| <= l} 2a_lm 2Y_lm with
 * the negative-m coefficients and functions from the real-field symmetry
 * (E_{l,-m} = (-1)^m conj(E_lm), sY_{l,-m} = (-1)^(m+s) (-s)lambda_lm exp(-i m phi)), slambda
 * recomputed for every pixel.  q, u: [npix] in ring order.
 */
void oracle_spin_alm2map_exact(int nrings, const int64_t *nphi, const double *theta, const double *phi0, int lmax,
                               int mmax, const double *E, const double *B, double *q, double *u)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int r = 0; r < nrings; ++r) {
        real *cp = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        real *cm = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        const int64_t o = s_ring_offset(nphi, r);
        for (int64_t j = 0; j < nphi[r]; ++j) {
            const real phi = (real)phi0[r] + 2.0L * SPI_L * (real)j / (real)nphi[r];
            real pr = 0, pi = 0;
            for (int m = 0; m <= mmax; ++m) {
                spin_lambda_column((real)theta[r], lmax, m, 2, cp);
                spin_lambda_column((real)theta[r], lmax, m, -2, cm);
                const real c = cosl((real)m * phi), sn = sinl((real)m * phi);
                const real sg = (m & 1) ? -1.0L : 1.0L;
                for (int l = (m > 2 ? m : 2); l <= lmax; ++l) {
                    const long i = s_alm_index(lmax, l, m);
                    const real er = (real)E[2 * i], ei = m > 0 ? (real)E[2 * i + 1] : 0.0L;
                    const real br = (real)B[2 * i], bi = m > 0 ? (real)B[2 * i + 1] : 0.0L;
                    /* +m: -(E + iB) 2lambda_lm exp(i m phi) */
                    const real ar = -(er - bi), ai = -(ei + br);
                    pr += cp[l - m] * (ar * c - ai * sn);
                    pi += cp[l - m] * (ar * sn + ai * c);
                    if (m > 0) {
                        /* -m: 2a_{l,-m} = -((-1)^m conj(E) + i (-1)^m conj(B)),
                           2Y_{l,-m} = (-1)^m (-2)lambda_lm exp(-i m phi) */
                        const real br2 = -sg * (er + bi), bi2 = -sg * (-ei + br);
                        const real f = sg * cm[l - m];
                        pr += f * (br2 * c + bi2 * sn);
                        pi += f * (bi2 * c - br2 * sn);
                    }
                }
            }
            q[o + j] = (double)pr;
            u[o + j] = (double)pi;
        }
        free(cp);
        free(cm);
    }
}

/*
 * Pixel-by-pixel spin-2 analysis from the definition: 2a_lm = sum w (Q + iU) conj(2Y_lm),
 * 2a'_lm = sum w (Q - iU) conj((-2)Y_lm), E = -(2a + 2a')/2, B = i (2a - 2a')/2, for m >= 0.
 */
void oracle_spin_map2alm_exact(int nrings, const int64_t *nphi, const double *theta, const double *phi0,
                               const double *w, int lmax, int mmax, const double *q, const double *u, double *E,
                               double *B)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int m = 0; m <= mmax; ++m) {
        real *cp = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        real *cm = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        const int n = lmax - m + 1;
        real *acc = (real *)calloc((size_t)n * 4, sizeof(real)); /* 2a re, im, 2a' re, im */
        for (int r = 0; r < nrings; ++r) {
            spin_lambda_column((real)theta[r], lmax, m, 2, cp);
            spin_lambda_column((real)theta[r], lmax, m, -2, cm);
            const int64_t o = s_ring_offset(nphi, r);
            for (int64_t j = 0; j < nphi[r]; ++j) {
                const real phi = (real)phi0[r] + 2.0L * SPI_L * (real)j / (real)nphi[r];
                const real c = cosl((real)m * phi), sn = sinl((real)m * phi);
                const real Q = (real)q[o + j], U = (real)u[o + j], wr = (real)w[r];
                /* (Q + iU) exp(-i m phi) and (Q - iU) exp(-i m phi) */
                const real ppr = Q * c + U * sn, ppi = U * c - Q * sn;
                const real pmr = Q * c - U * sn, pmi = -U * c - Q * sn;
                for (int jj = 0; jj < n; ++jj) {
                    acc[4 * jj + 0] += wr * cp[jj] * ppr;
                    acc[4 * jj + 1] += wr * cp[jj] * ppi;
                    acc[4 * jj + 2] += wr * cm[jj] * pmr;
                    acc[4 * jj + 3] += wr * cm[jj] * pmi;
                }
            }
        }
        for (int jj = 0; jj < n; ++jj) {
            const long i = s_alm_index(lmax, m + jj, m);
            const real ar = acc[4 * jj], ai = acc[4 * jj + 1], br = acc[4 * jj + 2], bi = acc[4 * jj + 3];
            E[2 * i] = (double)(-0.5L * (ar + br));
            E[2 * i + 1] = m == 0 ? 0.0 : (double)(-0.5L * (ai + bi));
            /* i (2a - 2a') / 2 */
            B[2 * i] = (double)(-0.5L * (ai - bi));
            B[2 * i + 1] = m == 0 ? 0.0 : (double)(0.5L * (ar - br));
        }
        free(cp);
        free(cm);
        free(acc);
    }
}
