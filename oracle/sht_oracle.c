/*
 * Oracle for the spherical harmonic transforms of Szydlarski, Esterie, Falcou,
 * Grigori and Stompor, "Parallel Spherical Harmonic Transforms on
 * heterogeneous architectures (GPUs/multi-core CPUs)" (arXiv:1106.0159).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow CPU statement of what
 * the transforms compute, used to check the CUDA library.  Only the test
 * suite, the smoke check and the CPU-baseline leg of the benchmark may load
 * it; the library never does, and this file shares no code with it.
 *
 * Arithmetic is long double throughout (x87 80-bit on x86-64, IEEE binary128
 * on aarch64).  The loops follow the paper's definitions directly:
 *
 *   lambda_{l m}(x)   Section 2.1, eqs. (assLegRec), (betaDef), (pmm), (pm1m):
 *                     the start value mu_m (1-x^2)^{m/2} is formed in log
 *                     space from lgamma and carried with an explicit binary
 *                     exponent, then the l-recurrence runs with that exponent
 *                     tracked separately (the rescaling of Section 2.1).
 *   synthesis         Section 2.1 eq. (alm2mapDef), with the real-field
 *                     symmetry a_{l,-m} = (-1)^m conj(a_{l m}),
 *                     Y_{l,-m} = (-1)^m conj(Y_{l m}) of Section 2.1.
 *   analysis          Section 2.1 eq. (map2almDef) with conj(Y) (the
 *                     continuous form, eq. (invers_continous), conjugates Y).
 *   separable forms   Section 2.2 eqs. (Delta2map), (DeltaDef), (almdef),
 *                     (almfftdef), with the phi sums done as direct sums over
 *                     the pixels of each ring (no FFT).
 *
 * Readings of garbled or silent passages (all listed in the design notes):
 *   - eq. (assLegRec): P_{l+2} = beta_{l+2} (x P_{l+1} - P_l / beta_{l+1});
 *     the printed "+" would give P_20 proportional to 3x^2+1.
 *   - eq. (pmm): the factor is (1-x^2)^{m/2} = sin^m(theta); with the
 *     printed exponent m, P_11 would not be sqrt(3/8pi) sin(theta).
 *   - eq. (pm1m): the coefficient is beta_{m+1,m} = sqrt(2m+3).
 *   - eqs. (Delta2map)/(almfftdef): the phase is exp(i m phi_j) with
 *     phi_j = phi0 + 2 pi j / nphi, the longitude of pixel j of the ring.
 *   - no Condon-Shortley factor: mu_m > 0, so lambda_{m m} > 0.
 *   - Im a_{l0} is ignored on input (real map).
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef long double real;

static const real PI_L = 3.14159265358979323846264338327950288L;

/* Section 2.1, eq. (betaDef). */
static real beta_lm(int l, int m)
{
    real L = (real)l, M = (real)m;
    return sqrtl((4.0L * L * L - 1.0L) / (L * L - M * M));
}

/* Section 2.1, eq. (pmm): ln mu_m with mu_m = sqrt((2m+1)!/(4 pi)) / (2^m m!). */
static real log_mu(int m)
{
    real M = (real)m;
    return 0.5L * (lgammal(2.0L * M + 2.0L) - logl(4.0L * PI_L)) - M * logl(2.0L) - lgammal(M + 1.0L);
}

/*
 * lambda_{l m}(cos theta) for l = m..lmax into out[0 .. lmax-m].
 * Values below the long double range come out as 0.
 */
static void lambda_column(real theta, int lmax, int m, real *out)
{
    int n = lmax - m + 1;
    if (n <= 0) return;
    real x = cosl(theta), s = sinl(theta);
    if (s < 0) s = -s;
    if (m > 0 && s == 0.0L) {
        for (int i = 0; i < n; ++i) out[i] = 0.0L;
        return;
    }
    /* start value P_mm = mu_m sin^m(theta) as v * 2^e with v in [1, 2) */
    real l2 = (log_mu(m) + (m > 0 ? (real)m * logl(s) : 0.0L)) / logl(2.0L);
    long e = (long)floorl(l2);
    real p_lm2 = 0.0L;                 /* P_{l-2}, scaled by 2^-e */
    real p_lm1 = exp2l(l2 - (real)e);  /* P_{l-1}, scaled by 2^-e */
    out[0] = ldexpl(p_lm1, (int)(e < -40000 ? -40000 : e));
    if (n == 1) return;
    /* eq. (pm1m): P_{m+1,m} = beta_{m+1,m} x P_{mm} */
    p_lm2 = p_lm1;
    p_lm1 = beta_lm(m + 1, m) * x * p_lm2;
    out[1] = ldexpl(p_lm1, (int)(e < -40000 ? -40000 : e));
    for (int l = m + 2; l <= lmax; ++l) {
        /* eq. (assLegRec) */
        real p = beta_lm(l, m) * (x * p_lm1 - p_lm2 / beta_lm(l - 1, m));
        p_lm2 = p_lm1;
        p_lm1 = p;
        /* keep the scaled pair inside the long double range */
        if (fabsl(p_lm1) > 0x1p+256L || fabsl(p_lm2) > 0x1p+256L) {
            p_lm1 = ldexpl(p_lm1, -256);
            p_lm2 = ldexpl(p_lm2, -256);
            e += 256;
        }
        out[l - m] = ldexpl(p_lm1, (int)(e < -40000 ? -40000 : e));
    }
}

static long alm_index(int lmax, int l, int m)
{
    return (long)m * (2L * lmax + 3L - m) / 2L + (l - m);
}

/* exp(i m phi) for m = 0..mmax: angle addition, re-seeded every 64 steps. */
static void phase_row(real phi, int mmax, real *c, real *s)
{
    real c1 = cosl(phi), s1 = sinl(phi);
    for (int m = 0; m <= mmax; ++m) {
        if ((m & 63) == 0) {
            c[m] = cosl((real)m * phi);
            s[m] = sinl((real)m * phi);
        } else {
            c[m] = c[m - 1] * c1 - s[m - 1] * s1;
            s[m] = s[m - 1] * c1 + c[m - 1] * s1;
        }
    }
}

static int64_t ring_offset(const int64_t *nphi, int r)
{
    int64_t o = 0;
    for (int i = 0; i < r; ++i) o += nphi[i];
    return o;
}

/* ------------------------------------------------------------------ */
/* exported entry points                                               */
/* ------------------------------------------------------------------ */

/* lambda_{l m}(cos theta), l = m..lmax, rounded to double. */
void oracle_lambda(double theta, int lmax, int m, double *out)
{
    int n = lmax - m + 1;
    if (n <= 0) return;
    real *col = (real *)malloc(sizeof(real) * (size_t)n);
    lambda_column((real)theta, lmax, m, col);
    for (int i = 0; i < n; ++i) out[i] = (double)col[i];
    free(col);
}

/* ln mu_m (for the tests). */
double oracle_log_mu(int m) { return (double)log_mu(m); }

/*
 * Section 2.2 eq. (DeltaDef), m >= 0: Delta^A_m(r) = sum_l a_lm lambda_lm(cos theta_r)
 * for the selected rings.  delta[(k*(mmax+1) + m)*2 + {0,1}] for ring rings[k].
 */
void oracle_delta_synth(int nrings, const double *theta, int lmax, int mmax,
                        const double *alm, int nsel, const int *rings, double *delta)
{
    (void)nrings;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nsel; ++k) {
        real *col = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        real th = (real)theta[rings[k]];
        for (int m = 0; m <= mmax; ++m) {
            lambda_column(th, lmax, m, col);
            real re = 0, im = 0;
            for (int l = m; l <= lmax; ++l) {
                long i = alm_index(lmax, l, m);
                re += (real)alm[2 * i] * col[l - m];
                if (m > 0) im += (real)alm[2 * i + 1] * col[l - m];
            }
            delta[((long)k * (mmax + 1) + m) * 2 + 0] = (double)re;
            delta[((long)k * (mmax + 1) + m) * 2 + 1] = (double)im;
        }
        free(col);
    }
}

/*
 * Section 2.2 eq. (Delta2map) with the m < 0 half of eq. (DeltaDef):
 * s(r, phi_j) = Delta_0 + 2 Re sum_{m>0} Delta_m exp(i m phi_j),
 * phi_j = phi0_r + 2 pi j / nphi_r.  Pixels of the selected rings are
 * written one ring after the other.
 */
void oracle_ring_synth(int nrings, const int64_t *nphi, const double *phi0, int mmax,
                       int nsel, const int *rings, const double *delta, double *out)
{
    (void)nrings;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nsel + 1));
    off[0] = 0;
    for (int k = 0; k < nsel; ++k) off[k + 1] = off[k] + nphi[rings[k]];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nsel; ++k) {
        int r = rings[k];
        int64_t n = nphi[r];
        real *c = (real *)malloc(sizeof(real) * (size_t)(mmax + 1));
        real *s = (real *)malloc(sizeof(real) * (size_t)(mmax + 1));
        const double *d = delta + (long)k * (mmax + 1) * 2;
        for (int64_t j = 0; j < n; ++j) {
            real phi = (real)phi0[r] + 2.0L * PI_L * (real)j / (real)n;
            phase_row(phi, mmax, c, s);
            real acc = (real)d[0];
            for (int m = 1; m <= mmax; ++m)
                acc += 2.0L * ((real)d[2 * m] * c[m] - (real)d[2 * m + 1] * s[m]);
            out[off[k] + j] = (double)acc;
        }
        free(c);
        free(s);
    }
    free(off);
}

/*
 * Section 2.1 eq. (alm2mapDef), evaluated pixel by pixel with lambda
 * recomputed for every pixel: s_n = sum_{l<=lmax} sum_{|m|<=min(l,mmax)} a_lm Y_lm(theta_n, phi_n),
 * with a_{l,-m} = (-1)^m conj(a_lm) and Y_{l,-m} = (-1)^m conj(Y_lm).
 */
void oracle_alm2map_exact(int nrings, const int64_t *nphi, const double *theta, const double *phi0,
                          int lmax, int mmax, const double *alm, double *map)
{
    int64_t npix = ring_offset(nphi, nrings);
    int *ring_of = (int *)malloc(sizeof(int) * (size_t)npix);
    int64_t *pix_in = (int64_t *)malloc(sizeof(int64_t) * (size_t)npix);
    {
        int64_t p = 0;
        for (int r = 0; r < nrings; ++r)
            for (int64_t j = 0; j < nphi[r]; ++j, ++p) { ring_of[p] = r; pix_in[p] = j; }
    }
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npix; ++p) {
        int r = ring_of[p];
        real th = (real)theta[r];
        real phi = (real)phi0[r] + 2.0L * PI_L * (real)pix_in[p] / (real)nphi[r];
        real *col = (real *)malloc(sizeof(real) * (size_t)(lmax + 1));
        real sre = 0, sim = 0;
        for (int m = 0; m <= mmax; ++m) {
            lambda_column(th, lmax, m, col);
            real cm = cosl((real)m * phi), sm = sinl((real)m * phi);
            for (int l = m; l <= lmax; ++l) {
                long i = alm_index(lmax, l, m);
                real are = (real)alm[2 * i], aim = (m == 0) ? 0.0L : (real)alm[2 * i + 1];
                real lam = col[l - m];
                /* + a_lm Y_lm */
                real yre = lam * cm, yim = lam * sm;
                sre += are * yre - aim * yim;
                sim += are * yim + aim * yre;
                if (m > 0) {
                    /* + a_{l,-m} Y_{l,-m} = conj(a_lm) conj(Y_lm) (the two (-1)^m cancel) */
                    sre += are * yre - aim * yim;
                    sim -= are * yim + aim * yre;
                }
            }
        }
        (void)sim; /* vanishes by the real-field symmetry */
        map[p] = (double)sre;
        free(col);
    }
    free(ring_of);
    free(pix_in);
}

/*
 * Section 2.1 eq. (map2almDef) with conj(Y): a_lm = sum_n w_n s_n conj(Y_lm(theta_n, phi_n)),
 * pixel by pixel with lambda recomputed for every pixel.  One m per thread.
 */
void oracle_map2alm_exact(int nrings, const int64_t *nphi, const double *theta, const double *phi0,
                          const double *w, int lmax, int mmax, const double *map, double *alm)
{
    #pragma omp parallel for schedule(dynamic, 1)
    for (int m = 0; m <= mmax; ++m) {
        int n = lmax - m + 1;
        real *col = (real *)malloc(sizeof(real) * (size_t)n);
        real *are = (real *)calloc((size_t)n, sizeof(real));
        real *aim = (real *)calloc((size_t)n, sizeof(real));
        int64_t p = 0;
        for (int r = 0; r < nrings; ++r) {
            real th = (real)theta[r];
            for (int64_t j = 0; j < nphi[r]; ++j, ++p) {
                lambda_column(th, lmax, m, col);
                real phi = (real)phi0[r] + 2.0L * PI_L * (real)j / (real)nphi[r];
                real ws = (real)w[r] * (real)map[p];
                real cm = cosl((real)m * phi), sm = sinl((real)m * phi);
                for (int l = m; l <= lmax; ++l) {
                    are[l - m] += ws * col[l - m] * cm;
                    aim[l - m] -= ws * col[l - m] * sm;
                }
            }
        }
        for (int l = m; l <= lmax; ++l) {
            long i = alm_index(lmax, l, m);
            alm[2 * i] = (double)are[l - m];
            alm[2 * i + 1] = (m == 0) ? 0.0 : (double)aim[l - m];
        }
        free(col);
        free(are);
        free(aim);
    }
}

/*
 * Section 2.2 eq. (almfftdef), read with the pixel longitude phi_j:
 * Delta^S_m(r) = w_r sum_j s(r, j) exp(-i m phi_j), for the selected m and
 * every ring.  delta[(k*nrings + r)*2 + {0,1}] for m = ms[k].
 */
void oracle_delta_anal(int nrings, const int64_t *nphi, const double *phi0, const double *w,
                       const double *map, int nm, const int *ms, double *delta)
{
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nrings + 1));
    off[0] = 0;
    for (int r = 0; r < nrings; ++r) off[r + 1] = off[r] + nphi[r];
    #pragma omp parallel for collapse(2) schedule(dynamic, 4)
    for (int k = 0; k < nm; ++k) {
        for (int r = 0; r < nrings; ++r) {
            int m = ms[k];
            int64_t n = nphi[r];
            real re = 0, im = 0;
            /* exp(-i m phi_j) = exp(-i m phi0) exp(-i 2 pi m j / n), angle addition over j */
            real step = 2.0L * PI_L * (real)m / (real)n;
            real cs = cosl(step), ss = sinl(step);
            real c = 0, s = 0;
            for (int64_t j = 0; j < n; ++j) {
                if ((j & 63) == 0) {
                    real ang = (real)m * ((real)phi0[r] + 2.0L * PI_L * (real)j / (real)n);
                    c = cosl(ang);
                    s = sinl(ang);
                } else {
                    real c2 = c * cs - s * ss;
                    s = s * cs + c * ss;
                    c = c2;
                }
                real v = (real)map[off[r] + j];
                re += v * c;
                im -= v * s;
            }
            delta[((long)k * nrings + r) * 2 + 0] = (double)((real)w[r] * re);
            delta[((long)k * nrings + r) * 2 + 1] = (double)((real)w[r] * im);
        }
    }
    free(off);
}

/*
 * Section 2.2 eq. (almdef): a_lm = sum_r Delta^S_m(r) lambda_lm(cos theta_r) for
 * the selected m.  Output for ms[k] is the (lmax - m + 1) complex values
 * l = m..lmax, written one m after the other.  Rings are summed in 64 fixed
 * chunks, then the chunks in order, so the result does not depend on the
 * thread count.
 */
void oracle_legendre_anal(int nrings, const double *theta, int lmax, int nm, const int *ms,
                          const double *delta, double *out)
{
    enum { NCHUNK = 64 };
    long o = 0;
    for (int k = 0; k < nm; ++k) {
        int m = ms[k];
        int n = lmax - m + 1;
        real *part = (real *)calloc((size_t)NCHUNK * n * 2, sizeof(real));
        #pragma omp parallel for schedule(dynamic, 1)
        for (int c = 0; c < NCHUNK; ++c) {
            real *col = (real *)malloc(sizeof(real) * (size_t)n);
            int r0 = (int)((long)nrings * c / NCHUNK), r1 = (int)((long)nrings * (c + 1) / NCHUNK);
            for (int r = r0; r < r1; ++r) {
                lambda_column((real)theta[r], lmax, m, col);
                real dre = (real)delta[((long)k * nrings + r) * 2];
                real dim = (real)delta[((long)k * nrings + r) * 2 + 1];
                for (int i = 0; i < n; ++i) {
                    part[((long)c * n + i) * 2 + 0] += dre * col[i];
                    part[((long)c * n + i) * 2 + 1] += dim * col[i];
                }
            }
            free(col);
        }
        for (int i = 0; i < n; ++i) {
            real re = 0, im = 0;
            for (int c = 0; c < NCHUNK; ++c) {
                re += part[((long)c * n + i) * 2 + 0];
                im += part[((long)c * n + i) * 2 + 1];
            }
            out[(o + i) * 2 + 0] = (double)re;
            out[(o + i) * 2 + 1] = (m == 0) ? 0.0 : (double)im;
        }
        o += n;
        free(part);
    }
}

/* Host threads the oracle's parallel loops use from now on (timing only: every result is the
 * same for any count, since each output value is summed by one thread in a fixed order).
 * Returns the previous count. */
int oracle_set_threads(int n)
{
    const int old = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return old;
}
