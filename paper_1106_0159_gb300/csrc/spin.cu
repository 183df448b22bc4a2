// Spin-2 (polarisation) transforms: the extension the paper names as future work (Section 6),
// built like the scalar path: a per-m Legendre step fused with its sum over l (synthesis) or over
// ring slots (analysis), around the scalar ring DFTs run on the Q and U maps.
//
// Functions.  sY_lm = slambda_lm(theta) exp(i m phi) for s = +-2, with slambda the spin-weighted
// functions in the normalisation of the scalar lambda_lm (no Condon-Shortley factor).  For l >= l0
// = max(m, 2) they obey the three-term recurrence of the Wigner d-functions,
//     slambda_{l+1} = A_l (x + m s / (l (l+1))) slambda_l - A_l B_l slambda_{l-1},
//     A_l = sqrt((2l+3)/(2l+1)) (l+1)(2l+1) / sqrt(((l+1)^2 - m^2)((l+1)^2 - 4)),
//     B_l = sqrt((2l+1)/(2l-1)) sqrt((l^2 - m^2)(l^2 - 4)) / (l (2l+1)),
// which is the scalar recurrence of eq. (assLegRec) with one extra term.  A and B depend on s only
// through s^2, so both spins share the normalisation y = slambda / c_l
// (c_{l0} = c_{l0+1} = 1, c_l = A_{l-1} B_{l-1} c_{l-2}) and the step
//     y_l = alpha_l (x + g_{l-1}) y_{l-1} - y_{l-2},   alpha_l = A_{l-1} c_{l-1} / c_l,
// with g of opposite sign for +2 and -2.  With u = 1 - cos(theta) (exact near the poles) the
// factor is alpha (1 +- g) - alpha u: the plan tabulates alpha, alpha (1 + g) and alpha (1 - g),
// and each spin costs two FP64 instructions per step, four for the pair.  Start values at l = l0:
//     +2: S_m sin(theta)^|m-2| sin(theta/2)^p,  -2: sigma S_m sin(theta)^|m-2| cos(theta/2)^p,
// p = 2 min(m, 2), sigma = -1 for m = 1 and +1 otherwise, S_m tabulated; the sin(theta) power is
// formed by binary powering with its exponent carried apart (the scalar start value), and the
// pair is rescaled together by 2^-512 exactly as in the scalar kernels.
//
// Maps and coefficients.  Q + iU = sum 2a_lm 2Y_lm with 2a_lm = -(E_lm + i B_lm) (Q - iU with -2),
// so with p = y+ + y-, q = y+ - y- and e = -(c/2) E, b = -(c/2) B:
//     Delta^Q_m = sum_l (e p + i b q),  Delta^U_m = sum_l (b p - i e q),
//     E_lm = -(c/2) sum_r (p Dq + i q Du),  B_lm = (c/2) sum_r (i q Dq - p Du),
// (Dq, Du the weighted ring sums of the Q and U maps, eq. almfftdef).  Under theta -> pi - theta
// slambda_lm -> (-1)^(l+m) (-s)lambda_lm, so p has the parity (-1)^(l+m) and q the opposite one:
// one recurrence serves a ring and its mirror, with terms collected into a "plus" sum P (same
// sign on both rings) and a "minus" sum M (Delta_N = P + M, Delta_S = P - M).
//
// Layouts: alm [nmaps][2][nalm] (E then B), maps [nmaps][2][npix] (Q then U), Delta
// [nmaps][2][nrings][mmax+1]; the ring stage therefore runs on 2 nmaps scalar maps.
#include "sht_internal.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace sht {
namespace {

#include "recurrence.cuh"

constexpr int SP_T = 128;   // ring slots (threads) per CTA
constexpr int SP_CH = 64;   // l per staged chunk
constexpr int SP_SUB = 16;  // steps between rescale tests
constexpr int SP_RED = 8;   // l per warp reduce-scatter round (analysis)

struct SpinArgs {
    const double2 *alm;   // synthesis: [nmaps][2][nalm]
    double2 *delta;       // synthesis out / analysis in: [nmaps][2][nrings][mmax+1]
    double2 *partial;     // analysis: [nblk][nmaps][2][nalm]
    const int *slotN, *slotS;
    const double *u, *s;
    const double4 *tab;   // [nalm] (alpha, alpha (1 + g), alpha (1 - g), c)
    const double *start;  // [mmax+1] S_m
    int nslots, nblk, lmax, mmax, nrings, nmaps;
    int64_t nalm;
};

// Start values of the pair at l0 = max(m, 2) as (y+, y-) 2^(512 k), and the seed state that
// makes the first step produce them (y_{l0-1} = 0, y_{l0-2} = -y_{l0}).
__device__ __forceinline__ void spin_seed(const SpinArgs &A, int m, int slot, double &p1, double &p2, double &m1,
                                          double &m2, int &k)
{
    const double u = A.u[slot];
    double y0;
    sectoral_start(A.s[slot], A.start[m], m >= 2 ? m - 2 : 2 - m, y0, k);
    const double h2 = 0.5 * u, c2 = 1.0 - 0.5 * u;  // sin^2(theta/2), cos^2(theta/2)
    double yp = y0, ym = y0;
    if (m >= 2) {
        yp *= h2 * h2;
        ym *= c2 * c2;
    } else if (m == 1) {
        yp *= h2;
        ym *= -c2;
    }
    p1 = 0.0;
    p2 = -yp;
    m1 = 0.0;
    m2 = -ym;
}

// one step of both recurrences from the staged coefficients
__device__ __forceinline__ void spin_step(double4 t, double u, double &p1, double &p2, double &m1, double &m2)
{
    const double fp = fma(-t.x, u, t.y);  // alpha (x + g)
    const double fm = fma(-t.x, u, t.z);  // alpha (x - g)
    const double yp = fma(fp, p1, -p2);
    const double ym = fma(fm, m1, -m2);
    p2 = p1;
    p1 = yp;
    m2 = m1;
    m1 = ym;
}

__device__ __forceinline__ bool spin_rescale(double &p1, double &p2, double &m1, double &m2, int &k)
{
    if (k < 0 && max(max(dexp(p1), dexp(p2)), max(dexp(m1), dexp(m2))) > RESCALE_THR) {
        p1 *= 0x1p-512;
        p2 *= 0x1p-512;
        m1 *= 0x1p-512;
        m2 *= 0x1p-512;
        k += 1;
        return true;
    }
    return false;
}

template <int NM>
__global__ void __launch_bounds__(SP_T) spin_synth_kernel(SpinArgs A)
{
    __shared__ double4 s_t[SP_CH];
    __shared__ double2 s_e[NM][SP_CH], s_b[NM][SP_CH];
    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    const int slot = blk * SP_T + threadIdx.x;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int l0 = max(m, 2);
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int64_t mstride = A.mmax + 1;

    double u = 0.0, p1 = 0.0, p2 = 0.0, m1 = 0.0, m2 = 0.0;
    int k = 0;
    if (active && l0 <= L) {
        u = A.u[slot];
        spin_seed(A, m, slot, p1, p2, m1, m2, k);
    }
    // Q plus / minus, U plus / minus sums of each map
    double QPr[NM], QPi[NM], QMr[NM], QMi[NM], UPr[NM], UPi[NM], UMr[NM], UMi[NM];
#pragma unroll
    for (int g = 0; g < NM; ++g) QPr[g] = QPi[g] = QMr[g] = QMi[g] = UPr[g] = UPi[g] = UMr[g] = UMi[g] = 0.0;

    for (int c0 = l0; c0 <= L; c0 += SP_CH) {
        const int nl = min(SP_CH, L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nl; i += SP_T) {
            const int64_t ix = base + (c0 - m) + i;
            const double4 t = A.tab[ix];
            s_t[i] = t;
            const double f = -0.5 * t.w;
#pragma unroll
            for (int g = 0; g < NM; ++g) {
                const double2 e = A.alm[(int64_t)(2 * g) * A.nalm + ix];
                const double2 b = A.alm[(int64_t)(2 * g + 1) * A.nalm + ix];
                s_e[g][i] = make_double2(f * e.x, m == 0 ? 0.0 : f * e.y);
                s_b[g][i] = make_double2(f * b.x, m == 0 ? 0.0 : f * b.y);
            }
        }
        __syncthreads();
        for (int j0 = 0; j0 < nl; j0 += SP_SUB) {
            const int jn = min(j0 + SP_SUB, nl);
            const bool scaled = __any_sync(0xffffffffu, k < 0);
            const bool any_live = __any_sync(0xffffffffu, active && k == 0);
            for (int j = j0; j < jn; ++j) {
                spin_step(s_t[j], u, p1, p2, m1, m2);
                if (!any_live) continue;
                const bool use = !scaled || k == 0;
                const double pp = use ? p1 + m1 : 0.0, qq = use ? p1 - m1 : 0.0;
                const bool even = ((c0 + j - m) & 1) == 0;  // l + m even: p in the plus sum
#pragma unroll
                for (int g = 0; g < NM; ++g) {
                    const double2 e = s_e[g][j], b = s_b[g][j];
                    // Q: e p + i b q;  U: b p - i e q
                    const double qpr = e.x * pp, qpi = e.y * pp, qqr = -b.y * qq, qqi = b.x * qq;
                    const double upr = b.x * pp, upi = b.y * pp, uqr = e.y * qq, uqi = -e.x * qq;
                    if (even) {
                        QPr[g] += qpr; QPi[g] += qpi; QMr[g] += qqr; QMi[g] += qqi;
                        UPr[g] += upr; UPi[g] += upi; UMr[g] += uqr; UMi[g] += uqi;
                    } else {
                        QMr[g] += qpr; QMi[g] += qpi; QPr[g] += qqr; QPi[g] += qqi;
                        UMr[g] += upr; UMi[g] += upi; UPr[g] += uqr; UPi[g] += uqi;
                    }
                }
            }
            if (scaled) spin_rescale(p1, p2, m1, m2, k);
        }
    }
    if (active) {
        const int rn = A.slotN[slot], rs = A.slotS[slot];
#pragma unroll
        for (int g = 0; g < NM; ++g) {
            double2 *dq = A.delta + (int64_t)(2 * g) * A.nrings * mstride;
            double2 *du = A.delta + (int64_t)(2 * g + 1) * A.nrings * mstride;
            if (rn >= 0 && SHT_CHK(rn < A.nrings && m <= A.mmax)) {
                dq[(int64_t)rn * mstride + m] = make_double2(QPr[g] + QMr[g], QPi[g] + QMi[g]);
                du[(int64_t)rn * mstride + m] = make_double2(UPr[g] + UMr[g], UPi[g] + UMi[g]);
            }
            if (rs >= 0 && SHT_CHK(rs < A.nrings && m <= A.mmax)) {
                dq[(int64_t)rs * mstride + m] = make_double2(QPr[g] - QMr[g], QPi[g] - QMi[g]);
                du[(int64_t)rs * mstride + m] = make_double2(UPr[g] - UMr[g], UPi[g] - UMi[g]);
            }
        }
    }
}

// afterwards every lane holds the warp total of value (lane & 7)
__device__ __forceinline__ double reduce_scatter8(double v[SP_RED])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = SP_RED / 2; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double send = up ? v[i] : v[i + h];
            const double keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    double r = v[0];
    r += __shfl_xor_sync(0xffffffffu, r, 8);
    r += __shfl_xor_sync(0xffffffffu, r, 16);
    return r;
}

// Analysis: one CTA per (m, 128 slots), NM maps.  Per l, every thread forms the four products of
// its slot, the warps reduce-scatter them over their 32 slots, and the CTA adds its warps and
// writes the block's partial E_lm, B_lm (coefficient -+c/2 applied), [blk][map][E|B][nalm].
template <int NM>
__global__ void __launch_bounds__(SP_T) spin_anal_kernel(SpinArgs A)
{
    constexpr int NW = SP_T / 32;
    __shared__ double4 s_t[SP_CH];
    __shared__ double s_red[NW][SP_CH][4 * NM];
    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    const int slot = blk * SP_T + threadIdx.x;
    const bool active = slot < A.nslots;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = A.lmax;
    const int l0 = max(m, 2);
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int64_t mstride = A.mmax + 1;
    double2 *part = A.partial + (int64_t)blk * A.nmaps * 2 * A.nalm;

    // l < l0: no spin-2 function
    for (int l = m + threadIdx.x; l < min(l0, L + 1); l += SP_T)
        for (int g = 0; g < A.nmaps; ++g) {
            part[(int64_t)(2 * g) * A.nalm + base + (l - m)] = make_double2(0.0, 0.0);
            part[(int64_t)(2 * g + 1) * A.nalm + base + (l - m)] = make_double2(0.0, 0.0);
        }
    if (l0 > L) return;

    double u = 0.0, p1 = 0.0, p2 = 0.0, m1 = 0.0, m2 = 0.0;
    int k = 0;
    // per map: Sigma and D of the weighted ring sums of Q and U over the slot's two rings
    double SQr[NM], SQi[NM], DQr[NM], DQi[NM], SUr[NM], SUi[NM], DUr[NM], DUi[NM];
#pragma unroll
    for (int g = 0; g < NM; ++g) SQr[g] = SQi[g] = DQr[g] = DQi[g] = SUr[g] = SUi[g] = DUr[g] = DUi[g] = 0.0;
    if (active) {
        u = A.u[slot];
        spin_seed(A, m, slot, p1, p2, m1, m2, k);
        const int rn = A.slotN[slot], rs = A.slotS[slot];
#pragma unroll
        for (int g = 0; g < NM; ++g) {
            const double2 *dq = A.delta + (int64_t)(2 * g) * A.nrings * mstride;
            const double2 *du = A.delta + (int64_t)(2 * g + 1) * A.nrings * mstride;
            double2 qn = make_double2(0.0, 0.0), qs = qn, un = qn, us = qn;
            if (rn >= 0 && SHT_CHK(rn < A.nrings)) {
                qn = dq[(int64_t)rn * mstride + m];
                un = du[(int64_t)rn * mstride + m];
            }
            if (rs >= 0 && SHT_CHK(rs < A.nrings)) {
                qs = dq[(int64_t)rs * mstride + m];
                us = du[(int64_t)rs * mstride + m];
            }
            SQr[g] = qn.x + qs.x; SQi[g] = qn.y + qs.y; DQr[g] = qn.x - qs.x; DQi[g] = qn.y - qs.y;
            SUr[g] = un.x + us.x; SUi[g] = un.y + us.y; DUr[g] = un.x - us.x; DUi[g] = un.y - us.y;
        }
    }

    for (int c0 = l0; c0 <= L; c0 += SP_CH) {
        const int nl = min(SP_CH, L - c0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nl; i += SP_T) s_t[i] = A.tab[base + (c0 - m) + i];
        __syncthreads();
        for (int j0 = 0; j0 < nl; j0 += SP_SUB) {
            const bool scaled = __any_sync(0xffffffffu, k < 0);
#pragma unroll
            for (int h = 0; h < SP_SUB / SP_RED; ++h) {
                const int jb = j0 + h * SP_RED;
                // [map][E re, E im, B re, B im][l]
                double v[NM][4][SP_RED];
#pragma unroll
                for (int jj = 0; jj < SP_RED; ++jj) {
                    const int j = jb + jj;
                    const bool inside = j < nl;
                    double pp = 0.0, qq = 0.0;
                    if (inside) {
                        spin_step(s_t[j], u, p1, p2, m1, m2);
                        if (active && (!scaled || k == 0)) {
                            pp = p1 + m1;
                            qq = p1 - m1;
                        }
                    }
                    const bool even = ((c0 + j - m) & 1) == 0;
#pragma unroll
                    for (int g = 0; g < NM; ++g) {
                        // even l + m: p with Sigma of Q (Qw) and D of U (Uw), q with D of Q and Sigma
                        // of U; odd: the other way round
                        const double qwr = even ? SQr[g] : DQr[g], qwi = even ? SQi[g] : DQi[g];
                        const double uwr = even ? SUr[g] : DUr[g], uwi = even ? SUi[g] : DUi[g];
                        const double qxr = even ? DQr[g] : SQr[g], qxi = even ? DQi[g] : SQi[g];
                        const double uxr = even ? DUr[g] : SUr[g], uxi = even ? DUi[g] : SUi[g];
                        // sum (p Qw + i q Ux) and sum (i q Qx - p Uw); the factors -c/2, c/2 come later
                        v[g][0][jj] = pp * qwr - qq * uxi;
                        v[g][1][jj] = pp * qwi + qq * uxr;
                        v[g][2][jj] = -qq * qxi - pp * uwr;
                        v[g][3][jj] = qq * qxr - pp * uwi;
                    }
                }
#pragma unroll
                for (int g = 0; g < NM; ++g)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const double r = reduce_scatter8(v[g][c]);
                        if (lane < SP_RED && jb + lane < SP_CH) s_red[warp][jb + lane][4 * g + c] = r;
                    }
            }
            if (scaled) spin_rescale(p1, p2, m1, m2, k);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nl * NM; i += SP_T) {
            const int j = i % nl, g = i / nl;
            double t[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int w = 0; w < NW; ++w)
#pragma unroll
                for (int c = 0; c < 4; ++c) t[c] += s_red[w][j][4 * g + c];
            const double hc = 0.5 * s_t[j].w;
            const int64_t ix = base + (c0 - m) + j;
            if (!SHT_CHK(ix < A.nalm)) continue;
            part[(int64_t)(2 * g) * A.nalm + ix] = make_double2(-hc * t[0], -hc * t[1]);
            part[(int64_t)(2 * g + 1) * A.nalm + ix] = make_double2(hc * t[2], hc * t[3]);
        }
    }
}

// E, B = sum over slot blocks in fixed order; Im at m = 0 is zero
__global__ void spin_reduce_kernel(const double2 *__restrict__ partial, double2 *__restrict__ alm, int nblk,
                                   int64_t nalm, int64_t nvec, int lmax)
{
    const int64_t total = nalm * nvec;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t % nalm;
        double re = 0.0, im = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const double2 v = partial[(int64_t)b * total + t];
            re += v.x;
            im += v.y;
        }
        alm[t] = make_double2(re, i <= lmax ? 0.0 : im);
    }
}

SpinArgs spin_args(const Plan &p)
{
    SpinArgs A{};
    A.slotN = p.d_slotN;
    A.slotS = p.d_slotS;
    A.u = p.d_u;
    A.s = p.d_s;
    A.tab = p.d_spin_tab;
    A.start = p.d_spin_start;
    A.nslots = p.nslots;
    A.nblk = (p.nslots + SP_T - 1) / SP_T;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    A.nrings = p.nrings;
    A.nalm = p.nalm;
    return A;
}

}  // namespace

// Spin-2 recurrence tables, long double on the host (once per plan, on first use).
cudaError_t build_spin_tables(Plan &p)
{
    if (p.d_spin_tab) return cudaSuccess;
    const int L = p.lmax, M = p.mmax;
    std::vector<double4> tab((size_t)p.nalm, make_double4(0.0, 0.0, 0.0, 0.0));
    std::vector<double> start((size_t)M + 1, 0.0);
    const long double PI_L = 3.14159265358979323846264338327950288L;
    for (int m = 0; m <= M; ++m) {
        const int l0 = std::max(m, 2);
        const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
        // S_m: +2 lambda_{l0, m} = S_m sin(theta)^|m-2| sin(theta/2)^(2 min(m, 2))
        const long double lnS =
            m >= 2 ? 0.5L * (logl(2.0L * m + 1.0L) + lgammal(2.0L * m + 1.0L) - logl(4.0L * PI_L) -
                             lgammal((long double)m + 3.0L) - lgammal((long double)m - 1.0L)) -
                         (m - 2) * logl(2.0L)
                   : 0.0L;
        if (m >= 2)
            start[m] = (double)expl(lnS);
        else if (m == 1)
            start[m] = (double)(2.0L * sqrtl(30.0L / (96.0L * PI_L)));   // K_1 / 2, K_1 = 4 sqrt(30 / 96 pi)
        else
            start[m] = (double)(1.5L * sqrtl(20.0L / (96.0L * PI_L)));   // K_0 / 4, K_0 = 6 sqrt(20 / 96 pi)
        if (l0 > L) continue;
        const long double mm = (long double)m * m;
        long double c2 = 1.0L, c1 = 1.0L;  // c_{l-2}, c_{l-1}
        tab[base + (l0 - m)] = make_double4(0.0, 0.0, 0.0, 1.0);
        for (int l = l0 + 1; l <= L; ++l) {
            const long double Lp = (long double)(l - 1), L1 = (long double)l;  // step l-1 -> l
            const long double A = sqrtl((2.0L * Lp + 3.0L) / (2.0L * Lp + 1.0L)) * L1 * (2.0L * Lp + 1.0L) /
                                  sqrtl((L1 * L1 - mm) * (L1 * L1 - 4.0L));
            long double c;
            if (l == l0 + 1) {
                c = 1.0L;
            } else {
                const long double B = sqrtl((2.0L * Lp + 1.0L) / (2.0L * Lp - 1.0L)) *
                                      sqrtl((Lp * Lp - mm) * (Lp * Lp - 4.0L)) / (Lp * (2.0L * Lp + 1.0L));
                c = A * B * c2;
            }
            const long double al = A * c1 / c;
            const long double g = 2.0L * (long double)m / (Lp * L1);
            tab[base + (l - m)] = make_double4((double)al, (double)(al * (1.0L + g)), (double)(al * (1.0L - g)),
                                               (double)c);
            c2 = c1;
            c1 = c;
        }
    }
    double4 *dt = nullptr;
    double *ds = nullptr;
    cudaError_t e = sht::dev_malloc(&dt, sizeof(double4) * tab.size());
    if (e == cudaSuccess) e = sht::dev_malloc(&ds, sizeof(double) * start.size());
    if (e == cudaSuccess) e = cudaMemcpy(dt, tab.data(), sizeof(double4) * tab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ds, start.data(), sizeof(double) * start.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dt);
        cudaFree(ds);
        return e;
    }
    p.d_spin_tab = dt;
    p.d_spin_start = ds;
    return cudaSuccess;
}

size_t spin_partial_bytes(const Plan &p, int nmaps)
{
    const int nblk = (p.nslots + SP_T - 1) / SP_T;
    return (size_t)nblk * nmaps * 2 * (size_t)p.nalm * sizeof(double2);
}

cudaError_t launch_spin_synth(const Plan &p, const double2 *alm, double2 *delta, int nmaps, cudaStream_t st,
                              int *nlaunch)
{
    *nlaunch = 0;
    SpinArgs A = spin_args(p);
    const unsigned grid = (unsigned)((p.mmax + 1) * A.nblk);
    const int64_t dstride = 2 * (int64_t)p.nrings * (p.mmax + 1);
    int g0 = 0;
    while (g0 < nmaps) {
        const int nm = nmaps - g0 >= 2 ? 2 : 1;
        A.alm = alm + (int64_t)g0 * 2 * p.nalm;
        A.delta = delta + (int64_t)g0 * dstride;
        A.nmaps = nm;
        if (nm == 2)
            spin_synth_kernel<2><<<grid, SP_T, 0, st>>>(A);
        else
            spin_synth_kernel<1><<<grid, SP_T, 0, st>>>(A);
        ++*nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        g0 += nm;
    }
    return cudaSuccess;
}

cudaError_t launch_spin_anal(const Plan &p, const double2 *delta, double2 *alm, double2 *partial, int nmaps,
                             cudaStream_t st, int *nlaunch)
{
    *nlaunch = 0;
    SpinArgs A = spin_args(p);
    const unsigned grid = (unsigned)((p.mmax + 1) * A.nblk);
    const int64_t dstride = 2 * (int64_t)p.nrings * (p.mmax + 1);
    int g0 = 0;
    while (g0 < nmaps) {
        const int nm = nmaps - g0 >= 2 ? 2 : 1;
        A.delta = const_cast<double2 *>(delta) + (int64_t)g0 * dstride;
        A.partial = partial;
        A.nmaps = nm;
        if (nm == 2)
            spin_anal_kernel<2><<<grid, SP_T, 0, st>>>(A);
        else
            spin_anal_kernel<1><<<grid, SP_T, 0, st>>>(A);
        ++*nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int64_t nvec = 2 * (int64_t)nm;
        const int rgrid = (int)std::min<int64_t>((nvec * p.nalm + 255) / 256, 152 * 16);
        spin_reduce_kernel<<<rgrid, 256, 0, st>>>(partial, alm + (int64_t)g0 * 2 * p.nalm, A.nblk, p.nalm, nvec,
                                                  p.lmax);
        ++*nlaunch;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        g0 += nm;
    }
    return cudaSuccess;
}

namespace {
SHT_CHECK_TAKE_DEF(take_check)
}  // namespace
cudaError_t take_check_word_spin(int *w) { return take_check(w); }

}  // namespace sht
