// Legendre stage of the transforms (Section 2.2 eqs. DeltaDef and almdef,
// Algorithms 1-2 step "core calculation", GPU form of Algorithms 5-6).
//
// Both kernels run one CTA per (m, block of ring slots), m ascending so the
// longest l-ranges start first.  A ring slot is a ring in the northern
// hemisphere together with its mirror ring (theta, pi - theta); one thread
// runs the l-recurrence once for both, using
// lambda_lm(-x) = (-1)^(l+m) lambda_lm(x): terms with l+m even are summed
// into E, odd ones into O, and Delta_N = E + O, Delta_S = E - O.
//
// The recurrence of eq. (assLegRec) (with the sign reading
// lambda_l = beta_l (x lambda_{l-1} - lambda_{l-2} / beta_{l-1})) is run in
// the normalised variable y_l = lambda_l / c_l, where c_m = c_{m+1} = 1 and
// c_l = (beta_l / beta_{l-1}) c_{l-2}.  Then
//     y_l = alpha_l x y_{l-1} - y_{l-2},   alpha_l = beta_l c_{l-1} / c_l,
// which costs two FP64 instructions per step: t = x y_{l-1} is formed as
// fma(-u, y, y) with u = 1 - cos(theta) (exact near the poles, where
// cos(theta) rounded to double would displace the ring by ~1e-16/sin(theta)),
// then y_l = fma(alpha_l, t, -y_{l-2}).  The factor c_l is folded into a_lm
// when it is staged (synthesis) or applied after the ring reduction
// (analysis).  The coefficient table stores mu_m at l = m and sqrt(2m+3)
// (eq. pm1m) at l = m + 1; seeding y_{m-1} = 0, y_{m-2} = -y_m lets the same
// step produce y_m and y_{m+1}.
//
// Rescaling (the scheme Section 2.1 leaves to HEALPix/S2HAT): the start
// value mu_m sin^m(theta) is formed by binary powering with its binary
// exponent carried in an int and split as y * 2^(512 k), k <= 0.  While
// k < 0 the pair (y_l, y_{l-1}) is multiplied by 2^-512 (k += 1) whenever
// its exponent passes 2^256; the test reads the exponent bits (integer pipe)
// once every 16 steps.  Terms are accumulated only at k = 0; terms with
// k < 0 are below 2^-224 and are dropped.  Once a whole warp has k = 0 the
// loop carries no tests at all.
//
// Polar slots.  Near a pole x = cos(theta) -> 1 and the recurrence is close
// to degenerate: a rounding error of relative size eps in y excites the
// second solution with amplitude ~eps/sin(theta), and over n steps the
// error in lambda grows to ~eps n^1.5 (1e-10 at theta = 4e-4, l = 4096).
// CTAs whose first slot has sin(theta) < 0.03 therefore run, for
// m <= mR, Reinsch's difference form in lambda itself:
//     D_l = (1 + rho_l) D_{l-1} + g_l lambda_{l-1},  lambda_l = lambda_{l-1} + D_l,
//     g_l = (beta_l - 2 - rho_l) - beta_l u,  rho_l = beta_l / beta_{l-1} - 1,
// with rho_l and b0_l = beta_l - 2 - rho_l tabulated from cancellation-free
// formulas; rounding errors then act on the small difference D instead of on
// lambda.  It costs four FP64 instructions per step instead of two.  For
// m > mR the values on these rings stay below the rescaling threshold for
// every l <= lmax, so the y form is used there.
#include "sht_internal.h"

#include <algorithm>
#include <vector>

namespace sht {
namespace {

#include "recurrence.cuh"

constexpr int SYN_T = 128;      // threads (= ring slots) per synthesis CTA
constexpr int ANA_T = 128;      // threads per analysis CTA
constexpr int CHL = 128;        // l-values staged per shared-memory chunk (multiple of 16)
constexpr int SUB = 16;         // steps between rescale tests
constexpr int RED_CL = 8;       // l-values per warp reduction round (analysis)

// Recurrence coefficients of one l-chunk in shared memory.
struct Coef {
    double al[CHL];               // y form: alpha_l
    double be[CHL], rh[CHL], b0[CHL];  // Reinsch form: beta_l, rho_l, b0_l
};

// One step of the recurrence.  y1 is the newest value; y2 is the previous
// value (y form) or the last difference D (Reinsch form).
template <bool REIN>
__device__ __forceinline__ double rec_step(const Coef &C, int j, double u, double &y1, double &y2)
{
    if (REIN) {
        const double g = fma(-C.be[j], u, C.b0[j]);
        const double t = fma(g, y1, y2);
        y2 = fma(C.rh[j], y2, t);
        y1 = y1 + y2;
        return y1;
    } else {
        const double t = fma(-u, y1, y1);
        const double y = fma(C.al[j], t, -y2);
        y2 = y1;
        y1 = y;
        return y;
    }
}

// State before l = m that makes the first two steps produce lambda_m and lambda_{m+1}.
template <bool REIN>
__device__ __forceinline__ void seed_state(double y0, double &y1, double &y2)
{
    y1 = 0.0;                  // value at l = m - 1
    y2 = REIN ? y0 : -y0;      // D_{m-1} = lambda_m (Reinsch) or y_{m-2} = -y_m
}

template <bool REIN>
__device__ __forceinline__ void stage_coef(Coef &C, const double *alpha, const double3 *rein, int64_t ix, int i)
{
    if (REIN) {
        const double3 c = rein[ix];
        C.be[i] = c.x;
        C.rh[i] = c.y;
        C.b0[i] = c.z;
    } else {
        C.al[i] = alpha[ix];
    }
}

struct SynArgs {
    const double2 *alm;   // [nmaps][nalm], first map of this launch
    double2 *delta;       // [nmaps][nrings][mmax+1]
    const int *slotN, *slotS;
    const double *u, *s;
    const double *alpha, *cfac;
    const double3 *rein;  // Reinsch coefficients for m <= mR
    const int *mflag;     // [mmax+1] 1 for the m this plan computes (null: all)
    int nslots, nblk, lmax, mmax, nrings, mR;
    int64_t nalm;
};

template <int NM, bool REIN>
__device__ __forceinline__ void synth_body(const SynArgs &A, int m, int blk, Coef &C, double2 (*s_a)[CHL])
{
    const int slot = blk * SYN_T + threadIdx.x;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;  // index(m, m)

    double u = 0.0, y1 = 0.0, y2 = 0.0;
    int k = 0;
    if (active) {
        u = A.u[slot];
        double y0;
        sectoral_start(A.s[slot], A.alpha[base], m, y0, k);
        seed_state<REIN>(y0, y1, y2);
    }

    double Er[NM], Ei[NM], Or[NM], Oi[NM];
#pragma unroll
    for (int g = 0; g < NM; ++g) Er[g] = Ei[g] = Or[g] = Oi[g] = 0.0;

    for (int l0 = m; l0 <= L; l0 += CHL) {
        const int nl = min(CHL, L - l0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nl; i += SYN_T) {
            const int64_t ix = base + (l0 - m) + i;
            stage_coef<REIN>(C, A.alpha, A.rein, ix, i);
            const double c = REIN ? 1.0 : A.cfac[ix];  // the y form sums c_l a_l y_l
#pragma unroll
            for (int g = 0; g < NM; ++g) {
                double2 a = A.alm[(int64_t)g * A.nalm + ix];
                s_a[g][i] = make_double2(c * a.x, m == 0 ? 0.0 : c * a.y);
            }
        }
        __syncthreads();

        for (int j0 = 0; j0 < nl; j0 += SUB) {
            const int jn = min(j0 + SUB, nl);
            const bool scaled = __any_sync(0xffffffffu, k < 0);
            if (!scaled) {
                int j = j0;
                for (; j + 1 < jn; j += 2) {
                    double y = rec_step<REIN>(C, j, u, y1, y2);
#pragma unroll
                    for (int g = 0; g < NM; ++g) {
                        const double2 a = s_a[g][j];
                        Er[g] = fma(a.x, y, Er[g]);
                        Ei[g] = fma(a.y, y, Ei[g]);
                    }
                    y = rec_step<REIN>(C, j + 1, u, y1, y2);
#pragma unroll
                    for (int g = 0; g < NM; ++g) {
                        const double2 a = s_a[g][j + 1];
                        Or[g] = fma(a.x, y, Or[g]);
                        Oi[g] = fma(a.y, y, Oi[g]);
                    }
                }
                if (j < jn) {  // ragged end: one even step
                    const double y = rec_step<REIN>(C, j, u, y1, y2);
#pragma unroll
                    for (int g = 0; g < NM; ++g) {
                        const double2 a = s_a[g][j];
                        Er[g] = fma(a.x, y, Er[g]);
                        Ei[g] = fma(a.y, y, Ei[g]);
                    }
                }
            } else {
                const bool any_live = __any_sync(0xffffffffu, active && k == 0);
                for (int j = j0; j < jn; ++j) {
                    const double y = rec_step<REIN>(C, j, u, y1, y2);
                    if (any_live) {
                        const double ya = (k == 0) ? y : 0.0;
                        if (((j + l0 - m) & 1) == 0) {
#pragma unroll
                            for (int g = 0; g < NM; ++g) {
                                const double2 a = s_a[g][j];
                                Er[g] = fma(a.x, ya, Er[g]);
                                Ei[g] = fma(a.y, ya, Ei[g]);
                            }
                        } else {
#pragma unroll
                            for (int g = 0; g < NM; ++g) {
                                const double2 a = s_a[g][j];
                                Or[g] = fma(a.x, ya, Or[g]);
                                Oi[g] = fma(a.y, ya, Oi[g]);
                            }
                        }
                    }
                }
                if (k < 0 && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                    y1 *= 0x1p-512;
                    y2 *= 0x1p-512;
                    k += 1;
                }
            }
        }
    }

    if (active) {
        const int rn = A.slotN[slot], rs = A.slotS[slot];
        const int64_t mstride = A.mmax + 1;
#pragma unroll
        for (int g = 0; g < NM; ++g) {
            double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
            if (rn >= 0 && SHT_CHK(rn < A.nrings && m <= A.mmax))
                d[(int64_t)rn * mstride + m] = make_double2(Er[g] + Or[g], Ei[g] + Oi[g]);
            if (rs >= 0 && SHT_CHK(rs < A.nrings && m <= A.mmax))
                d[(int64_t)rs * mstride + m] = make_double2(Er[g] - Or[g], Ei[g] - Oi[g]);
        }
    }
}

template <int NM>
__global__ void __launch_bounds__(SYN_T) legendre_synth_kernel(SynArgs A)
{
    __shared__ Coef C;
    __shared__ double2 s_a[NM][CHL];
    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    if (A.mflag && !A.mflag[m]) {  // an m this plan does not compute: Delta_m = 0 on these rings
        const int slot = blk * SYN_T + threadIdx.x;
        if (slot < A.nslots) {
            const int rn = A.slotN[slot], rs = A.slotS[slot];
            const int64_t mstride = A.mmax + 1;
            for (int g = 0; g < NM; ++g) {
                double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
                if (rn >= 0 && SHT_CHK(rn < A.nrings)) d[(int64_t)rn * mstride + m] = make_double2(0.0, 0.0);
                if (rs >= 0 && SHT_CHK(rs < A.nrings)) d[(int64_t)rs * mstride + m] = make_double2(0.0, 0.0);
            }
        }
        return;
    }
    const bool polar = m <= A.mR && A.s[blk * SYN_T] < POLAR_SIN;  // slots are sorted by colatitude
    if (polar)
        synth_body<NM, true>(A, m, blk, C, s_a);
    else
        synth_body<NM, false>(A, m, blk, C, s_a);
}

struct AnaArgs {
    const double2 *delta;  // [nmaps][nrings][mmax+1], first map of this launch
    double2 *partial;      // [nblk][nmaps_total][nalm]
    const int *slotN, *slotS;
    const double *u, *s;
    const double *alpha, *cfac;
    const double3 *rein;
    const int *mflag;      // [mmax+1] 1 for the m this plan computes (null: all)
    int nslots, nblk, lmax, mmax, nrings, mR;
    int64_t nalm;
    int64_t part_map_stride;   // nalm
    int64_t part_blk_stride;   // nmaps_total * nalm
};

// Reduce-scatter of RED_CL values per lane over the warp: afterwards every lane
// holds the warp total of value (lane & (RED_CL-1)).
__device__ __forceinline__ double warp_reduce_scatter8(double v[RED_CL])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int h = RED_CL / 2; h >= 1; h >>= 1) {
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

template <int NM, int K, bool REIN>
__device__ __forceinline__ void anal_body(const AnaArgs &A, int m, int blk, Coef &C,
                                          double (*s_red)[CHL][2 * NM])
{
    constexpr int NW = ANA_T / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int64_t mstride = A.mmax + 1;

    double u[K], y1[K], y2[K];
    int k[K];
    bool act[K];
    double Sr[K][NM], Si[K][NM], Dr[K][NM], Di[K][NM];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int slot = blk * (ANA_T * K) + q * ANA_T + threadIdx.x;
        u[q] = 0.0;
        y1[q] = 0.0;
        y2[q] = 0.0;
        k[q] = 0;
        act[q] = slot < A.nslots;
#pragma unroll
        for (int g = 0; g < NM; ++g) Sr[q][g] = Si[q][g] = Dr[q][g] = Di[q][g] = 0.0;
        if (act[q]) {
            u[q] = A.u[slot];
            double y0;
            sectoral_start(A.s[slot], A.alpha[base], m, y0, k[q]);
            seed_state<REIN>(y0, y1[q], y2[q]);
            const int rn = A.slotN[slot], rs = A.slotS[slot];
#pragma unroll
            for (int g = 0; g < NM; ++g) {
                const double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
                double2 dn = make_double2(0.0, 0.0), ds = make_double2(0.0, 0.0);
                if (rn >= 0) dn = d[(int64_t)rn * mstride + m];
                if (rs >= 0) ds = d[(int64_t)rs * mstride + m];
                Sr[q][g] = dn.x + ds.x;
                Si[q][g] = dn.y + ds.y;
                Dr[q][g] = dn.x - ds.x;
                Di[q][g] = dn.y - ds.y;
            }
        }
    }

    for (int l0 = m; l0 <= L; l0 += CHL) {
        const int nl = min(CHL, L - l0 + 1);
        __syncthreads();
        for (int i = threadIdx.x; i < nl; i += ANA_T) stage_coef<REIN>(C, A.alpha, A.rein, base + (l0 - m) + i, i);
        __syncthreads();

        for (int j0 = 0; j0 < nl; j0 += SUB) {
            bool scaled = false;
#pragma unroll
            for (int q = 0; q < K; ++q) scaled |= (k[q] < 0);
            scaled = __any_sync(0xffffffffu, scaled);
            // While every slot of the warp is still below the rescaling threshold its
            // terms are all dropped: only the recurrence runs and the warp's partial
            // sums for these l are zero.
            bool live = true;
            if (scaled) {
                bool mine = false;
#pragma unroll
                for (int q = 0; q < K; ++q) mine |= (act[q] && k[q] == 0);
                live = __any_sync(0xffffffffu, mine);
            }
            if (!live) {
                for (int j = j0; j < min(j0 + SUB, nl); ++j) {
#pragma unroll
                    for (int q = 0; q < K; ++q) rec_step<REIN>(C, j, u[q], y1[q], y2[q]);
                }
                if (lane < SUB) {
#pragma unroll
                    for (int g = 0; g < NM; ++g) {
                        s_red[warp][j0 + lane][2 * g] = 0.0;
                        s_red[warp][j0 + lane][2 * g + 1] = 0.0;
                    }
                }
            } else {
                // two rounds of RED_CL l-values per SUB block
#pragma unroll
                for (int h = 0; h < SUB / RED_CL; ++h) {
                    const int jb = j0 + h * RED_CL;
                    double vr[NM][RED_CL], vi[NM][RED_CL];
#pragma unroll
                    for (int jj = 0; jj < RED_CL; ++jj) {
                        const int j = jb + jj;
                        const bool inside = j < nl;
                        const bool even = ((jj & 1) == 0);  // l - m has the parity of jj
#pragma unroll
                        for (int g = 0; g < NM; ++g) vr[g][jj] = vi[g][jj] = 0.0;
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            double y = 0.0;
                            if (inside) y = rec_step<REIN>(C, j, u[q], y1[q], y2[q]);
                            const bool use = inside && (!scaled || k[q] == 0);
                            y = use ? y : 0.0;
#pragma unroll
                            for (int g = 0; g < NM; ++g) {
                                vr[g][jj] = fma(y, even ? Sr[q][g] : Dr[q][g], vr[g][jj]);
                                vi[g][jj] = fma(y, even ? Si[q][g] : Di[q][g], vi[g][jj]);
                            }
                        }
                    }
#pragma unroll
                    for (int g = 0; g < NM; ++g) {
                        const double rr = warp_reduce_scatter8(vr[g]);
                        const double ri = warp_reduce_scatter8(vi[g]);
                        if (lane < RED_CL) {
                            s_red[warp][jb + lane][2 * g] = rr;
                            s_red[warp][jb + lane][2 * g + 1] = ri;
                        }
                    }
                }
            }
            if (scaled) {
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    if (k[q] < 0 && max(dexp(y1[q]), dexp(y2[q])) > RESCALE_THR) {
                        y1[q] *= 0x1p-512;
                        y2[q] *= 0x1p-512;
                        k[q] += 1;
                    }
                }
            }
        }
        __syncthreads();
        // sum the warps and write this block's partial a_lm; the reduction multiplies
        // by c_l, so the Reinsch form (which sums lambda, not y) divides by it here
        for (int i = threadIdx.x; i < nl * NM; i += ANA_T) {
            const int j = i % nl, g = i / nl;
            double re = 0.0, im = 0.0;
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                re += s_red[w][j][2 * g];
                im += s_red[w][j][2 * g + 1];
            }
            const int64_t ix = base + (l0 - m) + j;
            if (REIN) {
                const double c = A.cfac[ix];
                re /= c;
                im /= c;
            }
            if (SHT_CHK(ix >= 0 && ix < A.nalm && blk < A.nblk))
                A.partial[(int64_t)blk * A.part_blk_stride + (int64_t)g * A.part_map_stride + ix] = make_double2(re, im);
        }
    }
}

template <int NM, int K>
__global__ void __launch_bounds__(ANA_T) legendre_anal_kernel(AnaArgs A)
{
    constexpr int NW = ANA_T / 32;
    __shared__ Coef C;
    __shared__ double s_red[NW][CHL][2 * NM];
    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    if (A.mflag && !A.mflag[m]) {  // an m this plan does not compute: zero partials
        const int64_t base = (int64_t)m * (2 * A.lmax + 3 - m) / 2;
        for (int i = threadIdx.x; i < (A.lmax - m + 1) * NM; i += ANA_T) {
            const int j = i % (A.lmax - m + 1), g = i / (A.lmax - m + 1);
            A.partial[(int64_t)blk * A.part_blk_stride + (int64_t)g * A.part_map_stride + base + j] =
                make_double2(0.0, 0.0);
        }
        return;
    }
    const bool polar = m <= A.mR && A.s[blk * (ANA_T * K)] < POLAR_SIN;
    if (polar)
        anal_body<NM, K, true>(A, m, blk, C, s_red);
    else
        anal_body<NM, K, false>(A, m, blk, C, s_red);
}

// a_lm = c_lm * sum over ring blocks (fixed order), Im a_l0 = 0
__global__ void reduce_blocks_kernel(const double2 *__restrict__ partial, const double *__restrict__ cfac,
                                     double2 *__restrict__ alm, int nblk, int64_t nalm, int nmaps, int lmax,
                                     int64_t blk_stride)
{
    const int64_t total = nalm * nmaps;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t g = t / nalm, i = t - g * nalm;
        double re = 0.0, im = 0.0;
        for (int b = 0; b < nblk; ++b) {
            const double2 v = partial[b * blk_stride + g * nalm + i];
            re += v.x;
            im += v.y;
        }
        const double c = cfac[i];
        alm[t] = make_double2(c * re, i <= lmax ? 0.0 : c * im);
    }
}

// ---------------------------------------------------------------- batched form (many plans)
//
// One persistent launch runs the Legendre tiles of many transforms (uneven lmax, any number of
// maps each): a tile is (job, first map, maps, m, slot block), the host sorts the tiles by their
// l-range, longest first (the min-max balancing of the paper's Section 4.2.1 carried over to a
// queue), and every CTA takes the next tile from a device counter until the queue is empty.

// tile: x = job, y = m, z = slot block, w = first map | (maps << 16)
__global__ void __launch_bounds__(SYN_T) legendre_synth_batch_kernel(const SynArgs *__restrict__ jobs,
                                                                     const int4 *__restrict__ tiles, int ntiles,
                                                                     int *counter)
{
    __shared__ Coef C;
    __shared__ double2 s_a[4][CHL];
    __shared__ int s_t;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_t = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= ntiles) break;
        const int4 T = tiles[t];
        SynArgs A = jobs[T.x];
        const int g0 = T.w & 0xffff, nm = T.w >> 16;
        A.alm += (int64_t)g0 * A.nalm;
        A.delta += (int64_t)g0 * A.nrings * (A.mmax + 1);
        const int m = T.y, blk = T.z;
        const bool polar = m <= A.mR && A.s[blk * SYN_T] < POLAR_SIN;
        if (nm == 4) {
            if (polar) synth_body<4, true>(A, m, blk, C, s_a); else synth_body<4, false>(A, m, blk, C, s_a);
        } else if (nm == 2) {
            if (polar) synth_body<2, true>(A, m, blk, C, s_a); else synth_body<2, false>(A, m, blk, C, s_a);
        } else {
            if (polar) synth_body<1, true>(A, m, blk, C, s_a); else synth_body<1, false>(A, m, blk, C, s_a);
        }
    }
}

// tile: x = job, y = m, z = slot block (K * 128 slots), w = first map | (maps << 16); the partial
// sums of job j go to its own buffer (A.partial), reduced afterwards by reduce_blocks_batch_kernel
template <int K>
__global__ void __launch_bounds__(ANA_T) legendre_anal_batch_kernel(const AnaArgs *__restrict__ jobs,
                                                                    const int4 *__restrict__ tiles, int ntiles,
                                                                    int *counter)
{
    constexpr int NW = ANA_T / 32;
    __shared__ Coef C;
    __shared__ double s_red_raw[NW * CHL * 4];
    __shared__ int s_t;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_t = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= ntiles) break;
        const int4 T = tiles[t];
        AnaArgs A = jobs[T.x];
        const int g0 = T.w & 0xffff, nm = T.w >> 16;
        A.delta += (int64_t)g0 * A.nrings * (A.mmax + 1);
        A.partial += (int64_t)g0 * A.part_map_stride;
        const int m = T.y, blk = T.z;
        const bool polar = m <= A.mR && A.s[blk * (ANA_T * K)] < POLAR_SIN;
        if (nm == 2) {
            auto *r = reinterpret_cast<double(*)[CHL][4]>(s_red_raw);
            if (polar) anal_body<2, K, true>(A, m, blk, C, r); else anal_body<2, K, false>(A, m, blk, C, r);
        } else {
            auto *r = reinterpret_cast<double(*)[CHL][2]>(s_red_raw);
            if (polar) anal_body<1, K, true>(A, m, blk, C, r); else anal_body<1, K, false>(A, m, blk, C, r);
        }
    }
}

// a_lm = c_lm * sum over ring blocks, for every job of the batch (one launch)
__global__ void reduce_blocks_batch_kernel(const BatchReduceJob *__restrict__ jobs, int njobs)
{
    for (int j = 0; j < njobs; ++j) {
        const BatchReduceJob J = jobs[j];
        const int64_t total = J.nalm * J.nmaps;
        for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
             t += (int64_t)gridDim.x * blockDim.x) {
            const int64_t g = t / J.nalm, i = t - g * J.nalm;
            double re = 0.0, im = 0.0;
            for (int b = 0; b < J.nblk; ++b) {
                const double2 v = J.partial[b * J.blk_stride + g * J.nalm + i];
                re += v.x;
                im += v.y;
            }
            const double c = J.cfac[i];
            J.alm[t] = make_double2(c * re, i <= J.lmax ? 0.0 : c * im);
        }
    }
}

int anal_slots_per_cta(const Plan &p) { return p.tune[SHT_TUNE_ANAL_SLOTS] * ANA_T; }

}  // namespace

cudaError_t launch_legendre_synth(const Plan &p, const double2 *alm, double2 *delta, int nmaps, cudaStream_t st,
                                  int *nlaunch)
{
    *nlaunch = 0;
    SynArgs A;
    A.slotN = p.d_slotN;
    A.slotS = p.d_slotS;
    A.u = p.d_u;
    A.s = p.d_s;
    A.alpha = p.d_alpha;
    A.cfac = p.d_cfac;
    A.rein = p.d_rein;
    A.mflag = p.d_mflag;
    A.mR = p.mR;
    A.nslots = p.nslots;
    A.nblk = (p.nslots + SYN_T - 1) / SYN_T;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    A.nrings = p.nrings;
    A.nalm = p.nalm;
    const unsigned grid = (unsigned)((p.mmax + 1) * A.nblk);
    const int64_t dstride = (int64_t)p.nrings * (p.mmax + 1);
    int g0 = 0;
    while (g0 < nmaps) {
        const int left = nmaps - g0;
        A.alm = alm + (int64_t)g0 * p.nalm;
        A.delta = delta + (int64_t)g0 * dstride;
        const int most = p.tune[SHT_TUNE_SYNTH_MAPS];
        if (left >= 4 && most >= 4) {
            legendre_synth_kernel<4><<<grid, SYN_T, 0, st>>>(A);
            g0 += 4;
        } else if (left >= 2 && most >= 2) {
            legendre_synth_kernel<2><<<grid, SYN_T, 0, st>>>(A);
            g0 += 2;
        } else {
            legendre_synth_kernel<1><<<grid, SYN_T, 0, st>>>(A);
            g0 += 1;
        }
        ++*nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t legendre_anal_partial_bytes(const Plan &p, int nmaps)
{
    const int per = anal_slots_per_cta(p);
    const int nblk = (p.nslots + per - 1) / per;
    return (size_t)nblk * (size_t)nmaps * (size_t)p.nalm * sizeof(double2);
}

int legendre_anal_default_slots(const Plan &p) { return p.nslots >= 4 * ANA_T ? 4 : 1; }

int legendre_anal_nblk(const Plan &p)
{
    const int per = anal_slots_per_cta(p);
    return (p.nslots + per - 1) / per;
}

cudaError_t launch_legendre_anal(const Plan &p, const double2 *delta, double2 *partial, int nmaps, cudaStream_t st,
                                 int *nlaunch)
{
    *nlaunch = 0;
    const int per = anal_slots_per_cta(p);
    AnaArgs A;
    A.slotN = p.d_slotN;
    A.slotS = p.d_slotS;
    A.u = p.d_u;
    A.s = p.d_s;
    A.alpha = p.d_alpha;
    A.cfac = p.d_cfac;
    A.rein = p.d_rein;
    A.mflag = p.d_mflag;
    A.mR = p.mR;
    A.nslots = p.nslots;
    A.nblk = (p.nslots + per - 1) / per;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    A.nrings = p.nrings;
    A.nalm = p.nalm;
    A.part_map_stride = p.nalm;
    A.part_blk_stride = (int64_t)nmaps * p.nalm;
    const unsigned grid = (unsigned)((p.mmax + 1) * A.nblk);
    const int64_t dstride = (int64_t)p.nrings * (p.mmax + 1);
    int g0 = 0;
    while (g0 < nmaps) {
        const int left = nmaps - g0;
        A.delta = delta + (int64_t)g0 * dstride;
        A.partial = partial + (int64_t)g0 * p.nalm;
        if (left >= 2 && p.tune[SHT_TUNE_ANAL_MAPS] >= 2) {
            if (per == 4 * ANA_T)
                legendre_anal_kernel<2, 4><<<grid, ANA_T, 0, st>>>(A);
            else
                legendre_anal_kernel<2, 1><<<grid, ANA_T, 0, st>>>(A);
            g0 += 2;
        } else {
            if (per == 4 * ANA_T)
                legendre_anal_kernel<1, 4><<<grid, ANA_T, 0, st>>>(A);
            else
                legendre_anal_kernel<1, 1><<<grid, ANA_T, 0, st>>>(A);
            g0 += 1;
        }
        ++*nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- batched form: host side

namespace {
template <class T>
cudaError_t upload_vec(T **dst, const std::vector<T> &v)
{
    cudaError_t e = dev_malloc(dst, sizeof(T) * std::max<size_t>(v.size(), 1));
    if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice);
    return e;
}

// tiles of every job, each job's maps cut into groups of at most `most`, sorted by l-range x maps
// (longest first; ties: lower job first)
std::vector<int4> batch_tiles(const std::vector<const Plan *> &plans, const std::vector<int> &nmaps, int most,
                              int slots_per_cta)
{
    struct Key {
        int64_t cost;
        int4 t;
    };
    std::vector<Key> keys;
    for (size_t j = 0; j < plans.size(); ++j) {
        const Plan &p = *plans[j];
        const int nblk = (p.nslots + slots_per_cta - 1) / slots_per_cta;
        for (int g0 = 0; g0 < nmaps[j]; g0 += most) {
            const int nm = std::min(most, nmaps[j] - g0);
            const int nmq = nm >= 4 ? 4 : nm >= 2 ? 2 : 1;  // the kernels take 4, 2 or 1 maps
            for (int g = g0; g < g0 + nm; g += nmq) {
                const int n = std::min(nmq, g0 + nm - g);
                const int q = n >= 4 ? 4 : n >= 2 ? 2 : 1;
                for (int m = 0; m <= p.mmax; ++m)
                    for (int b = 0; b < nblk; ++b)
                        keys.push_back({(int64_t)(p.lmax - m + 1) * q, make_int4((int)j, m, b, g | (q << 16))});
            }
        }
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) { return a.cost > b.cost; });
    std::vector<int4> out(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) out[i] = keys[i].t;
    return out;
}
}  // namespace

cudaError_t batch_legendre_synth_setup(const std::vector<const Plan *> &plans, const std::vector<const double2 *> &alm,
                                       const std::vector<double2 *> &delta, const std::vector<int> &nmaps,
                                       int maps_per_tile, BatchLaunch &L)
{
    std::vector<SynArgs> jobs(plans.size());
    for (size_t j = 0; j < plans.size(); ++j) {
        const Plan &p = *plans[j];
        SynArgs &A = jobs[j];
        A = SynArgs{};
        A.alm = alm[j];
        A.delta = delta[j];
        A.slotN = p.d_slotN;
        A.slotS = p.d_slotS;
        A.u = p.d_u;
        A.s = p.d_s;
        A.alpha = p.d_alpha;
        A.cfac = p.d_cfac;
        A.rein = p.d_rein;
        A.mflag = nullptr;
        A.mR = p.mR;
        A.nslots = p.nslots;
        A.nblk = (p.nslots + SYN_T - 1) / SYN_T;
        A.lmax = p.lmax;
        A.mmax = p.mmax;
        A.nrings = p.nrings;
        A.nalm = p.nalm;
    }
    const std::vector<int4> tiles = batch_tiles(plans, nmaps, maps_per_tile, SYN_T);
    L.ntiles = (int)tiles.size();
    cudaError_t e = upload_vec((SynArgs **)&L.jobs, jobs);
    if (e == cudaSuccess) e = upload_vec(&L.tiles, tiles);
    return e;
}

cudaError_t batch_legendre_anal_setup(const std::vector<const Plan *> &plans, const std::vector<const double2 *> &delta,
                                      const std::vector<double2 *> &partial, const std::vector<double2 *> &alm,
                                      const std::vector<int> &nmaps, int maps_per_tile, int slots_per_thread,
                                      BatchLaunch &L, BatchLaunch &R)
{
    const int per = slots_per_thread * ANA_T;
    std::vector<AnaArgs> jobs(plans.size());
    std::vector<BatchReduceJob> red(plans.size());
    for (size_t j = 0; j < plans.size(); ++j) {
        const Plan &p = *plans[j];
        AnaArgs &A = jobs[j];
        A = AnaArgs{};
        A.delta = delta[j];
        A.partial = partial[j];
        A.slotN = p.d_slotN;
        A.slotS = p.d_slotS;
        A.u = p.d_u;
        A.s = p.d_s;
        A.alpha = p.d_alpha;
        A.cfac = p.d_cfac;
        A.rein = p.d_rein;
        A.mflag = nullptr;
        A.mR = p.mR;
        A.nslots = p.nslots;
        A.nblk = (p.nslots + per - 1) / per;
        A.lmax = p.lmax;
        A.mmax = p.mmax;
        A.nrings = p.nrings;
        A.nalm = p.nalm;
        A.part_map_stride = p.nalm;
        A.part_blk_stride = (int64_t)nmaps[j] * p.nalm;
        red[j] = BatchReduceJob{partial[j], p.d_cfac, alm[j], A.nblk, p.nalm, nmaps[j], p.lmax,
                                (int64_t)nmaps[j] * p.nalm};
    }
    const std::vector<int4> tiles = batch_tiles(plans, nmaps, std::min(maps_per_tile, 2), per);
    L.ntiles = (int)tiles.size();
    L.k = slots_per_thread;
    R.ntiles = (int)plans.size();
    cudaError_t e = upload_vec((AnaArgs **)&L.jobs, jobs);
    if (e == cudaSuccess) e = upload_vec(&L.tiles, tiles);
    if (e == cudaSuccess) e = upload_vec((BatchReduceJob **)&R.jobs, red);
    return e;
}

size_t batch_anal_partial_bytes(const Plan &p, int nmaps, int slots_per_thread)
{
    const int per = slots_per_thread * ANA_T;
    return (size_t)((p.nslots + per - 1) / per) * nmaps * (size_t)p.nalm * sizeof(double2);
}

cudaError_t batch_legendre_synth_launch(const BatchLaunch &L, int *counter, int grid, cudaStream_t st)
{
    legendre_synth_batch_kernel<<<grid, SYN_T, 0, st>>>((const SynArgs *)L.jobs, L.tiles, L.ntiles, counter);
    return cudaGetLastError();
}

cudaError_t batch_legendre_anal_launch(const BatchLaunch &L, const BatchLaunch &R, int *counter, int grid,
                                       cudaStream_t st)
{
    if (L.k == 4)
        legendre_anal_batch_kernel<4><<<grid, ANA_T, 0, st>>>((const AnaArgs *)L.jobs, L.tiles, L.ntiles, counter);
    else
        legendre_anal_batch_kernel<1><<<grid, ANA_T, 0, st>>>((const AnaArgs *)L.jobs, L.tiles, L.ntiles, counter);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    reduce_blocks_batch_kernel<<<152 * 8, 256, 0, st>>>((const BatchReduceJob *)R.jobs, R.ntiles);
    return cudaGetLastError();
}

cudaError_t launch_block_reduce(const Plan &p, const double2 *partial, double2 *alm, int nmaps, cudaStream_t st)
{
    const int64_t total = p.nalm * nmaps;
    const int rgrid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    reduce_blocks_kernel<<<rgrid, 256, 0, st>>>(partial, p.d_cfac, alm, legendre_anal_nblk(p), p.nalm, nmaps, p.lmax,
                                                (int64_t)nmaps * p.nalm);
    return cudaGetLastError();
}

namespace {
SHT_CHECK_TAKE_DEF(take_check)
}  // namespace
cudaError_t take_check_word_legendre(int *w) { return take_check(w); }

}  // namespace sht
