// Precision form of the Legendre analysis (eq. almdef, Algorithm 5): the
// lambda recurrence stays in FP64; the products lambda * Delta^S and their
// sum over ring slots run on the FP32 pipe in double-float arithmetic.
//
// On this part FP32 issues 64 times faster than FP64 (2 FP64 FMA per SM per
// cycle).  A value v (FP64) is carried as hi + lo, two floats holding 48 bits
// of its 53-bit significand: hi the leading 24 bits (truncated), lo the next
// 24 of the remainder, both cut from the bit pattern with integer operations
// (an FP64 -> FP32 conversion would take an FP64 issue slot).  A product is
// formed exactly to ~2^-46 with FMA (ph = yh*xh, pl = fma(yh, xh, -ph) +
// yh*xl + yl*xh) and sums use TwoSum on the hi parts, so partial sums keep
// about 2^-44 relative accuracy, far inside the 1e-9 bar of this form.
//
// CTA: one m, 256 ring slots (one per thread, 8 warps).  Sigma = D_N + D_S
// and D = D_N - D_S for the maps of one launch (up to SHT_TUNE_DF_MAPS, 2 real columns
// each) sit in shared memory as double-float pairs.  Per group of 8 l, every lane forms its 8 products
// per column and a warp reduce-scatter (TwoSum) leaves each lane the warp
// total of one l; the eight warps' totals are added in shared memory and the
// block's partial a_lm (times 1/c, as in the FP64 kernel) is written as a
// double-float pair per component.  The fixed-order block reduction then
// converts and sums the blocks in FP64.
//
// Polar slots (the first 256 slots of a plan whose first ring has sin(theta) < 0.03, for
// m <= mR) run Reinsch's difference form of the recurrence in lambda itself (see legendre.cu:
// four FP64 instructions per step instead of two) in the REIN instantiation of the same kernel,
// which writes lambda-sums / c_lm in FP64 to a separate region that the block reduction reads in
// place of those blocks.
#include "sht_internal.h"

#include <algorithm>

namespace sht {
namespace {

constexpr int DF_T = 256;          // threads = slots per CTA
constexpr int DF_CHL = 32;         // l per shared-memory chunk (multiple of 8)
#ifndef DF_G_L
#define DF_G_L 8
#endif
constexpr int DF_G = DF_G_L;       // l per reduce-scatter round: 8 (16: fewer instructions, but 702 vs 677 ms at lmax 4096)
static_assert(DF_G == 8 || DF_G == 16, "DF_G is 8 or 16");
// Maps per launch: SHT_TUNE_DF_MAPS (16, 8 or 4; default 8).  Fewer maps: less shared memory and
// more CTAs per SM, but the FP64 recurrence runs once per launch.  lmax = 4096, HEALPix 2048, 16 maps
// on GB300: 16 maps per launch 809 ms, 8 maps 677 ms (two CTAs of 8 warps per SM), 4 maps 781 ms.
#include "recurrence.cuh"

// v -> hi + lo from the bit pattern (integer pipe).  Values below 2^-126 flush to zero
// (their share of any sum here is below 2^-100 of the largest term).
__device__ __forceinline__ float2 d2df(double v)
{
    const int hiw = __double2hiint(v);
    const unsigned low = (unsigned)__double2loint(v);
    const int ex = (hiw >> 20) & 0x7ff;
    const int e = ex - 1023;
    if (ex == 0 || e < -126) return make_float2(0.f, 0.f);
    const unsigned sign = (unsigned)hiw & 0x80000000u;
    // hi: sign, exponent, top 23 fraction bits (20 from the high word, 3 from the low word)
    const unsigned frac23 = (((unsigned)hiw & 0xFFFFFu) << 3) | (low >> 29);
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | frac23);
    // lo: the remaining 29 fraction bits times 2^(e - 52), rounded to 24 bits (zero when
    // 2^(e - 52) is below the normal float range; hi alone then carries 24 bits).  The 29-bit
    // integer becomes a float without a conversion instruction (those take an FP64 issue slot on
    // this part): its 13- and 16-bit halves exactly as (2^23 + h) - 2^23, then one FMA rounds once.
    const unsigned rem = low & 0x1FFFFFFFu;
    const float rh = __fsub_rn(__uint_as_float(0x4B000000u | (rem >> 16)), 8388608.0f);
    const float rl = __fsub_rn(__uint_as_float(0x4B000000u | (rem & 0xFFFFu)), 8388608.0f);
    const float sc = (e - 52 >= -126) ? __uint_as_float((unsigned)(e - 52 + 127) << 23) : 0.f;
    const float lo = __fmul_rn(__fmaf_rn(rh, 65536.0f, rl), sc);
    return make_float2(hi, sign ? -lo : lo);
}

__device__ __forceinline__ float2 df_mul(float2 y, float2 x)
{
    const float ph = y.x * x.x;
    float pl = fmaf(y.x, x.x, -ph);
    pl = fmaf(y.x, x.y, pl);
    pl = fmaf(y.y, x.x, pl);
    return make_float2(ph, pl);
}

__device__ __forceinline__ float2 df_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float err = (a.x - (s - bb)) + (b.x - bb);
    return make_float2(s, err + a.y + b.y);
}

__device__ __forceinline__ float2 shfl_xor_df(float2 v, int m)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Reduce-scatter of DF_G double-float values per lane over the warp: every lane ends with the
// warp total of value (lane & (DF_G - 1)).  The caller stores value i at v[i ^ (lane & (DF_G - 1))], so
// that in every halving round the value a lane keeps and the one it sends sit in fixed
// registers (no per-lane selects): after the round with partner lane ^ h, v[i] (i < h) holds
// both lanes' sums of value i ^ (lane & (DF_G - 1)).
__device__ __forceinline__ float2 warp_reduce_scatter_df(float2 v[DF_G])
{
#pragma unroll
    for (int h = DF_G / 2; h >= 1; h >>= 1) {
#pragma unroll
        for (int i = 0; i < h; ++i) v[i] = df_add(v[i], shfl_xor_df(v[i + h], h));
    }
    float2 r = v[0];
#pragma unroll
    for (int o = DF_G; o < 32; o <<= 1) r = df_add(r, shfl_xor_df(r, o));  // the other lane groups
    return r;
}

// v[i] <- v[i ^ b] for b = lane & (DF_G - 1) (log2 DF_G conditional swaps)
__device__ __forceinline__ void xor_permute(float2 v[DF_G], int b)
{
#pragma unroll
    for (int h = DF_G / 2; h >= 1; h >>= 1) {
        const bool sw = (b & h) != 0;
#pragma unroll
        for (int i = 0; i < DF_G; ++i) {
            if ((i & h) == 0) {
                const float2 a = v[i], c = v[i + h];
                v[i] = sw ? c : a;
                v[i + h] = sw ? a : c;
            }
        }
    }
}

struct DfArgs {
    const double2 *delta;  // [nmaps][nrings][mmax+1], first map of this group
    float4 *partial;       // [nblk][nmaps_total][nalm] as (re_hi, re_lo, im_hi, im_lo)
    double2 *polar;        // Reinsch form: a_lm / c_lm of slots 0 .. 255 at [map * polar_stride + index]
    int64_t polar_stride;
    const int *slotN, *slotS;
    const double *u, *s;
    const double *alpha, *cfac;
    const double3 *rein;   // Reinsch coefficients (beta_l, rho_l, b0_l) for m <= mR
    int nslots, nblk, lmax, mmax, nrings, mR, nmaps;
    int64_t nalm;
    int64_t part_blk_stride;  // nmaps_total * nalm
};

// float -> double from the bit pattern (integer pipe): normal floats exactly, zero and subnormals as 0
__device__ __forceinline__ double widen_f1(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xffu;
    const unsigned hi = (b & 0x80000000u) | ((ex + (1023u - 127u)) << 20) | ((b & 0x7FFFFFu) >> 3);
    return ex ? __hiloint2double((int)hi, (int)(b << 29)) : 0.0;
}
// hi + lo as one double: one DADD, no conversion instructions
__device__ __forceinline__ double widen_df(float2 a) { return widen_f1(a.x) + widen_f1(a.y); }

template <int N, bool REIN>
struct DfSmem {
    float2 X[2][N][DF_T];           // [parity: Sigma, D][column][slot]
    float2 red[DF_T / 32][N][DF_CHL];  // [warp][column][l]: l contiguous, no bank conflicts
    double co[REIN ? 3 : 1][DF_CHL];   // y form: alpha_l; Reinsch form: beta_l, rho_l, b0_l
};

// REIN = false: one CTA per (m, block of 256 slots), the y form, double-float partials.
// REIN = true:  one CTA per m <= mR on slots 0 .. 255 (A.nblk = 1), Reinsch's form, FP64 partials.
template <int N, bool REIN>
__global__ void __launch_bounds__(DF_T) legendre_anal_df_kernel(DfArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    DfSmem<N, REIN> &S = *reinterpret_cast<DfSmem<N, REIN> *>(smem_raw);

    constexpr int NW = DF_T / 32;
    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    if (!REIN && m <= A.mR && A.s[blk * DF_T] < POLAR_SIN) return;  // the REIN launch covers it
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int slot = blk * DF_T + tid;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int64_t mstride = A.mmax + 1;

    double u = 0.0, y1 = 0.0, y2 = 0.0;
    int k = 0;
    if (active) {
        u = A.u[slot];
        double y0;
        sectoral_start(A.s[slot], A.alpha[base], m, y0, k);
        y2 = REIN ? y0 : -y0;  // D_{m-1} = lambda_m (Reinsch) or y_{m-2} = -y_m, with y1 = 0
    }
    // Sigma and D of this slot, as double-float columns (2g: re, 2g+1: im)
    {
        const int rn = active ? A.slotN[slot] : -1, rs = active ? A.slotS[slot] : -1;
#pragma unroll
        for (int g = 0; g < N / 2; ++g) {
            double2 dn = make_double2(0.0, 0.0), ds = make_double2(0.0, 0.0);
            if (g < A.nmaps) {
                const double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
                if (rn >= 0) dn = d[(int64_t)rn * mstride + m];
                if (rs >= 0) ds = d[(int64_t)rs * mstride + m];
            }
            S.X[0][2 * g][tid] = d2df(dn.x + ds.x);
            S.X[0][2 * g + 1][tid] = d2df(dn.y + ds.y);
            S.X[1][2 * g][tid] = d2df(dn.x - ds.x);
            S.X[1][2 * g + 1][tid] = d2df(dn.y - ds.y);
        }
    }

    for (int l0 = m; l0 <= L; l0 += DF_CHL) {
        const int nl = min(DF_CHL, L - l0 + 1);
        __syncthreads();
        if (tid < DF_CHL) {
            if (REIN) {
                const double3 c = (tid < nl) ? A.rein[base + (l0 - m) + tid] : make_double3(0.0, 0.0, 0.0);
                S.co[0][tid] = c.x;
                S.co[1][tid] = c.y;
                S.co[2][tid] = c.z;
            } else {
                S.co[0][tid] = (tid < nl) ? A.alpha[base + (l0 - m) + tid] : 0.0;
            }
        }
        __syncthreads();
        for (int j0 = 0; j0 < DF_CHL; j0 += DF_G) {
            // 8 recurrence steps (past the end: no-op steps with zero values)
            const bool scaled = __any_sync(0xffffffffu, k < 0);
            float2 yv[DF_G];
            bool live = false;
#pragma unroll
            for (int jj = 0; jj < DF_G; ++jj) {
                const int j = j0 + jj;
                double y = 0.0;
                if (j < nl) {
                    if (REIN) {  // D_l = (1 + rho_l) D_{l-1} + g_l lambda_{l-1}, lambda_l = lambda_{l-1} + D_l
                        const double g = fma(-S.co[0][j], u, S.co[2][j]);
                        const double t = fma(g, y1, y2);
                        y2 = fma(S.co[1][j], y2, t);
                        y1 = y1 + y2;
                        y = y1;
                    } else {
                        const double t = fma(-u, y1, y1);
                        y = fma(S.co[0][j], t, -y2);
                        y2 = y1;
                        y1 = y;
                    }
                }
                const bool use = active && j < nl && !(scaled && k < 0);
                yv[jj] = use ? d2df(y) : make_float2(0.f, 0.f);
                live |= use;
            }
            if (((j0 + DF_G) & 15) == 0 && scaled && k < 0 && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                y1 *= 0x1p-512;
                y2 *= 0x1p-512;
                k += 1;
            }
            if (!__any_sync(0xffffffffu, live)) {
                if (lane < DF_G) {
#pragma unroll
                    for (int n = 0; n < N; ++n) S.red[warp][n][j0 + lane] = make_float2(0.f, 0.f);
                }
                continue;
            }
            // value i of this lane is step i ^ b, whose l - m parity is (i & 1) ^ (b & 1)
            const int b = lane & (DF_G - 1);
            xor_permute(yv, b);
            const int pe = b & 1;
#pragma unroll 4
            for (int n = 0; n < N; ++n) {
                const float2 xa = S.X[pe][n][tid], xb = S.X[pe ^ 1][n][tid];
                float2 p[DF_G];
#pragma unroll
                for (int i = 0; i < DF_G; ++i) p[i] = df_mul(yv[i], (i & 1) ? xb : xa);
                const float2 r = warp_reduce_scatter_df(p);
                if (lane < DF_G) S.red[warp][n][j0 + lane] = r;
            }
        }
        __syncthreads();
        // add the warps and write the block's partial: y sums as double-float pairs (the block
        // reduction multiplies by c_lm); Reinsch lambda sums divided by c_lm, in FP64
        for (int i = tid; i < nl * (N / 2); i += DF_T) {
            const int j = i % nl, g = i / nl;
            float2 re = S.red[0][2 * g][j], im = S.red[0][2 * g + 1][j];
#pragma unroll
            for (int w = 1; w < NW; ++w) {
                re = df_add(re, S.red[w][2 * g][j]);
                im = df_add(im, S.red[w][2 * g + 1][j]);
            }
            if (g < A.nmaps) {
                const int64_t ix = base + (l0 - m) + j;
                if (REIN) {
                    const double c = A.cfac[ix];
                    A.polar[(int64_t)g * A.polar_stride + ix] = make_double2(widen_df(re) / c, widen_df(im) / c);
                } else {
                    A.partial[(int64_t)blk * A.part_blk_stride + (int64_t)g * A.nalm + ix] =
                        make_float4(re.x, re.y, im.x, im.y);
                }
            }
        }
    }
}

// a_lm = c_lm * sum over blocks of (hi + lo).  The blocks are added in order as double-float
// pairs on the FP32 pipe (widening each partial to FP64 and adding there made this kernel
// FP64-bound: four conversions and four adds per complex value and block) and the sum is widened
// once.  Partial (block, map g, index i) sits at bk * blk_stride + g * map_stride + i * idx_stride:
// [block][map][index] from the double-float kernel, [block][index][map] from the tensor-core one;
// threads walk the innermost of the two.  For i < fp64_lim (m <= mR of a polar plan) the Reinsch
// kernel's FP64 partial polar[g * polar_stride + i], split into hi + lo, stands for blocks
// 0 .. polar_blocks - 1.
__global__ void reduce_blocks_df_kernel(const float4 *__restrict__ partial, const double2 *__restrict__ polar,
                                        int64_t polar_stride, int polar_blocks, const double *__restrict__ cfac,
                                        double2 *__restrict__ alm, int nblk, int64_t nalm, int nmaps, int lmax,
                                        int64_t blk_stride, int64_t map_stride, int64_t idx_stride, int64_t fp64_lim,
                                        int64_t i0, int64_t nidx)
{
    // coefficient indices i0 .. i0 + nidx - 1; the partial sums are indexed from i0
    const int64_t total = nidx * nmaps;
    const bool maps_inner = map_stride < idx_stride;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t g, il;
        if (maps_inner) {
            il = t / nmaps;
            g = t - il * nmaps;
        } else {
            g = t / nidx;
            il = t - g * nidx;
        }
        const int64_t i = i0 + il;
        const float4 *src = partial + g * map_stride + il * idx_stride;
        float2 re, im;
        int bk0 = 1;
        if (i < fp64_lim) {
            const double2 d = polar[g * polar_stride + i];
            re = d2df(d.x);
            im = d2df(d.y);
            bk0 = polar_blocks;
        } else {
            const float4 v = src[0];
            re = make_float2(v.x, v.y);
            im = make_float2(v.z, v.w);
        }
#pragma unroll 4
        for (int bk = bk0; bk < nblk; ++bk) {
            const float4 v = src[(int64_t)bk * blk_stride];
            re = df_add(re, make_float2(v.x, v.y));
            im = df_add(im, make_float2(v.z, v.w));
        }
        const double c = cfac[i];
        alm[g * nalm + i] = make_double2(c * widen_df(re), i <= lmax ? 0.0 : c * widen_df(im));
    }
}

// Polar slots of the precision-form synthesis (eq. DeltaDef): for m <= mR, slots 0 .. 127 (the
// first block of the tensor-core synthesis), Reinsch's form of the recurrence in FP64 and the
// sums E, O = sum over l of a_lm lambda_lm (l - m even, odd) in double-float on the FP32 pipe,
// for up to NM maps per launch; Delta_N = E + O, Delta_S = E - O.  One CTA per m.
constexpr int DFS_T = 128;  // threads = slots per CTA

struct DfSynArgs {
    const double2 *alm;    // [nmaps][nalm], first map of this launch
    double2 *delta;        // [nmaps][nrings][mmax+1]
    const int *slotN, *slotS;
    const double *u, *s, *alpha;
    const double3 *rein;   // Reinsch coefficients (beta_l, rho_l, b0_l) for m <= mR
    int nslots, lmax, mmax, nrings, nmaps;
    int64_t nalm;
};

template <int NM>
__global__ void __launch_bounds__(DFS_T) synth_df_polar_kernel(DfSynArgs A)
{
    __shared__ double co[3][DF_CHL];     // beta_l, rho_l, b0_l of the chunk
    __shared__ float4 sa[NM][DF_CHL];    // a_lm of the chunk as (re_hi, re_lo, im_hi, im_lo)
    const int m = blockIdx.x;
    const int tid = threadIdx.x;
    const int slot = (int)blockIdx.y * DFS_T + tid;  // block y of the polar slot blocks
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;

    double u = 0.0, y1 = 0.0, y2 = 0.0;  // y1: lambda_(l-1), y2: D_(l-1)
    int k = 0;
    if (active) {
        u = A.u[slot];
        double y0;
        sectoral_start(A.s[slot], A.alpha[base], m, y0, k);
        y2 = y0;  // D_(m-1) = lambda_m with lambda_(m-1) = 0
    }
    float2 acc[2][NM][2];  // [E, O][map][re, im]
#pragma unroll
    for (int p = 0; p < 2; ++p)
#pragma unroll
        for (int g = 0; g < NM; ++g) acc[p][g][0] = acc[p][g][1] = make_float2(0.f, 0.f);

    for (int l0 = m; l0 <= L; l0 += DF_CHL) {
        const int nl = min(DF_CHL, L - l0 + 1);
        __syncthreads();
        for (int i = tid; i < DF_CHL * (NM + 1); i += DFS_T) {
            const int row = i / DF_CHL, j = i - row * DF_CHL;
            const int64_t ix = base + (l0 - m) + j;
            if (row == 0) {
                const double3 c = (j < nl) ? A.rein[ix] : make_double3(0.0, 0.0, 0.0);
                co[0][j] = c.x;
                co[1][j] = c.y;
                co[2][j] = c.z;
            } else {
                const int g = row - 1;
                double2 a = make_double2(0.0, 0.0);
                if (j < nl && g < A.nmaps) a = A.alm[(int64_t)g * A.nalm + ix];
                const float2 re = d2df(a.x), im = d2df(m == 0 ? 0.0 : a.y);
                sa[g][j] = make_float4(re.x, re.y, im.x, im.y);
            }
        }
        __syncthreads();
        for (int j0 = 0; j0 < nl; j0 += 16) {
            const bool scaled = __any_sync(0xffffffffu, k < 0);
            const int jn = min(j0 + 16, nl);
            // steps in pairs: j even is l - m even (l0 - m is a multiple of 32), j + 1 odd
            for (int j = j0; j < jn; j += 2) {
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    if (j + p < jn) {
                        // D_l = (1 + rho_l) D_(l-1) + g_l lambda_(l-1), lambda_l = lambda_(l-1) + D_l
                        const double gl = fma(-co[0][j + p], u, co[2][j + p]);
                        const double t = fma(gl, y1, y2);
                        y2 = fma(co[1][j + p], y2, t);
                        y1 = y1 + y2;
                        const float2 yd = (active && !(scaled && k < 0)) ? d2df(y1) : make_float2(0.f, 0.f);
#pragma unroll
                        for (int g = 0; g < NM; ++g) {
                            const float4 a = sa[g][j + p];
                            acc[p][g][0] = df_add(acc[p][g][0], df_mul(yd, make_float2(a.x, a.y)));
                            acc[p][g][1] = df_add(acc[p][g][1], df_mul(yd, make_float2(a.z, a.w)));
                        }
                    }
                }
            }
            if (scaled && k < 0 && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                y1 *= 0x1p-512;
                y2 *= 0x1p-512;
                k += 1;
            }
        }
    }
    if (active) {
        const int rn = A.slotN[slot], rs = A.slotS[slot];
        const int64_t mstride = A.mmax + 1;
#pragma unroll
        for (int g = 0; g < NM; ++g) {
            if (g >= A.nmaps) continue;
            const double er = widen_df(acc[0][g][0]), ei = widen_df(acc[0][g][1]);
            const double orr = widen_df(acc[1][g][0]), oi = widen_df(acc[1][g][1]);
            double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
            if (rn >= 0 && SHT_CHK(rn < A.nrings && m <= A.mmax))
                d[(int64_t)rn * mstride + m] = make_double2(er + orr, ei + oi);
            if (rs >= 0 && SHT_CHK(rs < A.nrings && m <= A.mmax))
                d[(int64_t)rs * mstride + m] = make_double2(er - orr, ei - oi);
        }
    }
}

template <int N, bool REIN>
cudaError_t configure_df()
{
    const int smem = (int)sizeof(DfSmem<N, REIN>);
    cudaError_t e =
        cudaFuncSetAttribute(legendre_anal_df_kernel<N, REIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)  // all of the unified L1 as shared memory: as many CTAs per SM as it holds
        e = cudaFuncSetAttribute(legendre_anal_df_kernel<N, REIN>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

// grid: every (m, block) for the y form; m = 0 .. mR on block 0 for the Reinsch form
template <int N, bool REIN>
cudaError_t launch_df_group(const Plan &p, DfArgs A, cudaStream_t st)
{
    const unsigned grid = REIN ? (unsigned)(A.mR + 1) : (unsigned)((p.mmax + 1) * A.nblk);
    legendre_anal_df_kernel<N, REIN><<<grid, DF_T, (int)sizeof(DfSmem<N, REIN>), st>>>(A);
    return cudaGetLastError();
}

DfArgs df_args(const Plan &p)
{
    DfArgs A{};
    A.slotN = p.d_slotN;
    A.slotS = p.d_slotS;
    A.u = p.d_u;
    A.s = p.d_s;
    A.alpha = p.d_alpha;
    A.cfac = p.d_cfac;
    A.rein = p.d_rein;
    A.nslots = p.nslots;
    A.nblk = (p.nslots + DF_T - 1) / DF_T;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    A.nrings = p.nrings;
    A.mR = p.polar_first_slot ? p.mR : -1;
    A.nalm = p.nalm;
    return A;
}

}  // namespace

cudaError_t launch_reduce_blocks_df(const float4 *partial, const double2 *polar, int64_t polar_stride,
                                    int polar_blocks, const double *cfac, double2 *alm, int nblk, int64_t nalm,
                                    int nmaps, int lmax, int64_t blk_stride, int64_t map_stride, int64_t idx_stride,
                                    int64_t fp64_lim, cudaStream_t st, int64_t i0, int64_t nidx)
{
    if (nidx < 0) nidx = nalm - i0;
    const int64_t total = nidx * nmaps;
    const int rgrid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
    reduce_blocks_df_kernel<<<rgrid, 256, 0, st>>>(partial, polar, polar_stride, polar_blocks, cfac, alm, nblk, nalm,
                                                   nmaps, lmax, blk_stride, map_stride, idx_stride, fp64_lim, i0, nidx);
    return cudaGetLastError();
}

// The precision-form synthesis of the polar slots 0 .. 127 for m <= mR (nothing when the plan's
// first ring is not polar), up to 8 maps per launch.
cudaError_t launch_legendre_synth_df_polar(const Plan &p, const double2 *alm, double2 *delta, int nmaps,
                                           cudaStream_t st, int *nlaunch)
{
    *nlaunch = 0;
    if (p.mR < 0 || !p.polar_first_slot) return cudaSuccess;
    DfSynArgs A{};
    A.slotN = p.d_slotN;
    A.slotS = p.d_slotS;
    A.u = p.d_u;
    A.s = p.d_s;
    A.alpha = p.d_alpha;
    A.rein = p.d_rein;
    A.nslots = p.nslots;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    A.nrings = p.nrings;
    A.nalm = p.nalm;
    const int64_t dstride = (int64_t)p.nrings * (p.mmax + 1);
    for (int g0 = 0; g0 < nmaps;) {
        const int nm = std::min(8, nmaps - g0);
        A.nmaps = nm;
        A.alm = alm + (int64_t)g0 * p.nalm;
        A.delta = delta + (int64_t)g0 * dstride;
        if (nm > 4)
            synth_df_polar_kernel<8><<<dim3((unsigned)(p.mR + 1), (unsigned)p.polar_syn_blocks), DFS_T, 0, st>>>(A);
        else
            synth_df_polar_kernel<4><<<dim3((unsigned)(p.mR + 1), (unsigned)p.polar_syn_blocks), DFS_T, 0, st>>>(A);
        ++*nlaunch;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        g0 += nm;
    }
    return cudaSuccess;
}

cudaError_t configure_df_kernels()
{
    cudaError_t e = configure_df<32, false>();
    if (e == cudaSuccess) e = configure_df<16, false>();
    if (e == cudaSuccess) e = configure_df<8, false>();
    if (e == cudaSuccess) e = configure_df<32, true>();
    if (e == cudaSuccess) e = configure_df<16, true>();
    if (e == cudaSuccess) e = configure_df<8, true>();
    return e;
}

int legendre_anal_df_polar_slots() { return DF_T; }

// The Reinsch-form analysis of slots 0 .. 255 for m <= mR of a polar plan, in double-float:
// a_lm / c_lm of map g at polar[g * polar_stride + index], index < index(mR + 1, mR + 1),
// for groups of SHT_TUNE_DF_MAPS maps.
cudaError_t launch_legendre_anal_df_polar(const Plan &p, const double2 *delta, double2 *polar, int64_t polar_stride,
                                          int nmaps, cudaStream_t st, int *nlaunch)
{
    *nlaunch = 0;
    DfArgs A = df_args(p);
    if (A.mR < 0) return cudaSuccess;
    A.nblk = 1;
    A.polar_stride = polar_stride;
    const int64_t dstride = (int64_t)p.nrings * (p.mmax + 1);
    for (int g0 = 0; g0 < nmaps;) {
        const int nm = std::min(p.tune[SHT_TUNE_DF_MAPS], nmaps - g0);
        A.nmaps = nm;
        A.delta = delta + (int64_t)g0 * dstride;
        A.polar = polar + (int64_t)g0 * polar_stride;
        cudaError_t e = nm > 8 ? launch_df_group<32, true>(p, A, st)
                        : nm > 4 ? launch_df_group<16, true>(p, A, st)
                                 : launch_df_group<8, true>(p, A, st);
        ++*nlaunch;
        if (e != cudaSuccess) return e;
        g0 += nm;
    }
    return cudaSuccess;
}

int legendre_anal_df_nblk(const Plan &p) { return (p.nslots + DF_T - 1) / DF_T; }

size_t legendre_anal_df_partial_bytes(const Plan &p, int nmaps)
{
    return (size_t)legendre_anal_df_nblk(p) * (size_t)nmaps * (size_t)p.nalm * sizeof(float4);
}

// The precision-form analysis: double-float CTAs for every non-polar slot block, the Reinsch-form
// CTAs for block 0 when it is polar (m <= mR), then the block reduction.
cudaError_t launch_legendre_anal_df(const Plan &p, const double2 *delta, double2 *alm, void *partial, int nmaps,
                                    cudaStream_t st, int *nlaunch)
{
    *nlaunch = 0;
    DfArgs A = df_args(p);
    A.part_blk_stride = (int64_t)nmaps * p.nalm;
    const int64_t dstride = (int64_t)p.nrings * (p.mmax + 1);
    int g0 = 0;
    while (g0 < nmaps) {
        const int nm = std::min(p.tune[SHT_TUNE_DF_MAPS], nmaps - g0);
        A.nmaps = nm;
        A.delta = delta + (int64_t)g0 * dstride;
        A.partial = (float4 *)partial + (int64_t)g0 * p.nalm;
        cudaError_t e = nm > 8 ? launch_df_group<32, false>(p, A, st)
                        : nm > 4 ? launch_df_group<16, false>(p, A, st)
                                 : launch_df_group<8, false>(p, A, st);
        ++*nlaunch;
        if (e != cudaSuccess) return e;
        g0 += nm;
    }
    int64_t fp64_lim = 0;
    if (A.mR >= 0) {  // FP64 partials in place of block 0 for m <= mR (16 bytes, as a float4)
        int n = 0;
        cudaError_t e = launch_legendre_anal_df_polar(p, delta, (double2 *)partial, p.nalm, nmaps, st, &n);
        *nlaunch += n;
        if (e != cudaSuccess) return e;
        fp64_lim = (int64_t)(A.mR + 1) * (2 * (int64_t)p.lmax + 3 - (A.mR + 1)) / 2;  // index(mR+1, mR+1)
    }
    cudaError_t e = launch_reduce_blocks_df((const float4 *)partial, (const double2 *)partial, p.nalm, 1, p.d_cfac,
                                            alm, A.nblk, p.nalm, nmaps, p.lmax, A.part_blk_stride, p.nalm, 1,
                                            fp64_lim, st);
    ++*nlaunch;
    return e;
}

namespace {
SHT_CHECK_TAKE_DEF(take_check)
}  // namespace
cudaError_t take_check_word_df(int *w) { return take_check(w); }

}  // namespace sht
