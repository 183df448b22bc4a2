// Precision form of the Legendre synthesis (eq. DeltaDef): the lambda
// recurrence stays in FP64, the sum over l runs on the tensor cores.
//
// For one m, the sum Delta_m(r) = sum_l a_lm lambda_lm(r) over a block of 128
// ring slots and up to 16 maps is the matrix product of eq. (matrix_vec):
// [128 slots x l] . [l x 2 maps (re, im)], split by the parity of l - m into
// E (even) and O (odd) so that Delta_N = E + O, Delta_S = E - O.
//
// Exactness.  Both operands are cut into S = 7 balanced base-128 digits:
// v = 2^(E-6) sum_s d_s 2^(-7 s), |d_s| <= 64 (48 bits, rounded), with one
// scale exponent E per (m, slot block) for the recurrence values y = lambda / c
// and one per (m, map column) for c_lm a_lm.  The y exponent is the measured
// maximum of |y| over the block and all l (tc_ymax_kernel, once per plan,
// running the same recurrence): an a priori bound such as
// |lambda_lm| <= sqrt((2l+1)/4pi) can leave the leading digits empty by ten
// bits and push the significant bits into the small digit classes.  One scale
// per column is coarse for a red spectrum: at high l, c a is ~2^-12 of the
// column maximum and keeps ~12 bits fewer, which is why 7 digits are used (with
// 6 digits and products i + j <= 5 the map error reached 9e-10 of its RMS at
// lmax = 4096, spread evenly in relative terms over all m).
// Each digit d_s 2^(-7 s) is exact in bf16.  Products of digit pairs (i, j)
// with i + j <= 6 are accumulated by tcgen05.mma (kind::f16, bf16 inputs,
// FP32 accumulators in tensor memory) into five accumulators per parity:
// classes i + j = 0, 1, 2 and 3 each alone (class 0: integers of at most 2^24
// for up to 4096 terms, exact; classes 1-3: multiples of 2^-7w well inside 24
// bits, exact in practice) and classes 4..6 together.  The tensor core sums
// the 16 products of one MMA exactly when they share one scale, but it aligns
// a smaller addend to the accumulator and truncates: a probe showed products
// 2^-14 below the rest of their sum keeping only ~16 bits, and with classes 3-5
// merged the truncation bias reached 2.3e-9 of the output RMS at lmax = 4096
// (1.3e-10 with class 3 apart).  The epilogue adds the five in FP64 and
// applies 2^(E_y + E_a - 12).  Dropped products (i + j >= 7) and the 48-bit
// rounding stay near 2^-48 of the largest term.  Five accumulators of N
// columns per parity need 10 N <= 320 of the 512 tensor-memory columns, so
// one CTA runs per SM.
//
// Per CTA (one m, 128 slots, 416 threads in three warp groups), per chunk of 32 l:
//   1. the recurrence warps run 32 steps of the two-instruction y recurrence (see
//      legendre.cu), one slot per thread, and write the values to a y stage in shared memory;
//   2. the split warps cut each value into digits with integer and FP32 operations, store
//      them as the bf16 A tiles [parity][digit] of the chunk's stage and copy in the a_lm digit
//      tiles (prepared by tc_split_b_kernel);
//   3. one lane of the issuing warp issues the 2 x 28 MMAs (M = 128, N = 16 or 32, K = 16) and
//      commits them to the stage's mbarrier.
// y values and tiles are double-buffered, so the FP64 recurrence of chunk c + 1 runs while
// chunk c is split and multiplied: with one CTA per SM (tensor memory and shared memory
// both allow one), a single warp group could not keep the FP64 pipe busy between its
// integer work.
// Polar CTAs (Reinsch form, see legendre.cu) are left to the FP64 kernel.
#include "sht_internal.h"

#include <cuda_bf16.h>

#include <algorithm>

namespace sht {
namespace {

constexpr int TC_T = 128;           // slots per CTA = MMA M
#ifndef TC_DIGITS
#define TC_DIGITS 7
#endif
constexpr int TC_S = TC_DIGITS;     // digits per operand
static_assert(TC_S >= 6 && TC_S <= 7, "the digit split needs 53 - (7 S - 1) >= 1 and class-0 sums below 2^24");
constexpr int TC_CH = 32;           // l per chunk: 16 even + 16 odd
constexpr int TC_ATILE = 128 * 16 * 2;  // bytes of one [128 x 16] bf16 tile
constexpr long long WAIT_POLLS = 1ll << 26;
constexpr int TC_NCLS = 8;  // synthesis accumulator blocks per parity: digit classes 0 .. 7, one each
#ifndef TC_MAXW
#define TC_MAXW (TC_S - 1)  // highest digit class i + j accumulated
#endif

#include "recurrence.cuh"

__device__ __forceinline__ double pow2i_safe(int e)  // 2^e, 0 below the normal range
{
    return e < -1022 ? 0.0 : pow2i(min(e, 1023));
}

// sum over the S digit positions of 64 * 128^s: added to a signed F in (-2^B, 2^B], it makes
// every 7-bit field of the sum a digit plus 64 (the carries of the balanced representation are
// those of the one addition)
__host__ __device__ constexpr unsigned long long digit_bias()
{
    unsigned long long k = 0;
    for (int i = 0; i < TC_S; ++i) k = k * 128 + 64;
    return k;
}

// v * 2^(B - E), B = 7 S - 1 bits, rounded to the nearest integer, as S balanced base-128
// digits (most significant first), each returned as the float d_s * 2^(-7 s), so that
// v = 2^(E - 6) sum_s d_s 2^(-7 s) whatever S is.  |d_s| <= 64, and each float has at most
// 8 significant bits, so its upper 16 bits are its exact bf16.  Integer and FP32 pipes only:
// a field u = d + 64 becomes a float by OR-ing it into 2^23 and one exact FMA.
__device__ __forceinline__ void split_digits(double v, int E, float out[TC_S])
{
    constexpr int B = 7 * TC_S - 1;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    long long Fs = 0;
    if (ex != 0) {
        const int sh = 1075 - B + E - ex;  // v = mant 2^(ex - 1075)
        const unsigned long long mant = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
        unsigned long long F;
        if (sh >= 64)
            F = 0;
        else if (sh >= 53 - B)
            F = (mant + (1ull << (sh - 1))) >> sh;  // |v| < 2^E gives sh >= 53 - B, so F <= 2^B
        else
            F = (1ull << B) - 1;  // outside the bound: saturate
        Fs = (bits >> 63) ? -(long long)F : (long long)F;
    }
    const unsigned long long G = (unsigned long long)Fs + digit_bias();  // >= 0, top field <= 128
    const uint32_t lo = (uint32_t)G, hi = (uint32_t)(G >> 32);
#pragma unroll
    for (int i = 0; i < TC_S; ++i) {
        const int j = TC_S - 1 - i;  // field index, least significant first
        const int b0 = 7 * j;
        uint32_t u;
        if (j == TC_S - 1)
            u = (b0 >= 32) ? (hi >> (b0 - 32)) : __funnelshift_r(lo, hi, b0);  // top field: no mask
        else if (b0 + 7 <= 32)
            u = (lo >> b0) & 127u;
        else if (b0 >= 32)
            u = (hi >> (b0 - 32)) & 127u;
        else
            u = __funnelshift_r(lo, hi, b0) & 127u;
        const float sc = __int_as_float((127 - 7 * i) << 23);                   // 2^(-7 i)
        out[i] = fmaf(__uint_as_float(0x4B000000u | u), sc, -8388672.0f * sc);  // (u - 64) 2^(-7 i)
    }
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// a + b = s + e exactly (TwoSum), in _rn operations so that nothing is contracted
__device__ __forceinline__ float2 two_sum_rn(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return make_float2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// a + b for double-float pairs: TwoSum of the high parts, the low parts added, renormalised
__device__ __forceinline__ float2 df_add2(float2 a, float2 b)
{
    const float2 s = two_sum_rn(a.x, b.x);
    const float e = __fadd_rn(s.y, __fadd_rn(a.y, b.y));
    const float h = __fadd_rn(s.x, e);
    return make_float2(h, __fsub_rn(e, __fsub_rn(h, s.x)));
}

// float -> double from the bit pattern (integer pipe; an F2F conversion takes an FP64 issue slot):
// normal floats exactly, zero and subnormals (far below every value kept here) as 0
__device__ __forceinline__ double widen_f(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t ex = (b >> 23) & 0xffu;
    const uint32_t hi = (b & 0x80000000u) | ((ex + (1023u - 127u)) << 20) | ((b & 0x7FFFFFu) >> 3);
    return ex ? __hiloint2double((int)hi, (int)(b << 29)) : 0.0;
}

// the double-float v times 2^e as one double: the scaling in FP32 (exact) where both parts stay
// within its range, otherwise after widening
__device__ __forceinline__ double df_out(float2 v, int e)
{
    if (e >= -100 && e <= 96) {
        const float sc = __int_as_float((e + 127) << 23);
        return widen_f(__fmul_rn(v.x, sc)) + widen_f(__fmul_rn(v.y, sc));
    }
    return (widen_f(v.x) + widen_f(v.y)) * pow2i_safe(e);
}

// tcgen05 shared-memory matrix descriptor: K-major, no swizzle; lbo = byte stride between core
// matrices along K, sbo = along M/N; version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// kind::f16 instruction descriptor: F32 accumulate, BF16 A and B, both K-major, M = 128
template <int N>
__device__ __forceinline__ uint32_t umma_idesc()
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

// 1 in one lane of the (converged) warp, 0 in the others
__device__ __forceinline__ uint32_t elect_one()
{
    uint32_t e;
    asm volatile("{\n .reg .pred p;\n .reg .b32 r;\n elect.sync r|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(e));
    return e;
}

// the MMA and the commit issued by the lane with issue != 0 while the whole warp runs the code, so
// that descriptors and addresses stay warp-uniform
__device__ __forceinline__ void umma_bf16_by(uint32_t issue, uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                             uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.b32 p, %4, 0;\n setp.ne.b32 q, %5, 0;\n"
        " @q tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc), "r"(issue));
}

__device__ __forceinline__ void umma_commit_by(uint32_t issue, uint64_t *mbar)
{
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.b32 q, %1, 0;\n"
        " @q tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}" ::"r"(smem_u32(mbar)),
        "r"(issue));
}

// bounded wait for completion of the given phase parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t parity)
{
    const uint32_t a = smem_u32(mbar);
    for (long long it = 0; it < WAIT_POLLS; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");  // acquire: no shared-memory access moves above a successful wait
        if (done) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

// Synthesis operands.  B stacks two a_lm digits along N: stack sb = [B_(2 sb) | B_(2 sb + 1)]
// (N2 = 2N columns, digit 7 zero), so one MMA A_a x stack b/2 adds class a + b to accumulator block
// a + b and class a + b + 1 to block a + b + 1: the accumulators of a parity are one run of 8 blocks
// of N columns, block c holding class c only.
template <int N>
struct TcTile {
    static constexpr int N2 = 2 * N;                          // columns of one B stack
    static constexpr int B_TILE = N2 * 16 * 2;                // bytes of one [N2 x 16] stack
    static constexpr int NSTK = (TC_S + 1) / 2;               // stacks per parity
    static constexpr int B_CHUNK = 2 * NSTK * B_TILE;         // a_lm digits of one chunk
    static constexpr int A_BYTES = 2 * TC_S * TC_ATILE;
    static constexpr int TMEM_COLS = (2 * TC_NCLS * N <= 128) ? 128 : (2 * TC_NCLS * N <= 256) ? 256 : 512;
};

struct TcArgs {
    const double2 *alm;      // [nmaps][nalm], first map of this group
    double2 *delta;          // [nmaps][nrings][mmax+1] (synthesis: written; analysis: read)
    const int *slotN, *slotS;
    const double *u, *s;
    const double *alpha, *cfac;
    const int *Ey;           // [mmax+1][nblk] scale exponent of y per slot block
    const int *first;        // [mmax+1][nblk] first chunk with a kept y value (nch: none)
    const double2 *ck_y;     // [mmax+1][nblk][128] (y1, y2) at chunk first & ~1 (plan-time checkpoint)
    const int *ck_k;         // [mmax+1][nblk][128] rescaling exponent k there
    int *Ea;                 // [mmax+1][N] scale exponent of c a
    const int64_t *chunk_base;  // [mmax+1] first chunk of each m
    const int *chunk_m;      // [total chunks] m of each chunk
    uint4 *bdig;             // [total chunks][B_CHUNK / 16]
    float4 *partial;         // analysis: [nblk][nalm][nmaps] (re_hi, re_lo, im_hi, im_lo) of a_lm / c_lm per block
    int *status;             // device status word (bit 0: an mbarrier wait timed out)
    int nslots, nblk, lmax, mmax, nrings, mR, nmaps;
    int polar_slots;         // analysis: slots the Reinsch-form kernel covers for m <= mR (mR < 0: none)
    int64_t nalm;
    int m0;                  // analysis: first m of this launch (an m-slab)
    int64_t idx0, nalm_part; // analysis: partial sums hold the indices idx0 .. idx0 + nalm_part - 1
};

// ---------------------------------------------------------------- a_lm side

// E_a[m][n] with |c_lm a_lm| < 2^E_a for all l (from exponent fields, no FP64 work)
template <int N>
__global__ void tc_scale_kernel(TcArgs A)
{
    __shared__ int s_max[N];
    const int m = blockIdx.x;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    if (threadIdx.x < N) s_max[threadIdx.x] = 0;
    __syncthreads();
    int mx[N];
#pragma unroll
    for (int n = 0; n < N; ++n) mx[n] = 0;
    for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
        const int64_t ix = base + (l - m);
        const int ec = dexp(A.cfac[ix]);
#pragma unroll
        for (int g = 0; g < N / 2; ++g) {
            if (g < A.nmaps) {
                const double2 a = A.alm[(int64_t)g * A.nalm + ix];
                const int er = dexp(a.x), ei = (m == 0) ? 0 : dexp(a.y);
                if (er) mx[2 * g] = max(mx[2 * g], er + ec);
                if (ei) mx[2 * g + 1] = max(mx[2 * g + 1], ei + ec);
            }
        }
    }
#pragma unroll
    for (int n = 0; n < N; ++n) atomicMax(&s_max[n], mx[n]);
    __syncthreads();
    if (threadIdx.x < N) {
        const int e = s_max[threadIdx.x];
        A.Ea[m * N + threadIdx.x] = e ? e - 2044 : -1000;
    }
}

// digits of c_lm a_lm for one (m, chunk) in the tile layout of the MMA B operand:
// [parity][stack][N2 x 16] bf16 with digit s in stack s / 2 at columns n + N (s & 1), core matrix
// (n2/8, k/8) at ((k/8) (N2/8) + n2/8) * 64 elements; digit 7 is zero.  Thread (parity, k/8, n)
// cuts the 8 values k/8 .. k/8 + 7 of its column: each digit's 8 bf16 are one core-matrix row,
// 16 contiguous bytes, stored as one vector.
template <int N>
__global__ void tc_split_b_kernel(TcArgs A)
{
    const int64_t chunk = blockIdx.x;
    const int m = A.chunk_m[chunk];
    const int c = (int)(chunk - A.chunk_base[m]);
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    constexpr int N2 = TcTile<N>::N2;
    uint4 *out = A.bdig + chunk * (TcTile<N>::B_CHUNK / 16);
    for (int t = threadIdx.x; t < 2 * 2 * N; t += blockDim.x) {
        const int n = t % N, kh = (t / N) & 1, eo = t / (2 * N);
        const int g = n >> 1;
        const int E = A.Ea[m * N + n];
        uint32_t pk[TC_S][4];  // per digit, 8 bf16 as 4 pairs
#pragma unroll
        for (int kk = 0; kk < 8; kk += 2) {
            float d0[TC_S], d1[TC_S];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int l = m + TC_CH * c + 2 * (8 * kh + kk + h) + eo;
                double v = 0.0;
                if (l <= L && g < A.nmaps) {
                    const int64_t ix = base + (l - m);
                    const double2 a = A.alm[(int64_t)g * A.nalm + ix];
                    const double comp = (n & 1) ? (m == 0 ? 0.0 : a.y) : a.x;
                    v = A.cfac[ix] * comp;
                }
                split_digits(v, E, h ? d1 : d0);
            }
            // the digit floats are bf16-exact: a bf16 pair is the upper halves of two floats
#pragma unroll
            for (int s = 0; s < TC_S; ++s) pk[s][kk >> 1] = __byte_perm(__float_as_uint(d0[s]), __float_as_uint(d1[s]), 0x7632);
        }
#pragma unroll
        for (int s = 0; s < 2 * TcTile<N>::NSTK; ++s) {
            const int n2 = n + N * (s & 1);
            const int off = (kh * (N2 / 8) + (n2 >> 3)) * 64 + (n2 & 7) * 8;  // elements; a multiple of 8
            out[((eo * TcTile<N>::NSTK + (s >> 1)) * (N2 * 16) + off) / 8] =
                s < TC_S ? make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]) : make_uint4(0u, 0u, 0u, 0u);
        }
    }
}

// ---------------------------------------------------------------- y scale per (m, slot block)

// max over the block's slots and all l (terms kept: k = 0) of the biased exponent of y,
// written as E with |y| < 2^E (-1000 when every value is dropped), and the first chunk of 32 l
// in which any slot keeps a value (every earlier chunk contributes exactly zero).  Same
// recurrence, operation for operation (y' = (alpha x) y - y2 with alpha x = alpha - alpha u), as
// tc_synth_kernel, so that both see the same rescaling steps.
__global__ void __launch_bounds__(TC_T) tc_ymax_kernel(TcArgs A, int *Ey_out, int *first_out)
{
    __shared__ double s_al[TC_CH];
    __shared__ int s_max, s_first;
    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    const int tid = threadIdx.x;
    const int slot = blk * TC_T + tid;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int nch = (L - m + TC_CH) / TC_CH;
    if (tid == 0) {
        s_max = 0;
        s_first = nch;
    }
    double u = 0.0, y1 = 0.0, y2 = 0.0;
    int k = 0;
    if (active) {
        u = A.u[slot];
        double y0;
        sectoral_start(A.s[slot], A.alpha[base], m, y0, k);
        y2 = -y0;
    }
    int mx = 0, fc = nch;
    for (int c = 0; c < nch; ++c) {
        const int l0 = m + TC_CH * c;
        __syncthreads();
        if (tid < TC_CH) s_al[tid] = (l0 + tid <= L) ? A.alpha[base + (l0 - m) + tid] : 0.0;
        __syncthreads();
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const bool scaled = __any_sync(0xffffffffu, k < 0);
            for (int j = 16 * h; j < 16 * h + 16; ++j) {
                const double ax = fma(-s_al[j], u, s_al[j]);  // alpha x, off the dependency chain
                const double y = fma(ax, y1, -y2);
                y2 = y1;
                y1 = y;
                if (l0 + j <= L && !(scaled && k < 0)) {
                    mx = max(mx, dexp(y));
                    fc = min(fc, c);
                }
            }
            if (scaled && k < 0 && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                y1 *= 0x1p-512;
                y2 *= 0x1p-512;
                k += 1;
            }
        }
    }
    atomicMax(&s_max, active ? mx : 0);
    atomicMin(&s_first, active ? fc : nch);
    __syncthreads();
    if (tid == 0) {
        Ey_out[m * A.nblk + blk] = s_max ? s_max - 1022 : -1000;
        first_out[m * A.nblk + blk] = s_first;
    }
}

// The recurrence state (y1, y2, k) of every slot at the start of 32-l chunk first & ~1 (even, so
// that it also starts a 64-l chunk of the analysis), by the same recurrence, operation for
// operation, as tc_ymax_kernel.  The tensor-core kernels start there: the chunks before hold
// only dropped values, and skipping their recurrence saves about a fifth of the FP64 steps at
// lmax = 4096 on HEALPix.
__global__ void __launch_bounds__(TC_T) tc_ckpt_kernel(TcArgs A, const int *first, double2 *ck_y, int *ck_k)
{
    __shared__ double s_al[TC_CH];
    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    const int tid = threadIdx.x;
    const int slot = blk * TC_T + tid;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int nch = (L - m + TC_CH) / TC_CH;
    const int c0 = min(first[m * A.nblk + blk], nch) & ~1;
    double u = 0.0, y1 = 0.0, y2 = 0.0;
    int k = 0;
    if (active) {
        u = A.u[slot];
        double y0;
        sectoral_start(A.s[slot], A.alpha[base], m, y0, k);
        y2 = -y0;
    }
    for (int c = 0; c < c0; ++c) {
        const int l0 = m + TC_CH * c;
        __syncthreads();
        if (tid < TC_CH) s_al[tid] = (l0 + tid <= L) ? A.alpha[base + (l0 - m) + tid] : 0.0;
        __syncthreads();
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const bool scaled = __any_sync(0xffffffffu, k < 0);
            for (int j = 16 * h; j < 16 * h + 16; ++j) {
                const double ax = fma(-s_al[j], u, s_al[j]);
                const double y = fma(ax, y1, -y2);
                y2 = y1;
                y1 = y;
            }
            if (scaled && k < 0 && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                y1 *= 0x1p-512;
                y2 *= 0x1p-512;
                k += 1;
            }
        }
    }
    const int64_t ci = (int64_t)(m * A.nblk + blk) * TC_T + tid;
    ck_y[ci] = make_double2(y1, y2);
    ck_k[ci] = k;
}

// ---------------------------------------------------------------- the synthesis kernel

// named barriers (id 0 is __syncthreads): count = threads taking part, a multiple of 32
__device__ __forceinline__ void bar_sync(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int count)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ bool bar_red_and(int id, int count, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

enum : int { BAR_FULL = 2, BAR_EMPTY = 4, BAR_SPLIT = 6 };  // FULL, EMPTY: one per stage

template <int N>
struct TcWs {
    static constexpr int A_BYTES = TcTile<N>::A_BYTES;                    // one stage of A tiles
    static constexpr int B_CHUNK = TcTile<N>::B_CHUNK;                    // one stage of B tiles
    static constexpr int Y_BYTES = TC_CH * TC_T * 8;                      // one stage of y values
    static constexpr int OFF_B = 2 * A_BYTES;
    static constexpr int OFF_Y = OFF_B + 2 * B_CHUNK;
    static constexpr int OFF_BAR = OFF_Y + 2 * Y_BYTES;
    static constexpr int SMEM = OFF_BAR + 64 + 1024;                      // + alignment slack
};

constexpr int TC_NT = 3 * TC_T;  // threads per synthesis CTA: 4 recurrence warps + 8 split warps

// The recurrence warps (threads 0-127, thread r = slot r of the block) of the tensor-core kernels:
// from the plan-time checkpoint at chunk cfirst & ~1 (earlier chunks hold only dropped values)
// they run the two-instruction y recurrence and write each live chunk's 32 values (0 where
// dropped) to y stage q & 1, laid out [32 l][YS doubles].  alpha comes from a register of lane j
// (warp shuffle), loaded one chunk ahead.  Stages are handed over with named barriers over all
// TC_NT threads: FULL (arrive here, the split warps wait) and EMPTY (the split warps arrive,
// wait here, only where a later chunk reuses the stage).
template <int YS>
__device__ __forceinline__ void recurrence_warps(const TcArgs &A, int m, int blk, int r, bool active, int64_t base,
                                                 int nch, int cfirst, double *ybuf)
{
    const int lane = r & 31;
    const int L = A.lmax;
    const int c0 = cfirst & ~1;
    double u = 0.0, y1 = 0.0, y2 = 0.0;
    int k = 0;
    if (active) {
        u = A.u[blk * TC_T + r];
        const int64_t ci = (int64_t)(m * A.nblk + blk) * TC_T + r;
        const double2 st = A.ck_y[ci];
        y1 = st.x;
        y2 = st.y;
        k = A.ck_k[ci];
    }
    double al_next = (m + TC_CH * c0 + lane <= L) ? A.alpha[base + TC_CH * c0 + lane] : 0.0;
    for (int c = c0; c < nch; ++c) {
        const int l0 = m + TC_CH * c;
        const double al_cur = al_next;
        {
            const int ln = l0 + TC_CH + lane;
            al_next = (c + 1 < nch && ln <= L) ? A.alpha[base + (ln - m)] : 0.0;
        }
        const int q = c - cfirst;  // live chunk index
        double *yb = ybuf + (size_t)(q & 1) * TC_CH * YS;
        if (q >= 2) bar_sync(BAR_EMPTY + (q & 1), TC_NT);  // the split warps read chunk q - 2
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const bool scaled = __any_sync(0xffffffffu, k < 0);
            const bool drop = scaled && k < 0;
            // Groups of 8 steps: the 8 factors alpha x = alpha (1 - u) first (they do not depend on y),
            // then the chain of 8 dependent DFMAs, then the 8 stores.  Each step adds one DFMA to the
            // dependency chain, and a warp issues in order: a store right after its y would hold the
            // warp until y is ready and leave the FP64 pipe without the next factors to work on.
#pragma unroll
            for (int j0 = 16 * h; j0 < 16 * h + 16; j0 += 8) {
                double ax[8], yv[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const double a = __shfl_sync(0xffffffffu, al_cur, j0 + j);
                    ax[j] = fma(-a, u, a);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const double y = fma(ax[j], y1, -y2);
                    y2 = y1;
                    y1 = y;
                    yv[j] = y;
                }
                if (q >= 0) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) yb[(j0 + j) * YS + r] = drop ? 0.0 : yv[j];
                }
            }
            if (drop && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                y1 *= 0x1p-512;
                y2 *= 0x1p-512;
                k += 1;
            }
        }
        if (q >= 0) bar_arrive(BAR_FULL + (q & 1), TC_NT);
    }
}

// Warp groups per CTA (one m, 128 slots, 416 threads):
//   recurrence warps 0-3 (recurrence_warps): thread r runs the FP64 recurrence of slot r and
//     writes each chunk's 32 values to a double-buffered y stage in shared memory;
//   split warps 4-11: thread (par, r) cuts the 16 values of parity par of slot r into digits and
//     stores row r of the parity's A tiles (double-buffered); all of them copy the chunk's a_lm
//     digit tiles and arrive on the stage's full mbarrier; at the end they read tensor memory,
//     warps 4-7 for the first half of the columns and warps 8-11 for the second;
//   warp 12: waits on the full mbarrier, and one elected lane issues the chunk's 2 x 28 MMAs
//     (warp-uniform descriptors) and commits them to the stage's done mbarrier.
// Stages: the y buffer is handed over with named barriers (FULL: recurrence arrives, split
// waits; EMPTY: split arrives, recurrence waits, only where a later chunk reuses the stage);
// the A/B tiles of a stage are rewritten after the done mbarrier of the MMAs that read them.
template <int N>
__global__ void __launch_bounds__(TC_NT + 32, 1) tc_synth_kernel(TcArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    using W = TcWs<N>;
    unsigned char *sA = smem;                               // [stage][parity][digit][128 x 16] bf16
    unsigned char *sB = smem + W::OFF_B;                    // [stage][parity][digit][N x 16] bf16
    double *ybuf = (double *)(smem + W::OFF_Y);             // [stage][32 l][128 slots]
    uint64_t *mbar = (uint64_t *)(smem + W::OFF_BAR);       // done[stage]: the stage's MMAs complete
    uint64_t *full = mbar + 2;                              // full[stage]: the stage's tiles written
    uint32_t *tslot = (uint32_t *)(mbar + 4);

    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    if (m <= A.mR && A.s[blk * TC_T] < POLAR_SIN) return;  // Reinsch CTAs run in FP64

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool rec = warp < 4, issuer = warp == TC_NT / 32;
    const int sp = tid - TC_T;                              // split-thread index 0..255
    const int r = rec ? tid : (sp & (TC_T - 1));            // slot within the block
    const int par = rec ? 0 : (sp >> 7);                    // split threads: parity of l - m they cut
    const int slot = blk * TC_T + r;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int nch = (L - m + TC_CH) / TC_CH;
    const int cfirst = A.first[m * A.nblk + blk];           // chunks before it hold only dropped values
    const int nlive = nch - cfirst;

    if (nlive <= 0) {  // every value dropped: Delta_m is zero on these rings
        if (!rec && !issuer && par == 0 && active) {
            const int rn = A.slotN[slot], rs = A.slotS[slot];
            const int64_t mstride = A.mmax + 1;
            for (int g = 0; g < A.nmaps; ++g) {
                double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
                if (rn >= 0 && SHT_CHK(rn < A.nrings)) d[(int64_t)rn * mstride + m] = make_double2(0.0, 0.0);
                if (rs >= 0 && SHT_CHK(rs < A.nrings)) d[(int64_t)rs * mstride + m] = make_double2(0.0, 0.0);
            }
        }
        return;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TcTile<N>::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[i])), "r"(1));         // commit
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(TC_NT - TC_T)); // split threads
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;

    bool ok = true;
    if (rec) {
        recurrence_warps<TC_T>(A, m, blk, r, active, base, nch, cfirst, ybuf);
    } else if (issuer) {
        // ------------------------------------------------ MMA issue (one lane of the last warp)
        // per chunk: wait until the stage's tiles are written, issue its 2 x 16 MMAs (per parity eo,
        // A digit a against B stack b/2 for a + b <= 6) and commit them to the stage's done barrier.  The whole warp runs the loop with warp-uniform
        // descriptors; one elected lane issues.
        const uint32_t idesc = umma_idesc<TcTile<N>::N2>();
        const uint64_t dA0 = umma_desc(smem_u32(sA), 16 * 128, 128);
        const uint64_t dB0 = umma_desc(smem_u32(sB), (TcTile<N>::N2 / 8) * 128, 128);
        const uint32_t issue = elect_one();
        for (int q = 0; q < nlive; ++q) {
            const int st = q & 1;
            if (ok && !mbar_wait(&full[st], (uint32_t)((q >> 1) & 1))) ok = false;
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint64_t aS = dA0 + (uint64_t)((st * W::A_BYTES) >> 4);  // address field: bytes / 16
            const uint64_t bS = dB0 + (uint64_t)((st * W::B_CHUNK) >> 4);
#pragma unroll
            for (int eo = 0; eo < 2; ++eo) {
#pragma unroll
                for (int a = 0; a < TC_S; ++a) {
#pragma unroll
                    for (int b = 0; b + a <= TC_MAXW; b += 2) {
                        // classes a + b and a + b + 1 into blocks a + b, a + b + 1; the a = 0 MMAs of the
                        // first live chunk write blocks 0-7 once each, so they start the sums
                        const bool first = (q == 0) && (a == 0);
                        umma_bf16_by(issue, tmem + (uint32_t)((eo * TC_NCLS + a + b) * N),
                                     aS + (uint64_t)(((eo * TC_S + a) * TC_ATILE) >> 4),
                                     bS + (uint64_t)(((eo * TcTile<N>::NSTK + b / 2) * TcTile<N>::B_TILE) >> 4), idesc,
                                     first ? 0u : 1u);
                    }
                }
            }
            umma_commit_by(issue, &mbar[st]);
        }
        if (lane == 0 && !ok) atomicOr(A.status, 1);
    } else {
        // ------------------------------------------------ split group
        const int64_t chunk0 = A.chunk_base[m];
        const int Ey = A.Ey[m * A.nblk + blk];
        constexpr int NS = TC_NT - TC_T;                 // split threads
        constexpr int BTOT = TcTile<N>::B_CHUNK / 16;   // uint4 of one chunk's B tiles
        constexpr int BV = (BTOT + NS - 1) / NS;
        for (int q = 0; q < nlive; ++q) {
            const int c = cfirst + q;
            const int st = q & 1;
            unsigned char *a_st = sA + st * W::A_BYTES;
            unsigned char *b_st = sB + st * W::B_CHUNK;
            uint4 breg[BV];
            const uint4 *bsrc = A.bdig + (chunk0 + c) * BTOT;
#pragma unroll
            for (int i = 0; i < BV; ++i)
                if (i * NS + sp < BTOT) breg[i] = bsrc[i * NS + sp];
            bar_sync(BAR_FULL + st, TC_NT);  // y of chunk q is in its stage
            const double *yb = ybuf + (size_t)st * TC_CH * TC_T;
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                uint32_t pk[TC_S][4];  // 8 values of this parity per digit, bf16 pairs
#pragma unroll
                for (int qq = 0; qq < 8; qq += 2) {
                    float d0[TC_S], d1[TC_S];
                    split_digits(yb[(16 * h + 2 * qq + par) * TC_T + r], Ey, d0);
                    split_digits(yb[(16 * h + 2 * qq + 2 + par) * TC_T + r], Ey, d1);
                    // the digit floats are bf16-exact: a bf16 pair is the upper halves of two floats
#pragma unroll
                    for (int s = 0; s < TC_S; ++s)
                        pk[s][qq >> 1] = __byte_perm(__float_as_uint(d0[s]), __float_as_uint(d1[s]), 0x7632);
                }
                if (h == 1 && q + 2 < nlive) bar_arrive(BAR_EMPTY + st, TC_NT);  // y stage read
                // the MMAs of chunk q - 2 read this stage's tiles: wait (bounded) before rewriting them
                // (after the first half is cut, which only reads the y stage)
                if (h == 0 && q >= 2 && ok && !mbar_wait(&mbar[st], (uint32_t)(((q >> 1) - 1) & 1))) ok = false;
                // k-group h of this parity's A tiles: core matrix (slot/8, h), row slot%8
                const int off = ((h * 16) + (r >> 3)) * 128 + (r & 7) * 16;
#pragma unroll
                for (int s = 0; s < TC_S; ++s)
                    *(uint4 *)(a_st + (par * TC_S + s) * TC_ATILE + off) = make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
            }
#pragma unroll
            for (int i = 0; i < BV; ++i)
                if (i * NS + sp < BTOT) ((uint4 *)b_st)[i * NS + sp] = breg[i];
            asm volatile("fence.proxy.async.shared::cta;");
            asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[st])) : "memory");
        }
        // the last commits cover every MMA issued: wait (bounded) before TMEM is read
        if (ok && !mbar_wait(&mbar[(nlive - 1) & 1], (uint32_t)(((nlive - 1) >> 1) & 1))) ok = false;
        ok = bar_red_and(BAR_SPLIT, NS, ok);
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (ok) {
            // accumulators: column (eo * 8 + class) * N + n, lane = slot within the block; this thread
            // takes columns [par N/2, (par + 1) N/2)
            // The 8 class blocks are added as double-float pairs on the FP32 pipe, smallest class
            // first, and each sum is widened once (bit operations and one DADD): widening and adding
            // every block in FP64 took 512 FP64-pipe instructions per thread, about 65K cycles of a
            // CTA's end during which the SM (one CTA each) could not start the next one.
            constexpr int NH = N / 2;
            const int lw = warp & 3;  // this warp may read lanes 32 lw .. 32 lw + 31
            float2 fac[2][NH];
#pragma unroll
            for (int eo = 0; eo < 2; ++eo)
#pragma unroll
                for (int n = 0; n < NH; ++n) fac[eo][n] = make_float2(0.f, 0.f);
#pragma unroll
            for (int eo = 0; eo < 2; ++eo) {
#pragma unroll
                for (int cls = TC_NCLS - 1; cls >= 0; --cls) {
#pragma unroll
                    for (int n0 = 0; n0 < NH; n0 += 8) {
                        uint32_t v[8];
                        const uint32_t addr = tmem + ((uint32_t)(lw * 32) << 16) +
                                              (uint32_t)((eo * TC_NCLS + cls) * N + par * NH + n0);
                        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                                     : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                                       "=r"(v[6]), "=r"(v[7])
                                     : "r"(addr));
                        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                        for (int t = 0; t < 8; ++t) {
                            const float2 sm = two_sum_rn(fac[eo][n0 + t].x, __uint_as_float(v[t]));
                            fac[eo][n0 + t] = make_float2(sm.x, __fadd_rn(fac[eo][n0 + t].y, sm.y));
                        }
                    }
                }
            }
            // Delta_N = E + O, Delta_S = E - O in double-float, scaled by 2^(E_y + E_a - 12) and widened
            // once per value: 1 FP64 instruction per value instead of a DMUL and a DADD
            if (active) {
                const int rn = A.slotN[slot], rs = A.slotS[slot];
                const int64_t mstride = A.mmax + 1;
#pragma unroll
                for (int gg = 0; gg < NH / 2; ++gg) {
                    const int g = par * (NH / 2) + gg;  // map
                    if (g < A.nmaps) {
                        const int er = Ey + A.Ea[m * N + 2 * g] - 12, ei = Ey + A.Ea[m * N + 2 * g + 1] - 12;
                        const float2 Er = fac[0][2 * gg], Ei = fac[0][2 * gg + 1];
                        const float2 Or = fac[1][2 * gg], Oi = fac[1][2 * gg + 1];
                        double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
                        if (rn >= 0 && SHT_CHK(rn < A.nrings && m <= A.mmax))
                            d[(int64_t)rn * mstride + m] =
                                make_double2(df_out(df_add2(Er, Or), er), df_out(df_add2(Ei, Oi), ei));
                        if (rs >= 0 && SHT_CHK(rs < A.nrings && m <= A.mmax))
                            d[(int64_t)rs * mstride + m] = make_double2(
                                df_out(df_add2(Er, make_float2(-Or.x, -Or.y)), er),
                                df_out(df_add2(Ei, make_float2(-Oi.x, -Oi.y)), ei));
                    }
                }
            }
        } else if (sp == 0) {
            atomicOr(A.status, 1);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                                "r"(TcTile<N>::TMEM_COLS));
}

// ---------------------------------------------------------------- the analysis kernel
//
// a_lm = c_lm sum over ring slots of y_lm(slot) X_m(slot), X = Sigma = Delta_N + Delta_S for even
// l - m and X = D = Delta_N - Delta_S for odd (eq. almdef, Algorithm 5).  For one m and a block
// of 128 slots this is the product [columns x slots] . [slots x l] (eq. matrix_vec transposed),
// run on the tensor cores with the map columns as the matrix rows: 64 rows (Sigma and D, re and
// im, of up to 16 maps), K = 16 slots per MMA, N = 32 values of l (one 32-l chunk, its 16
// even-parity values first).  Each row keeps the columns of its parity; the other half is
// computed and dropped.  The X digits of the whole block (the A operand) are cut once per CTA and
// the y digits (B operand) per K-step, so one launch serves 16 maps with one pass of the FP64
// recurrence.
//
// Digits as in the synthesis: 7 balanced base-128 digits of y (per-(m, block) exponent of
// tc_ymax_kernel) and of X (per-(m, block, row) exponent measured in the CTA), products
// i + j <= 6.  A tcgen05 MMA of 64 rows costs as much as one of 128, and N = 64 about as much as
// N = 32 (measured: 46 and 48 cycles), so each MMA stacks two digits on both sides:
// A = [X_a ; X_(a+1)] (rows 0-63, 64-127) and B = [Y_b | Y_(b+1)] (columns 0-31, 32-63), a and b
// even, X_7 = Y_7 = 0.  Its four quadrants collect classes a + b, a + b + 1 (two) and a + b + 2,
// in the accumulator region of t = a + b (0, 2, 4, 6).  The ten MMAs with a + b <= 6 cover all
// 28 products (and some of classes 7 and 8) instead of 28 MMAs, and every quadrant holds one
// class: over 128 slots its sum stays below 2^22, exact in FP32.  A chunk's four regions
// (4 x 64 columns) are double-buffered in tensor memory, so the epilogue of chunk q - 1 runs
// while the MMAs of chunk q are issued.  It adds the quadrants as double-float pairs (FP32 pipe)
// and writes the block's partial a_lm / c_lm, [block][index][map], which the block reduction
// sums and multiplies by c_lm.
//
// CTA: one m, 128 slots, 416 threads.  Warps 0-3 run the recurrence (recurrence_warps, y stage of
// 32 l).  Split warps 4-11 cut the y values of each K-step into the double-buffered y tiles and
// signal each tile's full barrier; warp 12 waits for it, and one elected lane issues the K-step's
// 10 MMAs and commits them to the buffer's done barrier, so the split never waits for MMA issue.  The split
// warps also read the previous chunk's accumulators (and release them to the issuer through the
// set's free barrier).  With 128 rows, row r sits in tensor-memory lane r: lanes 0-63 hold the top
// halves and lanes 64-127 the bottom halves of the same 64 rows, so the warps of lane quarters
// 2, 3 pass their sums to those of quarters 0, 1 through shared memory.

constexpr int TA_R = 64;                          // rows: [Sigma | D] x 16 maps x (re, im)
constexpr int TA_MAPS = 16;                       // maps per launch
constexpr int TA_XD = TC_S + 1;                   // digits of y in shared memory (the last one zero)
constexpr int TA_XDX = TC_S;                      // digits of X in shared memory (no zero digit: see below)
constexpr int TA_REG = 4;                         // accumulator regions per chunk (t = 0, 2, 4, 6)
constexpr int TA_N = 2 * TC_CH;                   // MMA N: two y digits of one 32-l chunk
constexpr int TA_YS = TC_T + 4;                   // y stage row stride (doubles): conflict-free pair loads
constexpr int TA_XBYTES = TA_XDX * TA_R * TC_T * 2;  // X digits, [slot / 8][digit][row / 8] core matrices
constexpr int TA_XKB = TA_XDX * (TA_R / 8) * 128; // bytes between 8-slot groups of the X operand
constexpr int TA_BDIG = (TC_CH / 8) * 128;        // one digit of one 8-slot group of a K-step's y tile
constexpr int TA_BKB = TA_XD * TA_BDIG;           // bytes between the two 8-slot groups of a y tile
constexpr int TA_BTILE = 2 * TA_BKB;              // one K-step's y tile, [slot / 8][digit][l / 8] core matrices
constexpr int TA_NB = 5;                          // y tile buffers (K-steps in flight between split and MMA)
constexpr int TA_SK = 2;                          // K-steps a split thread cuts per iteration
static_assert((TC_T / 16) % TA_SK == 0 && TA_SK < TA_NB, "K-steps per split iteration");
constexpr int TA_ACC = TA_REG * TA_N;             // tensor-memory columns of one chunk's accumulators
constexpr int TA_OFF_B = TA_XBYTES;
constexpr int TA_OFF_Y = TA_OFF_B + TA_NB * TA_BTILE;
constexpr int TA_OFF_X = TA_OFF_Y + 2 * TC_CH * TA_YS * 8;
constexpr int TA_OFF_E = TA_OFF_X + TA_R * 16 * 8;
constexpr int TA_OFF_BAR = TA_OFF_E + TA_R * 4;
constexpr int TA_NBAR = 2 * TA_NB + 4;            // done[NB], full[NB], tfree[2], afull[2]
constexpr int TA_SMEM = TA_OFF_BAR + TA_NBAR * 8 + 16 + 128;
constexpr int TA_TMEM_COLS = 512;                 // two chunks of accumulators
constexpr int TA_NEPI = 4 * 32;                   // epilogue threads (one warp per tensor-memory lane quarter)
constexpr int TA_NT = TC_NT + TA_NEPI + 32;       // 4 recurrence + 8 split + 4 epilogue warps + 1 MMA-issuing warp
enum : int { BAR_EPI = 7, BAR_PREP = 8 };         // epilogue warps; split + epilogue warps after the X digits
static_assert(2 * TA_ACC <= TA_TMEM_COLS, "two accumulator sets fit the allocation");
static_assert(TA_SMEM > 114 * 1024 && TA_SMEM <= 227 * 1024, "one CTA per SM (it holds all tensor memory)");
static_assert(TC_S == 7 && TA_XD == 8, "the digit stacks pair digits 0-1, 2-3, 4-5, 6-7");
static_assert(TA_OFF_B + 1024 <= TA_SMEM, "the last X group's stack [X_6 ; next] stays in shared memory");
static_assert(TC_MAXW == 6, "regions t = 0, 2, 4, 6 cover the products of classes up to 6");

__device__ __forceinline__ float2 two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return make_float2(s, (a - (s - bb)) + (b - bb));
}

// a + b for double-float pairs (TwoSum on the high parts)
__device__ __forceinline__ float2 df_sum(float2 a, float2 b)
{
    const float2 s = two_sum(a.x, b.x);
    return make_float2(s.x, s.y + a.y + b.y);
}

// Columns 16 es .. 16 es + 15 (this row's parity) of both y-digit halves of the 4 accumulator
// regions of chunk buffer tb, this warp's lanes: regions 0 and 1 summed as double-float pairs in
// the order (region 0 half 0, region 0 half 1, region 1 half 0, ...), classes roughly in decreasing
// size, regions 2 and 3 summed in FP32 and added once; the loads go out four at a time and are
// waited for together.
__device__ __forceinline__ void read_regions(uint32_t tmem, int quarter, int tb, int es, float2 acc[16])
{
#pragma unroll
    for (int t = 0; t < 16; ++t) acc[t] = make_float2(0.f, 0.f);
#pragma unroll
    for (int h0 = 0; h0 < 2 * TA_REG; h0 += 4) {
        uint32_t v[4][16];
#pragma unroll
        for (int hh = 0; hh < 4; ++hh) {
            const int h = h0 + hh, reg = h >> 1, half = h & 1;
            const uint32_t addr = tmem + ((uint32_t)(32 * quarter) << 16) +
                                  (uint32_t)(tb * TA_ACC + reg * TA_N + half * TC_CH + 16 * es);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[hh][0]), "=r"(v[hh][1]), "=r"(v[hh][2]), "=r"(v[hh][3]), "=r"(v[hh][4]), "=r"(v[hh][5]),
                  "=r"(v[hh][6]), "=r"(v[hh][7]), "=r"(v[hh][8]), "=r"(v[hh][9]), "=r"(v[hh][10]), "=r"(v[hh][11]),
                  "=r"(v[hh][12]), "=r"(v[hh][13]), "=r"(v[hh][14]), "=r"(v[hh][15])
                : "r"(addr));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (h0 == 0) {  // regions t = 0, 2 (classes 0-4): double-float
#pragma unroll
            for (int hh = 0; hh < 4; ++hh)
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const float2 sm = two_sum(acc[t].x, __uint_as_float(v[hh][t]));
                    acc[t] = make_float2(sm.x, acc[t].y + sm.y);
                }
        } else {
            // regions t = 4, 6 (classes 4-8, at most about 2^-28 of the sum): added in FP32 (an error
            // near 2^-52 of the sum), then into the pair once.  The bottom half of region 6 (lane
            // quarters 2, 3: classes 7 and 8 only) is left out: X has no zero digit 7 in shared memory
            // (the a = 6 stack reads other digits there), and those classes lie near 2^-49 of the sum.
            const bool bottom = quarter >= 2;
#pragma unroll
            for (int t = 0; t < 16; ++t) {
                const float small = (__uint_as_float(v[0][t]) + __uint_as_float(v[1][t])) +
                                    (bottom ? 0.f : __uint_as_float(v[2][t]) + __uint_as_float(v[3][t]));
                const float2 sm = two_sum(acc[t].x, small);
                acc[t] = make_float2(sm.x, acc[t].y + sm.y);
            }
        }
    }
}

// CTA: one m, 128 slots, 544 threads in five roles.
//   warps 0-3   recurrence (recurrence_warps, double-buffered y stage of 32 l);
//   warps 4-11  split: cut the X digits of the block once, then per K-step (16 slots) the y values
//               into one of TA_NB y tiles, and arrive on its full barrier;
//   warp 16     MMA issue: per K-step wait for the tile, issue its 10 MMAs, commit them to the
//               tile's done barrier (the split waits on it before reusing the tile), and after the
//               last K-step of a chunk also to the accumulator set's afull barrier;
//   warps 12-15 epilogue, one per tensor-memory lane quarter: wait for afull, read the set, release
//               it (tfree), add the bottom halves (lane quarters 2, 3) to the top ones (0, 1) through
//               shared memory and write the block's partial a_lm / c_lm.
// Every barrier phase a warp waits for can run at most one phase ahead of that wait, so the
// parity tests are unambiguous; every mbarrier wait is bounded and the epilogue warps agree on
// their outcome (bar.red) so that their named barriers stay balanced.
__global__ void __launch_bounds__(TA_NT, 1) tc_anal_kernel(TcArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sX = smem;                               // X digits (A operand), K-major
    unsigned char *sY = smem + TA_OFF_B;                    // [buffer] y digit tiles, K-major (B operand)
    double *ybuf = (double *)(smem + TA_OFF_Y);             // [stage][32 l][TA_YS]
    float2 *xch = (float2 *)(smem + TA_OFF_X);              // [16 columns][64 rows] bottom-half sums
    int *sEx = (int *)(smem + TA_OFF_E);                    // [64] row exponents (biased, 0: all zero)
    uint64_t *mbar = (uint64_t *)(smem + TA_OFF_BAR);       // done[NB]: MMAs of a y tile complete
    uint64_t *full = mbar + TA_NB;                          // full[NB]: a y tile written
    uint64_t *tfree = full + TA_NB;                         // tfree[2]: an accumulator set read out
    uint64_t *afull = tfree + 2;                            // afull[2]: an accumulator set complete
    uint32_t *tslot = (uint32_t *)(afull + 2);

    const int m = A.m0 + (int)(blockIdx.x / A.nblk);
    const int blk = (int)(blockIdx.x % A.nblk);
    if (m <= A.mR && blk * TC_T < A.polar_slots) return;  // the Reinsch-form kernel covers these slots

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool rec = warp < 4, splitw = warp >= 4 && warp < 12, epi = warp >= 12 && warp < 16;
    const bool issuer = warp == 16;
    const int sp = tid - TC_T;                              // split-thread index 0..255
    const int r = rec ? tid : (sp & (TC_T - 1));            // slot within the block
    const int slot = blk * TC_T + r;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int nch = (L - m + TC_CH) / TC_CH;
    const int cfirst = A.first[m * A.nblk + blk];           // chunks before it hold only dropped values
    const int nlive = nch - cfirst;
    const int nm = A.nmaps;
    float4 *part = A.partial + (int64_t)blk * A.nalm_part * nm - A.idx0 * nm;  // this block's [index][map]

    // l before the first live chunk: zero partials
    {
        const int64_t dead = (int64_t)min(TC_CH * cfirst, L - m + 1) * nm;
        float4 *p0 = part + base * nm;
        for (int64_t t = tid; t < dead; t += TA_NT) p0[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (nlive <= 0) return;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TA_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < TA_NB; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar[i])), "r"(1));          // commit
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(2 * TC_T));   // split threads
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tfree[i])), "r"(TA_NEPI));  // epilogue
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&afull[i])), "r"(1));         // commit
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (tid < TA_R) sEx[tid] = 0;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;

    bool ok = true;
    if (rec) {
        recurrence_warps<TA_YS>(A, m, blk, r, active, base, nch, cfirst, ybuf);
    } else if (issuer) {
        // ------------------------------------------------ MMA issue (one lane of the last warp)
        // per chunk q: wait until accumulator set q & 1 is read out (chunk q - 2), then per K-step
        // until its y tile is written, issue its 10 MMAs and commit them to the tile's done barrier,
        // and after the chunk's last K-step to the set's afull barrier.  The whole warp runs the
        // loop (descriptors are base values plus constant offsets of the address field, kept
        // warp-uniform); one elected lane issues.
        const uint32_t idesc = umma_idesc<TA_N>();  // M = 128, N = 64
        const uint64_t dA0 = umma_desc(smem_u32(sX), TA_XKB, 128);
        const uint64_t dB0 = umma_desc(smem_u32(sY), TA_BKB, 128);
        const uint32_t issue = elect_one();
        for (int q = 0; q < nlive && ok; ++q) {
            const int st = q & 1;
            if (q >= 2 && ok && !mbar_wait(&tfree[st], (uint32_t)(((q - 2) >> 1) & 1))) ok = false;
            ok = __all_sync(0xffffffffu, ok);
            const uint32_t dt = tmem + (uint32_t)(st * TA_ACC);
#pragma unroll 1
            for (int kk = 0; kk < TC_T / 16 && ok; ++kk) {
                const int gk = 8 * q + kk, b = gk % TA_NB;
                if (!mbar_wait(&full[b], (uint32_t)((gk / TA_NB) & 1))) ok = false;
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint64_t aK = dA0 + (uint64_t)((kk * 2 * TA_XKB) >> 4);  // address field: bytes / 16
                const uint64_t bK = dB0 + (uint64_t)((b * TA_BTILE) >> 4);
#pragma unroll
                for (int t = 0; t <= TC_MAXW; t += 2) {
#pragma unroll
                    for (int i = 0; i <= t; i += 2) {  // [X_i ; X_(i+1)] against [Y_(t-i) | Y_(t-i+1)]
                        const int j = t - i;
                        umma_bf16_by(issue, dt + (uint32_t)((t / 2) * TA_N), aK + (uint64_t)((i * (TA_R / 8) * 128) >> 4),
                                     bK + (uint64_t)((j * TA_BDIG) >> 4), idesc, (kk == 0 && i == 0) ? 0u : 1u);
                    }
                }
                umma_commit_by(issue, &mbar[b]);
                if (kk == TC_T / 16 - 1) umma_commit_by(issue, &afull[st]);
            }
        }
        if (lane == 0 && !ok) atomicOr(A.status, 1);
    } else if (splitw) {
        // ------------------------------------------------ X digits, then the y tiles
        const int Ey = A.Ey[m * A.nblk + blk];
        const int hh = sp >> 7;  // this thread's maps: 8 hh .. 8 hh + 7 of slot r (uniform per warp)
        double xv[2][8][2];      // [Sigma, D][map][re, im] -> row 32 s + 2 g + c
        {
            const int rn = active ? A.slotN[slot] : -1, rs = active ? A.slotS[slot] : -1;
            const int64_t mstride = A.mmax + 1;
#pragma unroll
            for (int gg = 0; gg < 8; ++gg) {
                const int g = 8 * hh + gg;
                double2 dn = make_double2(0.0, 0.0), ds = make_double2(0.0, 0.0);
                if (g < nm) {
                    const double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
                    if (rn >= 0 && SHT_CHK(rn < A.nrings)) dn = d[(int64_t)rn * mstride + m];
                    if (rs >= 0 && SHT_CHK(rs < A.nrings)) ds = d[(int64_t)rs * mstride + m];
                }
                xv[0][gg][0] = dn.x + ds.x;
                xv[0][gg][1] = dn.y + ds.y;
                xv[1][gg][0] = dn.x - ds.x;
                xv[1][gg][1] = dn.y - ds.y;
            }
        }
        // row exponents: a warp's maximum first, then one shared atomic per row and warp
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int gg = 0; gg < 8; ++gg)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const unsigned e = __reduce_max_sync(0xffffffffu, (unsigned)dexp(xv[s][gg][c]));
                    if (lane == 0 && e) atomicMax(&sEx[32 * s + 2 * (8 * hh + gg) + c], (int)e);
                }
        // the zero digit Y_7 (the second half of the last stack of every y tile); X has no digit 7:
        // the stack [X_6 ; X_7] of the a = 6 MMA reads the next 8-slot group's first digit there,
        // whose products land only in the bottom half of region t = 6 (classes 7 and 8), which the
        // epilogue leaves out
        for (int t = sp; t < TA_NB * 2 * TA_BDIG / 16; t += 2 * TC_T) {  // [buffer][8-slot group]
            const int g2 = t / (TA_BDIG / 16), rest = t - g2 * (TA_BDIG / 16);
            *(uint4 *)(sY + g2 * TA_BKB + TC_S * TA_BDIG + rest * 16) = make_uint4(0u, 0u, 0u, 0u);
        }
        bar_sync(BAR_PREP, 2 * TC_T + TA_NEPI);  // row exponents complete (the epilogue reads them too)
        // A operand, K-major: element (row, k = r) of digit q in core matrix (q * 8 + row / 8) of
        // 8-slot group r / 8, so that digits q and q + 1 form one 128-row operand
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int gg = 0; gg < 8; ++gg)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int row = 32 * s + 2 * (8 * hh + gg) + c;
                    const int e = sEx[row];
                    float d[TC_S];
                    split_digits(xv[s][gg][c], e ? e - 1022 : -1000, d);
                    const int off = (r >> 3) * TA_XKB + (row >> 3) * 128 + (row & 7) * 16 + (r & 7) * 2;
                    // each digit float is bf16-exact: its upper half is the bf16 (no conversion instruction)
#pragma unroll
                    for (int q = 0; q < TC_S; ++q)
                        *(unsigned short *)(sX + off + q * (TA_R / 8) * 128) = (unsigned short)(__float_as_uint(d[q]) >> 16);
                }

        const int w8 = warp - 4;  // 0..7
        // y tile element pair of this thread per K-step: row n (l - l0 = 2 (n % 16) + n / 16),
        // slots 2 kp, 2 kp + 1 of 8-slot half kh
        const int kp = lane & 3, nlo = lane >> 2, nhi = w8 & 3, kh = w8 >> 2;
        const int n = 8 * nhi + nlo;
        const int jrow = 2 * (n & 15) + (n >> 4);
        const int boff = kh * TA_BKB + nhi * 128 + nlo * 16 + kp * 4;
        for (int q = 0; q < nlive; ++q) {
            const int st = q & 1;
            bar_sync(BAR_FULL + st, TC_NT);  // y of chunk q is in its stage
            const double *yb = ybuf + (size_t)st * TC_CH * TA_YS;
#pragma unroll 1
            for (int kk = 0; kk < TC_T / 16; kk += TA_SK) {
                // TA_SK K-steps at a time: 2 TA_SK independent values per thread (one K-step at a
                // time left the split warps latency-bound: 181 against 175 ms at lmax 4096, 16 maps)
                double2 yy[TA_SK];
#pragma unroll
                for (int u = 0; u < TA_SK; ++u)
                    yy[u] = *reinterpret_cast<const double2 *>(yb + jrow * TA_YS + 16 * (kk + u) + 8 * kh + 2 * kp);
#pragma unroll
                for (int u = 0; u < TA_SK; ++u) {
                    const int gk = 8 * q + kk + u, b = gk % TA_NB;
                    // the MMAs of K-step gk - NB read buffer b: wait (bounded) before rewriting it
                    if (gk >= TA_NB && ok && !mbar_wait(&mbar[b], (uint32_t)(((gk / TA_NB) - 1) & 1))) ok = false;
                }
                float d0[TA_SK][TC_S], d1[TA_SK][TC_S];
#pragma unroll
                for (int u = 0; u < TA_SK; ++u) {
                    split_digits(yy[u].x, Ey, d0[u]);
                    split_digits(yy[u].y, Ey, d1[u]);
                }
                if (kk + TA_SK == TC_T / 16 && q + 2 < nlive) bar_arrive(BAR_EMPTY + st, TC_NT);  // y stage read
#pragma unroll
                for (int u = 0; u < TA_SK; ++u) {
                    const int b = (8 * q + kk + u) % TA_NB;
                    unsigned char *yt = sY + b * TA_BTILE;
#pragma unroll
                    for (int s = 0; s < TC_S; ++s)
                        *(uint32_t *)(yt + s * TA_BDIG + boff) =
                            __byte_perm(__float_as_uint(d0[u][s]), __float_as_uint(d1[u][s]), 0x7632);
                    asm volatile("fence.proxy.async.shared::cta;");
                    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[b])) : "memory");
                }
            }
        }
        if (!ok && lane == 0) atomicOr(A.status, 1);
    } else if (epi) {
        // ------------------------------------------------ epilogue, one warp per lane quarter
        // lane quarter qd: row 32 (qd & 1) + lane, the top half (qd < 2) or the bottom half (qd >= 2)
        // of its sums; Sigma rows (qd even) keep the even l - m columns 0-15, D rows the odd 16-31
        const int qd = warp & 3, es = qd & 1;
        const int erow = 32 * es + lane;
        const int eg = lane >> 1, ec = lane & 1;
        bar_sync(BAR_PREP, 2 * TC_T + TA_NEPI);  // row exponents complete
        // value = (top + bottom) 2^(Ey + Ex - 12): a power of two, applied to hi and lo
        const int ex = sEx[erow];
        const int e = A.Ey[m * A.nblk + blk] + (ex ? ex - 1022 : -1000) - 12;
        const float sc = (e >= -126 && e <= 127) ? __int_as_float((e + 127) << 23) : 0.f;
        for (int q = 0; q < nlive; ++q) {
            const int tb = q & 1;
            if (ok && !mbar_wait(&afull[tb], (uint32_t)((q >> 1) & 1))) ok = false;
            ok = bar_red_and(BAR_EPI, TA_NEPI, ok);  // the four warps agree (tcgen05.ld is warp-wide)
            asm volatile("tcgen05.fence::after_thread_sync;");
            float2 acc[16];
            if (ok) read_regions(tmem, qd, tb, es, acc);
            asm volatile("tcgen05.fence::before_thread_sync;");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&tfree[tb])) : "memory");
            bar_sync(BAR_EPI, TA_NEPI);  // the top warps have read the previous chunk's exchange
            if (ok && qd >= 2) {
#pragma unroll
                for (int t = 0; t < 16; ++t) xch[t * TA_R + erow] = acc[t];
            }
            bar_sync(BAR_EPI, TA_NEPI);  // bottom sums in xch
            if (ok && qd < 2 && eg < nm) {
                const int l0 = m + TC_CH * (cfirst + q);
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const float2 v = df_sum(acc[t], xch[t * TA_R + erow]);
                    const int l = l0 + 2 * t + es;
                    if (l <= L && SHT_CHK(base + (l - m) >= A.idx0 && base + (l - m) < A.idx0 + A.nalm_part)) {
                        float2 *dst = reinterpret_cast<float2 *>(part + (base + (l - m)) * nm + eg) + ec;
                        *dst = make_float2(v.x * sc, v.y * sc);
                    }
                }
            }
        }
        if (!ok && lane == 0) atomicOr(A.status, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                                "r"(TA_TMEM_COLS));
}

template <int N>
cudaError_t launch_group(const Plan &p, TcArgs A, cudaStream_t st)
{
    const int64_t nchunks = p.tc_total_chunks;
    tc_scale_kernel<N><<<p.mmax + 1, 256, 0, st>>>(A);
    tc_split_b_kernel<N><<<(unsigned)nchunks, 4 * N, 0, st>>>(A);  // one thread per (parity, k half, column)
    // one CTA per SM: its shared memory (two stages of tiles and y values) is over half the SM's,
    // and its accumulators take more than half of the tensor memory
    static_assert(TcWs<N>::SMEM > 114 * 1024 && TcWs<N>::SMEM <= 227 * 1024, "one CTA per SM");
    StageEvents ev(p, SHT_STAGE_TC_SYNTH_KERNEL, st);
    tc_synth_kernel<N><<<(unsigned)((p.mmax + 1) * A.nblk), TC_NT + 32, TcWs<N>::SMEM, st>>>(A);
    p.launches[SHT_STAGE_TC_SYNTH_KERNEL] += 1;
    ev.done();
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_tc_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(tc_synth_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         TcWs<32>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_synth_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, TcWs<16>::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc_anal_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TA_SMEM);
    return e;
}

// index(mR + 1, mR + 1): the a_lm of m <= mR, which the Reinsch kernel covers on a polar block 0
static int64_t polar_alm_count(const Plan &p)
{
    const int mR = p.polar_first_slot ? p.mR : -1;
    return mR < 0 ? 0 : (int64_t)(mR + 1) * (2 * (int64_t)p.lmax + 3 - (mR + 1)) / 2;
}

// The tensor-core analysis runs in m-slabs of about equal coefficient counts, each followed by its
// block reduction, so that the partial sums of one slab only are held at a time: at lmax 4096 all
// 32 blocks x 16 maps x 16 B per coefficient would take 69 GB, a slab about 1/8 of that.  The
// first slab covers every m of the Reinsch-form polar slots.  Boundaries: first m of each slab,
// then mmax + 1.
static std::vector<int> anal_slabs(const Plan &p)
{
    const int nblk = (p.nslots + TC_T - 1) / TC_T;
    const int64_t full = (int64_t)nblk * TA_MAPS * p.nalm * (int64_t)sizeof(float4);
    const int ns = full <= (int64_t(2) << 30) ? 1 : 8;
    const int64_t L = p.lmax;
    auto idx = [&](int64_t m) { return m * (2 * L + 3 - m) / 2; };
    const int mR = p.polar_first_slot ? p.mR : -1;
    std::vector<int> b{0};
    for (int k = 1; k < ns; ++k) {
        const int64_t want = p.nalm * k / ns;
        int m = b.back() + 1;
        while (m <= p.mmax && idx(m) < want) ++m;
        m = std::max(m, mR + 1);
        if (m > b.back() && m <= p.mmax) b.push_back(m);
    }
    b.push_back(p.mmax + 1);
    return b;
}

static int64_t slab_max_count(const Plan &p)
{
    const std::vector<int> b = anal_slabs(p);
    const int64_t L = p.lmax;
    auto idx = [&](int64_t m) { return m * (2 * L + 3 - m) / 2; };
    int64_t mx = 0;
    for (size_t k = 0; k + 1 < b.size(); ++k) mx = std::max(mx, (b[k + 1] > p.mmax ? p.nalm : idx(b[k + 1])) - idx(b[k]));
    return mx;
}

// partial a_lm / c_lm per 128-slot block for one group of up to 16 maps and one m-slab,
// [block][index][map] float4, then the Reinsch-form partials of the first polar slots for
// m <= mR, [map][index] double2
size_t tc_anal_partial_bytes(const Plan &p, int nmaps)
{
    const int nblk = (p.nslots + TC_T - 1) / TC_T;
    const size_t nm = (size_t)std::min(nmaps, TA_MAPS);
    return (size_t)nblk * nm * (size_t)slab_max_count(p) * sizeof(float4) +
           nm * (size_t)polar_alm_count(p) * sizeof(double2);
}

// The precision-form analysis on the tensor cores: per group of up to 16 maps, the double-float
// Reinsch-form kernel for the polar slots (m <= mR), then per m-slab the tensor-core kernel for every
// other slot block and the fixed-order block reduction of that slab into a_lm.
cudaError_t launch_legendre_anal_tc(const Plan &p, const double2 *delta, double2 *alm, void *partial, int nmaps,
                                    cudaStream_t st, int *nlaunch)
{
    *nlaunch = 0;
    TcArgs A{};
    A.slotN = p.d_slotN;
    A.slotS = p.d_slotS;
    A.u = p.d_u;
    A.s = p.d_s;
    A.alpha = p.d_alpha;
    A.Ey = p.d_tc_Ey;
    A.first = p.d_tc_Ey + (size_t)(p.mmax + 1) * ((p.nslots + TC_T - 1) / TC_T);
    A.ck_y = p.d_tc_ck_y;
    A.ck_k = p.d_tc_ck_k;
    A.status = p.d_status;
    A.nslots = p.nslots;
    A.nblk = (p.nslots + TC_T - 1) / TC_T;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    A.nrings = p.nrings;
    A.mR = p.polar_first_slot ? p.mR : -1;
    A.polar_slots = legendre_anal_df_polar_slots();
    static_assert(TC_T == 128, "the polar slots cover whole 128-slot blocks");
    A.nalm = p.nalm;
    const int64_t dstride = (int64_t)p.nrings * (p.mmax + 1);
    const int64_t fp64_lim = polar_alm_count(p);
    const std::vector<int> slabs = anal_slabs(p);
    const int64_t smax = slab_max_count(p);
    const int64_t L = p.lmax;
    auto idx = [&](int64_t m) { return m * (2 * L + 3 - m) / 2; };
    for (int g0 = 0; g0 < nmaps; g0 += TA_MAPS) {
        const int nm = std::min(TA_MAPS, nmaps - g0);
        A.nmaps = nm;
        A.delta = const_cast<double2 *>(delta) + (int64_t)g0 * dstride;
        A.partial = (float4 *)partial;
        cudaError_t e;
        double2 *polar = nullptr;
        if (fp64_lim > 0) {
            int n = 0;
            polar = (double2 *)(A.partial + (int64_t)A.nblk * nm * smax);
            e = launch_legendre_anal_df_polar(p, A.delta, polar, fp64_lim, nm, st, &n);
            *nlaunch += n;
            if (e != cudaSuccess) return e;
        }
        for (size_t k = 0; k + 1 < slabs.size(); ++k) {
            const int mlo = slabs[k], mhi = slabs[k + 1];
            A.m0 = mlo;
            A.idx0 = idx(mlo);
            A.nalm_part = (mhi > p.mmax ? p.nalm : idx(mhi)) - A.idx0;
            {
                StageEvents ev(p, SHT_STAGE_TC_ANAL_KERNEL, st);
                tc_anal_kernel<<<(unsigned)((mhi - mlo) * A.nblk), TA_NT, TA_SMEM, st>>>(A);
                p.launches[SHT_STAGE_TC_ANAL_KERNEL] += 1;
                ev.done();
            }
            ++*nlaunch;
            e = cudaGetLastError();
            if (e != cudaSuccess) return e;
            // partial (block, map g, index i) at block * nalm_part nm + (i - idx0) nm + g
            e = launch_reduce_blocks_df(A.partial, polar, fp64_lim, A.polar_slots / TC_T, p.d_cfac,
                                        alm + (int64_t)g0 * p.nalm, A.nblk, p.nalm, nm, p.lmax,
                                        (int64_t)nm * A.nalm_part, 1, nm, fp64_lim, st, A.idx0, A.nalm_part);
            ++*nlaunch;
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Per-(m, slot block) y exponents for the precision form (synchronous, once per plan).
cudaError_t build_tc_scales(Plan &p)
{
    if (p.d_tc_Ey) return cudaSuccess;
    TcArgs A{};
    A.u = p.d_u;
    A.s = p.d_s;
    A.alpha = p.d_alpha;
    A.nslots = p.nslots;
    A.nblk = (p.nslots + TC_T - 1) / TC_T;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    int *ey = nullptr;  // [2][mmax + 1][nblk]: y exponents, then first live chunks
    const size_t n = (size_t)(p.mmax + 1) * A.nblk;
    cudaError_t e = sht::dev_malloc(&ey, sizeof(int) * 2 * n);
    if (e != cudaSuccess) return e;
    tc_ymax_kernel<<<(unsigned)n, TC_T>>>(A, ey, ey + n);
    e = cudaGetLastError();
    double2 *cky = nullptr;
    int *ckk = nullptr;
    if (e == cudaSuccess) e = sht::dev_malloc(&cky, sizeof(double2) * n * TC_T);
    if (e == cudaSuccess) e = sht::dev_malloc(&ckk, sizeof(int) * n * TC_T);
    if (e == cudaSuccess) {
        tc_ckpt_kernel<<<(unsigned)n, TC_T>>>(A, ey + n, cky, ckk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(ey);
        cudaFree(cky);
        cudaFree(ckk);
        return e;
    }
    p.d_tc_Ey = ey;
    p.d_tc_ck_y = cky;
    p.d_tc_ck_k = ckk;
    return cudaSuccess;
}

size_t tc_workspace_bytes(const Plan &p, int nmaps)
{
    if (nmaps <= 0) return 0;
    const int n = std::min(nmaps, p.tune[SHT_TUNE_TC_MAPS]) > 8 ? 32 : 16;
    const size_t bchunk = n > 16 ? (size_t)TcTile<32>::B_CHUNK : (size_t)TcTile<16>::B_CHUNK;
    return (size_t)p.tc_total_chunks * bchunk + (size_t)(p.mmax + 1) * 32 * sizeof(int) + 256;
}

// Synthesis Legendre stage in the precision form; scratch holds tc_workspace_bytes(p, nmaps).
cudaError_t launch_legendre_synth_tc(const Plan &p, const double2 *alm, double2 *delta, void *scratch, int nmaps,
                                     cudaStream_t st, int *nlaunch)
{
    *nlaunch = 0;
    TcArgs A{};
    A.slotN = p.d_slotN;
    A.slotS = p.d_slotS;
    A.u = p.d_u;
    A.s = p.d_s;
    A.alpha = p.d_alpha;
    A.cfac = p.d_cfac;
    A.Ey = p.d_tc_Ey;
    A.first = p.d_tc_Ey + (size_t)(p.mmax + 1) * ((p.nslots + TC_T - 1) / TC_T);
    A.ck_y = p.d_tc_ck_y;
    A.ck_k = p.d_tc_ck_k;
    A.chunk_base = p.d_tc_chunk_base;
    A.chunk_m = p.d_tc_chunk_m;
    A.status = p.d_status;
    A.nslots = p.nslots;
    A.nblk = (p.nslots + TC_T - 1) / TC_T;
    A.lmax = p.lmax;
    A.mmax = p.mmax;
    A.nrings = p.nrings;
    A.mR = p.mR;
    A.nalm = p.nalm;
    const int64_t dstride = (int64_t)p.nrings * (p.mmax + 1);
    int g0 = 0;
    while (g0 < nmaps) {
        const int nm = std::min(p.tune[SHT_TUNE_TC_MAPS], nmaps - g0);
        A.nmaps = nm;
        A.alm = alm + (int64_t)g0 * p.nalm;
        A.delta = delta + (int64_t)g0 * dstride;
        const int N = nm > 8 ? 32 : 16;
        const size_t bchunk = N == 32 ? (size_t)TcTile<32>::B_CHUNK : (size_t)TcTile<16>::B_CHUNK;
        A.bdig = (uint4 *)scratch;
        A.Ea = (int *)((char *)scratch + (size_t)p.tc_total_chunks * bchunk);
        cudaError_t e = (N == 32) ? launch_group<32>(p, A, st) : launch_group<16>(p, A, st);
        *nlaunch += 3;
        if (e != cudaSuccess) return e;
        g0 += nm;
    }
    return cudaSuccess;
}

namespace {
SHT_CHECK_TAKE_DEF(take_check)
}  // namespace
cudaError_t take_check_word_tc(int *w) { return take_check(w); }

}  // namespace sht
