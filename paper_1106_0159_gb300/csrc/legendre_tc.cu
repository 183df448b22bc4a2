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
// Per CTA (one m, 128 slots, one thread per slot), per chunk of 32 l:
//   1. every thread runs 32 steps of the two-instruction y recurrence
//      (see legendre.cu), splits each y into digits with integer operations
//      and stores them as two k-groups of the bf16 A tiles [parity][digit];
//      the a_lm digit tiles (prepared by tc_split_b_kernel) are copied in;
//   2. one thread issues the 2 x 28 MMAs (M = 128, N = 16 or 32, K = 16) and
//      commits them to an mbarrier, which the next chunk waits on before
//      overwriting the tiles.
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
constexpr int RESCALE_THR = 1023 + 256;
constexpr double POLAR_SIN = 0.03;  // must match legendre.cu
constexpr long long WAIT_POLLS = 1ll << 26;
#ifndef TC_NACC
#define TC_NACC 5       // accumulators per parity: classes 0 .. TC_NACC-2 alone, the rest together
#endif
#ifndef TC_MAXW
#define TC_MAXW (TC_S - 1)  // highest digit class i + j accumulated
#endif

__device__ __forceinline__ int dexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

__device__ __forceinline__ void normalise(double &v, int &e)
{
    int hi = __double2hiint(v);
    e += ((hi >> 20) & 0x7ff) - 1023;
    hi = (hi & 0x800fffff) | (1023 << 20);
    v = __hiloint2double(hi, __double2loint(v));
}

__device__ __forceinline__ double pow2i(int e) { return __hiloint2double((e + 1023) << 20, 0); }

__device__ __forceinline__ double pow2i_safe(int e)  // 2^e, 0 below the normal range
{
    return e < -1022 ? 0.0 : pow2i(min(e, 1023));
}

// mu_m sin^m(theta) as y0 * 2^(512 k) (same construction as legendre.cu)
__device__ void sectoral_start(double s, double mu, int m, double &y0, int &k)
{
    if (m > 0 && !(s > 1e-300)) {
        y0 = 0.0;
        k = 0;
        return;
    }
    double r = 1.0;
    int er = 0;
    double b = s;
    int eb = 0;
    if (m > 0) normalise(b, eb);
    for (int mm = m; mm; mm >>= 1) {
        if (mm & 1) {
            r *= b;
            er += eb;
            normalise(r, er);
        }
        if (mm > 1) {
            b *= b;
            eb *= 2;
            normalise(b, eb);
        }
    }
    int kk = (er >= 0) ? 0 : -((-er) >> 9);
    int rem = er - 512 * kk;
    y0 = mu * r * pow2i(rem);
    k = kk;
}

// |v| * 2^(B - E), B = 7 S - 1 bits, rounded to the nearest integer, as S balanced base-128
// digits (most significant first), each returned as the float d_s * 2^(-7 s), so that
// v = 2^(E - 6) sum_s d_s 2^(-7 s) whatever S is.  Integer pipe only.
__device__ __forceinline__ void split_digits(double v, int E, float out[TC_S])
{
    constexpr int B = 7 * TC_S - 1;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((bits >> 52) & 0x7ff);
    const bool neg = (bits >> 63) != 0;
    unsigned long long F = 0;
    if (ex != 0) {
        const int sh = 1075 - B + E - ex;  // v = mant 2^(ex - 1075)
        const unsigned long long mant = (bits & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull;
        if (sh >= 64)
            F = 0;
        else if (sh >= 53 - B)
            F = (mant + (1ull << (sh - 1))) >> sh;  // |v| < 2^E gives sh >= 53 - B, so F <= 2^B
        else
            F = (1ull << B) - 1;  // outside the bound: saturate
    }
    int d[TC_S];
#pragma unroll
    for (int s = TC_S - 1; s >= 1; --s) {
        const int dd = (int)((F + 64ull) & 127ull) - 64;
        F = (F - (unsigned long long)(long long)dd) >> 7;
        d[s] = dd;
    }
    d[0] = (int)F;
#pragma unroll
    for (int s = 0; s < TC_S; ++s) {
        const float f = (float)(neg ? -d[s] : d[s]);
        out[s] = f * __int_as_float((127 - 7 * s) << 23);  // exact power of two
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

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

__device__ __forceinline__ void umma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
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
            : "r"(a), "r"(parity));
        if (done) return true;
        if (it > 64) __nanosleep(32);
    }
    return false;
}

template <int N>
struct TcTile {
    static constexpr int B_TILE = N * 16 * 2;                 // bytes of one [N x 16] tile
    static constexpr int B_CHUNK = 2 * TC_S * B_TILE;         // a_lm digits of one chunk
    static constexpr int A_BYTES = 2 * TC_S * TC_ATILE;
    static constexpr int NACC = TC_NACC;                      // accumulators per parity
    static constexpr int TMEM_COLS = (2 * NACC * N <= 128) ? 128 : (2 * NACC * N <= 256) ? 256 : 512;
    static constexpr int SMEM = A_BYTES + B_CHUNK + 1024;
};

struct TcArgs {
    const double2 *alm;      // [nmaps][nalm], first map of this group
    double2 *delta;          // [nmaps][nrings][mmax+1]
    const int *slotN, *slotS;
    const double *u, *s;
    const double *alpha, *cfac;
    const int *Ey;           // [mmax+1][nblk] scale exponent of y per slot block
    const int *first;        // [mmax+1][nblk] first chunk with a kept y value (nch: none)
    int *Ea;                 // [mmax+1][N] scale exponent of c a
    const int64_t *chunk_base;  // [mmax+1] first chunk of each m
    const int *chunk_m;      // [total chunks] m of each chunk
    uint4 *bdig;             // [total chunks][B_CHUNK / 16]
    int *status;             // device status word (bit 0: an mbarrier wait timed out)
    int nslots, nblk, lmax, mmax, nrings, mR, nmaps;
    int64_t nalm;
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
// [parity][digit][N x 16] bf16, core matrix (n/8, k/8) at ((k/8) (N/8) + n/8) * 64 elements
template <int N>
__global__ void tc_split_b_kernel(TcArgs A)
{
    const int64_t chunk = blockIdx.x;
    const int m = A.chunk_m[chunk];
    const int c = (int)(chunk - A.chunk_base[m]);
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    __nv_bfloat16 *out = (__nv_bfloat16 *)(A.bdig + chunk * (TcTile<N>::B_CHUNK / 16));
    for (int t = threadIdx.x; t < 2 * 16 * N; t += blockDim.x) {
        const int n = t % N, k = (t / N) % 16, eo = t / (16 * N);
        const int l = m + TC_CH * c + 2 * k + eo;
        const int g = n >> 1;
        double v = 0.0;
        if (l <= L && g < A.nmaps) {
            const int64_t ix = base + (l - m);
            const double2 a = A.alm[(int64_t)g * A.nalm + ix];
            const double comp = (n & 1) ? (m == 0 ? 0.0 : a.y) : a.x;
            v = A.cfac[ix] * comp;
        }
        float d[TC_S];
        split_digits(v, A.Ea[m * N + n], d);
        const int off = ((k >> 3) * (N / 8) + (n >> 3)) * 64 + (n & 7) * 8 + (k & 7);
#pragma unroll
        for (int s = 0; s < TC_S; ++s) out[(eo * TC_S + s) * (N * 16) + off] = __float2bfloat16_rn(d[s]);
    }
}

// ---------------------------------------------------------------- y scale per (m, slot block)

// max over the block's slots and all l (terms kept: k = 0) of the biased exponent of y,
// written as E with |y| < 2^E (-1000 when every value is dropped), and the first chunk of 32 l
// in which any slot keeps a value (every earlier chunk contributes exactly zero).  Same
// recurrence, operation for operation, as tc_synth_kernel.
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
                const double t = fma(-u, y1, y1);
                const double y = fma(s_al[j], t, -y2);
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

// ---------------------------------------------------------------- the synthesis kernel

template <int N>
__global__ void __launch_bounds__(TC_T) tc_synth_kernel(TcArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                                   // [2][S][128 x 16] bf16
    unsigned char *sB = smem + TcTile<N>::A_BYTES;              // [2][S][N x 16] bf16
    uint64_t *mbar = (uint64_t *)(sB + TcTile<N>::B_CHUNK);
    uint32_t *tslot = (uint32_t *)(mbar + 1);
    __shared__ double s_al[TC_CH];

    const int m = blockIdx.x / A.nblk;
    const int blk = blockIdx.x - m * A.nblk;
    if (m <= A.mR && A.s[blk * TC_T] < POLAR_SIN) return;  // Reinsch CTAs run in FP64

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int slot = blk * TC_T + tid;
    const bool active = slot < A.nslots;
    const int L = A.lmax;
    const int64_t base = (int64_t)m * (2 * L + 3 - m) / 2;
    const int Ey = A.Ey[m * A.nblk + blk];

    double u = 0.0, y1 = 0.0, y2 = 0.0;
    int k = 0;
    if (active) {
        u = A.u[slot];
        double y0;
        sectoral_start(A.s[slot], A.alpha[base], m, y0, k);
        y1 = 0.0;
        y2 = -y0;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TcTile<N>::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;

    const int nch = (L - m + TC_CH) / TC_CH;
    const int cfirst = A.first[m * A.nblk + blk];  // chunks before it hold only dropped values
    const int64_t chunk0 = A.chunk_base[m];
    const uint32_t idesc = umma_idesc<N>();
    bool ok = true;
    int committed = -1;  // last chunk whose MMAs were committed

    for (int c = 0; c < nch; ++c) {
        const int l0 = m + TC_CH * c;
        if (tid < TC_CH) s_al[tid] = (l0 + tid <= L) ? A.alpha[base + (l0 - m) + tid] : 0.0;
        if (c < cfirst) {  // recurrence only: every value of this chunk is dropped
            __syncthreads();
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                const bool scaled = __any_sync(0xffffffffu, k < 0);
#pragma unroll
                for (int j = 16 * h; j < 16 * h + 16; ++j) {
                    const double t = fma(-u, y1, y1);
                    const double y = fma(s_al[j], t, -y2);
                    y2 = y1;
                    y1 = y;
                }
                if (scaled && k < 0 && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                    y1 *= 0x1p-512;
                    y2 *= 0x1p-512;
                    k += 1;
                }
            }
            __syncthreads();
            continue;
        }
        // this chunk's a_lm digit tiles, prefetched into registers
        constexpr int BTOT = TcTile<N>::B_CHUNK / 16;        // uint4 of the chunk's tiles
        constexpr int BV = (BTOT + TC_T - 1) / TC_T;          // per thread, the last one partial
        uint4 breg[BV];
        const uint4 *bsrc = A.bdig + (chunk0 + c) * BTOT;
#pragma unroll
        for (int i = 0; i < BV; ++i)
            if (i * TC_T + tid < BTOT) breg[i] = bsrc[i * TC_T + tid];
        __syncthreads();

#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            uint32_t pe[TC_S][4], po[TC_S][4];  // 8 even / 8 odd values per digit, bf16 pairs
            const bool scaled = __any_sync(0xffffffffu, k < 0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                float de[TC_S], dd[TC_S];
#pragma unroll
                for (int par = 0; par < 2; ++par) {
                    const int j = 16 * h + 2 * q + par;
                    const double t = fma(-u, y1, y1);
                    const double y = fma(s_al[j], t, -y2);
                    y2 = y1;
                    y1 = y;
                    const double yv = (scaled && k < 0) ? 0.0 : y;
                    split_digits(yv, Ey, par ? dd : de);
                }
                if ((q & 1) == 0) {
#pragma unroll
                    for (int s = 0; s < TC_S; ++s) {
                        pe[s][q >> 1] = pack_bf16x2(de[s], 0.f);
                        po[s][q >> 1] = pack_bf16x2(dd[s], 0.f);
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < TC_S; ++s) {
                        pe[s][q >> 1] = (pe[s][q >> 1] & 0xFFFFu) | (pack_bf16x2(de[s], 0.f) << 16);
                        po[s][q >> 1] = (po[s][q >> 1] & 0xFFFFu) | (pack_bf16x2(dd[s], 0.f) << 16);
                    }
                }
            }
            if (scaled && k < 0 && max(dexp(y1), dexp(y2)) > RESCALE_THR) {
                y1 *= 0x1p-512;
                y2 *= 0x1p-512;
                k += 1;
            }
            if (h == 0 && c > cfirst) {  // the previous chunk's MMAs still read the tiles
                if (!mbar_wait(mbar, (uint32_t)((c - 1 - cfirst) & 1))) ok = false;
            }
            // k-group h of every A tile: core matrix (slot/8, h), row slot%8
            const int off = ((h * 16) + (tid >> 3)) * 128 + (tid & 7) * 16;
#pragma unroll
            for (int s = 0; s < TC_S; ++s) {
                *(uint4 *)(sA + (0 * TC_S + s) * TC_ATILE + off) = make_uint4(pe[s][0], pe[s][1], pe[s][2], pe[s][3]);
                *(uint4 *)(sA + (1 * TC_S + s) * TC_ATILE + off) = make_uint4(po[s][0], po[s][1], po[s][2], po[s][3]);
            }
            if (h == 0) {
#pragma unroll
                for (int i = 0; i < BV; ++i)
                    if (i * TC_T + tid < BTOT) ((uint4 *)sB)[i * TC_T + tid] = breg[i];
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
#pragma unroll
            for (int eo = 0; eo < 2; ++eo) {
#pragma unroll
                for (int w = 0; w <= TC_MAXW; ++w) {
#pragma unroll
                    for (int i = 0; i <= w; ++i) {
                        const int j = w - i;
                        const int cls = w < TcTile<N>::NACC - 1 ? w : TcTile<N>::NACC - 1;
                        const bool first = (c == cfirst) && (i == 0) && (w <= TcTile<N>::NACC - 1);
                        const uint64_t ad = umma_desc(a0 + (eo * TC_S + i) * TC_ATILE, 16 * 128, 128);
                        const uint64_t bd = umma_desc(b0 + (eo * TC_S + j) * TcTile<N>::B_TILE, (N / 8) * 128, 128);
                        umma_bf16(tmem + (uint32_t)((eo * TcTile<N>::NACC + cls) * N), ad, bd, idesc, first ? 0u : 1u);
                    }
                }
            }
            umma_commit(mbar);
        }
        committed = c;
    }

    // wait (bounded) for the last committed MMAs, also on the error path, before TMEM is read or freed
    if (committed >= 0 && !mbar_wait(mbar, (uint32_t)((committed - cfirst) & 1))) ok = false;
    const bool any_mma = cfirst < nch;  // else every value was dropped and Delta is zero
    ok = __syncthreads_and(ok && (any_mma ? committed == nch - 1 : committed < 0));
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        // accumulators: column (eo * NACC + cls) * N + n, lane = slot within the block
        double acc[2][N];
#pragma unroll
        for (int eo = 0; eo < 2; ++eo)
#pragma unroll
            for (int n = 0; n < N; ++n) acc[eo][n] = 0.0;
#pragma unroll
        for (int eo = 0; eo < 2 && any_mma; ++eo) {
#pragma unroll
            for (int cls = 0; cls < TcTile<N>::NACC; ++cls) {
#pragma unroll
                for (int n0 = 0; n0 < N; n0 += 16) {
                    uint32_t r[16];
                    const uint32_t addr =
                        tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((eo * TcTile<N>::NACC + cls) * N + n0);
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(addr));
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc[eo][n0 + q] += (double)__uint_as_float(r[q]);
                }
            }
        }
        if (active) {
            const int rn = A.slotN[slot], rs = A.slotS[slot];
            const int64_t mstride = A.mmax + 1;
#pragma unroll
            for (int g = 0; g < N / 2; ++g) {
                if (g < A.nmaps) {
                    const double sr = pow2i_safe(Ey + A.Ea[m * N + 2 * g] - 12);
                    const double si = pow2i_safe(Ey + A.Ea[m * N + 2 * g + 1] - 12);
                    const double er = acc[0][2 * g] * sr, ei = acc[0][2 * g + 1] * si;
                    const double orr = acc[1][2 * g] * sr, oi = acc[1][2 * g + 1] * si;
                    double2 *d = A.delta + (int64_t)g * A.nrings * mstride;
                    if (rn >= 0) d[(int64_t)rn * mstride + m] = make_double2(er + orr, ei + oi);
                    if (rs >= 0) d[(int64_t)rs * mstride + m] = make_double2(er - orr, ei - oi);
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(A.status, 1);
    }
    (void)lane;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                                "r"(TcTile<N>::TMEM_COLS));
}

template <int N>
cudaError_t launch_group(const Plan &p, TcArgs A, cudaStream_t st)
{
    const int64_t nchunks = p.tc_total_chunks;
    tc_scale_kernel<N><<<p.mmax + 1, 256, 0, st>>>(A);
    tc_split_b_kernel<N><<<(unsigned)nchunks, 256, 0, st>>>(A);
    // at least 100 KB of shared memory per CTA keeps two CTAs per SM, which is what the
    // tensor memory holds (TMEM_COLS <= 256 of 512 columns each)
    const int smem = std::max(TcTile<N>::SMEM, TcTile<N>::TMEM_COLS > 256 ? 160 * 1024 : 100 * 1024);
    cudaError_t e = cudaFuncSetAttribute(tc_synth_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    tc_synth_kernel<N><<<(unsigned)((p.mmax + 1) * A.nblk), TC_T, smem, st>>>(A);
    return cudaGetLastError();
}

}  // namespace

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
    cudaError_t e = cudaMalloc(&ey, sizeof(int) * 2 * n);
    if (e != cudaSuccess) return e;
    tc_ymax_kernel<<<(unsigned)n, TC_T>>>(A, ey, ey + n);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(ey);
        return e;
    }
    p.d_tc_Ey = ey;
    return cudaSuccess;
}

size_t tc_workspace_bytes(const Plan &p, int nmaps)
{
    if (nmaps <= 0) return 0;
    const int n = nmaps > 8 ? 32 : 16;
    const size_t bchunk = (size_t)2 * TC_S * n * 16 * 2;
    return (size_t)p.tc_total_chunks * bchunk + (size_t)(p.mmax + 1) * 32 * sizeof(int) + 256;
}

// Synthesis Legendre stage in the precision form; scratch holds tc_workspace_bytes(p, min(nmaps, 16)).
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
        const int nm = std::min(16, nmaps - g0);
        A.nmaps = nm;
        A.alm = alm + (int64_t)g0 * p.nalm;
        A.delta = delta + (int64_t)g0 * dstride;
        const int N = nm > 8 ? 32 : 16;
        const size_t bchunk = (size_t)2 * TC_S * N * 16 * 2;
        A.bdig = (uint4 *)scratch;
        A.Ea = (int *)((char *)scratch + (size_t)p.tc_total_chunks * bchunk);
        cudaError_t e = (N == 32) ? launch_group<32>(p, A, st) : launch_group<16>(p, A, st);
        *nlaunch += 3;
        if (e != cudaSuccess) return e;
        g0 += nm;
    }
    return cudaSuccess;
}

}  // namespace sht
