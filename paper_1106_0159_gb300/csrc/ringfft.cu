// Ring stage of the transforms (Section 2.2 eqs. Delta2map and almfftdef,
// the FFT steps of Algorithms 1-2).
//
// Every pixel ring is a real sequence of nphi equidistant samples starting at
// phi0.  Two rings of equal length (normally a north/south mirror pair) share
// one complex DFT: ring A on the real part, ring B on the imaginary part.
//
// synthesis:  v_m = Delta_m exp(i m phi0) for 0 <= m <= mmax, folded into the
//             nphi bins (bin m mod nphi, and conj(v_m) into bin -m mod nphi),
//             then z_j = sum_k Z_k exp(+2 pi i j k / nphi).
// analysis:   S_k = sum_j s_j exp(-2 pi i j k / nphi),
//             Delta^S_m = w exp(-i m phi0) S_(m mod nphi).
//
// Each complex DFT is run by one CTA of a persistent grid in three
// CTA-private scratch buffers: Stockham passes of radix 4, 2, 3, 5, 7, 11 or
// 13 when nphi factors into those, otherwise Bluestein's chirp-z form with a
// power-of-two convolution.  The minus-sign DFT is taken as
// conj(DFT+(conj(x))).  Twiddles, chirps and Bluestein filters are plan
// tables built on the device at plan creation.
#include "sht_internal.h"

#include <algorithm>
#include <map>
#include <vector>

namespace sht {
namespace {

// Launch shape of the ring kernels: RING_CTAS_PER_SM x 152 persistent CTAs of RING_T threads.
// lmax 4096, HEALPix 2048, 16 maps, double-float DFTs (synthesis / analysis ms): 2 x 256: 57 / 47,
// 1 x 256: 80 / 62, 1 x 512: 58 / 49, 2 x 512: 47 / 39 (more threads per DFT, same scratch).
#ifndef RING_T
#define RING_T 512
#endif
#ifndef RING_CTAS_PER_SM
#define RING_CTAS_PER_SM 2
#endif
constexpr int FFT_T = RING_T;

#include "check.cuh"
constexpr int MAXR = 13;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 conjd(double2 a) { return make_double2(a.x, -a.y); }

// ---------------------------------------------------------------- arithmetic of the ring DFTs
//
// The DFT code below is written once over an arithmetic P: complex values P::C, table entries
// P::T, and the operations add, sub, mul (by a table entry or a value), conj and i-times.
//   F64: double2, the plain form.
//   DF:  a double-float complex (re hi, re lo, im hi, im lo) as float4, for the precision form.
//        A real is hi + lo with |lo| <= ulp(hi) / 2 (renormalised after every operation): sums by
//        TwoSum, products by an FMA two-product plus the cross terms, about 2^-44 relative.  On this
//        part FP32 issues 64 times faster than FP64, so the DFTs run about 5x faster at an accuracy
//        far inside the precision form's bar.  Inputs and outputs stay FP64.

struct F64 {
    using C = double2;
    using T = double2;
    static __device__ __forceinline__ C zero() { return make_double2(0.0, 0.0); }
    static __device__ __forceinline__ C add(C a, C b) { return cadd(a, b); }
    static __device__ __forceinline__ C sub(C a, C b) { return csub(a, b); }
    static __device__ __forceinline__ C mul(C a, T b) { return cmul(a, b); }
    static __device__ __forceinline__ C mulc(C a, C b) { return cmul(a, b); }
    static __device__ __forceinline__ C conj(C a) { return conjd(a); }
    static __device__ __forceinline__ C conjt(T a) { return conjd(a); }
    static __device__ __forceinline__ C itimes(C a) { return make_double2(-a.y, a.x); }
    static __device__ __forceinline__ C half(C a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
    static __device__ __forceinline__ C from(double2 v) { return v; }
    static __device__ __forceinline__ C from_re_im(double re, double im) { return make_double2(re, im); }
    static __device__ __forceinline__ double2 to(C v) { return v; }
    static __device__ __forceinline__ double re(C v) { return v.x; }
    static __device__ __forceinline__ double im(C v) { return v.y; }
};

// double-float helpers: a real is (hi, lo)
__device__ __forceinline__ float2 dfn_add(float2 a, float2 b)
{
    const float s = a.x + b.x;
    const float v = s - a.x;
    float e = (a.x - (s - v)) + (b.x - v);
    e += a.y + b.y;
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
__device__ __forceinline__ float2 dfn_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 dfn_mul(float2 a, float2 b)
{
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float h = p + e;
    return make_float2(h, e - (h - p));
}
// FP64 -> (hi, lo) from the bit pattern, on the integer pipe (an FP64 <-> FP32 conversion takes an
// FP64 issue slot): hi = sign, exponent and the top 23 fraction bits; lo = the remaining 29 bits,
// rounded to 24.  Below 2^-74 the remainder would leave the FP32 range: those (rare) values take
// the conversion instructions, and values below 2^-126 flush to zero.
__device__ __forceinline__ float2 dfn_from(double v)
{
    const int hiw = __double2hiint(v);
    const unsigned low = (unsigned)__double2loint(v);
    const int ex = (hiw >> 20) & 0x7ff;
    const int e = ex - 1023;
    if (ex == 0 || e < -126) return make_float2(0.f, 0.f);
    if (e < 52 - 126) {
        const float h = __double2float_rn(v);
        return make_float2(h, __double2float_rn(v - (double)h));
    }
    const unsigned sign = (unsigned)hiw & 0x80000000u;
    const unsigned frac23 = (((unsigned)hiw & 0xFFFFFu) << 3) | (low >> 29);
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | frac23);
    const unsigned rem = low & 0x1FFFFFFFu;
    const float sc = (e - 52 >= -126) ? __uint_as_float((unsigned)(e - 52 + 127) << 23) : 0.f;
    const float lo = (float)rem * sc;
    return make_float2(hi, sign ? -lo : lo);
}
// float -> double from the bit pattern (normal floats and zero, the only ones produced here)
__device__ __forceinline__ double dfn_widen(float f)
{
    const unsigned b = __float_as_uint(f);
    const unsigned ex = (b >> 23) & 0xffu;
    if (ex == 0) return 0.0;
    const unsigned hi = (b & 0x80000000u) | ((ex + (1023 - 127)) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(b << 29));
}
__device__ __forceinline__ double dfn_to(float2 a) { return dfn_widen(a.x) + dfn_widen(a.y); }

struct DF {
    using C = float4;   // (re hi, re lo, im hi, im lo)
    using T = float4;
    static __device__ __forceinline__ float2 R(C a) { return make_float2(a.x, a.y); }
    static __device__ __forceinline__ float2 I(C a) { return make_float2(a.z, a.w); }
    static __device__ __forceinline__ C mk(float2 r, float2 i) { return make_float4(r.x, r.y, i.x, i.y); }
    static __device__ __forceinline__ C zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
    static __device__ __forceinline__ C add(C a, C b) { return mk(dfn_add(R(a), R(b)), dfn_add(I(a), I(b))); }
    static __device__ __forceinline__ C sub(C a, C b)
    {
        return mk(dfn_add(R(a), dfn_neg(R(b))), dfn_add(I(a), dfn_neg(I(b))));
    }
    static __device__ __forceinline__ C mulc(C a, C b)
    {
        const float2 re = dfn_add(dfn_mul(R(a), R(b)), dfn_neg(dfn_mul(I(a), I(b))));
        const float2 im = dfn_add(dfn_mul(R(a), I(b)), dfn_mul(I(a), R(b)));
        return mk(re, im);
    }
    static __device__ __forceinline__ C mul(C a, T b) { return mulc(a, b); }
    static __device__ __forceinline__ C conj(C a) { return make_float4(a.x, a.y, -a.z, -a.w); }
    static __device__ __forceinline__ C conjt(T a) { return conj(a); }
    static __device__ __forceinline__ C itimes(C a) { return make_float4(-a.z, -a.w, a.x, a.y); }
    static __device__ __forceinline__ C half(C a) { return make_float4(0.5f * a.x, 0.5f * a.y, 0.5f * a.z, 0.5f * a.w); }
    static __device__ __forceinline__ C from(double2 v) { return mk(dfn_from(v.x), dfn_from(v.y)); }
    static __device__ __forceinline__ C from_re_im(double re, double im) { return mk(dfn_from(re), dfn_from(im)); }
    static __device__ __forceinline__ double2 to(C v) { return make_double2(dfn_to(R(v)), dfn_to(I(v))); }
    static __device__ __forceinline__ double re(C v) { return dfn_to(R(v)); }
    static __device__ __forceinline__ double im(C v) { return dfn_to(I(v)); }
};

// One Stockham pass: sub-transforms of length Lsub become length Lsub * p.
// Input  X[j * (n / Lsub) + q],  j < Lsub, q < n / Lsub
// Output Y[k * (n / (Lsub p)) + q'], k < Lsub p
template <class P>
__device__ void stockham_pass(const typename P::C *__restrict__ X, typename P::C *__restrict__ Y, int n, int Lsub,
                              int p, const typename P::T *__restrict__ tw)
{
    using C = typename P::C;
    const int nq = n / (Lsub * p);
    const int nbf = Lsub * nq;
    const int inStride = n / Lsub;
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int k1 = b / nq;
        const int q = b - k1 * nq;
        const C *src = X + (int64_t)k1 * inStride + q;
        C *dst = Y + (int64_t)k1 * nq + q;
        const int64_t ostride = (int64_t)Lsub * nq;
        if (p == 4) {
            C a0 = src[0], a1 = src[nq], a2 = src[2 * nq], a3 = src[3 * nq];
            if (k1) {
                const int t = k1 * nq;
                a1 = P::mul(a1, tw[t]);
                a2 = P::mul(a2, tw[2 * t]);
                a3 = P::mul(a3, tw[3 * t]);
            }
            const C s02 = P::add(a0, a2), d02 = P::sub(a0, a2);
            const C s13 = P::add(a1, a3), d13 = P::sub(a1, a3);
            const C id13 = P::itimes(d13);  // i * (a1 - a3)
            dst[0] = P::add(s02, s13);
            dst[ostride] = P::add(d02, id13);
            dst[2 * ostride] = P::sub(s02, s13);
            dst[3 * ostride] = P::sub(d02, id13);
        } else if (p == 2) {
            C a0 = src[0], a1 = src[nq];
            if (k1) a1 = P::mul(a1, tw[k1 * nq]);
            dst[0] = P::add(a0, a1);
            dst[ostride] = P::sub(a0, a1);
        } else {
            C a[MAXR];
            a[0] = src[0];
            for (int r = 1; r < p; ++r) {
                a[r] = src[(int64_t)r * nq];
                if (k1) a[r] = P::mul(a[r], tw[(int64_t)r * k1 * nq]);
            }
            const int wstep = n / p;  // exp(2 pi i / p) = tw[n / p]
            for (int k2 = 0; k2 < p; ++k2) {
                C acc = a[0];
                int e = 0;
                for (int r = 1; r < p; ++r) {
                    e += k2;
                    if (e >= p) e -= p;
                    acc = P::add(acc, P::mul(a[r], tw[(int64_t)e * wstep]));
                }
                dst[(int64_t)k2 * ostride] = acc;
            }
        }
    }
}

// Length-n DFT with the + sign on B0[0, n) (all threads of the CTA).  Returns
// the buffer that holds the result.  B1, B2 hold at least max(n, M) entries.
template <class P>
__device__ typename P::C *cta_dft(const FftLen &F, const typename P::T *__restrict__ tab, typename P::C *B0,
                                  typename P::C *B1, typename P::C *B2)
{
    using C = typename P::C;
    if (F.M == 0) {
        C *X = B0, *Y = B1;
        int Lsub = 1;
        for (int f = 0; f < F.nfac; ++f) {
            __syncthreads();
            stockham_pass<P>(X, Y, F.n, Lsub, F.fac[f], tab + F.tw);
            C *t = X;
            X = Y;
            Y = t;
            Lsub *= F.fac[f];
        }
        __syncthreads();
        return X;
    }
    const int n = F.n, M = F.M;
    const typename P::T *ch = tab + F.chirp;
    const typename P::T *filt = tab + F.filt;
    for (int j = threadIdx.x; j < M; j += blockDim.x) B1[j] = (j < n) ? P::mul(B0[j], ch[j]) : P::zero();
    C *X = B1, *Y = B2;
    int Lsub = 1;
    for (int f = 0; f < F.nfac; ++f) {
        __syncthreads();
        stockham_pass<P>(X, Y, M, Lsub, F.fac[f], tab + F.tw);
        C *t = X;
        X = Y;
        Y = t;
        Lsub *= F.fac[f];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < M; j += blockDim.x) X[j] = P::conj(P::mul(X[j], filt[j]));
    Lsub = 1;
    for (int f = 0; f < F.nfac; ++f) {
        __syncthreads();
        stockham_pass<P>(X, Y, M, Lsub, F.fac[f], tab + F.tw);
        C *t = X;
        X = Y;
        Y = t;
        Lsub *= F.fac[f];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) B0[k] = P::mul(P::conj(X[k]), ch[k]);
    __syncthreads();
    return B0;
}

template <class P>
struct RingArgs {
    const FftItem *items;
    const FftLen *lens;
    const typename P::T *tab;
    const typename P::T *phase;   // [nrings][mmax+1]
    const int64_t *ofs;
    const double *w;
    typename P::C *scratch;       // [grid][3][maxlen]
    int maxlen;
    int nitems, nmaps, nrings, mmax;
    int64_t npix;
    const double2 *delta_in;      // synthesis input
    double *map_out;              // synthesis output
    const double *map_in;         // analysis input
    double2 *delta_out;           // analysis output
};

// folded, phased spectrum bin k of one ring
template <class P>
__device__ __forceinline__ typename P::C fold_bin(const double2 *__restrict__ d, const typename P::T *__restrict__ ph,
                                                  int k, int n, int mmax)
{
    typename P::C c = P::zero();
    for (int m = k; m <= mmax; m += n) c = P::add(c, P::mul(P::from(d[m]), ph[m]));
    int m0 = (n - k) % n;
    if (m0 == 0) m0 = n;
    for (int m = m0; m <= mmax; m += n) c = P::add(c, P::conj(P::mul(P::from(d[m]), ph[m])));
    return c;
}

// one unit of the ring synthesis: map g of FFT item `item` (one or two rings)
template <class P>
__device__ void ring_synth_unit(const RingArgs<P> &A, int item, int g, typename P::C *B0, typename P::C *B1,
                                typename P::C *B2)
{
    using C = typename P::C;
    const int64_t mstride = A.mmax + 1;
    const FftItem it = A.items[item];
    const FftLen &F = A.lens[it.len_id];
    const int n = it.n;
    if (!SHT_CHK(it.ringA >= 0 && it.ringA < A.nrings && it.ringB < A.nrings && n <= A.maxlen && F.M <= A.maxlen &&
                 A.ofs[it.ringA] + n <= A.npix && (it.ringB < 0 || A.ofs[it.ringB] + n <= A.npix)))
        return;
    const double2 *dA = A.delta_in + ((int64_t)g * A.nrings + it.ringA) * mstride;
    const typename P::T *pA = A.phase + (int64_t)it.ringA * mstride;
    const double2 *dB = it.ringB >= 0 ? A.delta_in + ((int64_t)g * A.nrings + it.ringB) * mstride : nullptr;
    const typename P::T *pB = it.ringB >= 0 ? A.phase + (int64_t)it.ringB * mstride : nullptr;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const C ca = fold_bin<P>(dA, pA, k, n, A.mmax);
        C z = ca;
        if (dB) {
            const C cb = fold_bin<P>(dB, pB, k, n, A.mmax);
            z = P::add(ca, P::itimes(cb));  // C_A + i C_B
        }
        B0[k] = z;
    }
    __syncthreads();
    const C *X = cta_dft<P>(F, A.tab, B0, B1, B2);
    double *outA = A.map_out + (int64_t)g * A.npix + A.ofs[it.ringA];
    double *outB = it.ringB >= 0 ? A.map_out + (int64_t)g * A.npix + A.ofs[it.ringB] : nullptr;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const C z = X[j];
        outA[j] = P::re(z);
        if (outB) outB[j] = P::im(z);
    }
    __syncthreads();
}

template <class P>
__global__ void __launch_bounds__(FFT_T) ring_synth_kernel(RingArgs<P> A)
{
    using C = typename P::C;
    C *B0 = A.scratch + (int64_t)blockIdx.x * 3 * A.maxlen;
    C *B1 = B0 + A.maxlen, *B2 = B1 + A.maxlen;
    const int nunits = A.nitems * A.nmaps;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
        const int item = unit / A.nmaps, g = unit - item * A.nmaps;
        ring_synth_unit<P>(A, item, g, B0, B1, B2);
    }
}

// one unit of the ring analysis: map g of FFT item `item`
template <class P>
__device__ void ring_anal_unit(const RingArgs<P> &A, int item, int g, typename P::C *B0, typename P::C *B1,
                               typename P::C *B2)
{
    using C = typename P::C;
    const int64_t mstride = A.mmax + 1;
    const FftItem it = A.items[item];
    const FftLen &F = A.lens[it.len_id];
    const int n = it.n;
    if (!SHT_CHK(it.ringA >= 0 && it.ringA < A.nrings && it.ringB < A.nrings && n <= A.maxlen && F.M <= A.maxlen &&
                 A.ofs[it.ringA] + n <= A.npix && (it.ringB < 0 || A.ofs[it.ringB] + n <= A.npix)))
        return;
    const double *sA = A.map_in + (int64_t)g * A.npix + A.ofs[it.ringA];
    const double *sB = it.ringB >= 0 ? A.map_in + (int64_t)g * A.npix + A.ofs[it.ringB] : nullptr;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        B0[j] = P::from_re_im(sA[j], sB ? -sB[j] : 0.0);  // conj(s_A + i s_B)
    __syncthreads();
    const C *X = cta_dft<P>(F, A.tab, B0, B1, B2);  // conj(S)
    const typename P::T *pA = A.phase + (int64_t)it.ringA * mstride;
    double2 *oA = A.delta_out + ((int64_t)g * A.nrings + it.ringA) * mstride;
    const double wA = A.w[it.ringA];
    if (it.ringB < 0) {
        for (int m = threadIdx.x; m <= A.mmax; m += blockDim.x) {
            const C S = P::conj(X[m % n]);
            const double2 v = P::to(P::mulc(P::conjt(pA[m]), S));
            oA[m] = make_double2(wA * v.x, m == 0 ? 0.0 : wA * v.y);
        }
    } else {
        const typename P::T *pB = A.phase + (int64_t)it.ringB * mstride;
        double2 *oB = A.delta_out + ((int64_t)g * A.nrings + it.ringB) * mstride;
        const double wB = A.w[it.ringB];
        for (int m = threadIdx.x; m <= A.mmax; m += blockDim.x) {
            const int k = m % n;
            const int kc = (n - k) % n;
            const C S = P::conj(X[k]);
            const C Sc = X[kc];  // conj(S_{-k})
            const C SA = P::half(P::add(S, Sc));
            const C D = P::half(P::sub(S, Sc));
            const C SB = P::conj(P::itimes(P::conj(D)));  // D / (2 i) with D halved: -i D
            const double2 va = P::to(P::mulc(P::conjt(pA[m]), SA));
            const double2 vb = P::to(P::mulc(P::conjt(pB[m]), SB));
            oA[m] = make_double2(wA * va.x, m == 0 ? 0.0 : wA * va.y);
            oB[m] = make_double2(wB * vb.x, m == 0 ? 0.0 : wB * vb.y);
        }
    }
    __syncthreads();
}

template <class P>
__global__ void __launch_bounds__(FFT_T) ring_anal_kernel(RingArgs<P> A)
{
    using C = typename P::C;
    C *B0 = A.scratch + (int64_t)blockIdx.x * 3 * A.maxlen;
    C *B1 = B0 + A.maxlen, *B2 = B1 + A.maxlen;
    const int nunits = A.nitems * A.nmaps;
    for (int unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
        const int item = unit / A.nmaps, g = unit - item * A.nmaps;
        ring_anal_unit<P>(A, item, g, B0, B1, B2);
    }
}

// batched form: units (job, item, map) of many plans from one device counter, in the host's order
// (longest rings first); every CTA keeps its own three scratch buffers of `maxlen` entries
template <class P, bool SYNTH>
__global__ void __launch_bounds__(FFT_T) ring_batch_kernel(const RingArgs<P> *__restrict__ jobs,
                                                           const int4 *__restrict__ units, int nunits, int maxlen,
                                                           typename P::C *scratch, int *counter)
{
    using C = typename P::C;
    __shared__ int s_t;
    C *B0 = scratch + (int64_t)blockIdx.x * 3 * maxlen;
    C *B1 = B0 + maxlen, *B2 = B1 + maxlen;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_t = atomicAdd(counter, 1);
        __syncthreads();
        const int t = s_t;
        if (t >= nunits) break;
        const int4 U = units[t];
        if (SYNTH)
            ring_synth_unit<P>(jobs[U.x], U.y, U.z, B0, B1, B2);
        else
            ring_anal_unit<P>(jobs[U.x], U.y, U.z, B0, B1, B2);
    }
}

// double-float copies of FP64 tables (hi = rounded, lo = remainder rounded)
__global__ void df_table_kernel(const double2 *__restrict__ src, float4 *__restrict__ dst, int64_t n)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = src[t];
        const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
        dst[t] = make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
    }
}

// ---------------------------------------------------------------- plan tables

struct TabJob {
    int64_t off;
    int n;
    int kind;  // 0: exp(2 pi i k / n), k < n; 1: chirp exp(i pi j^2 / n), j < n
};

__global__ void fill_tables_kernel(const TabJob *jobs, int njobs, double2 *tab)
{
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const TabJob J = jobs[jb];
        for (int k = threadIdx.x; k < J.n; k += blockDim.x) {
            double s, c;
            if (J.kind == 0) {
                sincospi(2.0 * (double)k / (double)J.n, &s, &c);
            } else {
                const int64_t q = ((int64_t)k * k) % (2 * (int64_t)J.n);
                sincospi((double)q / (double)J.n, &s, &c);
            }
            tab[J.off + k] = make_double2(c, s);
        }
    }
}

__global__ void __launch_bounds__(FFT_T) bluestein_filter_kernel(const FftLen *lens, const int *ids, int nids,
                                                                 double2 *tab, double2 *scratch, int maxlen)
{
    double2 *B0 = scratch + (int64_t)blockIdx.x * 3 * maxlen;
    double2 *B1 = B0 + maxlen;
    for (int t = blockIdx.x; t < nids; t += gridDim.x) {
        const FftLen &F = lens[ids[t]];
        const int n = F.n, M = F.M;
        const double2 *ch = tab + F.chirp;
        // h'_d = conj(c_d) for 0 <= d < n, h'_{M-d} = conj(c_d) for 0 < d < n
        for (int j = threadIdx.x; j < M; j += blockDim.x) {
            double2 v = make_double2(0.0, 0.0);
            if (j < n)
                v = conjd(ch[j]);
            else if (j > M - n)
                v = conjd(ch[M - j]);
            B0[j] = v;
        }
        __syncthreads();
        double2 *X = B0, *Y = B1;
        int Lsub = 1;
        for (int f = 0; f < F.nfac; ++f) {
            __syncthreads();
            stockham_pass<F64>(X, Y, M, Lsub, F.fac[f], tab + F.tw);
            double2 *tmp = X;
            X = Y;
            Y = tmp;
            Lsub *= F.fac[f];
        }
        __syncthreads();
        const double inv = 1.0 / (double)M;
        for (int j = threadIdx.x; j < M; j += blockDim.x) {
            const double2 v = X[j];
            tab[F.filt + j] = make_double2(v.x * inv, v.y * inv);
        }
        __syncthreads();
    }
}

// exp(i m phi0_r), with m phi0 reduced modulo 2 pi in extra precision
__global__ void phase_table_kernel(const double *phi0, int nrings, int mmax, double2 *phase)
{
    const double TWO_PI_HI = 6.283185307179586232;      // 2 pi rounded to double
    const double TWO_PI_LO = 2.4492935982947064e-16;     // 2 pi - TWO_PI_HI
    const int64_t total = (int64_t)nrings * (mmax + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(t / (mmax + 1));
        const int m = (int)(t - (int64_t)r * (mmax + 1));
        const double p = phi0[r];
        const double hi = (double)m * p;
        const double lo = fma((double)m, p, -hi);          // m p = hi + lo exactly
        const double kq = rint(hi / TWO_PI_HI);
        double red = fma(-kq, TWO_PI_HI, hi);               // exact for |kq| < 2^20
        red = fma(-kq, TWO_PI_LO, red) + lo;
        double s, c;
        sincos(red, &s, &c);
        phase[t] = make_double2(c, s);
    }
}

bool factor_smooth(int n, std::vector<int> &fac)
{
    fac.clear();
    int r = n;
    while (r % 4 == 0) {
        fac.push_back(4);
        r /= 4;
    }
    while (r % 2 == 0) {
        fac.push_back(2);
        r /= 2;
    }
    for (int p : {3, 5, 7, 11, 13}) {
        while (r % p == 0) {
            fac.push_back(p);
            r /= p;
        }
    }
    return r == 1;
}

}  // namespace

size_t ring_scratch_bytes(const Plan &p) { return (size_t)ring_grid(p) * 3 * (size_t)p.fft_maxlen * sizeof(double2); }

int ring_grid(const Plan &p) { return std::max(1, std::min(p.nitems, RING_CTAS_PER_SM * 152)); }

namespace {

bool ring_df(const Plan &p) { return p.mode == SHT_MODE_SPLIT_BF16 && p.tune[SHT_TUNE_PREC_RING] && p.d_fft_tab_df; }

template <class P>
RingArgs<P> ring_args(const Plan &p, const typename P::T *tab, const typename P::T *phase, void *scratch, int nmaps)
{
    RingArgs<P> A{};
    A.items = p.d_items;
    A.lens = p.d_lens;
    A.tab = tab;
    A.phase = phase;
    A.ofs = p.d_ofs;
    A.w = p.d_w;
    A.scratch = (typename P::C *)scratch;
    A.maxlen = p.fft_maxlen;
    A.nitems = p.nitems;
    A.nmaps = nmaps;
    A.nrings = p.nrings;
    A.mmax = p.mmax;
    A.npix = p.npix;
    return A;
}

}  // namespace

// The ring stages run in double-float arithmetic in the precision form (unless SHT_TUNE_PREC_RING
// is 0), in FP64 otherwise.
cudaError_t launch_ring_synth_grid(const Plan &p, const double2 *delta, double *map, double2 *scratch, int nmaps,
                                   int grid, cudaStream_t st)
{
    if (ring_df(p)) {
        RingArgs<DF> A = ring_args<DF>(p, p.d_fft_tab_df, p.d_phase_df, scratch, nmaps);
        A.delta_in = delta;
        A.map_out = map;
        ring_synth_kernel<DF><<<grid, FFT_T, 0, st>>>(A);
    } else {
        RingArgs<F64> A = ring_args<F64>(p, p.d_fft_tab, p.d_phase, scratch, nmaps);
        A.delta_in = delta;
        A.map_out = map;
        ring_synth_kernel<F64><<<grid, FFT_T, 0, st>>>(A);
    }
    return cudaGetLastError();
}

cudaError_t launch_ring_synth(const Plan &p, const double2 *delta, double *map, double2 *scratch, int nmaps,
                              cudaStream_t st)
{
    return launch_ring_synth_grid(p, delta, map, scratch, nmaps, ring_grid(p), st);
}

cudaError_t launch_ring_anal(const Plan &p, const double *map, double2 *delta, double2 *scratch, int nmaps,
                             cudaStream_t st)
{
    if (ring_df(p)) {
        RingArgs<DF> A = ring_args<DF>(p, p.d_fft_tab_df, p.d_phase_df, scratch, nmaps);
        A.map_in = map;
        A.delta_out = delta;
        ring_anal_kernel<DF><<<ring_grid(p), FFT_T, 0, st>>>(A);
    } else {
        RingArgs<F64> A = ring_args<F64>(p, p.d_fft_tab, p.d_phase, scratch, nmaps);
        A.map_in = map;
        A.delta_out = delta;
        ring_anal_kernel<F64><<<ring_grid(p), FFT_T, 0, st>>>(A);
    }
    return cudaGetLastError();
}

// double-float copies of the DFT and phase tables for the precision form (synchronous, once)
cudaError_t build_df_ring_tables(Plan &p)
{
    if (p.d_fft_tab_df) return cudaSuccess;
    const int64_t nph = (int64_t)p.nrings * (p.mmax + 1);
    const int64_t ntab = std::max<int64_t>(p.fft_tab_len, 1);
    float4 *tab = nullptr, *ph = nullptr;
    cudaError_t e = sht::dev_malloc(&tab, sizeof(float4) * ntab);
    if (e == cudaSuccess) e = sht::dev_malloc(&ph, sizeof(float4) * nph);
    if (e == cudaSuccess) {
        df_table_kernel<<<152 * 8, 256>>>(p.d_fft_tab, tab, p.fft_tab_len);
        df_table_kernel<<<152 * 8, 256>>>(p.d_phase, ph, nph);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(tab);
        cudaFree(ph);
        return e;
    }
    p.d_fft_tab_df = tab;
    p.d_phase_df = ph;
    return cudaSuccess;
}

cudaError_t build_phase_table(Plan &p)
{
    cudaError_t e;
    double *d_phi0 = nullptr;
    const size_t bytes = (size_t)p.nrings * (p.mmax + 1) * sizeof(double2);
    if ((e = sht::dev_malloc(&p.d_phase, bytes)) != cudaSuccess) return e;
    if ((e = sht::dev_malloc(&d_phi0, p.nrings * sizeof(double))) != cudaSuccess) return e;
    e = cudaMemcpy(d_phi0, p.phi0.data(), p.nrings * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        phase_table_kernel<<<152 * 8, 256>>>(d_phi0, p.nrings, p.mmax, p.d_phase);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_phi0);
    return e;
}

// Items: ring slots whose two rings share a length become one item; others are singles.
// Longest first.  Lengths get their radices, tables and (Bluestein) filters.
cudaError_t build_fft_tables(Plan &p)
{
    std::vector<FftItem> items;
    for (int s = 0; s < p.nslots; ++s) {
        const int a = p.slotN[s], b = p.slotS[s];
        if (a >= 0 && b >= 0 && p.nphi[a] == p.nphi[b]) {
            items.push_back({a, b, -1, (int)p.nphi[a]});
        } else {
            if (a >= 0) items.push_back({a, -1, -1, (int)p.nphi[a]});
            if (b >= 0) items.push_back({b, -1, -1, (int)p.nphi[b]});
        }
    }
    std::stable_sort(items.begin(), items.end(), [](const FftItem &x, const FftItem &y) { return x.n > y.n; });

    std::map<int, int> len_id;
    std::vector<TabJob> jobs;
    std::vector<int> blue_ids;
    int64_t off = 0;
    int maxlen = 1;
    p.lens.clear();
    for (auto &it : items) {
        auto f = len_id.find(it.n);
        if (f != len_id.end()) {
            it.len_id = f->second;
            continue;
        }
        FftLen L{};
        L.n = it.n;
        std::vector<int> fac;
        if (factor_smooth(it.n, fac)) {
            L.M = 0;
            L.tw = off;
            jobs.push_back({off, it.n, 0});
            off += it.n;
            maxlen = std::max(maxlen, it.n);
        } else {
            int M = 1;
            while (M < 2 * it.n - 1) M <<= 1;
            factor_smooth(M, fac);
            L.M = M;
            L.tw = off;
            jobs.push_back({off, M, 0});
            off += M;
            L.chirp = off;
            jobs.push_back({off, it.n, 1});
            off += it.n;
            L.filt = off;
            off += M;
            maxlen = std::max(maxlen, M);
            blue_ids.push_back((int)p.lens.size());
        }
        if ((int)fac.size() > 24) return cudaErrorInvalidValue;
        L.nfac = (int)fac.size();
        for (size_t i = 0; i < fac.size(); ++i) L.fac[i] = fac[i];
        it.len_id = (int)p.lens.size();
        len_id[it.n] = it.len_id;
        p.lens.push_back(L);
    }
    p.nitems = (int)items.size();
    p.nlens = (int)p.lens.size();
    p.fft_maxlen = maxlen;
    p.fft_tab_len = off;

    cudaError_t e;
    TabJob *d_jobs = nullptr;
    int *d_blue = nullptr;
    double2 *d_scr = nullptr;
    if ((e = sht::dev_malloc(&p.d_items, sizeof(FftItem) * items.size())) != cudaSuccess) return e;
    if ((e = sht::dev_malloc(&p.d_lens, sizeof(FftLen) * p.lens.size())) != cudaSuccess) return e;
    if ((e = sht::dev_malloc(&p.d_fft_tab, sizeof(double2) * std::max<int64_t>(off, 1))) != cudaSuccess) return e;
    if ((e = cudaMemcpy(p.d_items, items.data(), sizeof(FftItem) * items.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    if ((e = cudaMemcpy(p.d_lens, p.lens.data(), sizeof(FftLen) * p.lens.size(), cudaMemcpyHostToDevice)) !=
        cudaSuccess)
        return e;
    if ((e = sht::dev_malloc(&d_jobs, sizeof(TabJob) * jobs.size())) != cudaSuccess) return e;
    e = cudaMemcpy(d_jobs, jobs.data(), sizeof(TabJob) * jobs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        fill_tables_kernel<<<(unsigned)std::min<size_t>(jobs.size(), 152 * 8), 256>>>(d_jobs, (int)jobs.size(),
                                                                                   p.d_fft_tab);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && !blue_ids.empty()) {
        const int g = (int)std::min<size_t>(blue_ids.size(), 152);
        e = sht::dev_malloc(&d_blue, sizeof(int) * blue_ids.size());
        if (e == cudaSuccess) e = cudaMemcpy(d_blue, blue_ids.data(), sizeof(int) * blue_ids.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = sht::dev_malloc(&d_scr, (size_t)g * 3 * maxlen * sizeof(double2));
        if (e == cudaSuccess) {
            bluestein_filter_kernel<<<g, FFT_T>>>(p.d_lens, d_blue, (int)blue_ids.size(), p.d_fft_tab, d_scr, maxlen);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_jobs);
    cudaFree(d_blue);
    cudaFree(d_scr);
    return e;
}

// ---------------------------------------------------------------- batched form: host side

cudaError_t batch_ring_setup(const std::vector<const Plan *> &plans, const std::vector<const void *> &in,
                             const std::vector<void *> &out, const std::vector<int> &nmaps, bool synth,
                             BatchLaunch &L, int &maxlen)
{
    std::vector<RingArgs<F64>> jobs(plans.size());
    struct Key {
        int n;
        int4 u;
    };
    std::vector<Key> keys;
    maxlen = 1;
    for (size_t j = 0; j < plans.size(); ++j) {
        const Plan &p = *plans[j];
        RingArgs<F64> A = ring_args<F64>(p, p.d_fft_tab, p.d_phase, nullptr, nmaps[j]);
        if (synth) {
            A.delta_in = (const double2 *)in[j];
            A.map_out = (double *)out[j];
        } else {
            A.map_in = (const double *)in[j];
            A.delta_out = (double2 *)out[j];
        }
        jobs[j] = A;
        maxlen = std::max(maxlen, p.fft_maxlen);
        std::vector<FftItem> items(p.nitems);
        cudaError_t e = cudaMemcpy(items.data(), p.d_items, sizeof(FftItem) * p.nitems, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        for (int i = 0; i < p.nitems; ++i) {
            const FftLen &F = p.lens[items[i].len_id];
            const int cost = F.M ? 3 * F.M : F.n;  // Bluestein runs three DFTs of length M
            for (int g = 0; g < nmaps[j]; ++g) keys.push_back({cost, make_int4((int)j, i, g, 0)});
        }
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) { return a.n > b.n; });
    std::vector<int4> units(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) units[i] = keys[i].u;
    L.ntiles = (int)units.size();
    cudaError_t e = dev_malloc((RingArgs<F64> **)&L.jobs, sizeof(RingArgs<F64>) * std::max<size_t>(jobs.size(), 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(L.jobs, jobs.data(), sizeof(RingArgs<F64>) * jobs.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = dev_malloc(&L.tiles, sizeof(int4) * std::max<size_t>(units.size(), 1));
    if (e == cudaSuccess && !units.empty())
        e = cudaMemcpy(L.tiles, units.data(), sizeof(int4) * units.size(), cudaMemcpyHostToDevice);
    return e;
}

cudaError_t batch_ring_launch(const BatchLaunch &L, bool synth, double2 *scratch, int maxlen, int *counter, int grid,
                              cudaStream_t st)
{
    if (synth)
        ring_batch_kernel<F64, true><<<grid, FFT_T, 0, st>>>((const RingArgs<F64> *)L.jobs, L.tiles, L.ntiles, maxlen,
                                                             scratch, counter);
    else
        ring_batch_kernel<F64, false><<<grid, FFT_T, 0, st>>>((const RingArgs<F64> *)L.jobs, L.tiles, L.ntiles,
                                                              maxlen, scratch, counter);
    return cudaGetLastError();
}

namespace {
SHT_CHECK_TAKE_DEF(take_check)
}  // namespace
cudaError_t take_check_word_ring(int *w) { return take_check(w); }

}  // namespace sht
