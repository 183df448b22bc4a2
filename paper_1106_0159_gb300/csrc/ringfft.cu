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
// Threads of the double-float DFT kernels that run one CTA per SM (shared-memory DFTs too large
// for two): 1024 at 64 registers each (lmax 4096, HEALPix 2048, 16 maps: synthesis / analysis
// 42.4 / 38.0 ms, against 46.4 / 38.8 with 512 threads at 128 registers); the FP64 ones keep 512.
constexpr int RING_DF_WIDE_T = 1024;

#include "check.cuh"
constexpr int MAXR = 13;

// Division by a divisor d fixed for a loop, without the integer divide: q = umulhi(b, M) with
// M = floor((2^32 - 1) / d) + 1 is floor(b / d) whenever b d < 2^32 (here b, d < 2^16).
// The constructor takes the largest b the loop divides; above the bound it divides plainly.
struct Div {
    unsigned M;
    int d;
    bool fast;
    __device__ __forceinline__ Div(int d_, int64_t bmax)
        : M(d_ > 1 ? 0xFFFFFFFFu / (unsigned)d_ + 1u : 0u), d(d_), fast(bmax * d_ < (1ll << 32))
    {
    }
    __device__ __forceinline__ int q(int b) const
    {
        return d > 1 ? (fast ? (int)__umulhi((unsigned)b, M) : b / d) : b;
    }
};

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
    static __device__ __forceinline__ T rot(T a, int q)  // i^q a
    {
        return q == 0 ? a : q == 1 ? make_double2(-a.y, a.x) : q == 2 ? make_double2(-a.x, -a.y) : make_double2(a.y, -a.x);
    }
    static __device__ __forceinline__ C half(C a) { return make_double2(0.5 * a.x, 0.5 * a.y); }
    using S = double;  // a real scalar
    static __device__ __forceinline__ S sfrom(double w) { return w; }
    static __device__ __forceinline__ C smul(C a, S w) { return make_double2(a.x * w, a.y * w); }
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
// a b + sg c d (sg = +-1) as one double-float: the two leading products exact by FMA, their sum by
// TwoSum, the four cross terms of the low parts added into the error term, one renormalisation
// (19 FP32 operations against 23 for two products and a sum)
__device__ __forceinline__ float2 dfn_dot2(float2 a, float2 b, float2 c, float2 d, float sg)
{
    const float p1 = a.x * b.x, p2 = sg * (c.x * d.x);
    const float e1 = fmaf(a.x, b.x, -p1), e2 = fmaf(sg * c.x, d.x, -p2);
    const float s = p1 + p2;
    const float v = s - p1;
    float t = (p1 - (s - v)) + (p2 - v);
    t += e1 + e2;
    t = fmaf(a.x, b.y, t);
    t = fmaf(a.y, b.x, t);
    t = fmaf(sg * c.x, d.y, t);
    t = fmaf(sg * c.y, d.x, t);
    const float h = s + t;
    return make_float2(h, t - (h - s));
}
// FP64 -> (hi, lo) from the bit pattern, on the integer pipe (an FP64 <-> FP32 conversion takes an
// FP64 issue slot, 1/64 of the FP32 rate on this part): hi = sign, exponent and the top 23 fraction
// bits; lo = the remaining 29 bits, rounded to 24.  Below 2^-74 the remainder would leave the FP32
// range and is dropped (|v| < 2^-74: an absolute error below 2^-97); below 2^-126 v flushes to zero.
// Such tiny values are common (the folded Delta_m of a polar ring past its turning point), so they
// take no conversion instruction either.
__device__ __forceinline__ float2 dfn_from(double v)
{
    const int hiw = __double2hiint(v);
    const unsigned low = (unsigned)__double2loint(v);
    const int ex = (hiw >> 20) & 0x7ff;
    const int e = ex - 1023;
    if (ex == 0 || e < -126) return make_float2(0.f, 0.f);
    const unsigned sign = (unsigned)hiw & 0x80000000u;
    const unsigned frac23 = (((unsigned)hiw & 0xFFFFFu) << 3) | (low >> 29);
    const float hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | frac23);
    if (e < 52 - 126) return make_float2(hi, 0.f);
    // the 29-bit remainder as a float rounded once: two exact 16- and 13-bit halves (2^23 + h - 2^23)
    // and one FMA, no integer-to-float conversion
    const unsigned rem = low & 0x1FFFFFFFu;
    const float rh = __uint_as_float(0x4B000000u | (rem >> 16)) - 8388608.0f;
    const float rl = __uint_as_float(0x4B000000u | (rem & 0xFFFFu)) - 8388608.0f;
    const float sc = (e - 52 >= -126) ? __uint_as_float((unsigned)(e - 52 + 127) << 23) : 0.f;
    const float lo = fmaf(rh, 65536.0f, rl) * sc;
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
        return mk(dfn_dot2(R(a), R(b), I(a), I(b), -1.f), dfn_dot2(R(a), I(b), I(a), R(b), 1.f));
    }
    static __device__ __forceinline__ C mul(C a, T b) { return mulc(a, b); }
    static __device__ __forceinline__ C conj(C a) { return make_float4(a.x, a.y, -a.z, -a.w); }
    static __device__ __forceinline__ C conjt(T a) { return conj(a); }
    static __device__ __forceinline__ C itimes(C a) { return make_float4(-a.z, -a.w, a.x, a.y); }
    static __device__ __forceinline__ T rot(T a, int q)  // i^q a
    {
        return q == 0 ? a
               : q == 1 ? make_float4(-a.z, -a.w, a.x, a.y)
               : q == 2 ? make_float4(-a.x, -a.y, -a.z, -a.w)
                        : make_float4(a.z, a.w, -a.x, -a.y);
    }
    static __device__ __forceinline__ C half(C a) { return make_float4(0.5f * a.x, 0.5f * a.y, 0.5f * a.z, 0.5f * a.w); }
    using S = float2;  // a real scalar, double-float
    static __device__ __forceinline__ S sfrom(double w) { return dfn_from(w); }
    static __device__ __forceinline__ C smul(C a, S w) { return mk(dfn_mul(R(a), w), dfn_mul(I(a), w)); }
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
    const Div by_nq(nq, nbf);
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int k1 = by_nq.q(b);
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

// ---------------------------------------------------------------- DFTs in shared memory
//
// In-place mixed-radix decimation in frequency: stage k (sub-transform length N_k, N_0 = n,
// N_(k+1) = N_k / p_k, stride m_k = N_k / p_k) takes, in every block of N_k entries, the p_k
// entries j + r m_k, forms their DFT of length p_k and multiplies output t by exp(2 pi i j t / N_k).
// Every butterfly reads and writes the same p_k places, so one buffer serves all stages; the
// spectrum ends in digit-reversed order (bin f = t_0 + p_0 t_1 + p_0 p_1 t_2 + ... at position
// t_0 m_0 + t_1 m_1 + ...), read back through a position table.  The transpose (decimation in
// time: the twiddles before the butterflies, stages in reverse order) takes digit-reversed input
// to natural order; Bluestein's convolution uses the pair, so it needs no reordering at all.
constexpr int DIF_MAXR = 13;

// exp(2 pi i e / n), e < n, from the plan's table in global memory
template <class P>
struct GlobalTw {
    const typename P::T *t;
    __device__ __forceinline__ typename P::T operator()(int64_t e) const { return t[e]; }
};
// ... or from its first quarter Q = n / 4 in shared memory: exp(2 pi i (q Q + r) / n) = i^q exp(2 pi i r / n)
template <class P>
struct QuarterTw {
    const typename P::T *t;
    int Q;
    Div byQ;
    __device__ __forceinline__ typename P::T operator()(int64_t e) const
    {
        const int q = byQ.q((int)e);
        return P::rot(t[(int)e - q * Q], q);
    }
};

template <class P, class TW>
__device__ void dif_stage(typename P::C *x, int nt, int n, int N, int p, const TW &tw)
{
    using C = typename P::C;
    const int m = N / p, tstep = n / N, per = n / p;
    const int nbf = nt * per;
    const Div by_per(per, nbf), by_m(m, per);
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int tr = nt > 1 ? by_per.q(b) : 0, w = b - tr * per;
        const int blk = by_m.q(w), j = w - blk * m;
        C *base = x + (int64_t)tr * n + (int64_t)blk * N + j;
        if (p == 4) {
            const C a0 = base[0], a1 = base[m], a2 = base[2 * m], a3 = base[3 * m];
            const C s02 = P::add(a0, a2), d02 = P::sub(a0, a2);
            const C s13 = P::add(a1, a3), d13 = P::sub(a1, a3);
            const C id13 = P::itimes(d13);
            C y1 = P::add(d02, id13), y2 = P::sub(s02, s13), y3 = P::sub(d02, id13);
            if (j) {
                y1 = P::mul(y1, tw((int64_t)j * tstep));
                y2 = P::mul(y2, tw((int64_t)2 * j * tstep));
                y3 = P::mul(y3, tw((int64_t)3 * j * tstep));
            }
            base[0] = P::add(s02, s13);
            base[m] = y1;
            base[2 * m] = y2;
            base[3 * m] = y3;
        } else if (p == 2) {
            const C a0 = base[0], a1 = base[m];
            C y1 = P::sub(a0, a1);
            if (j) y1 = P::mul(y1, tw((int64_t)j * tstep));
            base[0] = P::add(a0, a1);
            base[m] = y1;
        } else {
            C a[DIF_MAXR];
            for (int r = 0; r < p; ++r) a[r] = base[r * m];  // all p inputs held before any output
            const int wstep = n / p;  // exp(2 pi i / p) = tw(n / p)
            for (int t = 0; t < p; ++t) {
                C acc = a[0];
                int e = 0;
                for (int r = 1; r < p; ++r) {
                    e += t;
                    if (e >= p) e -= p;
                    acc = P::add(acc, P::mul(a[r], tw((int64_t)e * wstep)));
                }
                base[t * m] = (j && t) ? P::mul(acc, tw((int64_t)j * t * tstep)) : acc;
            }
        }
    }
}

// the transpose of dif_stage, for radix 2 or 4 (the Bluestein lengths are powers of two)
template <class P, class TW>
__device__ void dit_stage(typename P::C *x, int nt, int n, int N, int p, const TW &tw)
{
    using C = typename P::C;
    const int m = N / p, tstep = n / N, per = n / p;
    const int nbf = nt * per;
    const Div by_per(per, nbf), by_m(m, per);
    for (int b = threadIdx.x; b < nbf; b += blockDim.x) {
        const int tr = nt > 1 ? by_per.q(b) : 0, w = b - tr * per;
        const int blk = by_m.q(w), j = w - blk * m;
        C *base = x + (int64_t)tr * n + (int64_t)blk * N + j;
        if (p == 4) {
            C a0 = base[0], a1 = base[m], a2 = base[2 * m], a3 = base[3 * m];
            if (j) {
                a1 = P::mul(a1, tw((int64_t)j * tstep));
                a2 = P::mul(a2, tw((int64_t)2 * j * tstep));
                a3 = P::mul(a3, tw((int64_t)3 * j * tstep));
            }
            const C s02 = P::add(a0, a2), d02 = P::sub(a0, a2);
            const C s13 = P::add(a1, a3), d13 = P::sub(a1, a3);
            const C id13 = P::itimes(d13);
            base[0] = P::add(s02, s13);
            base[m] = P::add(d02, id13);
            base[2 * m] = P::sub(s02, s13);
            base[3 * m] = P::sub(d02, id13);
        } else {
            C a0 = base[0], a1 = base[m];
            if (j) a1 = P::mul(a1, tw((int64_t)j * tstep));
            base[0] = P::add(a0, a1);
            base[m] = P::sub(a0, a1);
        }
    }
}

// Length-n DFT with the + sign of D[0, n) in shared memory, in place, spectrum bin k left at
// D[perm[k]]; the split form uses Cb (bat Mb entries of shared memory) for Bluestein.  All
// threads of the CTA; returns after a barrier.
template <class P, class TW>
__device__ void smem_stages(const FftLen &F, const typename P::T *__restrict__ tab, typename P::C *D, typename P::C *Cb,
                            const TW &twn, int N, int k0)
{
    using C = typename P::C;
    const int n = F.n;
    if (F.split) {
        // stage 0, radix p: for every q < s the DFT of D[q + s r], r < p, by Bluestein, then the
        // stage twiddle exp(2 pi i q t / n), back into D[q + s t]
        const int p = F.rad[0], sN = n / p, Mb = F.Mb, lgM = __ffs(Mb) - 1;  // Mb a power of two
        const Div by_p(p, (int64_t)F.bat * p);
        const typename P::T *ch = tab + F.chirp_p, *twM = tab + F.tw_M, *fl = tab + F.filt_M;
        for (int q0 = 0; q0 < sN; q0 += F.bat) {
            const int nb = min(F.bat, sN - q0);
            for (int i = threadIdx.x; i < nb * Mb; i += blockDim.x) {
                const int tr = i >> lgM, r = i & (Mb - 1);
                Cb[i] = r < p ? P::mul(D[q0 + tr + sN * r], ch[r]) : P::zero();
            }
            int NM = Mb;
            for (int k = 0; k < F.nbr; ++k) {
                __syncthreads();
                dif_stage<P>(Cb, nb, Mb, NM, F.brad[k], GlobalTw<P>{twM});
                NM /= F.brad[k];
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nb * Mb; i += blockDim.x) Cb[i] = P::conj(P::mul(Cb[i], fl[i & (Mb - 1)]));
            for (int k = F.nbr - 1; k >= 0; --k) {
                NM *= F.brad[k];
                __syncthreads();
                dit_stage<P>(Cb, nb, Mb, NM, F.brad[k], GlobalTw<P>{twM});
            }
            __syncthreads();
            for (int i = threadIdx.x; i < nb * p; i += blockDim.x) {
                const int tr = by_p.q(i), t = i - tr * p, q = q0 + tr;
                C v = P::mul(P::conj(Cb[tr * Mb + t]), ch[t]);
                if (q && t) v = P::mul(v, twn((int64_t)q * t));
                D[q + sN * t] = v;
            }
            __syncthreads();
        }
        N = sN;
        k0 = 1;
    }
    for (int k = k0; k < F.nst; ++k) {
        __syncthreads();
        dif_stage<P>(D, 1, n, N, F.rad[k], twn);
        N /= F.rad[k];
    }
    __syncthreads();
}
template <class P>
__device__ void smem_dft(const FftLen &F, const typename P::T *__restrict__ tab, typename P::C *D, typename P::C *Cb)
{
    using C = typename P::C;
    using T = typename P::T;
    const int n = F.n;
    int N = n, k0 = 0;
    // the quarter-wave twiddle table after the data and the Bluestein buffers
    T *tq = (T *)(Cb + (F.split ? F.bat * F.Mb : 0));
    if (F.twq)
        for (int i = threadIdx.x; i < F.twq; i += blockDim.x) tq[i] = tab[F.tw_n + i];
    __syncthreads();
    if (F.twq)
        smem_stages<P>(F, tab, D, Cb, QuarterTw<P>{tq, F.twq, Div(F.twq, n)}, N, k0);
    else
        smem_stages<P>(F, tab, D, Cb, GlobalTw<P>{tab + F.tw_n}, N, k0);
}

__device__ __forceinline__ unsigned dynamic_smem_bytes()
{
    unsigned r;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}

// the shared-memory DFT of length F applies: the plan marks it, the launch asked for it and gave
// the shared memory it needs (otherwise the unit takes the global scratch path)
__device__ __forceinline__ bool smem_path(const FftLen &F, int use_sm)
{
    return F.sm && use_sm && (!F.split || F.bat >= 1) && F.smem_entries > 0 &&
           (unsigned)F.smem_entries <= dynamic_smem_bytes() / 16u;
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
    const int *perm;              // spectrum positions of the shared-memory DFTs
    int use_sm;                   // lengths with FftLen::sm take the shared-memory DFTs
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
    // the conjugate terms: -m = k mod n with m >= 1 (k < n)
    for (int m = n - k; m <= mmax; m += n) c = P::add(c, P::conj(P::mul(P::from(d[m]), ph[m])));
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
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const bool sm = smem_path(F, A.use_sm);
    C *D = sm ? (C *)ring_smem : B0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const C ca = fold_bin<P>(dA, pA, k, n, A.mmax);
        C z = ca;
        if (dB) {
            const C cb = fold_bin<P>(dB, pB, k, n, A.mmax);
            z = P::add(ca, P::itimes(cb));  // C_A + i C_B
        }
        D[k] = z;
    }
    double *outA = A.map_out + (int64_t)g * A.npix + A.ofs[it.ringA];
    double *outB = it.ringB >= 0 ? A.map_out + (int64_t)g * A.npix + A.ofs[it.ringB] : nullptr;
    if (sm) {
        smem_dft<P>(F, A.tab, D, D + n);
        const int *perm = A.perm + F.perm;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const C z = D[perm[j]];
            outA[j] = P::re(z);
            if (outB) outB[j] = P::im(z);
        }
    } else {
        __syncthreads();
        const C *X = cta_dft<P>(F, A.tab, B0, B1, B2);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const C z = X[j];
            outA[j] = P::re(z);
            if (outB) outB[j] = P::im(z);
        }
    }
    __syncthreads();
}

// MINB: CTAs per SM the register budget is set for (1 where the shared memory allows only one)
template <class P, int MINB, int NT = FFT_T>
__global__ void __launch_bounds__(NT, MINB) ring_synth_kernel(RingArgs<P> A)
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
    extern __shared__ __align__(16) unsigned char ring_smem[];
    const bool sm = smem_path(F, A.use_sm);
    C *D = sm ? (C *)ring_smem : B0;
    for (int j = threadIdx.x; j < n; j += blockDim.x)
        D[j] = P::from_re_im(sA[j], sB ? -sB[j] : 0.0);  // conj(s_A + i s_B)
    const C *X;       // conj(S): bin k at X[pos[k]] (pos the identity for the global path)
    const int *pos = nullptr;
    if (sm) {
        smem_dft<P>(F, A.tab, D, D + n);
        X = D;
        pos = A.perm + F.perm;
    } else {
        __syncthreads();
        X = cta_dft<P>(F, A.tab, B0, B1, B2);
    }
    const typename P::T *pA = A.phase + (int64_t)it.ringA * mstride;
    double2 *oA = A.delta_out + ((int64_t)g * A.nrings + it.ringA) * mstride;
    const typename P::S wA = P::sfrom(A.w[it.ringA]);  // the quadrature weight, applied before widening
    const Div by_n(n, A.mmax);
    if (it.ringB < 0) {
        for (int m = threadIdx.x; m <= A.mmax; m += blockDim.x) {
            const int k = m - n * by_n.q(m);
            const C S = P::conj(X[pos ? pos[k] : k]);
            const double2 v = P::to(P::smul(P::mulc(P::conjt(pA[m]), S), wA));
            oA[m] = make_double2(v.x, m == 0 ? 0.0 : v.y);
        }
    } else {
        const typename P::T *pB = A.phase + (int64_t)it.ringB * mstride;
        double2 *oB = A.delta_out + ((int64_t)g * A.nrings + it.ringB) * mstride;
        const typename P::S wB = P::sfrom(A.w[it.ringB]);
        for (int m = threadIdx.x; m <= A.mmax; m += blockDim.x) {
            const int k = m - n * by_n.q(m);
            const int kc = k ? n - k : 0;
            const C S = P::conj(X[pos ? pos[k] : k]);
            const C Sc = X[pos ? pos[kc] : kc];  // conj(S_{-k})
            const C SA = P::half(P::add(S, Sc));
            const C D = P::half(P::sub(S, Sc));
            const C SB = P::conj(P::itimes(P::conj(D)));  // D / (2 i) with D halved: -i D
            const double2 va = P::to(P::smul(P::mulc(P::conjt(pA[m]), SA), wA));
            const double2 vb = P::to(P::smul(P::mulc(P::conjt(pB[m]), SB), wB));
            oA[m] = make_double2(va.x, m == 0 ? 0.0 : va.y);
            oB[m] = make_double2(vb.x, m == 0 ? 0.0 : vb.y);
        }
    }
    __syncthreads();
}

template <class P, int MINB, int NT = FFT_T>
__global__ void __launch_bounds__(NT, MINB) ring_anal_kernel(RingArgs<P> A)
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
template <class P, bool SYNTH, int MINB>
__global__ void __launch_bounds__(FFT_T, MINB) ring_batch_kernel(const RingArgs<P> *__restrict__ jobs,
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

// Bluestein filters of the shared-memory path, moved from natural order into the DIF output order
struct PermJob {
    int64_t src, dst, pos;  // natural filter, permuted filter (tab), positions (int table)
    int M;
};
__global__ void permute_filter_kernel(const PermJob *jobs, int njobs, const int *pos, double2 *tab)
{
    for (int jb = blockIdx.x; jb < njobs; jb += gridDim.x) {
        const PermJob J = jobs[jb];
        for (int k = threadIdx.x; k < J.M; k += blockDim.x) tab[J.dst + pos[J.pos + k]] = tab[J.src + k];
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

// opt-in dynamic shared memory of one CTA on this part, less room for the kernels' static words
constexpr int RING_SMEM_CAP = 227 * 1024 - 256;

// every ring kernel may take up to RING_SMEM_CAP bytes of dynamic shared memory (set once)
cudaError_t ring_kernel_attributes()
{
    static cudaError_t done = [] {
        const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
        cudaError_t e = cudaSuccess;
        const void *k[] = {(const void *)ring_synth_kernel<F64, 1>,      (const void *)ring_synth_kernel<F64, 2>,
                           (const void *)ring_synth_kernel<DF, 1, RING_DF_WIDE_T>, (const void *)ring_synth_kernel<DF, 2>,
                           (const void *)ring_anal_kernel<F64, 1>,       (const void *)ring_anal_kernel<F64, 2>,
                           (const void *)ring_anal_kernel<DF, 1, RING_DF_WIDE_T>, (const void *)ring_anal_kernel<DF, 2>,
                           (const void *)ring_batch_kernel<F64, true, 1>, (const void *)ring_batch_kernel<F64, true, 2>,
                           (const void *)ring_batch_kernel<F64, false, 1>,
                           (const void *)ring_batch_kernel<F64, false, 2>};
        for (const void *f : k)
            if (e == cudaSuccess) e = cudaFuncSetAttribute(f, a, RING_SMEM_CAP);
        return e;
    }();
    return done;
}

// resident ring CTAs per SM at `smem` bytes of dynamic shared memory (the least over the kernels)
int ring_occupancy(int smem)
{
    int least = RING_CTAS_PER_SM, nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ring_synth_kernel<F64, 2>, FFT_T, smem) == cudaSuccess)
        least = std::min(least, nb);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ring_synth_kernel<DF, 2>, FFT_T, smem) == cudaSuccess)
        least = std::min(least, nb);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ring_anal_kernel<F64, 2>, FFT_T, smem) == cudaSuccess)
        least = std::min(least, nb);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, ring_anal_kernel<DF, 2>, FFT_T, smem) == cudaSuccess)
        least = std::min(least, nb);
    return std::max(1, least);
}

constexpr int RING_SMEM_HALF = 112 * 1024;  // two CTAs per SM, with room for static words

// Shared-memory form of a length-n DFT within `cap` complex entries: n = sm_part pb, sm_part smooth
// (its radices in sfac) and pb the product of the prime factors above 13; pb > 1 takes Bluestein
// DFTs of length pb on power-of-two buffers of Mb >= 2 pb - 1 entries, bat >= 1 at a time.  When
// 4 | n and room is left, the twq = n / 4 twiddles of the first quarter wave follow.  Returns
// whether it fits (entries = n + bat Mb + twq <= cap, at most 16 stages).
bool ring_sm_shape(int n, int64_t cap, int &pb, int &sm_part, int &Mb, int &bat, int &twq, int64_t &entries,
                   std::vector<int> &sfac)
{
    sm_part = 1;
    int r = n;
    for (int q : {2, 3, 5, 7, 11, 13})
        while (r % q == 0) {
            r /= q;
            sm_part *= q;
        }
    pb = r;
    factor_smooth(sm_part, sfac);
    Mb = 1;
    bat = 0;
    twq = 0;
    entries = n;
    if ((int)sfac.size() + (pb > 1) > 16 || n > cap) return false;
    if (pb > 1) {
        while (Mb < 2 * pb - 1) Mb <<= 1;
        if ((int64_t)n + Mb > cap) return false;
    }
    if (n % 4 == 0 && (int64_t)n + (pb > 1 ? Mb : 0) + n / 4 <= cap) twq = n / 4;
    if (pb > 1) {
        bat = (int)std::min<int64_t>(sm_part, (cap - n - twq) / Mb);
        entries = (int64_t)n + (int64_t)bat * Mb + twq;
    } else {
        entries = (int64_t)n + twq;
    }
    return bat >= 1 || pb == 1;
}

// Spectrum positions of the in-place DIF with radices r[0 .. k-1] over n: bin
// f = t_0 + r_0 t_1 + r_0 r_1 t_2 + ... sits at t_0 m_0 + t_1 m_1 + ..., m_s = n / (r_0 ... r_s).
void dif_positions(int n, const int *r, int k, int *pos)
{
    for (int f = 0; f < n; ++f) {
        int rem = f, N = n, at = 0;
        for (int s = 0; s < k; ++s) {
            const int m = N / r[s];
            at += (rem % r[s]) * m;
            rem /= r[s];
            N = m;
        }
        pos[f] = at;
    }
}

}  // namespace

namespace {

int ring_grid_max(const Plan &p) { return std::max(1, std::min(p.nitems, RING_CTAS_PER_SM * 152)); }

bool ring_df(const Plan &p) { return p.mode == SHT_MODE_SPLIT_BF16 && p.tune[SHT_TUNE_PREC_RING] && p.d_fft_tab_df; }

// Shared-memory DFTs: always with knob value 1; with the default 2 for the FP64 DFTs only.  The
// double-float DFTs are bound by the latency of their FP32 arithmetic, not by the scratch traffic, and
// ran faster through the global scratch at two CTAs per SM than in shared memory at one (lmax 4096,
// HEALPix 2048, 16 maps: 45 / 38 ms against 54 / 43 ms for synthesis / analysis).
bool ring_sm(const Plan &p)
{
    const int k = p.tune[SHT_TUNE_RING_SMEM];
    return p.ring_smem > 0 && (k == 1 || (k == 2 && !ring_df(p)));
}

// dynamic shared memory of one ring launch
int ring_smem_bytes(const Plan &p) { return ring_sm(p) ? p.ring_smem : 0; }

// one CTA per SM: the kernels built for one resident CTA (FP64: 512 threads at 128 registers,
// double-float: RING_DF_WIDE_T threads)
bool ring_wide(const Plan &p) { return ring_sm(p) && p.ring_occ < 2; }

}  // namespace

// global scratch for the lengths without the shared-memory path (and all lengths with it off)
size_t ring_scratch_bytes(const Plan &p)
{
    return (size_t)ring_grid_max(p) * 3 * (size_t)p.fft_maxlen * sizeof(double2);
}

// persistent grid: RING_CTAS_PER_SM CTAs per SM, fewer when the shared-memory DFTs leave room for fewer
int ring_grid(const Plan &p)
{
    const int g = ring_grid_max(p);
    return ring_sm(p) ? std::min(g, std::max(1, p.ring_occ) * 152) : g;
}

namespace {


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
    A.perm = p.d_fft_perm;
    A.use_sm = ring_sm(p) ? 1 : 0;
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
        if (ring_wide(p))
            ring_synth_kernel<DF, 1, RING_DF_WIDE_T><<<grid, RING_DF_WIDE_T, ring_smem_bytes(p), st>>>(A);
        else
            ring_synth_kernel<DF, 2><<<grid, FFT_T, ring_smem_bytes(p), st>>>(A);
    } else {
        RingArgs<F64> A = ring_args<F64>(p, p.d_fft_tab, p.d_phase, scratch, nmaps);
        A.delta_in = delta;
        A.map_out = map;
        if (ring_wide(p))
            ring_synth_kernel<F64, 1><<<grid, FFT_T, ring_smem_bytes(p), st>>>(A);
        else
            ring_synth_kernel<F64, 2><<<grid, FFT_T, ring_smem_bytes(p), st>>>(A);
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
        if (ring_wide(p))
            ring_anal_kernel<DF, 1, RING_DF_WIDE_T><<<ring_grid(p), RING_DF_WIDE_T, ring_smem_bytes(p), st>>>(A);
        else
            ring_anal_kernel<DF, 2><<<ring_grid(p), FFT_T, ring_smem_bytes(p), st>>>(A);
    } else {
        RingArgs<F64> A = ring_args<F64>(p, p.d_fft_tab, p.d_phase, scratch, nmaps);
        A.map_in = map;
        A.delta_out = delta;
        if (ring_wide(p))
            ring_anal_kernel<F64, 1><<<ring_grid(p), FFT_T, ring_smem_bytes(p), st>>>(A);
        else
            ring_anal_kernel<F64, 2><<<ring_grid(p), FFT_T, ring_smem_bytes(p), st>>>(A);
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
    std::vector<int> perm;           // int table of the shared-memory path
    std::vector<PermJob> pjobs;      // filters to move into DIF order
    struct Aux {
        int64_t chirp, tw, filt;
        int Mb, nbr, brad[16];
    };
    std::map<int, Aux> aux_of;       // Bluestein tables of the split stage, by its length
    std::vector<FftLen> pending_aux;  // their extra length entries, stored after the length in hand
    int64_t off = 0;
    int maxlen = 1, filt_maxlen = 1, smem_bytes = 0;
    p.lens.clear();
    // Shared memory of one launch: every CTA gets the largest need of the plan's lengths (one
    // Bluestein buffer per split length); the split lengths batch more Bluestein DFTs only within
    // that, or within half of the SM's shared memory when all fit there (two CTAs per SM).
    int64_t sm_budget = RING_SMEM_HALF / 16;
    for (const auto &it : items) {
        int pb, sm_part, Mb, bat, twq;
        int64_t need;
        std::vector<int> sf;
        if (ring_sm_shape(it.n, RING_SMEM_CAP / 16, pb, sm_part, Mb, bat, twq, need, sf))
            sm_budget = std::max(sm_budget, (int64_t)it.n + (pb > 1 ? Mb : 0) + twq);
    }
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

        // shared-memory path (ring_sm_shape), Bluestein DFTs of the split stage up to the budget
        int pb = 1, Mb = 1, bat = 0, sm_part = 1, twq = 0;
        int64_t entries = 0;
        std::vector<int> sfac;
        const bool fits = ring_sm_shape(it.n, sm_budget, pb, sm_part, Mb, bat, twq, entries, sfac);
        L.sm = 0;
        if (fits) {
            L.nst = 0;
            if (pb > 1) {
                auto a = aux_of.find(pb);
                if (a == aux_of.end()) {
                    Aux X{};
                    X.Mb = Mb;
                    std::vector<int> bf;
                    factor_smooth(X.Mb, bf);  // powers of 4 and at most one 2: at most 16 radices
                    X.nbr = (int)bf.size();
                    for (int i = 0; i < X.nbr; ++i) X.brad[i] = bf[i];
                    // natural-order tables and filter through an extra Bluestein length entry
                    FftLen B{};
                    B.n = pb;
                    B.M = X.Mb;
                    B.nfac = X.nbr;
                    for (int i = 0; i < X.nbr; ++i) B.fac[i] = bf[i];
                    X.tw = B.tw = off;
                    jobs.push_back({off, X.Mb, 0});
                    off += X.Mb;
                    X.chirp = B.chirp = off;
                    jobs.push_back({off, pb, 1});
                    off += pb;
                    B.filt = off;
                    off += X.Mb;
                    X.filt = off;
                    off += X.Mb;
                    const int64_t pos_at = (int64_t)perm.size();
                    perm.resize(perm.size() + X.Mb);
                    dif_positions(X.Mb, X.brad, X.nbr, perm.data() + pos_at);
                    pjobs.push_back({B.filt, X.filt, pos_at, X.Mb});
                    blue_ids.push_back((int)p.lens.size() + 1);  // stored right after L, below
                    filt_maxlen = std::max(filt_maxlen, X.Mb);
                    a = aux_of.emplace(pb, X).first;
                    pending_aux.push_back(B);
                }
                const Aux &X = a->second;
                L.split = 1;
                L.Mb = X.Mb;
                L.nbr = X.nbr;
                for (int i = 0; i < X.nbr; ++i) L.brad[i] = X.brad[i];
                L.chirp_p = X.chirp;
                L.tw_M = X.tw;
                L.filt_M = X.filt;
                L.bat = bat;
                L.rad[L.nst++] = pb;
            }
            for (int q : sfac) L.rad[L.nst++] = q;
            L.sm = 1;
            L.twq = twq;
            L.smem_entries = (int)entries;
            smem_bytes = std::max(smem_bytes, (int)entries * 16);
            if (L.M == 0) {
                L.tw_n = L.tw;
            } else {
                L.tw_n = off;
                jobs.push_back({off, it.n, 0});
                off += it.n;
            }
            L.perm = (int64_t)perm.size();
            perm.resize(perm.size() + it.n);
            dif_positions(it.n, L.rad, L.nst, perm.data() + L.perm);
        }
        it.len_id = (int)p.lens.size();
        len_id[it.n] = it.len_id;
        p.lens.push_back(L);
        for (const FftLen &B : pending_aux) p.lens.push_back(B);
        pending_aux.clear();
    }
    p.nitems = (int)items.size();
    p.nlens = (int)p.lens.size();
    p.fft_maxlen = maxlen;
    p.fft_tab_len = off;
    p.ring_smem = smem_bytes;
    maxlen = std::max(maxlen, filt_maxlen);  // scratch of the filter kernel

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
    PermJob *d_pj = nullptr;
    if (e == cudaSuccess && !perm.empty()) {
        e = sht::dev_malloc(&p.d_fft_perm, sizeof(int) * perm.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(p.d_fft_perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess && !pjobs.empty()) {
            e = sht::dev_malloc(&d_pj, sizeof(PermJob) * pjobs.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(d_pj, pjobs.data(), sizeof(PermJob) * pjobs.size(), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) {
                // after the filters: same (legacy default) stream
                permute_filter_kernel<<<(unsigned)std::min<size_t>(pjobs.size(), 152 * 8), 256>>>(
                    d_pj, (int)pjobs.size(), p.d_fft_perm, p.d_fft_tab);
                e = cudaGetLastError();
            }
        }
    }
    if (e == cudaSuccess) e = ring_kernel_attributes();
    if (e == cudaSuccess) p.ring_occ = ring_occupancy(p.ring_smem);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_jobs);
    cudaFree(d_blue);
    cudaFree(d_scr);
    cudaFree(d_pj);
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
    int smem = 0;
    for (size_t j = 0; j < plans.size(); ++j) {
        const Plan &p = *plans[j];
        RingArgs<F64> A = ring_args<F64>(p, p.d_fft_tab, p.d_phase, nullptr, nmaps[j]);
        A.use_sm = p.ring_smem > 0 ? 1 : 0;  // the batch always takes the shared-memory DFTs
        smem = std::max(smem, p.ring_smem);
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
            // Bluestein runs three DFTs of length M; the split form 2 s DFTs of length Mb
            const int cost = (F.sm && F.split) ? F.n + 2 * (F.n / F.rad[0]) * F.Mb : F.sm ? F.n : F.M ? 3 * F.M : F.n;
            for (int g = 0; g < nmaps[j]; ++g) keys.push_back({cost, make_int4((int)j, i, g, 0)});
        }
    }
    std::stable_sort(keys.begin(), keys.end(), [](const Key &a, const Key &b) { return a.n > b.n; });
    std::vector<int4> units(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) units[i] = keys[i].u;
    L.ntiles = (int)units.size();
    L.smem = smem;
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
    const RingArgs<F64> *J = (const RingArgs<F64> *)L.jobs;
    const bool wide = L.smem > RING_SMEM_HALF;  // one CTA per SM
    if (synth && wide)
        ring_batch_kernel<F64, true, 1><<<grid, FFT_T, L.smem, st>>>(J, L.tiles, L.ntiles, maxlen, scratch, counter);
    else if (synth)
        ring_batch_kernel<F64, true, 2><<<grid, FFT_T, L.smem, st>>>(J, L.tiles, L.ntiles, maxlen, scratch, counter);
    else if (wide)
        ring_batch_kernel<F64, false, 1><<<grid, FFT_T, L.smem, st>>>(J, L.tiles, L.ntiles, maxlen, scratch, counter);
    else
        ring_batch_kernel<F64, false, 2><<<grid, FFT_T, L.smem, st>>>(J, L.tiles, L.ntiles, maxlen, scratch, counter);
    return cudaGetLastError();
}

namespace {
SHT_CHECK_TAKE_DEF(take_check)
}  // namespace
cudaError_t take_check_word_ring(int *w) { return take_check(w); }

}  // namespace sht
