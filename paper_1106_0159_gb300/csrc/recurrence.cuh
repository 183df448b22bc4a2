// Pieces of the lambda recurrence shared by the FP64, double-float and tensor-core Legendre
// kernels (legendre.cu, legendre_df.cu, legendre_tc.cu): the exponent test of the rescaling
// scheme, the sectoral start value mu_m sin^m(theta) with its binary exponent carried apart
// (eq. pmm with the reading sin^m; rescaling as described in legendre.cu), and the two
// thresholds every kernel must agree on.  Included inside each file's anonymous namespace, so
// every translation unit keeps its own internal copy.
#pragma once

#include "check.cuh"

constexpr int RESCALE_THR = 1023 + 256;  // biased exponent of y that triggers a rescale by 2^-512
constexpr double POLAR_SIN = 0.03;       // slot blocks starting below this sin(theta) use the Reinsch form

// biased exponent field of v
__device__ __forceinline__ int dexp(double v) { return (__double2hiint(v) >> 20) & 0x7ff; }

// v in [1, 2) times 2^e  <-  v (positive, normal)
__device__ __forceinline__ void normalise(double &v, int &e)
{
    int hi = __double2hiint(v);
    e += ((hi >> 20) & 0x7ff) - 1023;
    hi = (hi & 0x800fffff) | (1023 << 20);
    v = __hiloint2double(hi, __double2loint(v));
}

__device__ __forceinline__ double pow2i(int e)  // 2^e for -1022 <= e <= 1023
{
    return __hiloint2double((e + 1023) << 20, 0);
}

// lambda_mm = mu_m sin^m(theta) as y0 * 2^(512 k), k <= 0, y0 < 2 mu_m (binary powering of
// sin(theta) with the exponent kept in an int); 0 at the pole for m > 0
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
    // r * 2^er, r in [1, 2), er <= 0;  k = ceil(er / 512)
    const int kk = (er >= 0) ? 0 : -((-er) >> 9);
    const int rem = er - 512 * kk;  // in (-512, 0]
    y0 = mu * r * pow2i(rem);
    k = kk;
}
