// Bounds checks of the checked build (nvcc -DSHT_CHECK), in place of a memory checker: before a
// kernel writes or reads global memory at an index computed from plan tables (ring, m, slot,
// coefficient index, pixel offset), SHT_CHK(cond) tests the index against its bounds; when the test
// fails it sets bit 1 of this translation unit's check word and the access is skipped.
// sht_plan_device_status folds every unit's word into bit 1 of the plan's status word.  In the
// normal build SHT_CHK is `true` and costs nothing.  Included inside each unit's anonymous
// namespace, so every translation unit has its own word.
#pragma once

#ifdef SHT_CHECK
__device__ int g_check_word;
__device__ __forceinline__ bool sht_chk_fail()
{
    atomicOr(&g_check_word, 2);
    return false;
}
#define SHT_CHK(cond) ((cond) ? true : sht_chk_fail())
// host: read this unit's word and clear it
#define SHT_CHECK_TAKE_DEF(name)                                                                    \
    cudaError_t name(int *w)                                                                        \
    {                                                                                               \
        int v = 0;                                                                                  \
        cudaError_t e = cudaMemcpyFromSymbol(&v, g_check_word, sizeof(int));                        \
        const int zero = 0;                                                                         \
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_check_word, &zero, sizeof(int));            \
        *w |= v;                                                                                    \
        return e;                                                                                   \
    }
#else
#define SHT_CHK(cond) true
#define SHT_CHECK_TAKE_DEF(name)                                                                    \
    cudaError_t name(int *) { return cudaSuccess; }
#endif
