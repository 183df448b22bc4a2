// Synthesis without any device allocation.
//
// Some callers cannot call cudaMalloc while they run a transform: code that
// runs inside another framework's memory pool or under a strict memory
// budget, or a caller that must not trigger the implicit device
// synchronisation a cudaMalloc/cudaFree may cause.  For them
// sht_alm2map_noalloc takes its scratch (the Delta intermediate, the
// precision form's digit tiles and the ring-FFT buffers) from one file-scope
// __device__ array instead of the plan's workspace.  It runs the plan's own
// arithmetic (sht_plan_set_mode), with the same kernels as sht_alm2map.
//
// The array is 64 MiB and exists on every GPU on which this library's module
// is loaded, for the life of the process.  Host code may not pass the
// array's symbol to a kernel (on the host it only names a stand-in object);
// its device address is looked up with cudaGetSymbolAddress once per device,
// on the first call made with that device current, and cached.
#include "sht_internal.h"

#include <algorithm>
#include <mutex>
#include <string>

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(64) << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" size_t sht_noalloc_scratch_bytes(void) { return NOALLOC_SCRATCH_BYTES; }

extern "C" sht_status sht_alm2map_noalloc(sht_plan_t plan, const void *alm, double *map, int nmaps, void *stream)
{
    if (!plan || nmaps < 0) return SHT_EINVAL;
    if (nmaps == 0) return SHT_OK;
    if (!alm || !map || alm == (const void *)map) return SHT_EINVAL;
    sht::Plan &p = plan->p;
    const bool prec = p.mode == SHT_MODE_SPLIT_BF16;
    if (prec && p.n_mlist > 0) {
        p.last_error = "sht_alm2map_noalloc: an m list is set: only the FP64 Legendre step computes a subset of m";
        return SHT_EUNSUPPORTED;
    }
    const size_t delta = ((size_t)nmaps * p.nrings * (p.mmax + 1) * sizeof(double2) + 255) & ~(size_t)255;
    const size_t per_cta = (size_t)3 * p.fft_maxlen * sizeof(double2);
    // the precision form's digit tiles of c_lm a_lm share the region after Delta with the ring
    // buffers (the Legendre step is done with them before the ring step starts)
    const size_t tc = prec ? sht::tc_workspace_bytes(p, nmaps) : 0;
    const size_t need = delta + std::max(per_cta, tc);
    if (need > NOALLOC_SCRATCH_BYTES) {
        p.last_error = "sht_alm2map_noalloc: " + std::to_string(nmaps) + " map(s) need " + std::to_string(need) +
                       " bytes of scratch; the static scratch holds " + std::to_string(NOALLOC_SCRATCH_BYTES) +
                       " bytes";
        return SHT_EINVAL;
    }
    int grid = sht::ring_grid(p);
    const size_t fit = (NOALLOC_SCRATCH_BYTES - delta) / per_cta;
    if ((size_t)grid > fit) grid = (int)fit;
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        p.last_error = std::string("sht_alm2map_noalloc: scratch address: ") + cudaGetErrorString(e);
        return SHT_ECUDA;
    }
    // Every Delta entry, digit tile and FFT buffer entry is written before it is read, so nothing
    // here needs clearing between calls.
    double2 *d = (double2 *)base;
    double2 *scratch = (double2 *)((char *)base + delta);
    cudaStream_t s = (cudaStream_t)stream;
    int n = 0;
    if (prec) {  // the plan's precision form, as sht_alm2map runs it
        e = sht::launch_legendre_synth_df_polar(p, (const double2 *)alm, d, nmaps, s, &n);
        p.launches[SHT_STAGE_LEGENDRE_SYNTH] += n;
        if (e == cudaSuccess) {
            e = sht::launch_legendre_synth_tc(p, (const double2 *)alm, d, scratch, nmaps, s, &n);
            p.launches[SHT_STAGE_LEGENDRE_SYNTH] += n;
        }
    } else {
        e = sht::launch_legendre_synth(p, (const double2 *)alm, d, nmaps, s, &n);
        p.launches[SHT_STAGE_LEGENDRE_SYNTH] += n;
    }
    if (e == cudaSuccess) {
        e = sht::launch_ring_synth_grid(p, d, map, scratch, nmaps, grid, s);
        p.launches[SHT_STAGE_RING_SYNTH] += 1;
    }
    if (e != cudaSuccess) {
        p.last_error = std::string("sht_alm2map_noalloc: ") + cudaGetErrorString(e);
        return SHT_ECUDA;
    }
    return SHT_OK;
}
