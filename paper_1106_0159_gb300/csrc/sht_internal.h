// Internal plan layout shared by the host plan code and the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "sht.h"

namespace sht {

// Every device allocation of the library goes through here: cudaMalloc, unless the host-side fault
// injector (sht_debug_fail_allocations_after) says this one fails, in which case it returns
// cudaErrorMemoryAllocation without allocating.
cudaError_t dev_malloc(void **ptr, size_t bytes);
template <class T>
cudaError_t dev_malloc(T **ptr, size_t bytes)
{
    return dev_malloc((void **)ptr, bytes);
}

// One complex FFT of length n on the ring stage: ring ringA rides on the real
// part and ringB (or -1) on the imaginary part (two real rings per complex
// transform).
struct FftItem {
    int ringA;
    int ringB;
    int len_id;   // index into the length table
    int n;
};

// Everything a CTA needs to run a length-n DFT with the + sign,
// y_k = sum_j x_j exp(+2 pi i j k / n).  Smooth n runs as Stockham passes
// with the radices fac[]; otherwise Bluestein with a power-of-two M.
struct FftLen {
    int n;
    int M;            // Bluestein convolution length, 0 when n is smooth
    int nfac;         // radices of n (smooth) or of M (Bluestein)
    int fac[24];
    int64_t tw;       // offset of exp(2 pi i k / n), k < n   (smooth) or of exp(2 pi i k / M), k < M (Bluestein)
    int64_t chirp;    // offset of exp(i pi j^2 / n), j < n   (Bluestein)
    int64_t filt;     // offset of FFT_M(h) / M, M entries      (Bluestein)
    // Shared-memory path (sm != 0; ringfft.cu): in-place DIF stages with radices rad[0 .. nst-1] over
    // the data in shared memory leave the spectrum in digit-reversed order, bin k at position
    // perm[k].  split != 0: stage 0 (radix p = rad[0], not smooth) runs as Bluestein DFTs of length p
    // in a second shared buffer, bat at a time: forward DIF of length Mb (radices brad), the filter
    // multiplied in the DIF output order, DIT back to natural order.
    int sm, nst, rad[16];
    int split, Mb, nbr, brad[16], bat;
    int64_t tw_n;     // exp(2 pi i k / n), k < n
    int64_t perm;     // offset into the int table: perm[k], k < n
    int64_t chirp_p;  // exp(i pi j^2 / p), j < p
    int64_t tw_M;     // exp(2 pi i k / Mb), k < Mb
    int64_t filt_M;   // filter of length Mb in DIF output order
    int smem_entries; // complex entries of shared memory the path takes: n + bat Mb + twq
    int twq;          // n / 4 when the quarter-wave table of exp(2 pi i k / n) is staged in shared memory, else 0
};

struct Plan {
    int lmax = 0, mmax = 0, nrings = 0;
    int64_t npix = 0, nalm = 0;
    int grid = 0;
    std::vector<int64_t> nphi, ofs;
    std::vector<double> theta, phi0, w;

    // ring slots after north/south pairing, ordered by colatitude of the north member
    int nslots = 0;
    std::vector<int> slotN, slotS;     // ring index or -1
    std::vector<double> slotTheta;     // colatitude used for lambda (northern hemisphere)

    // device tables
    int *d_slotN = nullptr, *d_slotS = nullptr;
    double *d_u = nullptr;      // 1 - cos(theta) per slot
    double *d_s = nullptr;      // sin(theta) per slot
    double *d_alpha = nullptr;  // [nalm] recurrence coefficients (see legendre.cu)
    double *d_cfac = nullptr;   // [nalm] lambda_lm = cfac * y_lm
    int mR = -1;                // Reinsch-form tables cover m <= mR
    double3 *d_rein = nullptr;  // [index(lmax, mR) + 1] (beta, rho, b0) for polar slots
    int64_t *d_ofs = nullptr;   // [nrings + 1]
    int *d_nphi = nullptr;      // [nrings]
    double *d_w = nullptr;      // [nrings]
    double2 *d_phase = nullptr; // [nrings][mmax + 1] exp(i m phi0_r)

    int nitems = 0;
    FftItem *d_items = nullptr;
    int nlens = 0;
    FftLen *d_lens = nullptr;
    std::vector<FftLen> lens;
    double2 *d_fft_tab = nullptr;
    float4 *d_fft_tab_df = nullptr;     // double-float copies for the precision form (built by set_mode)
    float4 *d_phase_df = nullptr;
    int64_t fft_tab_len = 0;
    int fft_maxlen = 0;         // per-CTA scratch length (complex entries, per buffer)
    int *d_fft_perm = nullptr;  // spectrum positions of the shared-memory DFTs
    int ring_smem = 0;          // dynamic shared memory of the ring kernels (bytes), 0: none fit
    int ring_occ = 1;           // ring CTAs resident per SM with that shared memory

    // precision form (split-bf16 contraction on the tensor cores)
    int mode = 0;                       // SHT_MODE_FP64 or SHT_MODE_SPLIT_BF16
    int64_t tc_total_chunks = 0;        // sum over m of ceil((lmax - m + 1) / 32)
    int64_t *d_tc_chunk_base = nullptr; // [mmax + 1]
    int *d_tc_chunk_m = nullptr;        // [tc_total_chunks]
    int *d_tc_Ey = nullptr;             // [2][mmax + 1][slot blocks]: scale exponent of y = lambda / c, first live chunk
    double2 *d_tc_ck_y = nullptr;       // [mmax + 1][slot blocks][128] recurrence state at the first live chunk & ~1
    int *d_tc_ck_k = nullptr;           // its rescaling exponents
    int *d_status = nullptr;            // device status word (bounded waits that gave up)
    int *d_mflag = nullptr;             // [mmax + 1] m computed by the FP64 Legendre steps (null: all)
    int n_mlist = 0;                    // number of listed m (0: all)
    double4 *d_spin_tab = nullptr;      // spin 2: [nalm] (alpha, alpha (1 + g), alpha (1 - g), c), built on first use
    double *d_spin_start = nullptr;     // spin 2: [mmax + 1] start coefficients S_m
    bool polar_first_slot = false;      // slot 0 runs the Reinsch form (sin(theta) < 0.03)
    int polar_syn_blocks = 0;     // leading 128-slot blocks whose first slot is polar (sin < 0.03): the
                                  // precision-form synthesis runs them in the Reinsch form for m <= mR

    // launch tuning (sht_tune): maps or slots per thread per launch
    int tune[SHT_TUNE_COUNT] = {4, 2, 4, 8, 16, 1, 1, 2};

    // workspace, grown on demand
    void *d_ws = nullptr;
    size_t ws_bytes = 0;

    // per-stage accounting: launches always, device time when enabled (stage ids as in sht.h;
    // the kernel-only stages are recorded by the launchers, which see a const plan)
    enum { NSTAGE = SHT_NSTAGES };
    bool timing = false;
    mutable int64_t launches[NSTAGE] = {};
    double stage_ms[NSTAGE] = {};
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    mutable std::vector<Pending> pending;
    mutable std::vector<cudaEvent_t> event_pool;

    std::string last_error;
};

// CUDA events recorded on the call's stream around a stage or one kernel launch while the plan's
// stage timing is on (sht_plan_set_stage_timing); done() queues the pair for sht_plan_stage_times.
struct StageEvents {
    const Plan &p;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr, b = nullptr;
    StageEvents(const Plan &pl, int st, cudaStream_t str);
    void done();
    ~StageEvents();
};

// launch helpers (legendre.cu, ringfft.cu); return cudaGetLastError(), count launches in *nlaunch
cudaError_t launch_legendre_synth(const Plan &p, const double2 *alm, double2 *delta, int nmaps, cudaStream_t st,
                                  int *nlaunch);
cudaError_t launch_legendre_anal(const Plan &p, const double2 *delta, double2 *partial, int nmaps, cudaStream_t st,
                                 int *nlaunch);
cudaError_t launch_block_reduce(const Plan &p, const double2 *partial, double2 *alm, int nmaps, cudaStream_t st);
int legendre_anal_nblk(const Plan &p);
int legendre_anal_default_slots(const Plan &p);  // default SHT_TUNE_ANAL_SLOTS for the plan's slot count
cudaError_t configure_tc_kernels();              // one-time function attributes (not stream work)
cudaError_t build_df_ring_tables(Plan &p);       // double-float DFT and phase tables (precision form)
cudaError_t configure_df_kernels();
size_t legendre_anal_partial_bytes(const Plan &p, int nmaps);
cudaError_t launch_ring_synth(const Plan &p, const double2 *delta, double *map, double2 *scratch, int nmaps,
                              cudaStream_t st);
cudaError_t launch_ring_anal(const Plan &p, const double *map, double2 *delta, double2 *scratch, int nmaps,
                             cudaStream_t st);
size_t ring_scratch_bytes(const Plan &p);
int ring_grid(const Plan &p);

// plan-time table builders (ringfft.cu); synchronous on the legacy stream
cudaError_t build_phase_table(Plan &p);
cudaError_t build_fft_tables(Plan &p);

int legendre_anal_df_nblk(const Plan &p);
size_t legendre_anal_df_partial_bytes(const Plan &p, int nmaps);
cudaError_t launch_legendre_anal_df(const Plan &p, const double2 *delta, double2 *alm, void *partial, int nmaps,
                                    cudaStream_t st, int *nlaunch);
size_t tc_workspace_bytes(const Plan &p, int nmaps);
// precision-form analysis on the tensor cores (groups of up to 16 maps, reduced per group)
cudaError_t launch_legendre_anal_tc(const Plan &p, const double2 *delta, double2 *alm, void *partial, int nmaps,
                                    cudaStream_t st, int *nlaunch);
size_t tc_anal_partial_bytes(const Plan &p, int nmaps);
// a_lm = c_lm * sum over blocks of double-float partials for the coefficient indices
// i0 .. i0 + nidx - 1 (nidx < 0: to nalm); partial (block, map, index i) at
// block * blk_stride + map * map_stride + (i - i0) * idx_stride; for i < fp64_lim blocks
// 0 .. polar_blocks - 1 are replaced by the FP64 partial polar[map * polar_stride + i]
cudaError_t launch_reduce_blocks_df(const float4 *partial, const double2 *polar, int64_t polar_stride,
                                    int polar_blocks, const double *cfac, double2 *alm, int nblk, int64_t nalm,
                                    int nmaps, int lmax, int64_t blk_stride, int64_t map_stride, int64_t idx_stride,
                                    int64_t fp64_lim, cudaStream_t st, int64_t i0 = 0, int64_t nidx = -1);
// precision-form Reinsch analysis of the first legendre_anal_df_polar_slots() slots for m <= mR
int legendre_anal_df_polar_slots();
cudaError_t launch_legendre_anal_df_polar(const Plan &p, const double2 *delta, double2 *polar, int64_t polar_stride,
                                          int nmaps, cudaStream_t st, int *nlaunch);
cudaError_t build_tc_scales(Plan &p);
cudaError_t launch_legendre_synth_tc(const Plan &p, const double2 *alm, double2 *delta, void *scratch, int nmaps,
                                     cudaStream_t st, int *nlaunch);
// precision-form synthesis of the polar slots 0 .. 127 for m <= mR (Reinsch form, double-float sums)
cudaError_t launch_legendre_synth_df_polar(const Plan &p, const double2 *alm, double2 *delta, int nmaps,
                                           cudaStream_t st, int *nlaunch);

// spin-2 transforms (spin.cu): Legendre steps on [nmaps][2] coefficient / Delta pairs
cudaError_t build_spin_tables(Plan &p);
size_t spin_partial_bytes(const Plan &p, int nmaps);
cudaError_t launch_spin_synth(const Plan &p, const double2 *alm, double2 *delta, int nmaps, cudaStream_t st,
                              int *nlaunch);
cudaError_t launch_spin_anal(const Plan &p, const double2 *delta, double2 *alm, double2 *partial, int nmaps,
                             cudaStream_t st, int *nlaunch);

// batched form (batch.cu, legendre.cu, ringfft.cu): one persistent launch per stage over the tiles
// of many plans, taken from a device counter in the host's order (longest first)
struct BatchLaunch {
    void *jobs = nullptr;     // device array of per-job kernel arguments
    int4 *tiles = nullptr;    // device tile list
    int ntiles = 0;
    int k = 1;                // analysis: ring slots per thread
    int smem = 0;             // ring DFTs: dynamic shared memory per CTA (bytes)
};
struct BatchReduceJob {
    const double2 *partial;
    const double *cfac;
    double2 *alm;
    int nblk;
    int64_t nalm;
    int nmaps;
    int lmax;
    int64_t blk_stride;
};
cudaError_t batch_legendre_synth_setup(const std::vector<const Plan *> &plans, const std::vector<const double2 *> &alm,
                                       const std::vector<double2 *> &delta, const std::vector<int> &nmaps,
                                       int maps_per_tile, BatchLaunch &L);
cudaError_t batch_legendre_anal_setup(const std::vector<const Plan *> &plans, const std::vector<const double2 *> &delta,
                                      const std::vector<double2 *> &partial, const std::vector<double2 *> &alm,
                                      const std::vector<int> &nmaps, int maps_per_tile, int slots_per_thread,
                                      BatchLaunch &L, BatchLaunch &R);
size_t batch_anal_partial_bytes(const Plan &p, int nmaps, int slots_per_thread);
cudaError_t batch_legendre_synth_launch(const BatchLaunch &L, int *counter, int grid, cudaStream_t st);
cudaError_t batch_legendre_anal_launch(const BatchLaunch &L, const BatchLaunch &R, int *counter, int grid,
                                       cudaStream_t st);
cudaError_t batch_ring_setup(const std::vector<const Plan *> &plans, const std::vector<const void *> &in,
                             const std::vector<void *> &out, const std::vector<int> &nmaps, bool synth,
                             BatchLaunch &L, int &maxlen);
cudaError_t batch_ring_launch(const BatchLaunch &L, bool synth, double2 *scratch, int maxlen, int *counter, int grid,
                              cudaStream_t st);

// bounds-check words of the checked build (bit 1; always 0 in the normal build): read and cleared
cudaError_t take_check_word_legendre(int *w);
cudaError_t take_check_word_df(int *w);
cudaError_t take_check_word_tc(int *w);
cudaError_t take_check_word_spin(int *w);
cudaError_t take_check_word_ring(int *w);

cudaError_t launch_ring_synth_grid(const Plan &p, const double2 *delta, double *map, double2 *scratch, int nmaps,
                                   int grid, cudaStream_t st);

}  // namespace sht

// the opaque handle of the C ABI
struct sht_plan_s {
    sht::Plan p;
};
