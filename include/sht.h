/*
 * sht.h -- C ABI of a single-GPU (sm_103a) spherical harmonic transform
 * library following Szydlarski, Esterie, Falcou, Grigori and Stompor,
 * "Parallel Spherical Harmonic Transforms on heterogeneous architectures
 * (GPUs/multi-core CPUs)", arXiv:1106.0159.
 *
 * Problem statement (Section 2.1, eqs. map2almDef and alm2mapDef; Section 2.2):
 *   synthesis  s(theta_r, phi_rj) = sum_{l<=lmax} sum_{|m|<=min(l,mmax)} a_lm Y_lm(theta_r, phi_rj)
 *   analysis   a_lm = sum_r w_r sum_j s(theta_r, phi_rj) conj(Y_lm(theta_r, phi_rj))
 * with Y_lm = lambda_lm(cos theta) exp(i m phi) (eq. YlmDef), lambda_lm the
 * normalised associated Legendre functions of eqs. (assLegRec)-(pm1m) without
 * a Condon-Shortley factor (lambda_mm > 0), a real map, so that
 * a_{l,-m} = (-1)^m conj(a_lm) and only m >= 0 is stored, and an
 * iso-latitude grid: ring r has nphi[r] equidistant pixels at
 * phi_rj = phi0[r] + 2 pi j / nphi[r] (Section 2.2).
 *
 * Layouts (all little-endian, no padding):
 *   alm   complex128 interleaved (re, im), [nmaps][nalm], m-major triangle:
 *         index(l, m) = m (2 lmax + 3 - m) / 2 + (l - m), 0 <= m <= mmax, m <= l <= lmax.
 *         Im a_l0 is ignored on input and written as 0 on output.
 *   map   double, [nmaps][npix], rings in the order given to sht_plan_create,
 *         pixel j of ring r at offset sum_{r' < r} nphi[r'] + j.
 *   delta complex128, [nmaps][nrings][mmax + 1]: Delta^A_m(r) of eq. (DeltaDef)
 *         (synthesis) or Delta^S_m(r) of eq. (almfftdef), weight included
 *         (analysis); ring order as for maps.
 *
 * Ownership and ordering: device pointers are owned by the caller and must
 * not alias; host arrays passed to the plan are copied.  Every transform call
 * is asynchronous and stream-ordered on `stream` (a cudaStream_t, NULL for
 * the legacy default stream).  Arguments are validated before anything is
 * enqueued; a call that returns an error has enqueued nothing and written
 * nothing.  A plan owns device tables and a scratch workspace that it grows
 * on demand; use one plan from one stream at a time.  CUDA failures map to
 * SHT_ECUDA and the CUDA error text is kept in the plan
 * (sht_plan_last_error).
 */
#ifndef SHT_H
#define SHT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sht_plan_s *sht_plan_t;

typedef enum {
    SHT_OK = 0,
    SHT_EINVAL = 1,        /* invalid argument (checked before any device work) */
    SHT_ENOMEM = 2,        /* host or device allocation failed */
    SHT_ECUDA = 3,         /* a CUDA call failed; see sht_plan_last_error */
    SHT_EUNSUPPORTED = 4,  /* valid but outside what this build implements */
    SHT_ETIMEOUT = 5       /* a bounded device wait gave up */
} sht_status;

typedef enum {
    SHT_GRID_CUSTOM = 0,
    SHT_GRID_HEALPIX = 1,
    SHT_GRID_GAUSS_LEGENDRE = 2
} sht_grid;

/*
 * Create a plan for rings (nphi[r], theta[r], phi0[r], w[r]), r < nrings,
 * and band limits lmax >= mmax >= 0 (Section 2.2; the weights w_n of
 * eq. map2almDef are taken per ring and applied to every pixel of the ring).
 * Host arrays, copied.  Rules: nrings >= 1, 1 <= nphi[r] <= 2^20,
 * 0 <= theta[r] <= pi, finite phi0 and w, lmax <= 16383.  Rings may come in
 * any order; rings mirrored about the equator are paired internally
 * (lambda_lm(-x) = (-1)^(l+m) lambda_lm(x)).  nphi may be smaller than
 * 2 mmax + 1, in which case the phi sums alias as the definition implies.
 * `grid` is informational.  Returns SHT_EINVAL for bad arguments,
 * SHT_ENOMEM / SHT_ECUDA when device set-up fails (nothing is leaked).
 */
sht_status sht_plan_create(sht_plan_t *out, sht_grid grid, int nrings,
                           const int64_t *nphi, const double *theta, const double *phi0,
                           const double *w, int lmax, int mmax);

/*
 * Arithmetic of the transforms:
 *   SHT_MODE_FP64        (default) every step in FP64.
 *   SHT_MODE_SPLIT_BF16  the precision form.  The lambda recurrence stays in FP64.  The sums of
 *                        eq. (matrix_vec) run on the tensor cores: the sum over l of the synthesis
 *                        and the sum over rings of the analysis, both operands cut into seven
 *                        balanced 7-bit digits, digit products accumulated in FP32 and combined in
 *                        FP64 or double-float.  The ring DFTs run in double-float on the FP32 pipe.
 *                        SHT_TUNE_PREC_ANAL and SHT_TUNE_PREC_RING select other kernels.  Relative
 *                        error against the exact transform <= 1e-9 of the output RMS.  Processes up
 *                        to 16 maps per pass over the recurrence.  Only the first 256 ring slots
 *                        (after north/south pairing, ordered from the poles) may lie within
 *                        sin(theta) < 0.03 of a pole; a grid with more polar slots (HEALPix
 *                        Nside >~ 7000) returns SHT_EUNSUPPORTED and stays in its old mode.
 * Switching to SHT_MODE_SPLIT_BF16 the first time runs one FP64 pass of the recurrence to
 * measure the scale of its values per (m, block of 128 ring slots) (synchronous; about the cost
 * of one single-map synthesis).  SHT_EINVAL for an unknown mode.
 */
typedef enum { SHT_MODE_FP64 = 0, SHT_MODE_SPLIT_BF16 = 1 } sht_mode;
sht_status sht_plan_set_mode(sht_plan_t plan, int mode);
int        sht_plan_mode(sht_plan_t plan);

/*
 * Device status word of the plan: bit 0 is set when a bounded wait inside a tensor-core kernel
 * gave up.  That kernel then skipped its output and released its resources, but MMAs it had
 * already issued may still have run, so treat the whole output of every call since the last
 * clear as untrusted, not only the block that timed out.  Waits for all work on the device
 * (cudaDeviceSynchronize, so kernels on non-blocking streams are finished too), then copies the
 * word to *status; clear != 0 resets it (and waits for the reset).  Returns SHT_ETIMEOUT while
 * bit 0 is set (read before the clear), SHT_OK otherwise.
 */
sht_status sht_plan_device_status(sht_plan_t plan, int *status, int clear);

/*
 * Restrict the FP64 Legendre steps of the plan to the listed m (the per-rank work of an
 * m-sharded transform, Section 4.1: the Legendre step of rank r covers its m and every ring, the
 * ring step its rings and every m).  With a list set, sht_legendre_synth / sht_alm2map compute
 * Delta_m only for listed m and write Delta_m = 0 for the others (a_lm of unlisted m is read as
 * zero), and sht_legendre_anal / sht_map2alm write a_lm = 0 for unlisted m.  The ring stages are
 * unchanged.  ms: host array of n distinct values in [0, mmax] (copied); n = 0 (ms may be NULL)
 * clears the list.  While a list is set, precision-form Legendre calls and the spin transforms
 * return SHT_EUNSUPPORTED.  Host call (synchronous copy of a flag table); SHT_EINVAL for a bad
 * list, which leaves the previous one in place.
 */
sht_status sht_plan_set_mlist(sht_plan_t plan, const int *ms, int n);

/*
 * Work accounting (host call, synchronous): the (l, m, ring-slot) recurrence steps of one pass,
 * *total = nalm * slots, and *live, those from the first 32-l chunk of each (m, block of 128
 * slots) in which some lambda is above the 2^-256 dropping threshold of the rescaling scheme
 * (steps before it contribute exactly zero and the precision-form kernels skip their sums).
 * Needs the tables made by the first switch to SHT_MODE_SPLIT_BF16; SHT_EINVAL before that.
 */
sht_status sht_plan_live_steps(sht_plan_t plan, int64_t *live, int64_t *total);

/*
 * Failure-path self test (no counterpart in the paper): enqueues on `stream` a one-block kernel
 * that waits, with a short poll budget, on an mbarrier nobody arrives at, the way the tensor-core
 * kernels wait for their MMAs; when the budget runs out it sets bit 0 of the plan's status word
 * and returns.  sht_plan_device_status then reports SHT_ETIMEOUT.  The GPU context stays usable.
 */
sht_status sht_plan_selftest_timeout(sht_plan_t plan, void *stream);

/* Free the plan, its device tables and workspace (synchronises the device). NULL is ignored. */
void sht_plan_destroy(sht_plan_t plan);

/*
 * Synthesis, Algorithm 2 (inverse transform): alm (device, [nmaps][nalm]
 * complex128) -> map (device, [nmaps][npix] double).  Runs the Legendre
 * step (eq. DeltaDef via eq. assLegRec) then the ring step (eq. Delta2map).
 */
sht_status sht_alm2map(sht_plan_t plan, const void *alm, double *map, int nmaps, void *stream);

/*
 * Analysis, Algorithm 1 (direct transform): map (device, [nmaps][npix]) ->
 * alm (device, [nmaps][nalm] complex128).  Runs the ring step (eq. almfftdef)
 * then the Legendre step (eq. almdef) and a fixed-order reduction over ring
 * blocks (deterministic: no atomics).
 */
sht_status sht_map2alm(sht_plan_t plan, const double *map, void *alm, int nmaps, void *stream);

/*
 * The transforms on caller-owned scratch (no counterpart in the paper): the same as sht_alm2map /
 * sht_map2alm, with the plan's own scratch replaced by `scratch` (device memory of at least
 * sht_workspace_bytes(plan, nmaps) bytes, 256-byte aligned, not shared with a call still in
 * flight).  One plan can then serve several streams at once, each with its own scratch: the
 * plan's tables are only read.  Calls on one plan must come from one host thread (the plan's
 * launch counters and stage timing are host state).  SHT_EINVAL for a missing, misaligned or too
 * small scratch, otherwise as sht_alm2map / sht_map2alm.
 */
sht_status sht_alm2map_ws(sht_plan_t plan, const void *alm, double *map, int nmaps, void *stream, void *scratch,
                          size_t scratch_bytes);
sht_status sht_map2alm_ws(sht_plan_t plan, const double *map, void *alm, int nmaps, void *stream, void *scratch,
                          size_t scratch_bytes);

/*
 * Spin-weighted (polarisation) transforms, the extension the paper names as future work
 * (Section 6), on the same plan and grid.  Only spin = 2 is implemented (SHT_EUNSUPPORTED
 * otherwise).  Functions sY_lm = slambda_lm(theta) exp(i m phi) in the normalisation of the scalar
 * lambda_lm (no Condon-Shortley factor): slambda_lm = sqrt((l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!))
 * sum_r C(l-s, r) C(l+s, r+s-m) (-1)^(l-r-s) sin(theta/2)^(2l-2r-s+m) cos(theta/2)^(2r+s-m).
 * Maps Q, U and coefficients E_lm, B_lm (l >= 2; entries with l < 2 are ignored on input and written
 * as 0; Im at m = 0 likewise):
 *   synthesis  Q + iU = sum_{l >= 2} sum_{|m| <= l} -(E_lm + i B_lm) 2Y_lm,
 *              with E_{l,-m} = (-1)^m conj(E_lm), B likewise (real Q, U);
 *   analysis   E_lm = -(2a_lm + 2a'_lm)/2, B_lm = i (2a_lm - 2a'_lm)/2 with
 *              2a_lm = sum_r w_r sum_j (Q + iU) conj(2Y_lm), 2a'_lm = sum_r w_r sum_j (Q - iU) conj((-2)Y_lm).
 * Layouts: alm complex128 [nmaps][2][nalm] (E then B, m-major triangle as above); map double
 * [nmaps][2][npix] (Q then U).  Arithmetic is FP64 for the Legendre step whatever the plan's mode
 * (the ring DFTs follow the mode, as in the scalar transforms); no Reinsch form on polar rings.
 * The first spin call on a plan builds its spin recurrence tables on the host and copies them to
 * the device (synchronous; 32 nalm bytes): make it before any stream capture.  Scratch grows on
 * demand to sht_spin_workspace_bytes(plan, nmaps).  Stream ordering and errors as sht_alm2map.
 */
sht_status sht_alm2map_spin(sht_plan_t plan, int spin, const void *alm, double *map, int nmaps, void *stream);
sht_status sht_map2alm_spin(sht_plan_t plan, int spin, const double *map, void *alm, int nmaps, void *stream);
size_t     sht_spin_workspace_bytes(sht_plan_t plan, int nmaps);

/* The four stages on their own (same layouts; delta as documented above). */
sht_status sht_legendre_synth(sht_plan_t plan, const void *alm, void *delta, int nmaps, void *stream); /* eq. DeltaDef */
sht_status sht_ring_synth(sht_plan_t plan, const void *delta, double *map, int nmaps, void *stream);    /* eq. Delta2map */
sht_status sht_ring_anal(sht_plan_t plan, const double *map, void *delta, int nmaps, void *stream);    /* eq. almfftdef */
sht_status sht_legendre_anal(sht_plan_t plan, const void *delta, void *alm, int nmaps, void *stream);  /* eq. almdef */

/* Sizes and indexing (pure host functions). */
int64_t sht_nalm(int lmax, int mmax);                 /* (mmax+1)(lmax+1) - mmax(mmax+1)/2, or -1 if invalid */
int64_t sht_alm_index(int lmax, int l, int m);        /* m (2 lmax + 3 - m)/2 + (l - m), or -1 if invalid */
int64_t sht_plan_npix(sht_plan_t plan);
int     sht_plan_nrings(sht_plan_t plan);
int     sht_plan_npairs(sht_plan_t plan);            /* ring slots after north/south pairing */
size_t  sht_workspace_bytes(sht_plan_t plan, int nmaps); /* scratch the transforms need for nmaps maps */

/*
 * Grow the plan's device scratch now to sht_workspace_bytes(plan, nmaps), so
 * that later calls with at most nmaps maps allocate nothing (a server keeps
 * its plans resident this way; the paper's memory estimate of Section 4.1
 * has the same parts: maps, a_lm and the Delta_m slabs).  Freeing a smaller
 * old scratch waits for the device.  SHT_EINVAL for a null plan or
 * nmaps < 1; SHT_ENOMEM (plan unchanged, old scratch released) when the
 * allocation fails.  Host call; no kernel runs.
 */
sht_status sht_plan_reserve(sht_plan_t plan, int nmaps);

/*
 * Launch tuning.  The paper has none: its tile sizes are fixed by its kernel
 * design.  Each knob bounds how many maps, or ring slots per thread, one
 * kernel launch takes.  Synthesis results are identical for every setting,
 * and the precision-form analysis is too (each map's sums keep their order).
 * The FP64 analysis order of the ring sums changes with the slots per thread,
 * so its results change within rounding.  The defaults are the settings
 * measured best on GB300 at lmax = 4096.  The scratch a call needs follows the
 * setting (sht_workspace_bytes); after a change, call sht_plan_reserve again
 * if calls must not allocate.  Host calls; SHT_EINVAL for a null plan, an
 * unknown knob or a value the knob does not take.
 */
typedef enum {
    SHT_TUNE_SYNTH_MAPS = 0, /* FP64 synthesis: maps per launch, 1, 2 or 4 (default 4) */
    SHT_TUNE_ANAL_MAPS = 1,  /* FP64 analysis: maps per launch, 1 or 2 (default 2) */
    SHT_TUNE_ANAL_SLOTS = 2, /* FP64 analysis: ring slots per thread, 1 or 4 (default 4, or 1 below 512 slots) */
    SHT_TUNE_DF_MAPS = 3,    /* precision-form analysis: maps per launch, 4, 8 or 16 (default 8) */
    SHT_TUNE_TC_MAPS = 4,    /* precision-form synthesis: maps per tensor-core launch, 8 or 16 (default 16) */
    SHT_TUNE_PREC_ANAL = 5,  /* precision-form analysis kernel: 0 double-float FP32, 1 tensor cores (default) */
    SHT_TUNE_PREC_RING = 6,  /* precision-form ring DFTs: 1 double-float FP32 (default), 0 FP64 */
    SHT_TUNE_RING_SMEM = 7,  /* ring DFTs: 1 in shared memory where the ring fits, 0 all through the
                                global scratch, 2 (default) shared memory for the FP64 DFTs and the
                                global scratch for the precision form's double-float DFTs; results
                                agree to rounding */
    SHT_TUNE_COUNT = 8
} sht_tune;
sht_status sht_plan_set_tuning(sht_plan_t plan, int knob, int value);
int sht_plan_tuning(sht_plan_t plan, int knob); /* the knob's value; -1 for a null plan or unknown knob */

/*
 * Batched form (no counterpart in the paper, which runs one transform at a time): many transforms
 * of one direction over plans of uneven lmax run as one persistent launch per stage.  The CTAs of a
 * launch take work tiles from a device queue in the order the host sorted them, longest first:
 * for the Legendre steps a tile is (transform, group of maps, m, block of ring slots), ordered by
 * its l-range times its maps (the min-max pairing of Section 4.2.1 turned into a queue); for the
 * ring steps a unit is (transform, ring pair, map), ordered by DFT length.  alm2map: Legendre
 * synthesis then ring synthesis; map2alm: ring analysis, Legendre analysis and the fixed-order
 * block reduction.  Job j is plans[j] on in[j] -> out[j] with nmaps[j] maps (device buffers in the
 * layouts of sht_alm2map / sht_map2alm; the batch keeps the pointers: write new inputs in place
 * between runs).  All plans must be in SHT_MODE_FP64 without an m list (SHT_EUNSUPPORTED
 * otherwise); the plans must outlive the batch.  The batch owns its Delta slabs, partial sums,
 * ring scratch and queue counters (allocated at creation, and again when a knob changes).
 * sht_batch_run enqueues only stream work on `stream` (a memset of the counters and the
 * launches), so it can be captured in a CUDA graph.  Results equal the one-plan calls bit for bit
 * (same kernels, same summation order), whatever the knobs.
 */
typedef struct sht_batch_s *sht_batch_t;
typedef enum {
    SHT_BATCH_SYNTH_MAPS = 0,  /* maps per Legendre synthesis tile: 1, 2 or 4 (default 4) */
    SHT_BATCH_LEG_CTAS = 1,    /* persistent Legendre CTAs per SM: 2, 4, 8 or 16 (default 8) */
    SHT_BATCH_RING_CTAS = 2,   /* persistent ring CTAs per SM: 1 to 4 (default 4) */
    SHT_BATCH_ANAL_MAPS = 3,   /* maps per Legendre analysis tile: 1 or 2 (default 2) */
    SHT_BATCH_ANAL_SLOTS = 4,  /* ring slots per thread of the analysis tiles: 1 or 4 (default 4) */
    SHT_BATCH_TUNE_COUNT = 5
} sht_batch_tune;
sht_status  sht_batch_create(sht_batch_t *out, int direction /* 0 alm2map, 1 map2alm */, int njobs,
                             const sht_plan_t *plans, const void *const *in, void *const *outs, const int *nmaps);
sht_status  sht_batch_set_tuning(sht_batch_t batch, int knob, int value); /* host call; rebuilds tiles and scratch */
int         sht_batch_tuning(sht_batch_t batch, int knob);
sht_status  sht_batch_run(sht_batch_t batch, void *stream);
int64_t     sht_batch_tiles(sht_batch_t batch, int stage); /* 0: Legendre tiles, 1: ring units; -1 if invalid */
const char *sht_batch_last_error(sht_batch_t batch);
void        sht_batch_destroy(sht_batch_t batch);          /* synchronises the device; NULL is ignored */

/*
 * Grid helpers (pure host).  HEALPix (Gorski et al. 2005, the grid of
 * Section 5): 4 nside - 1 rings north to south, caller arrays of that length,
 * equal weights 4 pi / (12 nside^2).  Gauss-Legendre: nrings rings at the
 * roots of P_nrings, north first, nphi pixels each, phi0 = 0,
 * w = 2 pi w_j / nphi with w_j the Gauss weights.  SHT_EINVAL on bad sizes.
 */
sht_status sht_geom_healpix(int nside, int64_t *nphi, double *theta, double *phi0, double *w);
sht_status sht_geom_gauss_legendre(int nrings, int64_t nphi, int64_t *nphi_out, double *theta,
                                   double *phi0, double *w);

/*
 * Per-stage accounting.  Kernel launches are always counted; with timing
 * enabled, every stage of every transform call is bracketed by CUDA events
 * recorded on the call's stream.  Stage ids (SHT_NSTAGES of them): 0 Legendre
 * synthesis, 1 ring synthesis, 2 ring analysis, 3 Legendre analysis, 4 ring-block
 * reduction of the FP64 analysis; 5 and 6 time one kernel alone, the main
 * tensor-core kernel of the precision-form synthesis (inside stage 0) and of the
 * precision-form analysis (inside stage 3), so that a roofline can divide by that
 * kernel's own time.  sht_plan_stage_times waits for the recorded events, adds
 * their durations to the running totals, and writes the totals
 * (ms[SHT_NSTAGES], launches[SHT_NSTAGES]); reset != 0 zeroes the totals afterwards.
 */
enum {
    SHT_STAGE_LEGENDRE_SYNTH = 0,
    SHT_STAGE_RING_SYNTH = 1,
    SHT_STAGE_RING_ANAL = 2,
    SHT_STAGE_LEGENDRE_ANAL = 3,
    SHT_STAGE_BLOCK_REDUCE = 4,
    SHT_STAGE_TC_SYNTH_KERNEL = 5,
    SHT_STAGE_TC_ANAL_KERNEL = 6,
    SHT_NSTAGES = 7
};
sht_status sht_plan_set_stage_timing(sht_plan_t plan, int enable);
sht_status sht_plan_stage_times(sht_plan_t plan, double *ms, int64_t *launches, int reset);

/*
 * Calibration (not part of the transforms): FP64 FMA throughput of the
 * current device in TFLOP/s (2 flops per FMA), from a short kernel of
 * independent FMA chains; the denominator of the Legendre stage's roofline.
 */
sht_status sht_fp64_fma_tflops(double *tflops);

/*
 * Synthesis for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a library service).  Same arguments, layouts, stream
 * ordering and arithmetic as sht_alm2map (the plan's mode: the FP64 path, or
 * the precision form's kernels on a SHT_MODE_SPLIT_BF16 plan), but the call
 * allocates nothing: its scratch (the Delta intermediate, then either the
 * precision form's digit tiles or the ring-FFT buffers) is a 64 MiB static
 * device array, sht_noalloc_scratch_bytes(), that every GPU loading this
 * library holds until the process exits.  Calls whose scratch
 * (16 nmaps nrings (mmax+1) bytes, rounded up to 256, plus the larger of one
 * ring-FFT buffer of 48 * max ring length bytes and, in the precision form,
 * the digit tiles of c_lm a_lm) exceeds it return SHT_EINVAL with the sizes
 * in sht_plan_last_error.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and caches it: make that
 * first call before any stream capture.  All calls share the one array, so
 * calls that overlap on the GPU (other streams, other threads, other plans)
 * race; serialise them.  The array keeps the last call's contents; nothing
 * in it needs to start at zero.
 */
sht_status sht_alm2map_noalloc(sht_plan_t plan, const void *alm, double *map, int nmaps, void *stream);
size_t     sht_noalloc_scratch_bytes(void);

/*
 * Host-side fault injection for tests (no counterpart in the paper): after n more successful device
 * allocations, the library's next allocation fails as if the device were out of memory (the call
 * returns cudaErrorMemoryAllocation internally, so the public call returns SHT_ENOMEM), and every
 * later one too, until the injector is switched off with a negative n.  Process-wide; returns the
 * previous setting.  Lets a test check that every allocation failure leaves nothing allocated.
 */
long sht_debug_fail_allocations_after(long n);

const char *sht_status_string(sht_status s);
const char *sht_plan_last_error(sht_plan_t plan);     /* "" when none */

#ifdef __cplusplus
}
#endif

#endif /* SHT_H */
