// Host side of the library: argument checks, plan construction (ring
// pairing, recurrence tables, ring-stage tables), workspace, and the C ABI
// entry points declared in include/sht.h.
#include "sht_internal.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>

namespace sht {

// allocations left before the injected failure; negative: no injection
static std::atomic<long> g_alloc_budget{-1};

cudaError_t dev_malloc(void **ptr, size_t bytes)
{
    long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) {
            *ptr = nullptr;
            return cudaErrorMemoryAllocation;
        }
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    return cudaMalloc(ptr, bytes);
}

static cudaEvent_t pool_event(const Plan &p)
{
    if (!p.event_pool.empty()) {
        cudaEvent_t e = p.event_pool.back();
        p.event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// NVTX range names of the stages (sht.h stage ids); the ranges mark where each stage is enqueued
// (header-only NVTX 3: without an attached tool the calls do nothing)
static const char *const kStageNames[SHT_NSTAGES] = {"sht legendre_synth", "sht ring_synth", "sht ring_anal",
                                                     "sht legendre_anal", "sht block_reduce", "sht tc_synth_kernel",
                                                     "sht tc_anal_kernel"};

StageEvents::StageEvents(const Plan &pl, int st, cudaStream_t str) : p(pl), stage(st), s(str)
{
    nvtxRangePushA(kStageNames[st]);
    if (p.timing) {
        a = pool_event(p);
        b = pool_event(p);
        if (a && b) cudaEventRecord(a, s);
    }
}

void StageEvents::done()
{
    if (a && b) {
        cudaEventRecord(b, s);
        p.pending.push_back({stage, a, b});
        a = b = nullptr;
    }
}

StageEvents::~StageEvents()
{
    if (a) p.event_pool.push_back(a);
    if (b) p.event_pool.push_back(b);
    nvtxRangePop();
}

}  // namespace sht

using sht::Plan;

namespace {

const double PI = 3.14159265358979323846;

bool is_finite(double v) { return std::isfinite(v); }

sht_status cuda_fail(Plan &p, cudaError_t e, const char *where)
{
    p.last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return (e == cudaErrorMemoryAllocation) ? SHT_ENOMEM : SHT_ECUDA;
}

void free_plan_device(Plan &p)
{
    void *ptrs[] = {p.d_slotN, p.d_slotS, p.d_u,     p.d_s,     p.d_alpha,   p.d_cfac,    p.d_ofs, p.d_nphi,
                    p.d_w,     p.d_phase, p.d_items, p.d_lens,  p.d_fft_tab, p.d_rein, p.d_ws,
                    p.d_tc_chunk_base, p.d_tc_chunk_m, p.d_tc_Ey, p.d_status, p.d_fft_tab_df, p.d_phase_df,
                    p.d_tc_ck_y, p.d_tc_ck_k, p.d_spin_tab, p.d_spin_start, p.d_mflag, p.d_fft_perm};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    p.d_slotN = p.d_slotS = nullptr;
    p.d_u = p.d_s = p.d_alpha = p.d_cfac = p.d_w = nullptr;
    p.d_ofs = nullptr;
    p.d_nphi = nullptr;
    p.d_phase = nullptr;
    p.d_items = nullptr;
    p.d_lens = nullptr;
    p.d_fft_tab = nullptr;
    p.d_rein = nullptr;
    p.d_ws = nullptr;
    p.d_tc_chunk_base = nullptr;
    p.d_tc_chunk_m = nullptr;
    p.d_tc_Ey = nullptr;
    p.d_status = nullptr;
    p.d_fft_tab_df = nullptr;
    p.d_phase_df = nullptr;
    p.d_tc_ck_y = nullptr;
    p.d_tc_ck_k = nullptr;
    p.d_spin_tab = nullptr;
    p.d_spin_start = nullptr;
    p.d_mflag = nullptr;
    p.n_mlist = 0;
    p.d_fft_perm = nullptr;
    p.ws_bytes = 0;
}

template <class T>
cudaError_t upload(T **dst, const T *src, size_t n)
{
    cudaError_t e = sht::dev_malloc((void **)dst, sizeof(T) * std::max<size_t>(n, 1));
    if (e != cudaSuccess) return e;
    if (n) e = cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
    return e;
}

// North/south pairing: rings whose colatitudes add to pi (within a few ulp of
// pi) share one lambda recurrence.  Every slot is evaluated at the northern
// colatitude of the pair.
void pair_rings(Plan &p)
{
    const double tol = 4e-15;
    std::vector<int> idx(p.nrings);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return p.theta[a] < p.theta[b]; });
    struct Slot {
        int n, s;
        double th;
    };
    std::vector<Slot> slots;
    auto single = [&](int r) {
        if (p.theta[r] <= 0.5 * PI)
            slots.push_back({r, -1, p.theta[r]});
        else
            slots.push_back({-1, r, PI - p.theta[r]});
    };
    int i = 0, j = p.nrings - 1;
    while (i <= j) {
        if (i == j) {
            single(idx[i]);
            break;
        }
        const int a = idx[i], b = idx[j];
        const double sum = p.theta[a] + p.theta[b];
        if (std::fabs(sum - PI) <= tol) {
            slots.push_back({a, b, p.theta[a]});
            ++i;
            --j;
        } else if (sum < PI) {
            single(a);
            ++i;
        } else {
            single(b);
            --j;
        }
    }
    std::stable_sort(slots.begin(), slots.end(), [](const Slot &x, const Slot &y) { return x.th < y.th; });
    p.nslots = (int)slots.size();
    p.slotN.resize(slots.size());
    p.slotS.resize(slots.size());
    p.slotTheta.resize(slots.size());
    for (size_t k = 0; k < slots.size(); ++k) {
        p.slotN[k] = slots[k].n;
        p.slotS[k] = slots[k].s;
        p.slotTheta[k] = slots[k].th;
    }
}

// Recurrence tables in the normalised variable y_l = lambda_l / c_l (see legendre.cu):
// alpha[index(m,m)] = mu_m, alpha[index(m+1,m)] = sqrt(2m+3) (eq. pm1m),
// alpha[index(l,m)] = beta_l c_{l-1} / c_l for l >= m+2 (eqs. assLegRec, betaDef),
// cfac[index(l,m)] = c_l with c_m = c_{m+1} = 1, c_l = (beta_l / beta_{l-1}) c_{l-2}.
void recurrence_tables(int lmax, int mmax, std::vector<double> &alpha, std::vector<double> &cfac)
{
    const int64_t nalm = sht_nalm(lmax, mmax);
    alpha.assign(nalm, 0.0);
    cfac.assign(nalm, 0.0);
    long double mu2 = 1.0L / (4.0L * 3.14159265358979323846264338327950288L);  // mu_0^2
    for (int m = 0; m <= mmax; ++m) {
        if (m > 0) mu2 *= (long double)(2 * m + 1) / (long double)(2 * m);  // eq. (pmm)
        const int64_t base = sht_alm_index(lmax, m, m);
        alpha[base] = (double)std::sqrt(mu2);
        cfac[base] = 1.0;
        if (m + 1 > lmax) continue;
        alpha[base + 1] = std::sqrt(2.0 * m + 3.0);
        cfac[base + 1] = 1.0;
        double c2 = 1.0, c1 = 1.0;            // c_{l-2}, c_{l-1}
        double bprev = std::sqrt(2.0 * m + 3.0);  // beta_{m+1,m}
        const double m2 = (double)m * m;
        for (int l = m + 2; l <= lmax; ++l) {
            const double L = (double)l;
            const double b = std::sqrt((4.0 * L * L - 1.0) / (L * L - m2));
            const double c = (b / bprev) * c2;
            alpha[base + (l - m)] = b * c1 / c;
            cfac[base + (l - m)] = c;
            c2 = c1;
            c1 = c;
            bprev = b;
        }
    }
}

// Reinsch-form tables for polar slots, m <= mR: (beta_l, rho_l, b0_l) with
// rho_l = beta_l / beta_{l-1} - 1 and b0_l = beta_l - 2 - rho_l, both from
// cancellation-free forms: delta_l = beta_l - 2 = (4m^2 - 1) / ((l^2 - m^2)(beta_l + 2)),
// rho_l = (delta_l - delta_{l-1}) / beta_{l-1}, b0_l = delta_l - rho_l.  Entries at
// l = m and l = m+1 seed the recurrence (see legendre.cu).
void reinsch_tables(int lmax, int mR, std::vector<double3> &rein)
{
    if (mR < 0) {
        rein.clear();
        return;
    }
    const int64_t n = sht_alm_index(lmax, lmax, mR) + 1;
    rein.assign(n, make_double3(0.0, 0.0, 0.0));
    for (int m = 0; m <= mR; ++m) {
        const int64_t base = sht_alm_index(lmax, m, m);
        rein[base] = make_double3(0.0, 0.0, 0.0);
        if (m + 1 > lmax) continue;
        const double b1 = std::sqrt(2.0 * m + 3.0);
        rein[base + 1] = make_double3(b1, -1.0, b1 - 1.0);
        const double m2 = (double)m * m, q = 4.0 * m2 - 1.0;
        double bprev = b1;
        double dprev = q / ((2.0 * m + 1.0) * (b1 + 2.0));  // beta_{m+1} - 2
        for (int l = m + 2; l <= lmax; ++l) {
            const double L = (double)l;
            const double b = std::sqrt((4.0 * L * L - 1.0) / (L * L - m2));
            const double d = q / ((L * L - m2) * (b + 2.0));
            const double rho = (d - dprev) / bprev;
            rein[base + (l - m)] = make_double3(b, rho, d - rho);
            bprev = b;
            dprev = d;
        }
    }
}

sht_status ensure_workspace(Plan &p, size_t need)
{
    if (p.ws_bytes >= need) return SHT_OK;
    if (p.d_ws) {
        cudaError_t e = cudaFree(p.d_ws);
        p.d_ws = nullptr;
        p.ws_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(p, e, "workspace free");
    }
    cudaError_t e = sht::dev_malloc(&p.d_ws, need);
    if (e != cudaSuccess) {
        p.d_ws = nullptr;
        cudaGetLastError();
        return cuda_fail(p, e, "workspace allocation");
    }
    p.ws_bytes = need;
    return SHT_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

size_t delta_bytes(const Plan &p, int nmaps) { return (size_t)nmaps * p.nrings * (p.mmax + 1) * sizeof(double2); }

sht_status check_call(sht_plan_t plan, const void *in, const void *out, int nmaps)
{
    if (!plan) return SHT_EINVAL;
    if (nmaps < 0) return SHT_EINVAL;
    if (nmaps > 0 && (!in || !out)) return SHT_EINVAL;
    if (nmaps > 0 && in == out) return SHT_EINVAL;
    return SHT_OK;
}



// --- stage runners: launches plus optional event bracketing on the call's stream
using sht::StageEvents;
using StageScope = StageEvents;

// tc_scratch: tc_workspace_bytes(p, min(nmaps, 16)) bytes, used in the precision form only
sht_status mlist_guard(Plan &p)
{
    if (p.n_mlist > 0 && p.mode != SHT_MODE_FP64) {
        p.last_error = "an m list is set: only the FP64 Legendre steps compute a subset of m";
        return SHT_EUNSUPPORTED;
    }
    return SHT_OK;
}

sht_status run_legendre_synth(Plan &p, const double2 *alm, double2 *delta, void *tc_scratch, int nmaps,
                              cudaStream_t s)
{
    if (sht_status g = mlist_guard(p)) return g;
    StageScope sc(p, 0, s);
    int n = 0;
    cudaError_t e;
    if (p.mode == SHT_MODE_SPLIT_BF16) {
        e = sht::launch_legendre_synth_df_polar(p, alm, delta, nmaps, s, &n);
        p.launches[0] += n;
        if (e == cudaSuccess) {
            e = sht::launch_legendre_synth_tc(p, alm, delta, tc_scratch, nmaps, s, &n);
            p.launches[0] += n;
        }
    } else {
        e = sht::launch_legendre_synth(p, alm, delta, nmaps, s, &n);
        p.launches[0] += n;
    }
    if (e != cudaSuccess) return cuda_fail(p, e, "legendre_synth");
    sc.done();
    return SHT_OK;
}

size_t synth_scratch_bytes(const Plan &p, int nmaps)
{
    return p.mode == SHT_MODE_SPLIT_BF16 ? sht::tc_workspace_bytes(p, nmaps) : 0;
}

size_t anal_partial_bytes(const Plan &p, int nmaps)
{
    if (p.mode != SHT_MODE_SPLIT_BF16) return sht::legendre_anal_partial_bytes(p, nmaps);
    return p.tune[SHT_TUNE_PREC_ANAL] ? sht::tc_anal_partial_bytes(p, nmaps)
                                      : sht::legendre_anal_df_partial_bytes(p, nmaps);
}

sht_status run_ring_synth(Plan &p, const double2 *delta, double *map, double2 *scratch, int nmaps, cudaStream_t s)
{
    StageScope sc(p, 1, s);
    cudaError_t e = sht::launch_ring_synth(p, delta, map, scratch, nmaps, s);
    p.launches[1] += 1;
    if (e != cudaSuccess) return cuda_fail(p, e, "ring_synth");
    sc.done();
    return SHT_OK;
}

sht_status run_ring_anal(Plan &p, const double *map, double2 *delta, double2 *scratch, int nmaps, cudaStream_t s)
{
    StageScope sc(p, 2, s);
    cudaError_t e = sht::launch_ring_anal(p, map, delta, scratch, nmaps, s);
    p.launches[2] += 1;
    if (e != cudaSuccess) return cuda_fail(p, e, "ring_anal");
    sc.done();
    return SHT_OK;
}

sht_status run_legendre_anal(Plan &p, const double2 *delta, double2 *alm, double2 *partial, int nmaps,
                             cudaStream_t s)
{
    if (sht_status g = mlist_guard(p)) return g;
    if (p.mode == SHT_MODE_SPLIT_BF16) {
        // precision form (reduction included): the l-sum contraction on the tensor cores, or
        // double-float products and slot sums on the FP32 pipe
        StageScope sc(p, 3, s);
        int n = 0;
        cudaError_t e = p.tune[SHT_TUNE_PREC_ANAL] ? sht::launch_legendre_anal_tc(p, delta, alm, partial, nmaps, s, &n)
                                                   : sht::launch_legendre_anal_df(p, delta, alm, partial, nmaps, s, &n);
        p.launches[3] += n;
        if (e != cudaSuccess) return cuda_fail(p, e, "legendre_anal");
        sc.done();
        return SHT_OK;
    }
    {
        StageScope sc(p, 3, s);
        int n = 0;
        cudaError_t e = sht::launch_legendre_anal(p, delta, partial, nmaps, s, &n);
        p.launches[3] += n;
        if (e != cudaSuccess) return cuda_fail(p, e, "legendre_anal");
        sc.done();
    }
    StageScope sc(p, 4, s);
    cudaError_t e = sht::launch_block_reduce(p, partial, alm, nmaps, s);
    p.launches[4] += 1;
    if (e != cudaSuccess) return cuda_fail(p, e, "block_reduce");
    sc.done();
    return SHT_OK;
}

}  // namespace

extern "C" {

int64_t sht_nalm(int lmax, int mmax)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax) return -1;
    return (int64_t)(mmax + 1) * (lmax + 1) - (int64_t)mmax * (mmax + 1) / 2;
}

int64_t sht_alm_index(int lmax, int l, int m)
{
    if (lmax < 0 || m < 0 || l < m || l > lmax) return -1;
    return (int64_t)m * (2 * (int64_t)lmax + 3 - m) / 2 + (l - m);
}

const char *sht_status_string(sht_status s)
{
    switch (s) {
    case SHT_OK: return "ok";
    case SHT_EINVAL: return "invalid argument";
    case SHT_ENOMEM: return "out of memory";
    case SHT_ECUDA: return "CUDA error";
    case SHT_EUNSUPPORTED: return "unsupported";
    case SHT_ETIMEOUT: return "device wait timed out";
    }
    return "unknown status";
}

const char *sht_plan_last_error(sht_plan_t plan) { return plan ? plan->p.last_error.c_str() : ""; }

int64_t sht_plan_npix(sht_plan_t plan) { return plan ? plan->p.npix : -1; }
int sht_plan_nrings(sht_plan_t plan) { return plan ? plan->p.nrings : -1; }
int sht_plan_npairs(sht_plan_t plan) { return plan ? plan->p.nslots : -1; }

size_t sht_workspace_bytes(sht_plan_t plan, int nmaps)
{
    if (!plan || nmaps <= 0) return 0;
    const Plan &p = plan->p;
    const size_t d = align256(delta_bytes(p, nmaps));
    const size_t r = align256(sht::ring_scratch_bytes(p));
    const size_t a = align256(anal_partial_bytes(p, nmaps));
    const size_t t = align256(synth_scratch_bytes(p, nmaps));
    return d + std::max(std::max(r, a), t);
}

sht_status sht_plan_set_tuning(sht_plan_t plan, int knob, int value)
{
    if (!plan) return SHT_EINVAL;
    bool ok = false;
    switch (knob) {
    case SHT_TUNE_SYNTH_MAPS: ok = value == 1 || value == 2 || value == 4; break;
    case SHT_TUNE_ANAL_MAPS: ok = value == 1 || value == 2; break;
    case SHT_TUNE_ANAL_SLOTS: ok = value == 1 || value == 4; break;
    case SHT_TUNE_DF_MAPS: ok = value == 4 || value == 8 || value == 16; break;
    case SHT_TUNE_TC_MAPS: ok = value == 8 || value == 16; break;
    case SHT_TUNE_PREC_ANAL: ok = value == 0 || value == 1; break;
    case SHT_TUNE_PREC_RING: ok = value == 0 || value == 1; break;
    case SHT_TUNE_RING_SMEM: ok = value >= 0 && value <= 2; break;
    default: ok = false;
    }
    if (!ok) return SHT_EINVAL;
    plan->p.tune[knob] = value;
    return SHT_OK;
}

int sht_plan_tuning(sht_plan_t plan, int knob)
{
    if (!plan || knob < 0 || knob >= SHT_TUNE_COUNT) return -1;
    return plan->p.tune[knob];
}

sht_status sht_plan_reserve(sht_plan_t plan, int nmaps)
{
    if (!plan || nmaps < 1) return SHT_EINVAL;
    return ensure_workspace(plan->p, sht_workspace_bytes(plan, nmaps));
}

sht_status sht_plan_set_mode(sht_plan_t plan, int mode)
{
    if (!plan || (mode != SHT_MODE_FP64 && mode != SHT_MODE_SPLIT_BF16)) return SHT_EINVAL;
    Plan &p = plan->p;
    if (mode == SHT_MODE_SPLIT_BF16) {
        // the Reinsch-form kernels of the precision form cover the first 256 slots (the analysis: one
        // CTA over slots 0 .. 255 per m; the synthesis: the leading polar 128-slot blocks)
        if (p.nslots > 256 && p.slotTheta[256] > 0.0 && std::sin(p.slotTheta[256]) < 0.03) return SHT_EUNSUPPORTED;
        cudaError_t e = sht::build_tc_scales(p);  // one FP64 pass of the recurrence, synchronous
        if (e == cudaSuccess) e = sht::build_df_ring_tables(p);
        if (e != cudaSuccess) return cuda_fail(p, e, "precision-form tables");
    }
    p.mode = mode;
    return SHT_OK;
}

int sht_plan_mode(sht_plan_t plan) { return plan ? plan->p.mode : -1; }

sht_status sht_plan_device_status(sht_plan_t plan, int *status, int clear)
{
    if (!plan || !status) return SHT_EINVAL;
    Plan &p = plan->p;
    // kernels on non-blocking streams do not order against the legacy stream of cudaMemcpy:
    // wait for the whole device first, so that no kernel can set the bit after the read
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, p.d_status, sizeof(int), cudaMemcpyDeviceToHost);
    // checked build: fold the kernels' bounds-check words into bit 1 (they are process-wide)
    int w = 0;
    if (e == cudaSuccess) e = sht::take_check_word_legendre(&w);
    if (e == cudaSuccess) e = sht::take_check_word_df(&w);
    if (e == cudaSuccess) e = sht::take_check_word_tc(&w);
    if (e == cudaSuccess) e = sht::take_check_word_spin(&w);
    if (e == cudaSuccess) e = sht::take_check_word_ring(&w);
    if (e == cudaSuccess) *status |= w;
    if (e == cudaSuccess && clear) e = cudaMemset(p.d_status, 0, sizeof(int));
    if (e == cudaSuccess && clear) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(p, e, "device status");
    return (*status & 1) ? SHT_ETIMEOUT : SHT_OK;
}

long sht_debug_fail_allocations_after(long n)
{
    return sht::g_alloc_budget.exchange(n < 0 ? -1 : n);
}

sht_status sht_plan_set_mlist(sht_plan_t plan, const int *ms, int n)
{
    if (!plan || n < 0 || (n > 0 && !ms)) return SHT_EINVAL;
    Plan &p = plan->p;
    if (n == 0) {
        if (p.d_mflag) {
            cudaError_t e = cudaFree(p.d_mflag);
            p.d_mflag = nullptr;
            if (e != cudaSuccess) return cuda_fail(p, e, "m list");
        }
        p.n_mlist = 0;
        return SHT_OK;
    }
    std::vector<int> flag((size_t)p.mmax + 1, 0);
    for (int i = 0; i < n; ++i) {
        if (ms[i] < 0 || ms[i] > p.mmax || flag[ms[i]]) return SHT_EINVAL;
        flag[ms[i]] = 1;
    }
    if (!p.d_mflag) {
        cudaError_t e = sht::dev_malloc(&p.d_mflag, sizeof(int) * flag.size());
        if (e != cudaSuccess) {
            p.d_mflag = nullptr;
            return cuda_fail(p, e, "m list");
        }
    }
    cudaError_t e = cudaMemcpy(p.d_mflag, flag.data(), sizeof(int) * flag.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(p, e, "m list");
    p.n_mlist = n;
    return SHT_OK;
}

sht_status sht_plan_live_steps(sht_plan_t plan, int64_t *live, int64_t *total)
{
    if (!plan || !live || !total) return SHT_EINVAL;
    Plan &p = plan->p;
    if (!p.d_tc_Ey) return SHT_EINVAL;  // the tables come with the first switch to the precision form
    const int nblk = (p.nslots + 127) / 128;
    std::vector<int> first((size_t)(p.mmax + 1) * nblk);
    cudaError_t e = cudaMemcpy(first.data(), p.d_tc_Ey + first.size(), sizeof(int) * first.size(),
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "live steps");
    int64_t lv = 0;
    for (int m = 0; m <= p.mmax; ++m)
        for (int b = 0; b < nblk; ++b) {
            const int64_t nl = (int64_t)(p.lmax - m + 1) - 32 * (int64_t)first[(size_t)m * nblk + b];
            const int64_t ns = std::min(128, p.nslots - 128 * b);
            if (nl > 0) lv += nl * ns;
        }
    *live = lv;
    *total = p.nalm * (int64_t)p.nslots;
    return SHT_OK;
}

sht_status sht_plan_create(sht_plan_t *out, sht_grid grid, int nrings, const int64_t *nphi, const double *theta,
                           const double *phi0, const double *w, int lmax, int mmax)
{
    if (!out) return SHT_EINVAL;
    *out = nullptr;
    if (nrings < 1 || !nphi || !theta || !phi0 || !w) return SHT_EINVAL;
    if (lmax < 0 || mmax < 0 || mmax > lmax || lmax > 16383) return SHT_EINVAL;
    if ((int)grid < 0 || (int)grid > 2) return SHT_EINVAL;
    for (int r = 0; r < nrings; ++r) {
        if (nphi[r] < 1 || nphi[r] > (1 << 20)) return SHT_EINVAL;
        if (!is_finite(theta[r]) || theta[r] < 0.0 || theta[r] > PI) return SHT_EINVAL;
        if (!is_finite(phi0[r]) || !is_finite(w[r])) return SHT_EINVAL;
        if (std::fabs(phi0[r]) > 1e3) return SHT_EINVAL;
    }
    sht_plan_s *h = new (std::nothrow) sht_plan_s();
    if (!h) return SHT_ENOMEM;
    Plan &p = h->p;
    p.lmax = lmax;
    p.mmax = mmax;
    p.nrings = nrings;
    p.grid = (int)grid;
    p.nalm = sht_nalm(lmax, mmax);
    p.nphi.assign(nphi, nphi + nrings);
    p.theta.assign(theta, theta + nrings);
    p.phi0.assign(phi0, phi0 + nrings);
    p.w.assign(w, w + nrings);
    p.ofs.resize(nrings + 1);
    p.ofs[0] = 0;
    for (int r = 0; r < nrings; ++r) p.ofs[r + 1] = p.ofs[r] + nphi[r];
    p.npix = p.ofs[nrings];

    pair_rings(p);
    std::vector<double> u(p.nslots), s(p.nslots);
    for (int k = 0; k < p.nslots; ++k) {
        const double th = p.slotTheta[k];
        const double h2 = std::sin(0.5 * th);
        u[k] = 2.0 * h2 * h2;  // 1 - cos(theta), accurate near the pole
        s[k] = std::sin(th);
    }
    std::vector<double> alpha, cfac;
    recurrence_tables(lmax, mmax, alpha, cfac);
    bool any_polar = false;
    for (int k = 0; k < p.nslots; ++k) any_polar |= (s[k] < 0.03);
    p.mR = any_polar ? std::min(mmax, lmax / 10 + 64) : -1;
    std::vector<double3> rein;
    reinsch_tables(lmax, p.mR, rein);
    p.polar_first_slot = p.mR >= 0 && s[0] < 0.03;
    p.polar_syn_blocks = 0;
    if (p.mR >= 0)
        while (p.polar_syn_blocks * 128 < p.nslots && s[p.polar_syn_blocks * 128] < 0.03) ++p.polar_syn_blocks;
    p.tune[SHT_TUNE_ANAL_SLOTS] = sht::legendre_anal_default_slots(p);
    // precision form: 32-l chunks per m
    std::vector<int64_t> chunk_base(mmax + 1);
    int64_t nchunks = 0;
    for (int m = 0; m <= mmax; ++m) {
        chunk_base[m] = nchunks;
        nchunks += (lmax - m + 32) / 32;
    }
    p.tc_total_chunks = nchunks;
    std::vector<int> chunk_m(nchunks);
    for (int m = 0; m <= mmax; ++m)
        for (int64_t c = chunk_base[m]; c < (m < mmax ? chunk_base[m + 1] : nchunks); ++c) chunk_m[c] = m;
    std::vector<int> nphi32(nrings);
    for (int r = 0; r < nrings; ++r) nphi32[r] = (int)nphi[r];

    cudaError_t e = cudaSuccess;
    const char *where = "plan upload";
    if (e == cudaSuccess) e = upload(&p.d_slotN, p.slotN.data(), p.slotN.size());
    if (e == cudaSuccess) e = upload(&p.d_slotS, p.slotS.data(), p.slotS.size());
    if (e == cudaSuccess) e = upload(&p.d_u, u.data(), u.size());
    if (e == cudaSuccess) e = upload(&p.d_s, s.data(), s.size());
    if (e == cudaSuccess) e = upload(&p.d_alpha, alpha.data(), alpha.size());
    if (e == cudaSuccess) e = upload(&p.d_cfac, cfac.data(), cfac.size());
    if (e == cudaSuccess && p.mR >= 0) e = upload(&p.d_rein, rein.data(), rein.size());
    if (e == cudaSuccess) e = upload(&p.d_tc_chunk_base, chunk_base.data(), chunk_base.size());
    if (e == cudaSuccess) e = upload(&p.d_tc_chunk_m, chunk_m.data(), chunk_m.size());
    if (e == cudaSuccess) {
        const int zero = 0;
        e = upload(&p.d_status, &zero, 1);
    }
    if (e == cudaSuccess) e = upload(&p.d_ofs, p.ofs.data(), p.ofs.size());
    if (e == cudaSuccess) e = upload(&p.d_nphi, nphi32.data(), nphi32.size());
    if (e == cudaSuccess) e = upload(&p.d_w, p.w.data(), p.w.size());
    if (e == cudaSuccess) {  // function attributes once, so that calls enqueue stream work only
        where = "kernel attributes";
        e = sht::configure_tc_kernels();
        if (e == cudaSuccess) e = sht::configure_df_kernels();
    }
    if (e == cudaSuccess) {
        where = "phase table";
        e = sht::build_phase_table(p);
    }
    if (e == cudaSuccess) {
        where = "ring tables";
        e = sht::build_fft_tables(p);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        sht_status st = (e == cudaErrorMemoryAllocation) ? SHT_ENOMEM : SHT_ECUDA;
        if (e == cudaErrorInvalidValue && std::string(where) == "ring tables") st = SHT_EUNSUPPORTED;
        free_plan_device(p);
        delete h;
        (void)where;
        return st;
    }
    *out = h;
    return SHT_OK;
}

void sht_plan_destroy(sht_plan_t plan)
{
    if (!plan) return;
    cudaDeviceSynchronize();
    for (auto &pe : plan->p.pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    for (cudaEvent_t e : plan->p.event_pool) cudaEventDestroy(e);
    free_plan_device(plan->p);
    delete plan;
}

sht_status sht_legendre_synth(sht_plan_t plan, const void *alm, void *delta, int nmaps, void *stream)
{
    sht_status st = check_call(plan, alm, delta, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    st = ensure_workspace(p, align256(synth_scratch_bytes(p, nmaps)));
    if (st != SHT_OK) return st;
    return run_legendre_synth(p, (const double2 *)alm, (double2 *)delta, p.d_ws, nmaps, (cudaStream_t)stream);
}

sht_status sht_ring_synth(sht_plan_t plan, const void *delta, double *map, int nmaps, void *stream)
{
    sht_status st = check_call(plan, delta, map, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    st = ensure_workspace(p, align256(sht::ring_scratch_bytes(p)));
    if (st != SHT_OK) return st;
    return run_ring_synth(p, (const double2 *)delta, map, (double2 *)p.d_ws, nmaps, (cudaStream_t)stream);
}

sht_status sht_ring_anal(sht_plan_t plan, const double *map, void *delta, int nmaps, void *stream)
{
    sht_status st = check_call(plan, map, delta, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    st = ensure_workspace(p, align256(sht::ring_scratch_bytes(p)));
    if (st != SHT_OK) return st;
    return run_ring_anal(p, map, (double2 *)delta, (double2 *)p.d_ws, nmaps, (cudaStream_t)stream);
}

sht_status sht_legendre_anal(sht_plan_t plan, const void *delta, void *alm, int nmaps, void *stream)
{
    sht_status st = check_call(plan, delta, alm, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    st = ensure_workspace(p, align256(anal_partial_bytes(p, nmaps)));
    if (st != SHT_OK) return st;
    return run_legendre_anal(p, (const double2 *)delta, (double2 *)alm, (double2 *)p.d_ws, nmaps,
                             (cudaStream_t)stream);
}

sht_status sht_alm2map(sht_plan_t plan, const void *alm, double *map, int nmaps, void *stream)
{
    sht_status st = check_call(plan, alm, map, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    const size_t d = align256(delta_bytes(p, nmaps));
    st = ensure_workspace(p, d + std::max(align256(sht::ring_scratch_bytes(p)), align256(synth_scratch_bytes(p, nmaps))));
    if (st != SHT_OK) return st;
    double2 *delta = (double2 *)p.d_ws;
    double2 *scratch = (double2 *)((char *)p.d_ws + d);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_legendre_synth(p, (const double2 *)alm, delta, scratch, nmaps, s);
    if (st != SHT_OK) return st;
    return run_ring_synth(p, delta, map, scratch, nmaps, s);
}

sht_status sht_map2alm(sht_plan_t plan, const double *map, void *alm, int nmaps, void *stream)
{
    sht_status st = check_call(plan, map, alm, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    const size_t d = align256(delta_bytes(p, nmaps));
    const size_t r = align256(sht::ring_scratch_bytes(p));
    const size_t a = align256(anal_partial_bytes(p, nmaps));
    st = ensure_workspace(p, d + std::max(r, a));
    if (st != SHT_OK) return st;
    double2 *delta = (double2 *)p.d_ws;
    double2 *scratch = (double2 *)((char *)p.d_ws + d);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_ring_anal(p, map, delta, scratch, nmaps, s);
    if (st != SHT_OK) return st;
    return run_legendre_anal(p, delta, (double2 *)alm, scratch, nmaps, s);
}

// Spin-2 transforms (see the header and spin.cu).
static sht_status spin_prepare(Plan &p, int spin)
{
    if (p.n_mlist > 0) {
        p.last_error = "an m list is set: the spin transforms compute every m";
        return SHT_EUNSUPPORTED;
    }
    if (spin != 2) {
        p.last_error = "spin-weighted transforms: only spin 2 is implemented";
        return SHT_EUNSUPPORTED;
    }
    cudaError_t e = sht::build_spin_tables(p);
    if (e != cudaSuccess) return cuda_fail(p, e, "spin tables");
    return SHT_OK;
}

size_t sht_spin_workspace_bytes(sht_plan_t plan, int nmaps)
{
    if (!plan || nmaps <= 0) return 0;
    const Plan &p = plan->p;
    return align256(delta_bytes(p, 2 * nmaps)) +
           std::max(align256(sht::ring_scratch_bytes(p)), align256(sht::spin_partial_bytes(p, std::min(nmaps, 2))));
}

sht_status sht_alm2map_spin(sht_plan_t plan, int spin, const void *alm, double *map, int nmaps, void *stream)
{
    sht_status st = check_call(plan, alm, map, nmaps);
    if (st != SHT_OK) return st;
    Plan &p = plan->p;
    if ((st = spin_prepare(p, spin)) != SHT_OK || nmaps == 0) return st;
    st = ensure_workspace(p, sht_spin_workspace_bytes(plan, nmaps));
    if (st != SHT_OK) return st;
    const size_t d = align256(delta_bytes(p, 2 * nmaps));
    double2 *delta = (double2 *)p.d_ws;
    double2 *scratch = (double2 *)((char *)p.d_ws + d);
    cudaStream_t s = (cudaStream_t)stream;
    {
        StageScope sc(p, SHT_STAGE_LEGENDRE_SYNTH, s);
        int n = 0;
        cudaError_t e = sht::launch_spin_synth(p, (const double2 *)alm, delta, nmaps, s, &n);
        p.launches[SHT_STAGE_LEGENDRE_SYNTH] += n;
        if (e != cudaSuccess) return cuda_fail(p, e, "spin legendre_synth");
        sc.done();
    }
    return run_ring_synth(p, delta, map, scratch, 2 * nmaps, s);
}

sht_status sht_map2alm_spin(sht_plan_t plan, int spin, const double *map, void *alm, int nmaps, void *stream)
{
    sht_status st = check_call(plan, map, alm, nmaps);
    if (st != SHT_OK) return st;
    Plan &p = plan->p;
    if ((st = spin_prepare(p, spin)) != SHT_OK || nmaps == 0) return st;
    st = ensure_workspace(p, sht_spin_workspace_bytes(plan, nmaps));
    if (st != SHT_OK) return st;
    const size_t d = align256(delta_bytes(p, 2 * nmaps));
    double2 *delta = (double2 *)p.d_ws;
    double2 *scratch = (double2 *)((char *)p.d_ws + d);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_ring_anal(p, map, delta, scratch, 2 * nmaps, s);
    if (st != SHT_OK) return st;
    StageScope sc(p, SHT_STAGE_LEGENDRE_ANAL, s);
    int n = 0;
    cudaError_t e = sht::launch_spin_anal(p, delta, (double2 *)alm, scratch, nmaps, s, &n);
    p.launches[SHT_STAGE_LEGENDRE_ANAL] += n;
    if (e != cudaSuccess) return cuda_fail(p, e, "spin legendre_anal");
    sc.done();
    return SHT_OK;
}

// The same transforms on caller-owned scratch (see the header).
static sht_status check_ws(sht_plan_t plan, int nmaps, void *scratch, size_t scratch_bytes)
{
    if (!scratch || ((uintptr_t)scratch & 255u)) return SHT_EINVAL;
    if (scratch_bytes < sht_workspace_bytes(plan, nmaps)) return SHT_EINVAL;
    return SHT_OK;
}

sht_status sht_alm2map_ws(sht_plan_t plan, const void *alm, double *map, int nmaps, void *stream, void *scratch,
                          size_t scratch_bytes)
{
    sht_status st = check_call(plan, alm, map, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    if ((st = check_ws(plan, nmaps, scratch, scratch_bytes)) != SHT_OK) return st;
    const size_t d = align256(delta_bytes(p, nmaps));
    double2 *delta = (double2 *)scratch;
    double2 *sc = (double2 *)((char *)scratch + d);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_legendre_synth(p, (const double2 *)alm, delta, sc, nmaps, s);
    if (st != SHT_OK) return st;
    return run_ring_synth(p, delta, map, sc, nmaps, s);
}

sht_status sht_map2alm_ws(sht_plan_t plan, const double *map, void *alm, int nmaps, void *stream, void *scratch,
                          size_t scratch_bytes)
{
    sht_status st = check_call(plan, map, alm, nmaps);
    if (st != SHT_OK || nmaps == 0) return st;
    Plan &p = plan->p;
    if ((st = check_ws(plan, nmaps, scratch, scratch_bytes)) != SHT_OK) return st;
    const size_t d = align256(delta_bytes(p, nmaps));
    double2 *delta = (double2 *)scratch;
    double2 *sc = (double2 *)((char *)scratch + d);
    cudaStream_t s = (cudaStream_t)stream;
    st = run_ring_anal(p, map, delta, sc, nmaps, s);
    if (st != SHT_OK) return st;
    return run_legendre_anal(p, delta, (double2 *)alm, sc, nmaps, s);
}

sht_status sht_plan_set_stage_timing(sht_plan_t plan, int enable)
{
    if (!plan) return SHT_EINVAL;
    plan->p.timing = enable != 0;
    return SHT_OK;
}

sht_status sht_plan_stage_times(sht_plan_t plan, double *ms, int64_t *launches, int reset)
{
    if (!plan) return SHT_EINVAL;
    Plan &p = plan->p;
    sht_status st = SHT_OK;
    for (auto &pe : p.pending) {
        cudaError_t e = cudaEventSynchronize(pe.b);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pe.a, pe.b);
        if (e != cudaSuccess) {
            st = cuda_fail(p, e, "stage timing");
        } else {
            p.stage_ms[pe.stage] += t;
        }
        p.event_pool.push_back(pe.a);
        p.event_pool.push_back(pe.b);
    }
    p.pending.clear();
    for (int i = 0; i < Plan::NSTAGE; ++i) {
        if (ms) ms[i] = p.stage_ms[i];
        if (launches) launches[i] = p.launches[i];
        if (reset) {
            p.stage_ms[i] = 0.0;
            p.launches[i] = 0;
        }
    }
    return st;
}

// ------------------------------------------------------------------ grids

sht_status sht_geom_healpix(int nside, int64_t *nphi, double *theta, double *phi0, double *w)
{
    if (nside < 1 || nside > (1 << 13) || !nphi || !theta || !phi0 || !w) return SHT_EINVAL;
    const int nr = 4 * nside - 1;
    const double npix = 12.0 * nside * (double)nside;
    for (int k = 0; k < nr; ++k) {
        const int i = k + 1;
        const int north = (i <= 2 * nside) ? i : 4 * nside - i;
        double th, p0;
        int64_t n;
        if (north < nside) {
            n = 4 * north;
            th = 2.0 * std::asin(north / (std::sqrt(6.0) * nside));
            p0 = PI / (4.0 * north);
        } else {
            n = 4 * (int64_t)nside;
            const double z = 4.0 / 3.0 - 2.0 * north / (3.0 * nside);
            th = std::acos(z);
            p0 = ((i - nside) % 2 == 0) ? PI / (4.0 * nside) : 0.0;
        }
        if (i > 2 * nside) th = PI - th;
        nphi[k] = n;
        theta[k] = th;
        phi0[k] = p0;
        w[k] = 4.0 * PI / npix;
    }
    return SHT_OK;
}

// Gauss-Legendre nodes by Newton's method on P_N(cos theta) in the colatitude itself, from the
// asymptotic guess theta = pi (j + 3/4) / (N + 1/2); weights 2 sin^2(theta) / (N P_{N-1}(x))^2
// (at a root, (1 - x^2) P_N'(x) = N P_{N-1}(x)), with no 1 - x^2 cancellation near the poles.
// The southern half mirrors the northern one.
static void legendre_pair(int N, double th, double &pn, double &pn1)
{
    if (N == 0) {
        pn = 1.0;
        pn1 = 0.0;
        return;
    }
    const double x = std::cos(th);
    double p0 = 1.0, p1 = x;  // P_{l-1}, P_l
    if (x > 0.5) {
        // near the pole: Reinsch's difference form with u = 1 - x = 2 sin^2(theta/2) exact, so that
        // rounding acts on D_l = P_l - P_{l-1}:  D_{l+1} = (l D_l - (2l+1) u P_l) / (l+1)
        const double h = std::sin(0.5 * th);
        const double u = 2.0 * h * h;
        p1 = 1.0 - u;
        double d = -u;
        for (int l = 1; l < N; ++l) {
            d = (l * d - (2.0 * l + 1.0) * u * p1) / (l + 1.0);
            p0 = p1;
            p1 += d;
        }
    } else {
        for (int l = 1; l < N; ++l) {
            const double p2 = ((2.0 * l + 1.0) * x * p1 - l * p0) / (l + 1.0);
            p0 = p1;
            p1 = p2;
        }
    }
    pn = p1;
    pn1 = p0;
}

sht_status sht_geom_gauss_legendre(int nrings, int64_t nphi, int64_t *nphi_out, double *theta, double *phi0, double *w)
{
    if (nrings < 1 || nrings > (1 << 16) || nphi < 1 || nphi > (1 << 20) || !nphi_out || !theta || !phi0 || !w)
        return SHT_EINVAL;
    const int N = nrings;
    for (int j = 0; j < (N + 1) / 2; ++j) {
        const int js = N - 1 - j;
        double th = PI * (j + 0.75) / (N + 0.5);
        if (js == j) {
            th = 0.5 * PI;  // odd N: the equator is a node
        } else {
            int converged = 0;
            for (int it = 0; it < 100; ++it) {
                const double x = std::cos(th), sn = std::sin(th);
                double pn, pn1;
                legendre_pair(N, th, pn, pn1);
                // d P_N(cos theta) / d theta = -N (P_{N-1} - x P_N) / sin(theta)
                const double dth = pn * sn / (N * (pn1 - x * pn));
                th += dth;
                if (std::fabs(dth) <= 1e-16 * th) {
                    if (++converged >= 2) break;
                }
            }
        }
        const double sn = std::sin(th);
        double pn, pn1;
        legendre_pair(N, th, pn, pn1);
        const double wg = 2.0 * sn * sn / ((N * pn1) * (N * pn1));
        theta[j] = th;
        w[j] = 2.0 * PI * wg / (double)nphi;
        if (js != j) {
            theta[js] = PI - th;
            w[js] = w[j];
        }
    }
    for (int r = 0; r < N; ++r) {
        nphi_out[r] = nphi;
        phi0[r] = 0.0;
    }
    return SHT_OK;
}

}  // extern "C"
