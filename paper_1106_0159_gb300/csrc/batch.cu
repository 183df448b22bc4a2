// Batched form: many transforms of one direction, over plans of uneven lmax, each stage one
// persistent launch whose CTAs take tiles from a device queue, longest first.  The paper runs one
// transform at a time; this is the batching of its per-m work units across transforms.
//
// alm2map:  Legendre synthesis tiles of every job -> ring synthesis units of every job;
// map2alm:  ring analysis units -> Legendre analysis tiles -> block reduction of every job.
// The batch owns its Delta slabs, partial sums, scratch and queue counters; sht_batch_run only
// enqueues stream work (three memsets and the launches), so it can be captured in a CUDA graph and
// replayed with new inputs written in place.
#include "sht_internal.h"

#include <algorithm>
#include <string>
#include <vector>

struct sht_batch_s {
    int direction = 0;                       // 0 alm2map, 1 map2alm
    std::vector<const sht::Plan *> plans;
    std::vector<int> nmaps;
    std::vector<const void *> in;
    std::vector<void *> out;
    int tune[SHT_BATCH_TUNE_COUNT] = {4, 8, 4, 2, 4};
    // device state, rebuilt when a knob changes
    void *d_ws = nullptr;                    // Delta slabs, then partial sums / ring scratch
    size_t ws_bytes = 0;
    int *d_counters = nullptr;               // one queue counter per launch
    sht::BatchLaunch leg, red, ring;
    int maxlen = 1;
    double2 *ring_scratch = nullptr;
    bool ready = false;
    std::string last_error;
};

namespace {

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

void free_launch(sht::BatchLaunch &L)
{
    cudaFree(L.jobs);
    cudaFree(L.tiles);
    L = sht::BatchLaunch{};
}

void release(sht_batch_s &b)
{
    cudaFree(b.d_ws);
    cudaFree(b.d_counters);
    b.d_ws = nullptr;
    b.d_counters = nullptr;
    b.ws_bytes = 0;
    free_launch(b.leg);
    free_launch(b.red);
    free_launch(b.ring);
    b.ring_scratch = nullptr;
    b.ready = false;
}

int ring_ctas(const sht_batch_s &b) { return 152 * std::max(1, b.tune[SHT_BATCH_RING_CTAS]); }

sht_status prepare(sht_batch_s &b)
{
    if (b.ready) return SHT_OK;
    release(b);
    const size_t nj = b.plans.size();
    std::vector<size_t> doff(nj);
    size_t off = 0;
    for (size_t j = 0; j < nj; ++j) {
        doff[j] = off;
        off += al256((size_t)b.nmaps[j] * b.plans[j]->nrings * (b.plans[j]->mmax + 1) * sizeof(double2));
    }
    const int k = b.tune[SHT_BATCH_ANAL_SLOTS];
    std::vector<size_t> poff(nj);
    size_t pend = off;
    if (b.direction == 1)
        for (size_t j = 0; j < nj; ++j) {
            poff[j] = pend;
            pend += al256(sht::batch_anal_partial_bytes(*b.plans[j], b.nmaps[j], k));
        }
    int maxlen = 1;
    for (auto *p : b.plans) maxlen = std::max(maxlen, p->fft_maxlen);
    // ring scratch after the Delta slabs; the analysis partials do not overlap it (the ring stage of
    // map2alm runs before the Legendre stage, but keeping both lets a graph replay them back to back)
    const size_t scratch_off = al256(pend);
    const size_t need = scratch_off + (size_t)ring_ctas(b) * 3 * maxlen * sizeof(double2);
    cudaError_t e = sht::dev_malloc(&b.d_ws, need);
    if (e == cudaSuccess) e = sht::dev_malloc(&b.d_counters, 4 * sizeof(int));
    if (e != cudaSuccess) {
        b.last_error = std::string("batch workspace: ") + cudaGetErrorString(e);
        release(b);
        return e == cudaErrorMemoryAllocation ? SHT_ENOMEM : SHT_ECUDA;
    }
    b.ws_bytes = need;
    b.maxlen = maxlen;
    b.ring_scratch = (double2 *)((char *)b.d_ws + scratch_off);
    std::vector<double2 *> delta(nj), partial(nj);
    std::vector<const double2 *> cdelta(nj);
    for (size_t j = 0; j < nj; ++j) {
        delta[j] = (double2 *)((char *)b.d_ws + doff[j]);
        cdelta[j] = delta[j];
        partial[j] = (double2 *)((char *)b.d_ws + poff[j]);
    }
    int ml = 0;
    if (b.direction == 0) {
        std::vector<const double2 *> alm(nj);
        std::vector<const void *> rin(nj);
        std::vector<void *> rout(nj);
        for (size_t j = 0; j < nj; ++j) {
            alm[j] = (const double2 *)b.in[j];
            rin[j] = delta[j];
            rout[j] = b.out[j];
        }
        e = sht::batch_legendre_synth_setup(b.plans, alm, delta, b.nmaps, b.tune[SHT_BATCH_SYNTH_MAPS], b.leg);
        if (e == cudaSuccess) e = sht::batch_ring_setup(b.plans, rin, rout, b.nmaps, true, b.ring, ml);
    } else {
        std::vector<double2 *> alm(nj);
        std::vector<void *> rout(nj);
        for (size_t j = 0; j < nj; ++j) {
            alm[j] = (double2 *)b.out[j];
            rout[j] = delta[j];
        }
        e = sht::batch_ring_setup(b.plans, b.in, rout, b.nmaps, false, b.ring, ml);
        if (e == cudaSuccess)
            e = sht::batch_legendre_anal_setup(b.plans, cdelta, partial, alm, b.nmaps, b.tune[SHT_BATCH_ANAL_MAPS], k,
                                               b.leg, b.red);
    }
    if (e != cudaSuccess) {
        b.last_error = std::string("batch set-up: ") + cudaGetErrorString(e);
        release(b);
        return e == cudaErrorMemoryAllocation ? SHT_ENOMEM : SHT_ECUDA;
    }
    b.ready = true;
    return SHT_OK;
}

}  // namespace

extern "C" {

sht_status sht_batch_create(sht_batch_t *out, int direction, int njobs, const sht_plan_t *plans, const void *const *in,
                            void *const *outs, const int *nmaps)
{
    if (!out) return SHT_EINVAL;
    *out = nullptr;
    if ((direction != 0 && direction != 1) || njobs < 1 || !plans || !in || !outs || !nmaps) return SHT_EINVAL;
    for (int j = 0; j < njobs; ++j) {
        if (!plans[j] || !in[j] || !outs[j] || nmaps[j] < 1 || nmaps[j] > 0xffff || in[j] == outs[j])
            return SHT_EINVAL;
        if (plans[j]->p.mode != SHT_MODE_FP64 || plans[j]->p.n_mlist > 0) return SHT_EUNSUPPORTED;
    }
    sht_batch_s *b = new (std::nothrow) sht_batch_s();
    if (!b) return SHT_ENOMEM;
    b->direction = direction;
    for (int j = 0; j < njobs; ++j) {
        b->plans.push_back(&plans[j]->p);
        b->nmaps.push_back(nmaps[j]);
        b->in.push_back(in[j]);
        b->out.push_back(outs[j]);
    }
    sht_status st = prepare(*b);
    if (st != SHT_OK) {
        delete b;
        return st;
    }
    *out = b;
    return SHT_OK;
}

sht_status sht_batch_set_tuning(sht_batch_t b, int knob, int value)
{
    if (!b) return SHT_EINVAL;
    bool ok = false;
    switch (knob) {
    case SHT_BATCH_SYNTH_MAPS: ok = value == 1 || value == 2 || value == 4; break;
    case SHT_BATCH_LEG_CTAS: ok = value == 2 || value == 4 || value == 8 || value == 16; break;
    case SHT_BATCH_RING_CTAS: ok = value >= 1 && value <= 4; break;
    case SHT_BATCH_ANAL_MAPS: ok = value == 1 || value == 2; break;
    case SHT_BATCH_ANAL_SLOTS: ok = value == 1 || value == 4; break;
    default: ok = false;
    }
    if (!ok) return SHT_EINVAL;
    if (b->tune[knob] != value) {
        b->tune[knob] = value;
        b->ready = false;
        // rebuild now (synchronous), so that sht_batch_run only enqueues stream work
        sht_status st = prepare(*b);
        if (st != SHT_OK) return st;
    }
    return SHT_OK;
}

int sht_batch_tuning(sht_batch_t b, int knob)
{
    if (!b || knob < 0 || knob >= SHT_BATCH_TUNE_COUNT) return -1;
    return b->tune[knob];
}

sht_status sht_batch_run(sht_batch_t b, void *stream)
{
    if (!b) return SHT_EINVAL;
    if (!b->ready) return SHT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, 4 * sizeof(int), s);
    const int lgrid = 152 * b->tune[SHT_BATCH_LEG_CTAS];
    if (b->direction == 0) {
        if (e == cudaSuccess) e = sht::batch_legendre_synth_launch(b->leg, b->d_counters, lgrid, s);
        if (e == cudaSuccess)
            e = sht::batch_ring_launch(b->ring, true, b->ring_scratch, b->maxlen, b->d_counters + 1, ring_ctas(*b), s);
    } else {
        if (e == cudaSuccess)
            e = sht::batch_ring_launch(b->ring, false, b->ring_scratch, b->maxlen, b->d_counters + 1, ring_ctas(*b),
                                       s);
        if (e == cudaSuccess) e = sht::batch_legendre_anal_launch(b->leg, b->red, b->d_counters, lgrid, s);
    }
    if (e != cudaSuccess) {
        b->last_error = std::string("batch run: ") + cudaGetErrorString(e);
        return SHT_ECUDA;
    }
    return SHT_OK;
}

int64_t sht_batch_tiles(sht_batch_t b, int stage)
{
    if (!b) return -1;
    if (stage == 0) return b->leg.ntiles;
    if (stage == 1) return b->ring.ntiles;
    return -1;
}

const char *sht_batch_last_error(sht_batch_t b) { return b ? b->last_error.c_str() : ""; }

void sht_batch_destroy(sht_batch_t b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    release(*b);
    delete b;
}

}  // extern "C"
