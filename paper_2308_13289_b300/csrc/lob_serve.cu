// lob_serve.cu -- the serving tick executor: continuous batching of
// simulation episodes over the books of one engine context.  Host code only:
// a tick issues the caller's device generator, the engine's processing and
// the levels of the advanced books on two streams, through a ring of pinned
// upload buffers, so the host can run several ticks ahead of the GPU.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>
#include <utility>
#include <vector>

#include "../../include/lob.h"
#include "lob_engine.h"

struct lob_serve {
    lob_serve_desc d{};
    int S = 0;
    // slot state: the running episode's progress (steps done, steps, messages a step)
    std::vector<uint8_t> active;
    std::vector<int64_t> step, n_steps;
    std::vector<int32_t> mps;
    std::vector<int32_t> free_slots;                       // popped from the back
    std::vector<std::pair<int32_t, uint64_t>> restart;     // (slot, stream id) admitted since the last tick
    // one tick's upload, int64 words, packed to the tick's own sizes (n active, r restarts):
    // offsets [n+1] | counts [n] | active slots (int32) [n] | stream ids [r] | restart slots (int32) [r]
    int64_t max_words = 0;
    int64_t* d_pack[2] = {nullptr, nullptr};
    struct Entry {
        int64_t* h = nullptr;
        cudaEvent_t copied = nullptr, g0 = nullptr, g1 = nullptr, t0 = nullptr, t1 = nullptr;
        bool busy = false, timed = false;
        int32_t n = 0;
    };
    std::vector<Entry> ring;
    int64_t* h_ring = nullptr;
    int pos = 0;
    cudaEvent_t ev_gen[2] = {nullptr, nullptr};   // windows of buffer k written
    cudaEvent_t ev_used[2] = {nullptr, nullptr};  // windows of buffer k consumed
    int64_t tick = 0;
    std::vector<float> proc_ms, gen_ms;
    std::vector<int32_t> n_in_tick;
};

namespace {

int64_t words_of(int64_t n, int64_t r) { return (n + 1) + n + (n + 1) / 2 + r + (r + 1) / 2; }

// Wait until a ring entry's upload has been read and, for a timed tick, its
// processing has finished; record the tick's times.
int retire(lob_serve* s, lob_serve::Entry& e)
{
    cudaError_t err = cudaEventSynchronize(e.copied);
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_serve: upload");
    if (e.timed) {
        err = cudaEventSynchronize(e.t1);
        if (err != cudaSuccess) return lob_cuda_fail(err, "lob_serve: tick");
        float p = 0.f, g = 0.f;
        err = cudaEventElapsedTime(&p, e.t0, e.t1);
        if (err == cudaSuccess) err = cudaEventElapsedTime(&g, e.g0, e.g1);
        if (err != cudaSuccess) return lob_cuda_fail(err, "lob_serve: elapsed time");
        s->proc_ms.push_back(p);
        s->gen_ms.push_back(g);
        s->n_in_tick.push_back(e.n);
    }
    e.busy = e.timed = false;
    return LOB_OK;
}

int retire_all(lob_serve* s)
{
    // oldest first, so the recorded ticks stay in order
    const int R = (int)s->ring.size();
    for (int i = 0; i < R; ++i) {
        lob_serve::Entry& e = s->ring[(s->pos + i) % R];
        if (e.busy) {
            const int rc = retire(s, e);
            if (rc != LOB_OK) return rc;
        }
    }
    return LOB_OK;
}

void release(lob_serve* s)
{
    for (auto& e : s->ring) {
        for (cudaEvent_t ev : {e.copied, e.g0, e.g1, e.t0, e.t1})
            if (ev) cudaEventDestroy(ev);
    }
    for (int k = 0; k < 2; ++k) {
        if (s->ev_gen[k]) cudaEventDestroy(s->ev_gen[k]);
        if (s->ev_used[k]) cudaEventDestroy(s->ev_used[k]);
        if (s->d_pack[k]) cudaFree(s->d_pack[k]);
    }
    if (s->h_ring) cudaFreeHost(s->h_ring);
    delete s;
}

}  // namespace

extern "C" {

int lob_serve_create(lob_serve** out, const lob_serve_desc* d)
{
    if (!out || !d) {
        lob_set_error("lob_serve_create: null argument");
        return LOB_E_INVAL;
    }
    *out = nullptr;
    if (!d->engine || !d->gen_params || !d->gen_init || !d->gen_advance || !d->d_geo_px ||
        !d->d_geo_q || !d->d_gen_states || !d->d_gen_pools || !d->d_win0 || !d->d_win1 ||
        !d->d_bid_px || !d->d_bid_qty || !d->d_ask_px || !d->d_ask_qty || !d->d_trade_counts ||
        d->slots < 1 || d->slots != d->engine->cfg.n_books || d->max_msgs < 0 || d->depth < 1 ||
        d->depth > 64 || d->ring < 1 || d->ring > 64) {
        lob_set_error("lob_serve_create: invalid descriptor (slots=%d, max_msgs=%d, depth=%d, "
                      "ring=%d)", d->slots, d->max_msgs, d->depth, d->ring);
        return LOB_E_INVAL;
    }
    lob_serve* s = new (std::nothrow) lob_serve;
    if (!s) {
        lob_set_error("lob_serve_create: out of host memory");
        return LOB_E_NOMEM;
    }
    s->d = *d;
    const int S = s->S = d->slots;
    s->active.assign(S, 0);
    s->step.assign(S, 0);
    s->n_steps.assign(S, 0);
    s->mps.assign(S, 0);
    s->free_slots.reserve(S);
    for (int i = S - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->restart.reserve(S);
    s->max_words = words_of(S, S);
    cudaError_t err = cudaSuccess;
    for (int k = 0; k < 2 && err == cudaSuccess; ++k) {
        err = cudaMalloc(&s->d_pack[k], (size_t)s->max_words * 8);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->ev_gen[k], cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&s->ev_used[k], cudaEventDisableTiming);
    }
    if (err == cudaSuccess)
        err = cudaHostAlloc(&s->h_ring, (size_t)d->ring * s->max_words * 8, cudaHostAllocDefault);
    s->ring.resize(d->ring);
    for (int i = 0; i < d->ring && err == cudaSuccess; ++i) {
        lob_serve::Entry& e = s->ring[i];
        e.h = s->h_ring + (int64_t)i * s->max_words;
        err = cudaEventCreateWithFlags(&e.copied, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventCreate(&e.g0);
        if (err == cudaSuccess) err = cudaEventCreate(&e.g1);
        if (err == cudaSuccess) err = cudaEventCreate(&e.t0);
        if (err == cudaSuccess) err = cudaEventCreate(&e.t1);
    }
    if (err != cudaSuccess) {
        release(s);
        return lob_cuda_fail(err, "lob_serve_create");
    }
    *out = s;
    return LOB_OK;
}

int lob_serve_admit(lob_serve* s, uint64_t stream_id, int64_t n_steps, int32_t msgs_per_step,
                    int32_t* slot_out)
{
    if (!s || !slot_out || n_steps < 0 || msgs_per_step < 0 || msgs_per_step > s->d.max_msgs) {
        lob_set_error("lob_serve_admit: invalid argument (n_steps=%lld, msgs_per_step=%d)",
                      (long long)n_steps, msgs_per_step);
        return LOB_E_INVAL;
    }
    if (s->free_slots.empty()) {
        *slot_out = -1;
        lob_set_error("lob_serve_admit: no free slot");
        return LOB_E_STATE;
    }
    const int32_t slot = s->free_slots.back();
    s->free_slots.pop_back();
    s->active[slot] = 1;
    s->step[slot] = 0;
    s->n_steps[slot] = n_steps;
    s->mps[slot] = msgs_per_step;
    s->restart.emplace_back(slot, stream_id);
    *slot_out = slot;
    return LOB_OK;
}

int lob_serve_tick(lob_serve* s, int32_t timing, int32_t collect, int32_t* h_active,
                   int32_t* n_active, int32_t* h_finished, int32_t* n_finished,
                   int64_t* n_msgs)
{
    if (!s || !n_active || !h_finished || !n_finished || !n_msgs) {
        lob_set_error("lob_serve_tick: null argument");
        return LOB_E_INVAL;
    }
    *n_active = *n_finished = 0;
    *n_msgs = 0;
    lob_serve::Entry& e = s->ring[s->pos];
    if (e.busy) {
        const int rc = retire(s, e);
        if (rc != LOB_OK) return rc;
    }
    // the tick's upload, packed to its own sizes
    int64_t* buf = e.h;
    int32_t n = 0;
    for (int slot = 0; slot < s->S; ++slot) n += s->active[slot];
    if (n == 0) return LOB_OK;
    const int32_t r = (int32_t)s->restart.size();
    const int64_t o_cnt = n + 1, o_ids = o_cnt + n, o_sid = o_ids + (n + 1) / 2,
                  o_rid = o_sid + r, words = words_of(n, r);
    int32_t* ids = reinterpret_cast<int32_t*>(buf + o_ids);
    int64_t acc = 0;
    buf[0] = 0;
    for (int slot = 0, i = 0; slot < s->S; ++slot) {
        if (!s->active[slot]) continue;
        ids[i] = slot;
        buf[o_cnt + i] = s->mps[slot];
        acc += s->mps[slot];
        buf[1 + i] = acc;
        ++i;
    }
    int32_t* rid = reinterpret_cast<int32_t*>(buf + o_rid);
    for (int32_t i = 0; i < r; ++i) {
        rid[i] = s->restart[i].first;
        buf[o_sid + i] = (int64_t)s->restart[i].second;
    }
    s->restart.clear();
    s->pos = (s->pos + 1) % (int)s->ring.size();

    const int k = (int)(s->tick & 1);
    int64_t* dp = s->d_pack[k];
    const int64_t* d_off = dp;
    const int64_t* d_cnt = dp + o_cnt;
    const int32_t* d_ids = reinterpret_cast<const int32_t*>(dp + o_ids);
    const uint64_t* d_sid = reinterpret_cast<const uint64_t*>(dp + o_sid);
    const int32_t* d_rid = reinterpret_cast<const int32_t*>(dp + o_rid);
    void* win = k == 0 ? s->d.d_win0 : s->d.d_win1;
    cudaStream_t gs = (cudaStream_t)s->d.gen_stream, ps = (cudaStream_t)s->d.proc_stream;
    const lob_serve_desc& d = s->d;

    // generator stream: this tick's windows (buffer k is free once the
    // processing two ticks back has consumed it)
    cudaError_t err = cudaStreamWaitEvent(gs, s->ev_used[k], 0);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(dp, buf, (size_t)words * 8, cudaMemcpyHostToDevice, gs);
    if (err == cudaSuccess) err = cudaEventRecord(e.copied, gs);
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_serve_tick: upload");
    e.busy = true;
    e.timed = timing != 0;
    e.n = n;
    if (timing && (err = cudaEventRecord(e.g0, gs)) != cudaSuccess)
        return lob_cuda_fail(err, "lob_serve_tick: event");
    if (r && d.gen_init(d.gen_params, r, d_rid, d_sid, d.d_gen_states, gs) != 0) {
        lob_set_error("lob_serve_tick: generator initialisation failed");
        return LOB_E_CUDA;
    }
    if (d.gen_advance(d.gen_params, d.d_geo_px, d.d_geo_q, n, d_ids, d.d_gen_states,
                      d.d_gen_pools, d_cnt, d_off, win, gs) != 0) {
        lob_set_error("lob_serve_tick: generator failed");
        return LOB_E_CUDA;
    }
    if (timing) err = cudaEventRecord(e.g1, gs);
    if (err == cudaSuccess) err = cudaEventRecord(s->ev_gen[k], gs);
    // processing stream: reset the admitted books, apply the windows, write
    // the levels of the books just advanced
    if (err == cudaSuccess) err = cudaStreamWaitEvent(ps, s->ev_gen[k], 0);
    if (err == cudaSuccess && timing) err = cudaEventRecord(e.t0, ps);
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_serve_tick: stream order");
    int rc = LOB_OK;
    if (r) rc = lob_reset_books(d.engine, d_rid, r, ps);
    if (rc == LOB_OK)
        rc = lob_process_batch(d.engine, reinterpret_cast<const lob_msg_t*>(win), d_off, d_ids, n,
                               ps);
    if (rc == LOB_OK)
        rc = lob_get_levels_books(d.engine, d_ids, n, d.depth, d.d_bid_px, d.d_bid_qty,
                                  d.d_ask_px, d.d_ask_qty, ps);
    if (rc == LOB_OK && collect) rc = lob_get_trades(d.engine, nullptr, d.d_trade_counts, ps);
    if (rc != LOB_OK) return rc;
    if (timing) err = cudaEventRecord(e.t1, ps);
    if (err == cudaSuccess) err = cudaEventRecord(s->ev_used[k], ps);
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_serve_tick: event");
    s->tick += 1;

    // every active episode advanced one step; those at their last step leave
    int32_t nf = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t slot = ids[i];
        if (h_active) h_active[i] = slot;
        if (++s->step[slot] >= s->n_steps[slot]) {
            h_finished[nf++] = slot;
            s->active[slot] = 0;
            s->free_slots.push_back(slot);
        }
    }
    *n_active = n;
    *n_finished = nf;
    *n_msgs = acc;
    return LOB_OK;
}

int lob_serve_ready(lob_serve* s)
{
    if (!s) {
        lob_set_error("lob_serve_ready: null executor");
        return LOB_E_INVAL;
    }
    const lob_serve::Entry& e = s->ring[s->pos];
    if (!e.busy) return 1;
    for (cudaEvent_t ev : {e.copied, e.timed ? e.t1 : e.copied}) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaErrorNotReady) return 0;
        if (q != cudaSuccess) return lob_cuda_fail(q, "lob_serve_ready");
    }
    return 1;
}

int lob_serve_timings(lob_serve* s, float* proc_ms, float* gen_ms, int32_t* n_in_tick,
                      int32_t cap, int32_t* count)
{
    if (!s || !count || cap < 0 || (cap > 0 && (!proc_ms || !gen_ms || !n_in_tick))) {
        lob_set_error("lob_serve_timings: invalid argument");
        return LOB_E_INVAL;
    }
    const int rc = retire_all(s);
    if (rc != LOB_OK) return rc;
    const int32_t total = (int32_t)s->proc_ms.size();
    *count = total;
    if (cap < total) return LOB_OK;  // sizes only; nothing is cleared
    for (int32_t i = 0; i < total; ++i) {
        proc_ms[i] = s->proc_ms[i];
        gen_ms[i] = s->gen_ms[i];
        n_in_tick[i] = s->n_in_tick[i];
    }
    s->proc_ms.clear();
    s->gen_ms.clear();
    s->n_in_tick.clear();
    return LOB_OK;
}

int lob_serve_destroy(lob_serve* s)
{
    if (!s) return LOB_OK;
    const int rc = retire_all(s);
    release(s);
    return rc;
}

}  // extern "C"
