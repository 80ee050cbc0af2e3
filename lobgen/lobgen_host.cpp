// lobgen_host.cpp -- host (CPU) side of the seeded order-flow generator.
//
// C ABI used through ctypes by the test-suite, the benchmark and the CPU
// checker.  Books are independent streams, so generation is split across
// std::thread workers by book; the output does not depend on the thread count.
#include <stdint.h>
#include <string.h>
#include <algorithm>
#include <thread>
#include <vector>

#include "lobgen_core.h"

static_assert(sizeof(lobgen_msg_t) == 32, "message record must be 32 bytes");
static_assert(sizeof(lobgen_pool_entry_t) == 16, "pool entry must be 16 bytes");
static_assert(sizeof(lobgen_state_t) == 40, "state layout");
static_assert(sizeof(lobgen_params_t) == 72, "params layout");

template <class F>
static void parallel_books(int32_t n_books, int32_t n_threads, F&& body)
{
    if (n_threads <= 1 || n_books <= 1) {
        for (int32_t b = 0; b < n_books; ++b) body(b);
        return;
    }
    int32_t nt = std::min(n_threads, n_books);
    std::vector<std::thread> pool;
    pool.reserve(nt);
    for (int32_t t = 0; t < nt; ++t) {
        pool.emplace_back([&, t]() {
            for (int32_t b = t; b < n_books; b += nt) body(b);
        });
    }
    for (auto& th : pool) th.join();
}

extern "C" {

int lobgen_abi_version(void) { return 1; }

// Initialise `n_books` generator states; book b uses stream id stream_ids[b]
// (or b when stream_ids is NULL).
int lobgen_init(const lobgen_params_t* p, int32_t n_books, const uint64_t* stream_ids,
                lobgen_state_t* states)
{
    if (!p || !states || n_books < 0) return -1;
    if (p->pool_cap < 1 || p->pool_cap > 4096) return -1;
    for (int32_t b = 0; b < n_books; ++b)
        lg_init_state(p, stream_ids ? stream_ids[b] : (uint64_t)b, &states[b]);
    return 0;
}

// Draw counts[b] further messages of book b into out[out_offsets[b] ...].
// pools is [n_books][p->pool_cap].
int lobgen_advance(const lobgen_params_t* p, const uint64_t* geo_px, const uint64_t* geo_q,
                   int32_t n_books, lobgen_state_t* states, lobgen_pool_entry_t* pools,
                   const int64_t* counts, const int64_t* out_offsets, lobgen_msg_t* out,
                   int32_t n_threads)
{
    if (!p || !geo_px || !geo_q || !states || !pools || !counts || !out_offsets || !out)
        return -1;
    parallel_books(n_books, n_threads, [&](int32_t b) {
        lobgen_state_t s = states[b];
        lobgen_pool_entry_t* pool = pools + (int64_t)b * p->pool_cap;
        lobgen_msg_t* o = out + out_offsets[b];
        for (int64_t k = 0; k < counts[b]; ++k) o[k] = lg_next(p, geo_px, geo_q, &s, pool);
        states[b] = s;
    });
    return 0;
}

// One-shot: fresh state per book, book b gets offsets[b+1]-offsets[b]
// messages written contiguously at out + offsets[b].
int lobgen_generate(const lobgen_params_t* p, const uint64_t* geo_px, const uint64_t* geo_q,
                    int32_t n_books, const uint64_t* stream_ids, const int64_t* offsets,
                    lobgen_msg_t* out, int32_t n_threads)
{
    if (!p || !geo_px || !geo_q || !offsets || !out || n_books < 0) return -1;
    if (p->pool_cap < 1 || p->pool_cap > 4096) return -1;
    parallel_books(n_books, n_threads, [&](int32_t b) {
        std::vector<lobgen_pool_entry_t> pool((size_t)p->pool_cap);
        lobgen_state_t s;
        lg_init_state(p, stream_ids ? stream_ids[b] : (uint64_t)b, &s);
        lobgen_msg_t* o = out + offsets[b];
        int64_t n = offsets[b + 1] - offsets[b];
        for (int64_t k = 0; k < n; ++k) o[k] = lg_next(p, geo_px, geo_q, &s, pool.data());
    });
    return 0;
}

// Agent draws for steps [0, n_steps) of envs [0, n_envs): out[step][env].
int lobgen_agent_draws(uint64_t seed, int32_t n_envs, int32_t n_steps, uint32_t* out)
{
    if (!out || n_envs < 0 || n_steps < 0) return -1;
    for (int32_t t = 0; t < n_steps; ++t)
        for (int32_t e = 0; e < n_envs; ++e)
            out[(int64_t)t * n_envs + e] = lg_agent_draw(seed, (uint64_t)e, (uint64_t)t);
    return 0;
}

}  // extern "C"
