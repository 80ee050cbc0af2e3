/*
 * lobgen_core.h -- seeded synthetic order-flow generator (shared input source).
 *
 * This module produces the message streams that stand in for the LOBSTER
 * replay data of Sec. 5.1.1 (TSLA / AMZN message files, not available here).
 * It holds no order-book arithmetic: it never looks at a book, never matches,
 * never decides whether an order rests.  It only draws messages
 * m = [T, S, Q, P, OID, TID, time] (Sec. 4.2, eq. message) from a seeded,
 * counter-based random source, so that the host (CPU checker, benchmarks) and
 * the device (serving loop, RL episodes) can produce bit-identical streams.
 *
 * Random source: SplitMix64's output function (Steele, Lea & Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) used as a keyed
 * hash of (seed, stream, message index, draw index).  All sampling is integer
 * only: categorical draws compare the high 32 bits against uint32 cut points,
 * geometric draws invert the CDF through a uint64 threshold table that the
 * host computes once and both sides read, uniform draws use multiply-shift.
 *
 * The same source compiles as C (host) and as CUDA (__host__ __device__).
 */
#ifndef LOBGEN_CORE_H
#define LOBGEN_CORE_H

#include <stdint.h>

#ifdef __CUDACC__
#define LG_FN __host__ __device__ __forceinline__
#else
#define LG_FN static inline
#endif

/* Message record as written to the stream: 32 bytes, little endian,
 * {int32 type, side, price, qty, oid, tid; int64 time_ns}.  type: 1 limit,
 * 2 partial cancel, 3 delete, 4 market; side: +1 bid (buy), -1 ask (sell). */
typedef struct {
    int32_t type, side, price, qty, oid, tid;
    int64_t time_ns;
} lobgen_msg_t;

/* One remembered limit order that a later cancel or delete may target. */
typedef struct {
    int32_t oid, qty, price, side;
} lobgen_pool_entry_t;

/* Stream parameters (identical for every book of a workload). */
typedef struct {
    uint64_t seed;
    uint32_t cut_add;         /* P(add) * 2^32                                  */
    uint32_t cut_cancel;      /* (P(add) + P(partial cancel)) * 2^32            */
    uint32_t cut_delete;      /* (P(add) + P(cancel) + P(delete)) * 2^32        */
    uint32_t cut_mid_down;    /* r32 <  cut_mid_down -> mid - 1                 */
    uint32_t cut_mid_up;      /* r32 >= cut_mid_up   -> mid + 1                 */
    uint32_t cut_marketable;  /* r32 <  cut_marketable -> aggressive limit      */
    int32_t  start_mid;       /* 10000 ticks                                    */
    int32_t  tid_max;         /* trader ids U{1..tid_max}                       */
    int32_t  dt_max;          /* time step 1 + U{0..dt_max-1} ns                */
    int32_t  pool_cap;        /* remembered ids for cancel targeting (<= 4096)  */
    int32_t  geo_px_kmax;     /* price offset G truncated at this value         */
    int32_t  geo_q_kmax;      /* qty G truncated at this value                  */
    int64_t  t0_ns;           /* first message time base                        */
    int32_t  first_oid;       /* OIDs count up from here                        */
    int32_t  pad_;
} lobgen_params_t;

/* Per-book generator state (the pool lives in a separate array). */
typedef struct {
    int64_t  time_ns;
    uint64_t key;             /* per-book key derived from (seed, stream id)    */
    uint64_t index;           /* messages drawn so far                          */
    int32_t  mid;
    int32_t  next_oid;
    int32_t  pool_count;
    int32_t  pad_;
} lobgen_state_t;

/* ---- random source --------------------------------------------------- */

/* SplitMix64 output function of x + golden gamma (written from the paper's
 * description of the generator: one Weyl step followed by the variant-13
 * xor-shift-multiply finaliser). */
LG_FN uint64_t lg_mix(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

LG_FN uint64_t lg_stream_key(uint64_t seed, uint64_t stream)
{
    return lg_mix(lg_mix(seed) ^ (stream * 0xD1B54A32D192ED03ull));
}

/* draw number `d` (0..15) of item `idx` of the stream with key `key` */
LG_FN uint64_t lg_draw(uint64_t key, uint64_t idx, uint32_t d)
{
    return lg_mix(key ^ lg_mix((idx << 4) | (uint64_t)(d & 15u)));
}

LG_FN uint32_t lg_hi32(uint64_t r) { return (uint32_t)(r >> 32); }

/* uniform on {0..n-1}, n >= 1 (multiply-shift on the high 32 bits) */
LG_FN uint32_t lg_uniform(uint64_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)lg_hi32(r) * (uint64_t)n) >> 32);
}

/* Geometric on {0,1,..,kmax} by inverse CDF: the smallest k with r < thr[k],
 * kmax if r >= thr[kmax-1].  thr[k] = floor(F(k) * 2^64) is increasing. */
LG_FN int32_t lg_geometric(uint64_t r, const uint64_t* thr, int32_t kmax)
{
    int32_t lo = 0, hi = kmax;
    while (lo < hi) {
        int32_t m = (lo + hi) >> 1;
        if (r < thr[m]) hi = m; else lo = m + 1;
    }
    return lo;
}

/* ---- the stream ------------------------------------------------------- */

LG_FN void lg_init_state(const lobgen_params_t* p, uint64_t stream_id,
                         lobgen_state_t* s)
{
    s->time_ns = p->t0_ns;
    s->key = lg_stream_key(p->seed, stream_id);
    s->index = 0;
    s->mid = p->start_mid;
    s->next_oid = p->first_oid;
    s->pool_count = 0;
    s->pad_ = 0;
}

/* Draw the next message of one book's stream.
 * Draw slots: 0 mid step, 1 type, 2 side, 3 price offset, 4 marketable,
 * 5 quantity, 6 trader id, 7 pool slot, 8 time step. */
LG_FN lobgen_msg_t lg_next(const lobgen_params_t* p, const uint64_t* geo_px,
                           const uint64_t* geo_q, lobgen_state_t* s,
                           lobgen_pool_entry_t* pool)
{
    const uint64_t key = s->key, i = s->index;
    lobgen_msg_t m;

    /* exogenous mid-price walk, one step per message */
    uint32_t rm = lg_hi32(lg_draw(key, i, 0));
    int32_t mid = s->mid;
    if (rm < p->cut_mid_down) mid -= 1;
    else if (rm >= p->cut_mid_up) mid += 1;
    if (mid < 1) mid = 1;
    s->mid = mid;

    uint32_t rt = lg_hi32(lg_draw(key, i, 1));
    int32_t type = rt < p->cut_add ? 1 : rt < p->cut_cancel ? 2
                 : rt < p->cut_delete ? 3 : 4;
    if ((type == 2 || type == 3) && s->pool_count == 0) type = 1;

    int32_t side = (lg_draw(key, i, 2) >> 63) ? 1 : -1;
    int32_t tid = 1 + (int32_t)lg_uniform(lg_draw(key, i, 6), (uint32_t)p->tid_max);

    m.type = type;
    m.tid = tid;
    if (type == 1) {
        int32_t g = lg_geometric(lg_draw(key, i, 3), geo_px, p->geo_px_kmax);
        int aggressive = lg_hi32(lg_draw(key, i, 4)) < p->cut_marketable;
        int32_t price = aggressive ? (side == 1 ? mid + g : mid - g)
                                   : (side == 1 ? mid - 1 - g : mid + 1 + g);
        if (price < 1) price = 1;
        int32_t qty = 1 + lg_geometric(lg_draw(key, i, 5), geo_q, p->geo_q_kmax);
        int32_t oid = s->next_oid++;
        m.side = side; m.price = price; m.qty = qty; m.oid = oid;
        lobgen_pool_entry_t e; e.oid = oid; e.qty = qty; e.price = price; e.side = side;
        if (s->pool_count < p->pool_cap) {
            pool[s->pool_count++] = e;
        } else {
            pool[lg_uniform(lg_draw(key, i, 7), (uint32_t)p->pool_cap)] = e;
        }
    } else if (type == 2 || type == 3) {
        uint32_t j = lg_uniform(lg_draw(key, i, 7), (uint32_t)s->pool_count);
        lobgen_pool_entry_t e = pool[j];
        m.side = e.side; m.price = e.price; m.oid = e.oid;
        if (type == 2) {
            m.qty = e.qty >= 2 ? 1 + (int32_t)lg_uniform(lg_draw(key, i, 5), (uint32_t)(e.qty - 1)) : 1;
        } else {
            m.qty = e.qty;
            pool[j] = pool[s->pool_count - 1];
            s->pool_count -= 1;
        }
    } else {
        m.side = side;
        m.price = 0;
        m.qty = 1 + lg_geometric(lg_draw(key, i, 5), geo_q, p->geo_q_kmax);
        m.oid = s->next_oid++;
    }
    s->time_ns += 1 + (int64_t)lg_uniform(lg_draw(key, i, 8), (uint32_t)p->dt_max);
    m.time_ns = s->time_ns;
    s->index = i + 1;
    return m;
}

/* Random draws of the synthetic execution agent for one (env, step):
 * bits 0-1 = number of child orders - 1 (U{1..4}); bits 2+3k..4+3k = action
 * of child k, U{0..5}: 0..4 = offset -2..+2 ticks from the best ask,
 * 5 = market order. */
LG_FN uint32_t lg_agent_draw(uint64_t seed, uint64_t env, uint64_t step)
{
    uint64_t key = lg_stream_key(seed ^ 0xA6E17A6E17A6E17Aull, env);
    uint32_t n = lg_uniform(lg_draw(key, step, 0), 4);
    uint32_t w = n;
    for (uint32_t k = 0; k < 4; ++k)
        w |= lg_uniform(lg_draw(key, step, 1 + k), 6) << (2 + 3 * k);
    return w;
}

#endif /* LOBGEN_CORE_H */
