// lob_process.cuh -- the processing kernel of the batched order-book engine.
//
// A persistent grid of warps; each warp pulls a work item (one book's message
// segment, Sec. 4.3 batching over independent books) from a device work queue,
// stages the book and the segment's messages in shared memory with 1-D bulk
// asynchronous copies (double-buffered chunks completed on mbarriers), applies
// the messages in order with the warp routines of lob_core.cuh, and writes the
// book back.  Uneven segment lengths balance through the queue; the queue
// resets itself when the last warp leaves.  Included by lob_engine.cu only.
#pragma once

#include "../../include/lob.h"
#include "lob_core.cuh"

namespace {

using namespace lob;

constexpr uint64_t kWaitNs = 2000000000ull;  // bounded wait for a staged chunk: 2 s

struct ProcArgs {
    const Msg* msgs;
    const int64_t* offsets;  // [n_items+1] boundaries, or starts when `counts_in` is set
    const int64_t* counts_in;
    const int32_t* book_ids;
    int32_t n_items;
    int32_t n_books;
    char* state;
    int32_t* counts;
    Trade* trades;
    int64_t* tcounts;
    int64_t* stats;
    int32_t* status;
    int32_t* queue;
    int32_t cap, rule, trade_cap, append, chunk, pad_;
    uint64_t wait_ns;
    int32_t* l1;  // level-1 trace [message][4], or null
};

// Each of the two chunk buffers holds one message more than a chunk, so the
// message loop can always load the next message (the one past a chunk's end
// is read and never used) without a bounds test.
__host__ __device__ constexpr int chunk_stride(int chunk) { return (chunk + 1) * 32; }

template <int K>
__host__ __device__ constexpr int warp_smem_bytes(int chunk)
{
    return ((Geo<K>::BOOK_BYTES + 2 * chunk_stride(chunk) + 16) + 127) / 128 * 128;
}

// threads per CTA the processing kernel is compiled for (bounds registers)
template <int K>
constexpr int max_threads() { return K >= 4 ? 256 : 512; }

// kTrace: also write the level-1 state after every message; kSnap: the
// snapshot cancel rule (LOB_FLAG_SNAPSHOT_CANCELS).  Each combination is its
// own instantiation, so the default one carries neither.
template <int K, bool kTrace, bool kSnap>
__global__ void __launch_bounds__(max_threads<K>(), 1) k_process(ProcArgs a)
{
    using Book = typename BookPolicy<K>::type;
    extern __shared__ __align__(128) char smem[];
    const int l = lane_id();
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int chunk = a.chunk;
    char* base = smem + warp * warp_smem_bytes<K>(chunk);
    char* image = base;  // staged book image (the whole book for the shared-memory policy)
    char* msgbuf = base + Geo<K>::BOOK_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(msgbuf + 2 * chunk_stride(chunk));
    const int total_warps = gridDim.x * W;

    if (l == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    __syncwarp();

    uint32_t g = 0;  // chunks consumed by this warp: stage g&1, parity (g>>1)&1
    bool failed = false;
    while (!failed) {
        int item = 0;
        if (l == 0) item = atomicAdd(&a.queue[0], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.n_items) break;
        const int b = a.book_ids ? a.book_ids[item] : item;
        if (b < 0 || b >= a.n_books) {
            if (l == 0) atomicOr(a.status, LOB_STATUS_BAD_BOOK);
            continue;
        }
        const int64_t lo = a.offsets[item];
        const int64_t hi = a.counts_in ? lo + a.counts_in[item] : a.offsets[item + 1];
        if (hi < lo) {
            if (l == 0) atomicOr(a.status, LOB_STATUS_BAD_SEGMENT);
            continue;
        }
        TradeSink ts{a.trades + (int64_t)b * a.trade_cap, a.append ? a.tcounts[b] : 0,
                     a.trade_cap};
        const int64_t nmsg = hi - lo;
        if (nmsg == 0) {
            __syncwarp();
            if (l == 0) a.tcounts[b] = ts.count;
            continue;
        }
        const int nchunks = (int)((nmsg + chunk - 1) / chunk);
        char* gbook = a.state + (int64_t)b * Geo<K>::BOOK_BYTES;
        if (l == 0) {
            fence_proxy_async();
            for (int c = 0; c < 2 && c < nchunks; ++c) {
                const uint32_t st = (g + c) & 1;
                const int64_t c0 = lo + (int64_t)c * chunk;
                const uint32_t cnt = (uint32_t)min((int64_t)chunk, hi - c0);
                mbar_expect_tx(&bar[st], cnt * 32 + (c == 0 ? Geo<K>::BOOK_BYTES : 0));
                if (c == 0) bulk_g2s(image, gbook, Geo<K>::BOOK_BYTES, &bar[st]);
                bulk_g2s(msgbuf + st * chunk_stride(chunk), a.msgs + c0, cnt * 32, &bar[st]);
            }
        }
        int n_bid = a.counts[2 * b], n_ask = a.counts[2 * b + 1];
        Counters ctr{0, l};
        Tally tally;
        NoObs obs;
        const int64_t tcount0 = ts.count;
        Book bk;
        if constexpr (!Book::kInRegisters) bk.base = image;
        // book-independent counters, accumulated by the pre-pass per lane
        int32_t c_kind[5] = {0, 0, 0, 0, 0};  // noop, invalid, limit, cancel, market
        int64_t q_limit = 0, q_market = 0;
        for (int c = 0; c < nchunks; ++c) {
            const uint32_t st = (g + c) & 1, par = ((g + c) >> 1) & 1;
            if (!mbar_wait_bounded(&bar[st], par, a.wait_ns)) {
                // give up on this warp: record it, let in-flight copies land
                if (l == 0) atomicOr(a.status, LOB_STATUS_TIMEOUT);
                const int last = min(c + 1, nchunks - 1);
                for (int d = c; d <= last; ++d)
                    mbar_wait_bounded(&bar[(g + d) & 1], ((g + d) >> 1) & 1, a.wait_ns);
                failed = true;
                break;
            }
            if (c == 0) bk.from_image(image);
            int4* mb = reinterpret_cast<int4*>(msgbuf + st * chunk_stride(chunk));
            const int cnt = (int)min((int64_t)chunk, hi - (lo + (int64_t)c * chunk));
            // pre-pass, 32 messages at a time: validate and classify (the part of
            // Sec. 4.2 that does not depend on the book); the dispatch code
            // replaces the type word in the staged copy
            for (int i = l; i < cnt; i += 32) {
                const int4 h = mb[2 * i];
                int kind = 0;
                const int32_t op = classify(h.x, h.y, h.z, h.w, kind);
                mb[2 * i].x = op;
                c_kind[0] += kind == CTR_NOOP;
                c_kind[1] += kind == CTR_INVALID;
                c_kind[2] += kind == CTR_LIMIT;
                c_kind[3] += kind == CTR_CANCEL;
                c_kind[4] += kind == CTR_MARKET;
                q_limit += kind == CTR_LIMIT ? h.w : 0;
                q_market += kind == CTR_MARKET ? h.w : 0;
            }
            __syncwarp();
            // the book-dependent part, strictly in order
            int4 na = mb[0], nb = mb[1];
            for (int i = 0; i < cnt; ++i) {
                const int4 ha = na, hb = nb;
                na = mb[2 * i + 2];  // past the chunk's end: the padding message, unused
                nb = mb[2 * i + 3];
                apply_message<K, false>(bk, n_bid, n_ask, a.cap, a.rule, ha.x, ha.z, ha.w, hb.x, hb.y,
                                 hb.z, hb.w, ts, tally, obs, kSnap);
                check_book<K>(bk, n_bid, n_ask, a.cap, a.status);
                if constexpr (kTrace) {
                    const int4 top = level1_book<K>(bk, n_bid, n_ask);
                    if (l == 0) reinterpret_cast<int4*>(a.l1)[lo + (int64_t)c * chunk + i] = top;
                }
            }
            __syncwarp();
            if (c + 2 < nchunks && l == 0) {
                fence_proxy_async();
                const int64_t c0 = lo + (int64_t)(c + 2) * chunk;
                const uint32_t cn = (uint32_t)min((int64_t)chunk, hi - c0);
                mbar_expect_tx(&bar[st], cn * 32);
                bulk_g2s(msgbuf + st * chunk_stride(chunk), a.msgs + c0, cn * 32, &bar[st]);
            }
        }
        if (failed) break;
        g += (uint32_t)nchunks;
        // write the book back
        bk.to_image(image);
        __syncwarp();
        const int4* src = reinterpret_cast<const int4*>(image);
        int4* dst = reinterpret_cast<int4*>(gbook);
#pragma unroll 4
        for (int i = l; i < Geo<K>::BOOK_BYTES / 16; i += 32) dst[i] = src[i];
        ctr.add(CTR_MSGS, nmsg);
        ctr.add(CTR_TRADES, ts.count - tcount0);
        ctr.add(CTR_TRADES_DROPPED, max(ts.count - a.trade_cap, (int64_t)0) -
                                        max(tcount0 - a.trade_cap, (int64_t)0));
        ctr.add(CTR_TRADED_QTY, tally.traded_qty);
        ctr.add(CTR_RESTED, tally.rested);
        ctr.add(CTR_REJECTED, tally.rejected);
        ctr.add(CTR_REJECTED_QTY, tally.rejected_qty);
        ctr.add(CTR_EVICTED, tally.evicted);
        ctr.add(CTR_EVICTED_QTY, tally.evicted_qty);
        ctr.add(CTR_CANCEL_HIT, tally.cancel_hit);
        ctr.add(CTR_CANCELLED_QTY, tally.cancelled_qty);
        ctr.add(CTR_MARKET_DISCARDED_QTY, tally.discarded_qty);
        ctr.add(CTR_NOOP, __reduce_add_sync(kFull, (unsigned)c_kind[0]));
        ctr.add(CTR_INVALID, __reduce_add_sync(kFull, (unsigned)c_kind[1]));
        ctr.add(CTR_LIMIT, __reduce_add_sync(kFull, (unsigned)c_kind[2]));
        ctr.add(CTR_CANCEL, __reduce_add_sync(kFull, (unsigned)c_kind[3]));
        ctr.add(CTR_MARKET, __reduce_add_sync(kFull, (unsigned)c_kind[4]));
        ctr.add(CTR_LIMIT_QTY, warp_sum64(q_limit));
        ctr.add(CTR_MARKET_QTY, warp_sum64(q_market));
        // a cancel that found no live order is a miss
        const int64_t n_cancel = __shfl_sync(kFull, ctr.v, CTR_CANCEL);
        const int64_t n_hit = __shfl_sync(kFull, ctr.v, CTR_CANCEL_HIT);
        ctr.add(CTR_CANCEL_MISS, n_cancel - n_hit);
        if (l < kNumCtr) a.stats[(int64_t)b * kNumCtr + l] += ctr.v;
        if (l == 0) {
            a.counts[2 * b] = n_bid;
            a.counts[2 * b + 1] = n_ask;
            a.tcounts[b] = ts.count;
        }
        __syncwarp();
    }
    // leave the queue; the last warp out resets it for the next launch
    if (l == 0) {
        __threadfence();
        const int done = atomicAdd(&a.queue[1], 1);
        if (done == total_warps - 1) {
            a.queue[0] = 0;
            a.queue[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace
