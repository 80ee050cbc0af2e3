// lob_env.cu -- execution-environment steps (Sec. 5) fused into one kernel.
//
// A warp owns one environment (= one book of a lob_ctx).  For each step it
// stages the step's window of data messages in shared memory (bulk copy,
// double-buffered across steps), replays them with the book kept on chip,
// runs the synthetic execution agent (child sell orders, or the final cancel
// and market sell), and writes the step's top levels, agent fills and VWAP
// reward.  One launch can run many consecutive steps (the book never leaves
// the SM between them); a single-step launch is what a CUDA graph captures.
#include <cuda_runtime.h>
#include <stdint.h>

#include <new>

#include "../../include/lob.h"
#include "lob_core.cuh"
#include "lob_engine.h"

using namespace lob;

struct EnvStateDev {
    int64_t submitted, executed, last_time;
    int32_t id_counter, last_ask;
    double p_init;
};
static_assert(sizeof(EnvStateDev) == 40, "env state layout");

struct lob_env {
    lob_ctx* book = nullptr;
    lob_env_config_t cfg;
    EnvStateDev* d_state = nullptr;
    int64_t* d_seg_flag = nullptr;  // per environment: last segment finished (see k_env)
    int chunk = 0;        // staged messages per step (msgs_per_step rounded up to 8)
    int warps = 4;
    int per_sm_v[8] = {1, 1, 1, 1, 1, 1, 1, 1};  // resident CTAs per SM of each
                                                // (trace, snap, segmented) variant
    int smem_per_cta = 0;
    int64_t launches = 0;
    int32_t last_segments = 0;  // segments per environment of the last lob_env_run
};

namespace {

constexpr uint64_t kEnvWaitNs = 2000000000ull;
constexpr int kLevelScratch = 128 * 8 + 64 * 4;  // two prefix words and a price per level
constexpr int kAgentRecs = 8;  // staged agent orders of one step (at most 4 + 1)

struct EnvArgs {
    const Msg* replay;
    int64_t stride_env;
    int32_t msgs_per_step, step0, n_run, n_envs;
    const uint32_t* draws;
    char* state;
    int32_t* counts;
    Trade* trades;
    int64_t* tcounts;
    int64_t* stats;
    int32_t* status;
    int32_t* queue;
    int32_t cap, rule, trade_cap, chunk;
    EnvStateDev* env;
    int32_t n_steps, parent, agent_tid, depth, p_fallback, pad_;
    double lambda;
    float* reward;
    int32_t *bid_px, *bid_qty, *ask_px, *ask_qty;
    int64_t* fills;
    uint64_t wait_ns;
    int32_t* l1;  // [n_run][n_envs][msgs_per_step][4] or null
    const float* actions;  // [n_run][n_envs][4] policy sizes, or null (stand-in draws)
    int32_t passive_ticks, tick;
    int32_t n_seg, pad2_;  // segments each environment's steps are split into (1 = whole run)
    int64_t* seg_flag;     // [n_envs] (epoch << 8) | segments of this launch finished
};

// Acquire load / release store of a 64-bit flag in global memory (gpu scope).
__device__ __forceinline__ int64_t ld_acquire_gpu(const int64_t* p)
{
    int64_t v;
    asm volatile("ld.acquire.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_gpu(int64_t* p, int64_t v)
{
    asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// order this thread's generic-proxy view of global memory before its later
// async-proxy (bulk copy) reads of it
__device__ __forceinline__ void fence_proxy_async_global()
{
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// Each of the two step buffers holds one message more than a step, and the
// agent buffer more than a step's agent orders, so the message loop always
// loads the next message (past the end: padding, never used) without a test.
__host__ __device__ constexpr int env_stage_stride(int chunk) { return (chunk + 1) * 32; }

template <int K>
__host__ __device__ constexpr int env_warp_smem(int chunk)
{
    return ((Geo<K>::BOOK_BYTES + 2 * env_stage_stride(chunk) + 16 + kLevelScratch +
             kAgentRecs * 32) + 127) / 128 * 128;
}

// kTrace: the kernel also writes the level-1 state after every data message;
// kSnap: the snapshot cancel rule (LOB_FLAG_SNAPSHOT_CANCELS).  Separate
// instantiations, so the default loop carries neither.
// Work items: in the kSeg instantiation (n_seg > 1) every environment's run
// is split into n_seg
// segments of consecutive steps, handed out segment by segment over all
// environments (item = segment * n_envs + env), so that the last round of a
// persistent grid is not left with a few whole episodes while the other
// warps idle.  A segment starts from the book, counts and agent state the
// previous segment of its environment wrote back; it waits (bounded) on that
// environment's flag, which the previous segment releases with the launch's
// epoch, a device counter that every launch advances when its last warp
// leaves (so a replayed CUDA graph never reads a stale flag).
// Register-resident books (K <= 4) run in CTAs of four warps, bounded so that
// three CTAs fit an SM (at most 168 registers a thread, no spills): twelve
// environments' serial chains per SM instead of the eight that 186 registers
// allowed, 20 % less time per episode.  (CTAs of one or two warps measured
// no faster at 186 registers, and slower at 144-152 with 13-14 per SM.)
template <int K, bool kTrace, bool kSnap, bool kSeg>
__global__ void __launch_bounds__(K >= 8 ? 256 : 128, K >= 8 ? 1 : 3) k_env(EnvArgs a)
{
    using Book = typename BookPolicy<K>::type;
    extern __shared__ __align__(128) char smem[];
    const int l = lane_id();
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int chunk = a.chunk;
    char* base = smem + warp * env_warp_smem<K>(chunk);
    char* image = base;
    char* msgbuf = base + Geo<K>::BOOK_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(msgbuf + 2 * env_stage_stride(chunk));
    unsigned long long* lq =
        reinterpret_cast<unsigned long long*>(msgbuf + 2 * env_stage_stride(chunk) + 16);
    int32_t* lp = reinterpret_cast<int32_t*>(lq + 128);
    int4* agent_buf = reinterpret_cast<int4*>(lp + 64);
    const int total_warps = gridDim.x * W;
    const uint32_t bytes = (uint32_t)a.msgs_per_step * 32;

    if (l == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
        fence_proxy_async();
    }
    __syncwarp();

    uint32_t g = 0;
    bool failed = false;
    const int64_t epoch = kSeg ? (int64_t)*reinterpret_cast<volatile int32_t*>(&a.queue[2]) : 0;
    while (!failed) {
        int item = 0;
        if (l == 0) item = atomicAdd(&a.queue[0], 1);
        item = __shfl_sync(kFull, item, 0);
        if (item >= a.n_envs * a.n_seg) break;
        constexpr bool segmented = kSeg;
        int seg = 0, b = item, r0 = 0, r1 = a.n_run;
        if (segmented) {  // (n_run * n_seg < 2^31, checked on the host)
            seg = item / a.n_envs;
            b = item - seg * a.n_envs;
            r0 = seg * a.n_run / a.n_seg;
            r1 = (seg + 1) * a.n_run / a.n_seg;
        }
        char* gbook = a.state + (int64_t)b * Geo<K>::BOOK_BYTES;
        const Msg* my = a.replay + (int64_t)b * a.stride_env;
        if (segmented && seg > 0) {
            // the previous segment of this environment must have written back
            bool ok = true;
            if (l == 0) {
                const int64_t want = (epoch << 8) | seg;
                if (ld_acquire_gpu(&a.seg_flag[b]) != want) {
                    const uint64_t t0 = global_ns();
                    while (ld_acquire_gpu(&a.seg_flag[b]) != want) {
                        if (global_ns() - t0 > a.wait_ns) {
                            ok = false;
                            break;
                        }
                    }
                }
                if (ok) fence_proxy_async_global();
                else atomicOr(a.status, LOB_STATUS_TIMEOUT);
            }
            if (!__shfl_sync(kFull, ok ? 1 : 0, 0)) continue;  // skip it (status set)
        }
        if (l == 0) {
            fence_proxy_async();
            for (int c = 0; c < 2 && c < r1 - r0; ++c) {
                const uint32_t st = (g + c) & 1;
                mbar_expect_tx(&bar[st], bytes + (c == 0 ? Geo<K>::BOOK_BYTES : 0));
                if (c == 0) bulk_g2s(image, gbook, Geo<K>::BOOK_BYTES, &bar[st]);
                bulk_g2s(msgbuf + st * env_stage_stride(chunk),
                         my + (int64_t)(a.step0 + r0 + c) * a.msgs_per_step, bytes, &bar[st]);
            }
        }
        int n_bid, n_ask;
        EnvStateDev es;
        if (segmented) {
            // written by another SM in this launch: read through L2, never a
            // stale line of this SM's L1
            n_bid = __ldcg(&a.counts[2 * b]);
            n_ask = __ldcg(&a.counts[2 * b + 1]);
            const int64_t* src = reinterpret_cast<const int64_t*>(&a.env[b]);
            int64_t w[5];
#pragma unroll
            for (int k = 0; k < 5; ++k) w[k] = __ldcg(src + k);
            memcpy(&es, w, sizeof(es));
        } else {
            n_bid = a.counts[2 * b];
            n_ask = a.counts[2 * b + 1];
            es = a.env[b];
        }
        Counters ctr{0, l};
        Tally tally;
        Book bk;
        if constexpr (!Book::kInRegisters) bk.base = image;
        int32_t c_kind[5] = {0, 0, 0, 0, 0};  // noop, invalid, limit, cancel, market (per lane)
        int64_t q_limit = 0, q_market = 0, n_msgs = 0;
        int64_t n_trades = 0, n_dropped = 0;
        TradeSink ts{a.trades + (int64_t)b * a.trade_cap, 0, a.trade_cap};
        for (int r = r0; r < r1; ++r) {
            const int t = a.step0 + r;
            const int rr = r - r0;  // step within this work item
            const uint32_t st = (g + rr) & 1, par = ((g + rr) >> 1) & 1;
            if (!mbar_wait_bounded(&bar[st], par, a.wait_ns)) {
                if (l == 0) atomicOr(a.status, LOB_STATUS_TIMEOUT);
                const int last = min(rr + 1, r1 - r0 - 1);
                for (int d = rr; d <= last; ++d)
                    mbar_wait_bounded(&bar[(g + d) & 1], ((g + d) >> 1) & 1, a.wait_ns);
                failed = true;
                break;
            }
            if (rr == 0) bk.from_image(image);
            int4* mb = reinterpret_cast<int4*>(msgbuf + st * env_stage_stride(chunk));
            const int cnt = a.msgs_per_step;
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
            // 1. replay the step's data messages (trade log restarts each step)
            ts.count = 0;
            VwapObs obs;
            obs.agent_tid = a.agent_tid;
            const int64_t traded0 = tally.traded_qty;
            // last data time of the window (agent orders carry it)
            if (cnt > 0) {
                const int4 hl = mb[2 * (cnt - 1) + 1];
                es.last_time = (int64_t)(((uint64_t)(uint32_t)hl.w << 32) | (uint32_t)hl.z);
            }
            n_msgs += cnt;
            // phase 0: the window's data messages; phase 1: the agent's orders,
            // staged as records and run through the same (not unrolled) loop
#pragma unroll 1
            for (int phase = 0; phase < 2; ++phase) {
                const int4* src = mb;
                int count = cnt;
                if (phase == 1) {
                    src = agent_buf;
                    count = 0;
                    const int32_t tlo = (int32_t)(uint32_t)(uint64_t)es.last_time;
                    const int32_t thi = (int32_t)(uint32_t)((uint64_t)es.last_time >> 32);
                    auto stage = [&](int32_t op, int32_t price, int32_t q) {
                        const int32_t oid = (int32_t)((1u << 30) + (uint32_t)es.id_counter);
                        es.id_counter += 1;
                        es.submitted += q;
                        if (l == 0) {
                            agent_buf[2 * count] = make_int4(op, -1, price, q);
                            agent_buf[2 * count + 1] = make_int4(oid, a.agent_tid, tlo, thi);
                            if (op == OP_MARKET_ASK) {
                                c_kind[4] += 1;
                                q_market += q;
                            } else {
                                c_kind[2] += 1;
                                q_limit += q;
                            }
                        }
                        count += 1;
                    };
                    // initial mid of the episode (after the first data window)
                    if (t == 0) {
                        const int32_t bb = n_bid > 0 ? bk.template best_px<0>(n_bid) : 0;
                        const int32_t ba = n_ask > 0 ? bk.template best_px<1>(n_ask) : 0;
                        if (n_bid > 0 && n_ask > 0)
                            es.p_init = __ddiv_rn(__dadd_rn((double)bb, (double)ba), 2.0);
                        else if (n_bid > 0)
                            es.p_init = (double)bb;
                        else if (n_ask > 0)
                            es.p_init = (double)ba;
                        else
                            es.p_init = (double)a.p_fallback;
                    }
                    if (t < a.n_steps - 1 && a.actions != nullptr) {
                        // policy sizes at the four prices (Sec. 5.2.3), prices read
                        // once from the book after the data messages
                        if (n_ask > 0) es.last_ask = bk.template best_px<1>(n_ask);
                        const float* av = a.actions + ((int64_t)r * a.n_envs + b) * 4;
                        const int64_t pb = n_bid > 0 ? bk.template best_px<0>(n_bid) : -1;
                        const int64_t pa = n_ask > 0 ? bk.template best_px<1>(n_ask) : -1;
                        int32_t px[4];
                        px[0] = (int32_t)pb;  // far touch
                        if (n_bid > 0 && n_ask > 0) {
                            const int64_t two_t = 2 * (int64_t)a.tick;  // mid, up to the grid
                            px[1] = (int32_t)((pb + pa + two_t - 1) / two_t * a.tick);
                        } else {
                            px[1] = (int32_t)(n_bid > 0 ? pb : pa);
                        }
                        px[2] = (int32_t)pa;  // near touch
                        const int64_t pp = pa + (int64_t)a.passive_ticks * a.tick;
                        px[3] = (n_ask > 0 && pp <= kMaxInt) ? (int32_t)pp : -1;
                        int64_t remaining = (int64_t)a.parent - es.submitted;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const double x = (double)av[k];
                            int64_t q = 0;
                            if (x >= 1.0 && remaining > 0) {
                                const double w = floor(x);
                                q = w >= (double)remaining ? remaining : (int64_t)w;
                            }
                            if (px[k] <= 0 || q <= 0) continue;
                            stage(OP_LIMIT_ASK, px[k], (int32_t)q);
                            remaining -= q;
                        }
                    } else if (t < a.n_steps - 1) {
                        if (n_ask > 0) es.last_ask = bk.template best_px<1>(n_ask);
                        const int64_t remaining = (int64_t)a.parent - es.submitted;
                        const int64_t steps_left = (int64_t)a.n_steps - t;
                        const int64_t target =
                            remaining > 0 ? (remaining + steps_left - 1) / steps_left : 0;
                        const uint32_t w = a.draws[(int64_t)r * a.n_envs + b];
                        const int nchild = (int)(w & 3u) + 1;
                        const int64_t base_q = target / nchild, extra = target % nchild;
                        for (int k = 0; k < nchild; ++k) {
                            const int32_t q = (int32_t)(base_q + (k == 0 ? extra : 0));
                            if (q <= 0) continue;
                            const int32_t act = (int32_t)((w >> (2 + 3 * k)) & 7u);
                            if (act == 5)
                                stage(OP_MARKET_ASK, 0, q);
                            else
                                stage(OP_LIMIT_ASK, max(1, es.last_ask + act - 2), q);
                        }
                    } else {
                        // last step: cancel the agent's resting orders in priority order
                        while (n_ask > 0) {
                            SideVec<K> tmp;
                            SideVec<K>& v = bk.template acquire<1>(tmp);
                            int jj = -1;
#pragma unroll
                            for (int j = K - 1; j >= 0; --j)
                                if (l * K + j < n_ask && v.tid[j] == a.agent_tid) jj = j;
                            const unsigned hit = __ballot_sync(kFull, jj >= 0);
                            if (hit == 0) break;
                            const int L = __ffs(hit) - 1;
                            const int j_hit = __shfl_sync(kFull, jj, L);
                            const int p = L * K + j_hit;
                            const int32_t q = __shfl_sync(kFull, pick<K>(v.q, j_hit), L);
                            shift_out<K>(v.px, p, n_ask);
                            shift_out<K>(v.q, p, n_ask);
                            shift_out<K>(v.oid, p, n_ask);
                            shift_out<K>(v.tid, p, n_ask);
                            shift_out<K>(v.tlo, p, n_ask);
                            shift_out<K>(v.thi, p, n_ask);
                            bk.template release<1>(v, lane_touches<K>(p, n_ask - 1));
                            if constexpr (!Book::kInRegisters) __syncwarp();
                            n_ask -= 1;
                            bk.template refresh_best<1>();
                            tally.cancel_hit += 1;
                            tally.cancelled_qty += q;
                            if (l == 0) c_kind[3] += 1;
                            n_msgs += 1;
                        }
                        // ... then sell what is left at market
                        const int64_t left =
                            (int64_t)a.parent - (es.executed + warp_sum64(obs.aq));
                        if (left > 0) stage(OP_MARKET_ASK, 0, (int32_t)left);
                    }
                    n_msgs += count;
                    __syncwarp();
                }
                int4 na = src[0], nb = src[1];
                for (int i = 0; i < count; ++i) {
                    const int4 ha = na, hb = nb;
                    na = src[2 * i + 2];  // past the end: padding, unused
                    nb = src[2 * i + 3];
                    apply_message<K, true>(bk, n_bid, n_ask, a.cap, a.rule, ha.x, ha.z, ha.w, hb.x,
                                     hb.y, hb.z, hb.w, ts, tally, obs, kSnap);
                    check_book<K>(bk, n_bid, n_ask, a.cap, a.status);
                    if (kTrace && phase == 0) {
                        const int4 top = level1_book<K>(bk, n_bid, n_ask);
                        if (l == 0)
                            reinterpret_cast<int4*>(a.l1)[((int64_t)r * a.n_envs + b) *
                                                              a.msgs_per_step + i] = top;
                    }
                }
            }
            n_trades += ts.count;
            n_dropped += max(ts.count - (int64_t)a.trade_cap, (int64_t)0);
            // 4. fills and reward (eqs. rewardfunc, vwap), IEEE double
            const int64_t sq = tally.traded_qty - traded0;
            const int64_t spq = warp_sum64(obs.spq);
            const int64_t aq = warp_sum64(obs.aq);
            const int64_t apq = warp_sum64(obs.apq);
            es.executed += aq;
            const int64_t o = (int64_t)r * a.n_envs + b;
            if (l == 0) {
                double rew = 0.0;
                if (sq > 0 && aq > 0) {
                    const double vwap = __ddiv_rn((double)spq, (double)sq);
                    const double adv = __dsub_rn((double)apq, __dmul_rn((double)aq, vwap));
                    const double drift =
                        __dmul_rn(a.lambda, __dmul_rn((double)aq, __dsub_rn(vwap, es.p_init)));
                    rew = __dadd_rn(adv, drift);
                }
                a.reward[o] = (float)rew;
                a.fills[2 * o] = aq;
                a.fills[2 * o + 1] = apq;
            }
            // 5. top levels of both sides
            {
                int32_t vpx[K], vq[K];
                priority_px_q<K, 0>(bk, n_bid, vpx, vq);
                emit_levels<K>(vpx, vq, n_bid, a.depth, lq, lp, a.bid_px + o * a.depth,
                               a.bid_qty + o * a.depth);
                priority_px_q<K, 1>(bk, n_ask, vpx, vq);
                emit_levels<K>(vpx, vq, n_ask, a.depth, lq, lp, a.ask_px + o * a.depth,
                               a.ask_qty + o * a.depth);
            }
            __syncwarp();
            if (r + 2 < r1 && l == 0) {
                fence_proxy_async();
                mbar_expect_tx(&bar[st], bytes);
                bulk_g2s(msgbuf + st * env_stage_stride(chunk), my + (int64_t)(t + 2) * a.msgs_per_step, bytes,
                         &bar[st]);
            }
        }
        if (failed) break;
        g += (uint32_t)(r1 - r0);
        bk.to_image(image);
        __syncwarp();
        const int4* src = reinterpret_cast<const int4*>(image);
        int4* dst = reinterpret_cast<int4*>(gbook);
#pragma unroll 4
        for (int i = l; i < Geo<K>::BOOK_BYTES / 16; i += 32) dst[i] = src[i];
        // counters: data messages, agent orders and agent cancels all count
        ctr.add(CTR_MSGS, n_msgs);
        ctr.add(CTR_NOOP, __reduce_add_sync(kFull, (unsigned)c_kind[0]));
        ctr.add(CTR_INVALID, __reduce_add_sync(kFull, (unsigned)c_kind[1]));
        ctr.add(CTR_LIMIT, __reduce_add_sync(kFull, (unsigned)c_kind[2]));
        ctr.add(CTR_CANCEL, __reduce_add_sync(kFull, (unsigned)c_kind[3]));
        ctr.add(CTR_MARKET, __reduce_add_sync(kFull, (unsigned)c_kind[4]));
        ctr.add(CTR_LIMIT_QTY, warp_sum64(q_limit));
        ctr.add(CTR_MARKET_QTY, warp_sum64(q_market));
        ctr.add(CTR_TRADES, n_trades);
        ctr.add(CTR_TRADES_DROPPED, n_dropped);
        ctr.add(CTR_TRADED_QTY, tally.traded_qty);
        ctr.add(CTR_RESTED, tally.rested);
        ctr.add(CTR_REJECTED, tally.rejected);
        ctr.add(CTR_REJECTED_QTY, tally.rejected_qty);
        ctr.add(CTR_EVICTED, tally.evicted);
        ctr.add(CTR_EVICTED_QTY, tally.evicted_qty);
        ctr.add(CTR_CANCEL_HIT, tally.cancel_hit);
        ctr.add(CTR_CANCELLED_QTY, tally.cancelled_qty);
        ctr.add(CTR_MARKET_DISCARDED_QTY, tally.discarded_qty);
        const int64_t n_cancel = __shfl_sync(kFull, ctr.v, CTR_CANCEL);
        const int64_t n_hit = __shfl_sync(kFull, ctr.v, CTR_CANCEL_HIT);
        ctr.add(CTR_CANCEL_MISS, n_cancel - n_hit);
        // counters of consecutive segments may be added on different SMs: in L2
        if (l < kNumCtr) {
            int64_t* dst = &a.stats[(int64_t)b * kNumCtr + l];
            if (segmented)
                atomicAdd(reinterpret_cast<unsigned long long*>(dst), (unsigned long long)ctr.v);
            else
                *dst += ctr.v;
        }
        if (l == 0) {
            a.counts[2 * b] = n_bid;
            a.counts[2 * b + 1] = n_ask;
            a.tcounts[b] = ts.count;
            a.env[b] = es;
        }
        if (segmented) {
            // release this segment: every lane's write-back first
            __threadfence();
            __syncwarp();
            if (l == 0) st_release_gpu(&a.seg_flag[b], (epoch << 8) | (seg + 1));
        }
        __syncwarp();
    }
    if (l == 0) {
        __threadfence();
        const int done = atomicAdd(&a.queue[1], 1);
        if (done == total_warps - 1) {
            a.queue[0] = 0;
            a.queue[1] = 0;
            if (kSeg) a.queue[2] += 1;  // the next segmented launch's epoch
            __threadfence();
        }
    }
}

// Observation vector (Sec. 5.2.2) from one step's level-1 trace and the
// environment state: one CTA per environment (grid-stride over environments),
// thread k handles message k of the step.  The row (6M + 8 floats) is built in
// shared memory and written with 16-byte stores when its size and the
// output's alignment allow (M even, 16-byte aligned obs),
// so the store pipe issues a quarter of the instructions of per-feature stores.
__global__ void k_env_observe(const EnvStateDev* __restrict__ env, const Msg* __restrict__ replay,
                              int64_t stride_env, const int4* __restrict__ l1, int32_t M,
                              int32_t n_envs, int64_t passive_off, int32_t parent,
                              float* __restrict__ obs)
{
    extern __shared__ __align__(16) float srow[];
    const int64_t row = 6 * (int64_t)M + 8;
    const int64_t kSec = 1000000000;
    const int k = threadIdx.x;
    const bool vec = (row & 3) == 0 && (reinterpret_cast<uintptr_t>(obs) & 15u) == 0;
    // a best ask (1 .. INT32_MAX) plus an offset in 0 .. INT32_MAX stays below 2^32
    const bool small_off = passive_off >= 0 && passive_off <= 0x7fffffffLL;
    for (int b = blockIdx.x; b < n_envs; b += gridDim.x) {
        if (k < M) {
            const int4 r = l1[(int64_t)b * M + k];  // best bid price, its qty, best ask price, its qty
            const bool hb = r.x > 0, ha = r.z > 0;
            // Every per-message feature in 32-bit arithmetic, with the bits of
            // the binary64 definitions (the FP64 pipe of this GPU is narrow):
            // the mid of two prices is RN(bid + ask) / 2 -- the sum is exact
            // below 2^32 and halving commutes with rounding to float --, the
            // spread and the quantity imbalance fit in int32 (both operands
            // lie in 0 .. INT32_MAX), and the passive price fits in uint32
            // whenever the offset does (decided once per launch).
            float midf = -1.0f;
            if (hb && ha)
                midf = __uint2float_rn((uint32_t)r.x + (uint32_t)r.z) * 0.5f;
            else if (hb)
                midf = __int2float_rn(r.x);
            else if (ha)
                midf = __int2float_rn(r.z);
            float passive = -1.0f;
            if (ha) {
                const int64_t pp = (int64_t)r.z + passive_off;
                passive = small_off ? __uint2float_rn((uint32_t)pp) : __ll2float_rn(pp);
            }
            srow[k] = __int2float_rn(r.x);
            srow[M + k] = __int2float_rn(r.z);
            srow[2 * M + k] = midf;
            srow[3 * M + k] = passive;
            srow[4 * M + k] = hb && ha ? __int2float_rn(r.z - r.x) : -1.0f;
            srow[5 * M + 8 + k] = __int2float_rn(r.w - r.y);
            if (k == M - 1) {
                double mid = -1.0;  // the last mid in binary64 for the drift feature
                if (hb && ha)
                    mid = __dmul_rn(__dadd_rn((double)r.x, (double)r.z), 0.5);
                else if (hb)
                    mid = (double)r.x;
                else if (ha)
                    mid = (double)r.z;
                const EnvStateDev es = env[b];
                const int64_t t_init = replay[(int64_t)b * stride_env].time_ns;
                const int64_t tc = es.last_time, te = es.last_time - t_init;
                float* sc = srow + 5 * M;
                sc[0] = __ll2float_rn(tc / kSec);
                sc[1] = __ll2float_rn(tc % kSec);
                sc[2] = __ll2float_rn(te / kSec);
                sc[3] = __ll2float_rn(te % kSec);
                sc[4] = __double2float_rn(es.p_init);
                sc[5] = __double2float_rn(mid >= 0.0 ? __dsub_rn(mid, es.p_init) : 0.0);
                sc[6] = __int2float_rn(parent);
                sc[7] = __ll2float_rn(es.executed);
            }
        }
        __syncthreads();
        float* o = obs + (int64_t)b * row;
        if (vec) {
            const float4* src = reinterpret_cast<const float4*>(srow);
            float4* dst = reinterpret_cast<float4*>(o);
            for (int i = k; i < (int)(row >> 2); i += blockDim.x) dst[i] = src[i];
        } else {
            for (int i = k; i < (int)row; i += blockDim.x) o[i] = srow[i];
        }
        __syncthreads();
    }
}

// Segments per environment for a launch of n_run steps on `warps` resident
// warps: the split whose rounds of equal segments, ceil(n_envs*S/warps)/S
// whole runs, finish first; 1 when every environment has a warp to itself,
// and never segments shorter than 8 steps.
int env_segments(int n_envs, int n_run, int warps)
{
    if (warps < 1 || n_envs <= warps || n_run < 16 || n_envs > (1 << 26) || n_run > (1 << 26))
        return 1;
    int best = 1;
    double best_cost = (double)((n_envs + warps - 1) / warps);
    for (int S = 2; S <= 16 && n_run / S >= 8; ++S) {
        const double cost = (double)(((int64_t)n_envs * S + warps - 1) / warps) / S;
        if (cost < best_cost * 0.99) {
            best = S;
            best_cost = cost;
        }
    }
    return best;
}

const void* env_kernel(int K, bool trace, bool snap, bool seg)
{
#define LOB_ENV_KS(k, sg)                                                                  \
    return trace ? (snap ? reinterpret_cast<const void*>(&k_env<k, true, true, sg>)         \
                         : reinterpret_cast<const void*>(&k_env<k, true, false, sg>))       \
                 : (snap ? reinterpret_cast<const void*>(&k_env<k, false, true, sg>)        \
                         : reinterpret_cast<const void*>(&k_env<k, false, false, sg>))
#define LOB_ENV_K(k)          \
    if (seg) {                \
        LOB_ENV_KS(k, true);  \
    } else {                  \
        LOB_ENV_KS(k, false); \
    }
    switch (K) {
    case 1: LOB_ENV_K(1);
    case 2: LOB_ENV_K(2);
    case 4: LOB_ENV_K(4);
    case 8: LOB_ENV_K(8);
    default: LOB_ENV_K(16);
    }
#undef LOB_ENV_K
#undef LOB_ENV_KS
}

int env_smem(int K, int chunk)
{
    switch (K) {
    case 1: return env_warp_smem<1>(chunk);
    case 2: return env_warp_smem<2>(chunk);
    case 4: return env_warp_smem<4>(chunk);
    case 8: return env_warp_smem<8>(chunk);
    default: return env_warp_smem<16>(chunk);
    }
}

__global__ void k_env_reset(EnvStateDev* st, int32_t n, int32_t fallback)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    EnvStateDev s;
    s.submitted = 0;
    s.executed = 0;
    s.last_time = 0;
    s.id_counter = 0;
    s.last_ask = fallback;
    s.p_init = 0.0;
    st[i] = s;
}

__global__ void k_env_state(const EnvStateDev* st, int32_t n, int64_t* out, double* p_init)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const EnvStateDev s = st[i];
    if (out) {
        out[5 * (int64_t)i + 0] = s.submitted;
        out[5 * (int64_t)i + 1] = s.executed;
        out[5 * (int64_t)i + 2] = s.id_counter;
        out[5 * (int64_t)i + 3] = s.last_ask;
        out[5 * (int64_t)i + 4] = s.last_time;
    }
    if (p_init) p_init[i] = s.p_init;
}

}  // namespace

extern "C" {

int lob_env_create(lob_env** out, lob_ctx* book, const lob_env_config_t* cfg, void* stream)
{
    if (!out || !book || !cfg || cfg->n_steps < 1 || cfg->parent_qty < 0 || cfg->depth < 1 ||
        cfg->depth > 64 || cfg->msgs_per_step < 1 || cfg->msgs_per_step > 1024 ||
        cfg->p_init_fallback < 1 || cfg->passive_ticks < 0 || cfg->tick_size < 1) {
        lob_set_error("lob_env_create: invalid argument");
        return LOB_E_INVAL;
    }
    lob_env* e = new (std::nothrow) lob_env();
    if (!e) {
        lob_set_error("lob_env_create: host allocation failed");
        return LOB_E_NOMEM;
    }
    e->book = book;
    e->cfg = *cfg;
    e->chunk = (cfg->msgs_per_step + 7) / 8 * 8;
    const int K = book->K;
    e->warps = K >= 8 ? 2 : 4;
    e->smem_per_cta = env_smem(K, e->chunk) * e->warps;
    int max_optin = 0;
    cudaError_t err = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                             book->device);
    if (err == cudaSuccess && e->smem_per_cta > max_optin) {
        delete e;
        lob_set_error("lob_env_create: %d messages per step do not fit in shared memory",
                      cfg->msgs_per_step);
        return LOB_E_INVAL;
    }
    for (int v = 0; v < 8 && err == cudaSuccess; ++v) {
        const void* fn = env_kernel(K, (v & 1) != 0, (v & 2) != 0, (v & 4) != 0);
        err = lob_raise_smem_limit(fn, e->smem_per_cta);
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&e->per_sm_v[v], fn,
                                                                32 * e->warps, e->smem_per_cta);
        if (e->per_sm_v[v] < 1) e->per_sm_v[v] = 1;
    }
    if (err == cudaSuccess)
        err = cudaMalloc(&e->d_state, sizeof(EnvStateDev) * (size_t)book->cfg.n_books);
    if (err == cudaSuccess)
        err = cudaMalloc(&e->d_seg_flag, sizeof(int64_t) * (size_t)book->cfg.n_books);
    if (err == cudaSuccess)
        err = cudaMemsetAsync(e->d_seg_flag, 0, sizeof(int64_t) * (size_t)book->cfg.n_books,
                              (cudaStream_t)stream);
    if (err != cudaSuccess) {
        delete e;
        return lob_cuda_fail(err, "lob_env_create");
    }
    int rc = lob_env_reset(e, stream);
    if (rc != LOB_OK) {
        lob_env_destroy(e);
        return rc;
    }
    *out = e;
    return LOB_OK;
}

int lob_env_destroy(lob_env* e)
{
    if (!e) return LOB_OK;
    cudaError_t err = cudaSuccess;
    if (e->d_state) {
        err = cudaDeviceSynchronize();
        cudaError_t e2 = cudaFree(e->d_state);
        if (err == cudaSuccess) err = e2;
    }
    if (e->d_seg_flag) {
        cudaError_t e2 = cudaFree(e->d_seg_flag);
        if (err == cudaSuccess) err = e2;
    }
    delete e;
    return err == cudaSuccess ? LOB_OK : lob_cuda_fail(err, "lob_env_destroy");
}

int lob_env_reset(lob_env* e, void* stream)
{
    if (!e) {
        lob_set_error("lob_env_reset: null environment");
        return LOB_E_INVAL;
    }
    const int n = e->book->cfg.n_books;
    k_env_reset<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(e->d_state, n,
                                                                   e->cfg.p_init_fallback);
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? LOB_OK : lob_cuda_fail(err, "lob_env_reset");
}

int lob_env_run(lob_env* e, const lob_msg_t* d_replay, int64_t stride_env, int32_t step0,
                int32_t n_run, const uint32_t* d_draws, const float* d_actions, float* d_reward,
                int32_t* d_bid_px, int32_t* d_bid_qty, int32_t* d_ask_px, int32_t* d_ask_qty,
                int64_t* d_fills, int32_t* d_l1, void* stream)
{
    // exactly one agent source: the stand-in's draws or the policy's actions
    if (!e || !d_replay || (!d_draws == !d_actions) || !d_reward || !d_bid_px || !d_bid_qty ||
        !d_ask_px || !d_ask_qty || !d_fills || n_run < 1 || step0 < 0 ||
        step0 + n_run > e->cfg.n_steps ||
        stride_env < (int64_t)e->cfg.n_steps * e->cfg.msgs_per_step) {
        lob_set_error("lob_env_run: invalid argument (step0=%d n_run=%d)", step0, n_run);
        return LOB_E_INVAL;
    }
    if (((uintptr_t)d_replay & 15u) != 0 || ((uintptr_t)d_l1 & 15u) != 0) {
        lob_set_error("lob_env_run: messages and trace must be 16-byte aligned");
        return LOB_E_INVAL;
    }
    lob_ctx* c = e->book;
    EnvArgs a;
    a.replay = reinterpret_cast<const Msg*>(d_replay);
    a.stride_env = stride_env;
    a.msgs_per_step = e->cfg.msgs_per_step;
    a.step0 = step0;
    a.n_run = n_run;
    a.n_envs = c->cfg.n_books;
    a.draws = d_draws;
    a.state = c->d_state;
    a.counts = c->d_counts;
    a.trades = reinterpret_cast<Trade*>(c->d_trades);
    a.tcounts = c->d_tcounts;
    a.stats = c->d_stats;
    a.status = c->d_status;
    a.queue = c->d_queue;
    a.cap = c->cfg.capacity;
    a.rule = c->cfg.overflow_rule;
    a.trade_cap = c->cfg.trade_capacity;
    a.chunk = e->chunk;
    a.env = e->d_state;
    a.n_steps = e->cfg.n_steps;
    a.parent = e->cfg.parent_qty;
    a.agent_tid = e->cfg.agent_tid;
    a.depth = e->cfg.depth;
    a.p_fallback = e->cfg.p_init_fallback;
    a.pad_ = 0;
    a.lambda = e->cfg.lambda;
    a.reward = d_reward;
    a.bid_px = d_bid_px;
    a.bid_qty = d_bid_qty;
    a.ask_px = d_ask_px;
    a.ask_qty = d_ask_qty;
    a.fills = d_fills;
    a.wait_ns = kEnvWaitNs;
    a.l1 = d_l1;
    a.actions = d_actions;
    a.passive_ticks = e->cfg.passive_ticks;
    a.tick = e->cfg.tick_size;
    const int W = e->warps;
    int grid = (a.n_envs + W - 1) / W;
    const bool snap = (c->cfg.flags & LOB_FLAG_SNAPSHOT_CANCELS) != 0;
    const int variant = (d_l1 != nullptr ? 1 : 0) | (snap ? 2 : 0);
    int resident = c->num_sms * e->per_sm_v[variant];
    if (grid > resident) grid = resident;
    a.n_seg = env_segments(a.n_envs, n_run, grid * W);
    if (a.n_seg > 1) {  // the segmented instantiation's own occupancy
        resident = c->num_sms * e->per_sm_v[variant | 4];
        grid = (a.n_envs + W - 1) / W;
        if (grid > resident) grid = resident;
        a.n_seg = env_segments(a.n_envs, n_run, grid * W);
    }
    e->last_segments = a.n_seg;
    a.pad2_ = 0;
    a.seg_flag = e->d_seg_flag;
    void* args[] = {&a};
    cudaError_t err = cudaLaunchKernel(env_kernel(c->K, d_l1 != nullptr, snap, a.n_seg > 1),
                                       dim3(grid),
                                       dim3(32 * W), args,
                                       (size_t)e->smem_per_cta, (cudaStream_t)stream);
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_env_run launch");
    c->launches += 1;
    e->launches += 1;
    return LOB_OK;
}

int32_t lob_env_segments(const lob_env* e) { return e ? e->last_segments : -1; }

int lob_env_observe(lob_env* e, const lob_msg_t* d_replay, int64_t stride_env,
                    const int32_t* d_l1, float* d_obs, void* stream)
{
    if (!e || !d_replay || !d_l1 || !d_obs ||
        stride_env < (int64_t)e->cfg.n_steps * e->cfg.msgs_per_step) {
        lob_set_error("lob_env_observe: invalid argument");
        return LOB_E_INVAL;
    }
    if (((uintptr_t)d_l1 & 15u) != 0 || ((uintptr_t)d_replay & 7u) != 0) {
        lob_set_error("lob_env_observe: trace must be 16-byte and messages 8-byte aligned");
        return LOB_E_INVAL;
    }
    lob_ctx* c = e->book;
    const int M = e->cfg.msgs_per_step;
    const int threads = (M + 31) / 32 * 32;  // msgs_per_step <= 1024
    const int grid = c->cfg.n_books < c->num_sms * 16 ? c->cfg.n_books : c->num_sms * 16;
    const size_t smem = (size_t)(6 * M + 8) * sizeof(float);  // at most 24.6 KB (M <= 1024)
    k_env_observe<<<grid, threads, smem, (cudaStream_t)stream>>>(
        e->d_state, reinterpret_cast<const Msg*>(d_replay), stride_env,
        reinterpret_cast<const int4*>(d_l1), M, c->cfg.n_books,
        (int64_t)e->cfg.passive_ticks * e->cfg.tick_size, e->cfg.parent_qty, d_obs);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_env_observe launch");
    c->launches += 1;
    return LOB_OK;
}

int lob_env_get_state(lob_env* e, int64_t* d_state, double* d_p_init, void* stream)
{
    if (!e) {
        lob_set_error("lob_env_get_state: null environment");
        return LOB_E_INVAL;
    }
    const int n = e->book->cfg.n_books;
    k_env_state<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(e->d_state, n, d_state,
                                                                   d_p_init);
    cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? LOB_OK : lob_cuda_fail(err, "lob_env_get_state");
}

}  // extern "C"
