// lob_literal.cu -- the paper's own book formulation on the GPU (an ablation).
//
// Sec. 4, eqs. 1-2: each side is an UNSORTED array of N slots
// [P, Q, OID, TID, time], an empty slot holding -1 in every field.  Every
// operation is a full-array one, as Sec. 4.1 describes them:
//   add    : write the order into an empty slot (the full-side rule picks the
//            worst order by a full scan when none is empty);
//   cancel : find the OID by a full scan and subtract the quantity;
//   match  : repeatedly take Best(o) -- a full arg-max (bids) / arg-min (asks)
//            over the prices, earliest arrival among equal prices -- while the
//            aggressor has quantity left and the prices cross; after every fill
//            and every operation, every slot with Q <= 0 is reset to -1.
// With all_branches = 1 a message also pays what `vmap` makes the paper pay
// (Sec. 4.3): the limit, cancel and market branches all run, each on its own
// copy of the book, and the message's own branch is kept (a select).
//
// One warp per book; a book and two scratch copies live in shared memory;
// slot s of a side sits in lane s % 32.  Results are the same as the engine's
// (sorted sides) and the oracle's: books, trades and trade counts.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lob.h"
#include "lob_core.cuh"
#include "lob_engine.h"

namespace {

using lob::kFull;
using lob::kMaxInt;
using lob::lane_id;
using lob::Msg;
using lob::Trade;

constexpr int kLitWarps = 4;

template <int K>
struct LitGeo {
    static constexpr int NP = 32 * K;           // slots per side
    static constexpr int P = 0, Q = 4 * NP, OID = 8 * NP, TID = 12 * NP, ARR = 16 * NP,
                         T = 20 * NP;           // byte offsets inside a side
    static constexpr int SIDE = 28 * NP;
    static constexpr int BOOK = 2 * SIDE;       // side 0 bids, side 1 asks
};

template <int K>
struct LitSide {
    char* b;
    __device__ __forceinline__ int32_t* P() const { return reinterpret_cast<int32_t*>(b + LitGeo<K>::P); }
    __device__ __forceinline__ int32_t* Q() const { return reinterpret_cast<int32_t*>(b + LitGeo<K>::Q); }
    __device__ __forceinline__ int32_t* OID() const { return reinterpret_cast<int32_t*>(b + LitGeo<K>::OID); }
    __device__ __forceinline__ int32_t* TID() const { return reinterpret_cast<int32_t*>(b + LitGeo<K>::TID); }
    __device__ __forceinline__ int32_t* ARR() const { return reinterpret_cast<int32_t*>(b + LitGeo<K>::ARR); }
    __device__ __forceinline__ int64_t* T() const { return reinterpret_cast<int64_t*>(b + LitGeo<K>::T); }
};

template <int K>
__device__ __forceinline__ LitSide<K> lit_side(char* book, int x)
{
    return LitSide<K>{book + x * LitGeo<K>::SIDE};
}

struct LitArgs {
    const Msg* msgs;
    const int64_t* offsets;
    int32_t n_books, cap, trade_cap, rule, all_branches;
    Trade* trades;
    int64_t* trade_counts;
    int32_t *price, *qty, *oid, *tid;
    int64_t* time;
    int32_t* count;
};

// every field of every slot = -1
template <int K>
__device__ __forceinline__ void lit_clear(char* book)
{
    int4* d = reinterpret_cast<int4*>(book);
    for (int i = lane_id(); i < LitGeo<K>::BOOK / 16; i += 32) d[i] = make_int4(-1, -1, -1, -1);
    __syncwarp();
}

template <int K>
__device__ __forceinline__ void lit_copy(char* dst, const char* src)
{
    const int4* s = reinterpret_cast<const int4*>(src);
    int4* d = reinterpret_cast<int4*>(dst);
#pragma unroll 4
    for (int i = lane_id(); i < LitGeo<K>::BOOK / 16; i += 32) d[i] = s[i];
    __syncwarp();
}

// Best(o) (or, with worst = true, the full-side rule's worst order) by a full
// scan: each lane over its slots, then warp reductions of the price and of the
// arrival among the orders at that price.  Slot, or -1 for an empty side.
template <int K>
__device__ __forceinline__ int lit_extreme(LitSide<K> s, int cap, bool is_bid, bool worst)
{
    const int l = lane_id();
    const bool hi = is_bid != worst;  // the extreme is the highest price
    int32_t bp = 0;
    int32_t ba = 0;
    int bs = -1;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = l + 32 * j;
        if (x < cap) {
            const int32_t p = s.P()[x];
            if (p != -1) {
                const int32_t a = s.ARR()[x];
                const bool better_p = hi ? p > bp : p < bp;
                const bool better_a = worst ? a > ba : a < ba;
                if (bs < 0 || better_p || (p == bp && better_a)) {
                    bp = p;
                    ba = a;
                    bs = x;
                }
            }
        }
    }
    const int32_t wp = hi ? __reduce_max_sync(kFull, bs >= 0 ? bp : INT32_MIN)
                          : __reduce_min_sync(kFull, bs >= 0 ? bp : INT32_MAX);
    const bool at = bs >= 0 && bp == wp;
    // arrivals are >= 0: the earliest is the minimum, the latest the maximum
    const int32_t wa = worst ? __reduce_max_sync(kFull, at ? ba : -1)
                             : __reduce_min_sync(kFull, at ? ba : INT32_MAX);
    const unsigned hit = __ballot_sync(kFull, at && ba == wa);
    if (hit == 0) return -1;
    return __shfl_sync(kFull, bs, __ffs(hit) - 1);
}

// slot holding `oid` (a live order), or -1
template <int K>
__device__ __forceinline__ int lit_find(LitSide<K> s, int cap, int32_t oid)
{
    const int l = lane_id();
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = l + 32 * j;
        const unsigned hit = __ballot_sync(kFull, x < cap && s.P()[x] != -1 && s.OID()[x] == oid);
        if (hit) return 32 * j + __ffs(hit) - 1;
    }
    return -1;
}

template <int K>
__device__ __forceinline__ int lit_first_empty(LitSide<K> s, int cap)
{
    const int l = lane_id();
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int x = l + 32 * j;
        const unsigned hit = __ballot_sync(kFull, x < cap && s.P()[x] == -1);
        if (hit) return 32 * j + __ffs(hit) - 1;
    }
    return -1;
}

// every slot of both sides with Q <= 0 back to -1 (Sec. 4.1 cleanup)
template <int K>
__device__ __forceinline__ void lit_cleanup(char* book, int cap)
{
    const int l = lane_id();
#pragma unroll
    for (int x2 = 0; x2 < 2; ++x2) {
        const LitSide<K> s = lit_side<K>(book, x2);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int x = l + 32 * j;
            if (x < cap && s.P()[x] != -1 && s.Q()[x] <= 0) {
                s.P()[x] = -1;
                s.Q()[x] = -1;
                s.OID()[x] = -1;
                s.TID()[x] = -1;
                s.ARR()[x] = -1;
                s.T()[x] = -1;
            }
        }
    }
    __syncwarp();
}

struct LitLog {
    Trade* log;
    int64_t n;
    int32_t cap;
};

// matching loop against the side opposite to the aggressor; returns max(0, Q_a)
template <int K>
__device__ int32_t lit_match(char* book, int cap, const Msg& m, int32_t P_a, bool emit,
                             LitLog& lg)
{
    const bool buy = m.side == 1;
    const LitSide<K> s = lit_side<K>(book, buy ? 1 : 0);
    int32_t Q_a = m.qty;
#pragma unroll 1
    for (;;) {
        if (Q_a <= 0) break;
        const int x = lit_extreme<K>(s, cap, !buy, false);
        if (x < 0) break;
        const int32_t P_s = s.P()[x];
        if (buy ? P_a < P_s : P_a > P_s) break;
        const int32_t Q_s = s.Q()[x];
        const int32_t Q_s_new = Q_s - Q_a > 0 ? Q_s - Q_a : 0;
        const int32_t Q_a_new = Q_a - Q_s;
        if (emit) {
            if (lane_id() == 0 && lg.n < lg.cap) {
                Trade t;
                t.price = P_s;
                t.qty = Q_s - Q_s_new;
                t.oid_aggr = m.oid;
                t.oid_stand = s.OID()[x];
                t.tid_aggr = m.tid;
                t.tid_stand = s.TID()[x];
                t.time_ns = m.time_ns;
                lg.log[lg.n] = t;
            }
            lg.n += 1;
        }
        __syncwarp();
        if (lane_id() == 0) s.Q()[x] = Q_s_new;
        __syncwarp();
        Q_a = Q_a_new;
        lit_cleanup<K>(book, cap);
    }
    return Q_a > 0 ? Q_a : 0;
}

template <int K>
__device__ void lit_add(char* book, int cap, int rule, const Msg& m, int32_t Q, int32_t arrival)
{
    const bool bid = m.side == 1;
    const LitSide<K> s = lit_side<K>(book, bid ? 0 : 1);
    int x = lit_first_empty<K>(s, cap);
    if (x < 0) {
        const int w = lit_extreme<K>(s, cap, bid, true);
        const int32_t pw = s.P()[w];
        const bool better = bid ? m.price > pw : m.price < pw;
        if (rule != LOB_OVERFLOW_EVICT || !better) return;  // rejected
        x = w;                                              // evicted
    }
    __syncwarp();
    if (lane_id() == 0) {
        s.P()[x] = m.price;
        s.Q()[x] = Q;
        s.OID()[x] = m.oid;
        s.TID()[x] = m.tid;
        s.ARR()[x] = arrival;
        s.T()[x] = m.time_ns;
    }
    __syncwarp();
}

template <int K>
__device__ void lit_cancel(char* book, int cap, const Msg& m)
{
    const LitSide<K> s = lit_side<K>(book, m.side == 1 ? 0 : 1);
    const int x = lit_find<K>(s, cap, m.oid);
    if (x < 0) return;  // unknown id: no-op
    __syncwarp();
    if (lane_id() == 0) s.Q()[x] = s.Q()[x] - m.qty;
    __syncwarp();
    lit_cleanup<K>(book, cap);
}

enum { BR_NONE = 0, BR_LIMIT = 1, BR_CANCEL = 2, BR_MARKET = 3 };

// one branch of the message dispatch (Sec. 4.2) on `book`; trades and the
// arrival counter advance only when `emit`
template <int K>
__device__ void lit_branch(int br, char* book, const LitArgs& a, const Msg& m, bool emit,
                           LitLog& lg, int32_t& arrival)
{
    if (br == BR_LIMIT) {
        const int32_t rest = lit_match<K>(book, a.cap, m, m.price, emit, lg);
        if (rest > 0) {
            lit_add<K>(book, a.cap, a.rule, m, rest, arrival);
            if (emit) arrival += 1;
        }
    } else if (br == BR_CANCEL) {
        lit_cancel<K>(book, a.cap, m);
    } else if (br == BR_MARKET) {
        lit_match<K>(book, a.cap, m, m.side == -1 ? 0 : kMaxInt, emit, lg);
    }
    lit_cleanup<K>(book, a.cap);
}

template <int K>
__global__ void __launch_bounds__(32 * kLitWarps) k_literal(LitArgs a)
{
    extern __shared__ __align__(16) char smem[];
    const int l = lane_id();
    const int warp = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    char* bufs = smem + (size_t)warp * 3 * LitGeo<K>::BOOK;
    for (int b = blockIdx.x * W + warp; b < a.n_books; b += gridDim.x * W) {
        int cur = 0;
        char* book = bufs;
        lit_clear<K>(book);
        LitLog lg{a.trades + (int64_t)b * a.trade_cap, 0, a.trade_cap};
        int32_t arrival = 0;
        const int64_t lo = a.offsets[b], hi = a.offsets[b + 1];
#pragma unroll 1
        for (int64_t k = lo; k < hi; ++k) {
            const Msg m = a.msgs[k];  // the same record in every lane
            int br = BR_NONE;
            const bool valid = m.type >= 1 && m.type <= 4 && (m.side == 1 || m.side == -1) &&
                               m.qty > 0 && !(m.type == 1 && m.price <= 0);
            if (valid) br = m.type == 1 ? BR_LIMIT : m.type == 4 ? BR_MARKET : BR_CANCEL;
            if (!a.all_branches) {
                if (br != BR_NONE) lit_branch<K>(br, book, a, m, true, lg, arrival);
                continue;
            }
            // vmap-style: all three branches, each on a copy; keep the message's own
            int keep = cur;
            int spare = (cur + 1) % 3;
#pragma unroll 1
            for (int t = BR_LIMIT; t <= BR_MARKET; ++t) {
                char* dst = bufs + (size_t)spare * LitGeo<K>::BOOK;
                lit_copy<K>(dst, book);
                lit_branch<K>(t, dst, a, m, t == br, lg, arrival);
                if (t == br) {
                    keep = spare;
                    spare = 3 - cur - spare;  // the buffer that is neither kept nor current
                }
            }
            cur = keep;
            book = bufs + (size_t)cur * LitGeo<K>::BOOK;
        }
        // outputs: trade count, -1 past the stored trades, canonical book
        if (l == 0) a.trade_counts[b] = lg.n;
        const int64_t stored = lg.n < a.trade_cap ? lg.n : a.trade_cap;
        int32_t* tr = reinterpret_cast<int32_t*>(a.trades + (int64_t)b * a.trade_cap);
        for (int64_t i = stored * 8 + l; i < (int64_t)a.trade_cap * 8; i += 32) tr[i] = -1;
#pragma unroll 1
        for (int x2 = 0; x2 < 2; ++x2) {
            const LitSide<K> s = lit_side<K>(book, x2);
            const bool bid = x2 == 0;
            int live = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int x = l + 32 * j;
                live += (x < a.cap && s.P()[x] != -1) ? 1 : 0;
            }
            const int n = __reduce_add_sync(kFull, live);
            const int64_t base = ((int64_t)b * 2 + x2) * a.cap;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int x = l + 32 * j;
                if (x < a.cap && s.P()[x] != -1) {
                    const int32_t p = s.P()[x], ar = s.ARR()[x];
                    int rank = 0;  // live orders ahead of this one in priority
                    for (int y = 0; y < a.cap; ++y) {
                        const int32_t py = s.P()[y];
                        if (py == -1) continue;
                        const bool ahead = bid ? py > p : py < p;
                        rank += (ahead || (py == p && s.ARR()[y] < ar)) ? 1 : 0;
                    }
                    a.price[base + rank] = p;
                    a.qty[base + rank] = s.Q()[x];
                    a.oid[base + rank] = s.OID()[x];
                    a.tid[base + rank] = s.TID()[x];
                    a.time[base + rank] = s.T()[x];
                }
            }
            for (int i = n + l; i < a.cap; i += 32) {
                a.price[base + i] = -1;
                a.qty[base + i] = -1;
                a.oid[base + i] = -1;
                a.tid[base + i] = -1;
                a.time[base + i] = -1;
            }
            if (l == 0) a.count[b * 2 + x2] = n;
        }
        __syncwarp();
    }
}

const void* literal_kernel(int K)
{
    switch (K) {
    case 1: return reinterpret_cast<const void*>(&k_literal<1>);
    case 2: return reinterpret_cast<const void*>(&k_literal<2>);
    default: return reinterpret_cast<const void*>(&k_literal<4>);
    }
}

int literal_book_bytes(int K) { return 56 * 32 * K; }

}  // namespace

int lob_literal_process(const lob_msg_t* d_msgs, const int64_t* d_offsets, int32_t n_books,
                        int32_t capacity, int32_t trade_capacity, int32_t overflow_rule,
                        int32_t all_branches, lob_trade_t* d_trades, int64_t* d_trade_counts,
                        int32_t* d_price, int32_t* d_qty, int32_t* d_oid, int32_t* d_tid,
                        int64_t* d_time, int32_t* d_count, void* stream)
{
    if (n_books < 0 || capacity < 1 || capacity > 128 || trade_capacity < 0 ||
        (overflow_rule != LOB_OVERFLOW_EVICT && overflow_rule != LOB_OVERFLOW_REJECT) ||
        (all_branches != 0 && all_branches != 1) || !d_offsets || !d_trade_counts ||
        !d_price || !d_qty || !d_oid || !d_tid || !d_time || !d_count ||
        (trade_capacity > 0 && !d_trades)) {
        lob_set_error("lob_literal_process: invalid argument");
        return LOB_E_INVAL;
    }
    if (((uintptr_t)d_msgs & 15u) != 0) {
        lob_set_error("lob_literal_process: messages must be 16-byte aligned");
        return LOB_E_INVAL;
    }
    if (n_books == 0) return LOB_OK;
    const int K = capacity <= 32 ? 1 : capacity <= 64 ? 2 : 4;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem = 3 * literal_book_bytes(K) * kLitWarps;
    if (err == cudaSuccess) err = lob_raise_smem_limit(literal_kernel(K), smem);
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, literal_kernel(K),
                                                            32 * kLitWarps, smem);
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_literal_process setup");
    LitArgs a;
    a.msgs = reinterpret_cast<const Msg*>(d_msgs);
    a.offsets = d_offsets;
    a.n_books = n_books;
    a.cap = capacity;
    a.trade_cap = trade_capacity;
    a.rule = overflow_rule;
    a.all_branches = all_branches;
    a.trades = reinterpret_cast<Trade*>(d_trades);
    a.trade_counts = d_trade_counts;
    a.price = d_price;
    a.qty = d_qty;
    a.oid = d_oid;
    a.tid = d_tid;
    a.time = d_time;
    a.count = d_count;
    int grid = (n_books + kLitWarps - 1) / kLitWarps;
    const int resident = sms * (per_sm > 0 ? per_sm : 1);
    if (grid > resident) grid = resident;
    void* args[] = {&a};
    err = cudaLaunchKernel(literal_kernel(K), dim3(grid), dim3(32 * kLitWarps), args, (size_t)smem,
                           (cudaStream_t)stream);
    return err == cudaSuccess ? LOB_OK : lob_cuda_fail(err, "lob_literal_process launch");
}
