// lob_core.cuh -- warp-level order-book operations for sm_103a.
//
// One warp owns one book.  Each side of the book (Sec. 4, eqs. 1-2: arrays of
// N orders [P, Q, OID, TID, time]) is held in shared memory SORTED BY PRIORITY:
// slot 0 is Best(o) of eq. best_price (highest bid / lowest ask) and orders of
// equal price sit in arrival order.  The paper keeps its arrays unsorted because
// vmap turns every branch into a select and re-sorting would run on every message
// (Sec. 4.3); a warp takes only the branch a message needs, so here the sorted
// form is cheaper: the best order is slot 0, an insert or delete moves the tail
// by one slot, and a multi-level match is one prefix scan instead of a loop.
//
// Blocked layout: capacity rounded up to C = 32*K slots, lane l holds slots
// [l*K, l*K + K) of every field, so a lane reads its slots with 128-bit shared
// loads and the warp never needs a barrier to move data between lanes (a
// one-slot shift passes a single value per field through a shuffle).
//
// Field arrays of one side, in bytes from the side's base:
//   px[C] int32 | qty[C] int32 | oid[C] int32 | tid[C] int32 | tm[C] int64
// A book is [bid side][ask side] = 48*C bytes, the same layout in HBM and in
// shared memory, so staging a book is one contiguous bulk copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace lob {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kMaxK = 16;        // capacity <= 512
constexpr int kNumCtr = 20;      // per-book counters (order fixed by the C ABI)
constexpr int32_t kMaxInt = 2147483647;
constexpr int32_t kSnapshotOidMax = -9000;  // orders from a level snapshot: OID <= -9000

enum : int {
    CTR_MSGS = 0, CTR_LIMIT, CTR_CANCEL, CTR_MARKET, CTR_NOOP, CTR_INVALID, CTR_TRADES,
    CTR_TRADED_QTY, CTR_RESTED, CTR_REJECTED, CTR_REJECTED_QTY, CTR_EVICTED, CTR_EVICTED_QTY,
    CTR_CANCEL_HIT, CTR_CANCELLED_QTY, CTR_CANCEL_MISS, CTR_MARKET_DISCARDED_QTY, CTR_LIMIT_QTY,
    CTR_MARKET_QTY, CTR_TRADES_DROPPED
};

struct Msg {  // 32-byte message record {type, side, price, qty, oid, tid, time_ns}
    int32_t type, side, price, qty, oid, tid;
    int64_t time_ns;
};
struct Trade {  // 32-byte trade record
    int32_t price, qty, oid_aggr, oid_stand, tid_aggr, tid_stand;
    int64_t time_ns;
};
static_assert(sizeof(Msg) == 32 && sizeof(Trade) == 32, "record sizes");

template <int K>
struct Geo {
    static constexpr int C = 32 * K;
    static constexpr int PX = 0, QTY = 4 * C, OID = 8 * C, TID = 12 * C, TM = 16 * C;
    static constexpr int SIDE_BYTES = 24 * C;
    static constexpr int BOOK_BYTES = 2 * SIDE_BYTES;
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_barrier_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy shared accesses before later
// async-proxy (bulk copy) accesses
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared, completion signalled on `bar` (bytes % 16 == 0,
// both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after `limit_ns` of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// ------------------------------------------------------- lane-vector helpers

template <int K>
__device__ __forceinline__ void ld_vec(const int32_t* arr, int32_t (&v)[K])
{
    const int l = lane_id();
    if constexpr (K == 1) {
        v[0] = arr[l];
    } else if constexpr (K == 2) {
        int2 t = reinterpret_cast<const int2*>(arr)[l];
        v[0] = t.x; v[1] = t.y;
    } else {
        const int4* q = reinterpret_cast<const int4*>(arr) + l * (K / 4);
#pragma unroll
        for (int i = 0; i < K / 4; ++i) {
            int4 t = q[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    }
}

template <int K>
__device__ __forceinline__ void st_vec(int32_t* arr, const int32_t (&v)[K])
{
    const int l = lane_id();
    if constexpr (K == 1) {
        arr[l] = v[0];
    } else if constexpr (K == 2) {
        reinterpret_cast<int2*>(arr)[l] = make_int2(v[0], v[1]);
    } else {
        int4* q = reinterpret_cast<int4*>(arr) + l * (K / 4);
#pragma unroll
        for (int i = 0; i < K / 4; ++i)
            q[i] = make_int4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
    }
}

template <int K>
__device__ __forceinline__ void ld_vec(const int64_t* arr, int64_t (&v)[K])
{
    const int l = lane_id();
    if constexpr (K == 1) {
        v[0] = arr[l];
    } else {
        const longlong2* q = reinterpret_cast<const longlong2*>(arr) + l * (K / 2);
#pragma unroll
        for (int i = 0; i < K / 2; ++i) {
            longlong2 t = q[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    }
}

template <int K>
__device__ __forceinline__ void st_vec(int64_t* arr, const int64_t (&v)[K])
{
    const int l = lane_id();
    if constexpr (K == 1) {
        arr[l] = v[0];
    } else {
        longlong2* q = reinterpret_cast<longlong2*>(arr) + l * (K / 2);
#pragma unroll
        for (int i = 0; i < K / 2; ++i) q[i] = make_longlong2(v[2 * i], v[2 * i + 1]);
    }
}

// min(a + b, INT32_MAX) for a, b in [0, INT32_MAX] (no wrap: a + b < 2^32)
__device__ __forceinline__ uint32_t sat_add(uint32_t a, uint32_t b)
{
    return min(a + b, (uint32_t)kMaxInt);
}

// ---------------------------------------------------------------- primitives

// Insert `val` into a lane's slots, the place given per slot: in[j + 1] says
// whether slot l*K+j keeps its order (it ranks before the new one), in[0] the
// same of the slot to its left (slot -1 keeps).  A slot that does not keep
// takes `val` when its left neighbour keeps and the neighbour's order when it
// does not; `prev` is the left neighbour's last slot, fetched beforehand
// (__shfl_up_sync(kFull, v[K - 1], 1)) so that the shuffle can be issued
// before the place is known.  Slots at or past the new count hold no order and
// every reader bounds its slots by the count, so they take whatever the shift
// brings.
template <int K, typename T>
__device__ __forceinline__ void shift_in_pred(T (&v)[K], const bool (&in)[K + 1], T val, T prev)
{
    T nv[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        T left = (j == 0) ? prev : v[j - 1];
        nv[j] = in[j + 1] ? v[j] : (in[j] ? val : left);
    }
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = nv[j];
}

// shift_out with the right neighbour's first slot already fetched
// (next = __shfl_down_sync(kFull, v[0], 1)); slots past the new count take
// whatever the shift brings, as in shift_in_pred.
template <int K, typename T>
__device__ __forceinline__ void shift_out_next(T (&v)[K], int p, T next)
{
    const int l = lane_id();
    T nv[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int s = l * K + j;
        T right = (j == K - 1) ? next : v[j + 1];
        nv[j] = (s >= p) ? right : v[j];
    }
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = nv[j];
}

// Shift slots [p+1, n) left by one (slot p disappears).
template <int K, typename T>
__device__ __forceinline__ void shift_out(T (&v)[K], int p, int n)
{
    const int l = lane_id();
    T next = __shfl_down_sync(kFull, v[0], 1);
    T nv[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int s = l * K + j;
        T right = (j == K - 1) ? next : v[j + 1];
        nv[j] = (s >= p && s < n - 1) ? right : v[j];
    }
#pragma unroll
    for (int j = 0; j < K; ++j) v[j] = nv[j];
}

// New slot s takes old slot s + m (0 < m): the first m slots disappear.
// Slots at or past n - m are left undefined (they are beyond the new count).
template <int K, typename T>
__device__ __forceinline__ void drop_front(T (&v)[K], int m)
{
    const int l = lane_id();
    const int a = m / K, b = m % K;  // K is a power of two
    T r[K];
#pragma unroll
    for (int j = 0; j < K; ++j) r[j] = v[j];
    // rotate lane-locally by b (warp-uniform): r[j] = v[(j + b) % K], by
    // selects on the bits of b
#pragma unroll
    for (int bit = 1; bit < K; bit <<= 1) {
        const bool on = (b & bit) != 0;
        T t[K];
#pragma unroll
        for (int j = 0; j < K; ++j) t[j] = on ? r[(j + bit) % K] : r[j];
#pragma unroll
        for (int j = 0; j < K; ++j) r[j] = t[j];
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int src = (l + a + ((j + b) >= K ? 1 : 0)) & 31;
        v[j] = __shfl_sync(kFull, r[j], src);
    }
}

// Does this lane own a slot in [lo, hi)?
template <int K>
__device__ __forceinline__ bool lane_touches(int lo, int hi)
{
    const int s0 = lane_id() * K;
    return s0 + K > lo && s0 < hi;
}

// ------------------------------------------------------------ side vectors

// The K slots a lane owns on one side, every field.
template <int K>
struct SideVec {
    int32_t px[K], q[K], oid[K], tid[K];
    int32_t tlo[K], thi[K];  // time stamp, low and high 32 bits
};

// v[r] for a run-time r in [0, K) by a tree of selects on the bits of r (a
// plain indexed read, or a chain of equality selects that the compiler folds
// back into one, would force the lane's registers into local memory).
template <int K, typename T>
__device__ __forceinline__ T pick(const T (&v)[K], int r)
{
    T t[K];
#pragma unroll
    for (int j = 0; j < K; ++j) t[j] = v[j];
#pragma unroll
    for (int w = 1; w < K; w <<= 1) {
        const bool hi = (r & w) != 0;
#pragma unroll
        for (int j = 0; j + w < K; j += 2 * w) t[j] = hi ? t[j + w] : t[j];
    }
    return t[0];
}

// Value of slot s (warp-uniform s) broadcast to every lane.
template <int K, typename T>
__device__ __forceinline__ T slot_value(const T (&v)[K], int s)
{
    return __shfl_sync(kFull, pick<K>(v, s % K), s / K);
}

// Side X: 0 = bids (priority = higher price first), 1 = asks (lower first).
// A resting price `a` ranks at least as well as an incoming price `p`; on the
// opposite side of an aggressor this is exactly the crossing test (Sec. 4.1:
// a buy crosses while P_a >= P_s, a sell while P_a <= P_s).
template <int X>
__device__ __forceinline__ bool at_least(int32_t a, int32_t p)
{
    return X == 0 ? a >= p : a <= p;
}

// ------------------------------------------------------- storage policies
//
// RegBook: both sides stay in registers for a whole message stream (each lane
// keeps its K slots of every field, blocked: lane l holds ranks l*K..l*K+K-1);
// used for K <= 4.  SmemBook: the staged image in shared memory, a lane's
// slots moved through registers on demand (acquire/release); the base of
// GroupBook (K = 8, 16), whose own operations work group by group in place.
// The book operations below are written once against these policies.

template <int K>
struct RegBook {
    SideVec<K> s[2];
    int32_t bp[2];  // each side's best price (slot 0), warp-uniform; stale while the side is empty
    static constexpr bool kInRegisters = true;
    static constexpr bool kGrouped = false;
    // the side itself is modified in place; `tmp` is unused
    template <int X> __device__ __forceinline__ SideVec<K>& acquire(SideVec<K>&) { return s[X]; }
    template <int X> __device__ __forceinline__ void release(const SideVec<K>&, bool) {}
    template <int X> __device__ __forceinline__ int32_t best_px(int) const { return bp[X]; }
    // re-read side X's best price after an operation that may have changed slot 0
    template <int X> __device__ __forceinline__ void refresh_best()
    {
        bp[X] = __shfl_sync(kFull, s[X].px[0], 0);
    }
    template <int X> __device__ __forceinline__ void set_best(int32_t p) { bp[X] = p; }
    // qty of slot p held by lane L at position jj
    template <int X> __device__ __forceinline__ void set_qty(int L, int jj, int p, int32_t q)
    {
        const int l = lane_id();
#pragma unroll
        for (int j = 0; j < K; ++j)
            if (l == L && j == jj) s[X].q[j] = q;
    }
    // fill from / spill to a staged book image in shared memory
    __device__ __forceinline__ void from_image(const char* img)
    {
        load_side(img, s[0]);
        load_side(img + Geo<K>::SIDE_BYTES, s[1]);
        refresh_best<0>();
        refresh_best<1>();
    }
    __device__ __forceinline__ void to_image(char* img) const
    {
        store_side(img, s[0]);
        store_side(img + Geo<K>::SIDE_BYTES, s[1]);
    }
    static __device__ __forceinline__ void load_side(const char* b, SideVec<K>& v)
    {
        ld_vec<K>(reinterpret_cast<const int32_t*>(b + Geo<K>::PX), v.px);
        ld_vec<K>(reinterpret_cast<const int32_t*>(b + Geo<K>::QTY), v.q);
        ld_vec<K>(reinterpret_cast<const int32_t*>(b + Geo<K>::OID), v.oid);
        ld_vec<K>(reinterpret_cast<const int32_t*>(b + Geo<K>::TID), v.tid);
        int64_t t[K];
        ld_vec<K>(reinterpret_cast<const int64_t*>(b + Geo<K>::TM), t);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            v.tlo[j] = (int32_t)(uint32_t)(uint64_t)t[j];
            v.thi[j] = (int32_t)(uint32_t)((uint64_t)t[j] >> 32);
        }
    }
    static __device__ __forceinline__ void store_side(char* b, const SideVec<K>& v)
    {
        st_vec<K>(reinterpret_cast<int32_t*>(b + Geo<K>::PX), v.px);
        st_vec<K>(reinterpret_cast<int32_t*>(b + Geo<K>::QTY), v.q);
        st_vec<K>(reinterpret_cast<int32_t*>(b + Geo<K>::OID), v.oid);
        st_vec<K>(reinterpret_cast<int32_t*>(b + Geo<K>::TID), v.tid);
        int64_t t[K];
#pragma unroll
        for (int j = 0; j < K; ++j)
            t[j] = (int64_t)(((uint64_t)(uint32_t)v.thi[j] << 32) | (uint32_t)v.tlo[j]);
        st_vec<K>(reinterpret_cast<int64_t*>(b + Geo<K>::TM), t);
    }
};

template <int K>
struct SmemBook {
    char* base;  // staged book image in shared memory
    static constexpr bool kInRegisters = false;
    static constexpr bool kGrouped = false;
    template <int X> __device__ __forceinline__ char* side() const { return base + X * Geo<K>::SIDE_BYTES; }
    // the lane's slots are moved through `tmp` and written back on release
    template <int X> __device__ __forceinline__ SideVec<K>& acquire(SideVec<K>& tmp)
    {
        RegBook<K>::load_side(side<X>(), tmp);
        return tmp;
    }
    template <int X> __device__ __forceinline__ void release(const SideVec<K>& v, bool touch)
    {
        if (touch) RegBook<K>::store_side(side<X>(), v);
    }
    template <int X> __device__ __forceinline__ int32_t best_px(int) const
    {
        return reinterpret_cast<const int32_t*>(side<X>() + Geo<K>::PX)[0];
    }
    template <int X> __device__ __forceinline__ void set_qty(int L, int, int p, int32_t q)
    {
        if (lane_id() == L) reinterpret_cast<int32_t*>(side<X>() + Geo<K>::QTY)[p] = q;
    }
    template <int X> __device__ __forceinline__ void refresh_best() {}
    template <int X> __device__ __forceinline__ void set_best(int32_t) {}
    __device__ __forceinline__ void from_image(const char*) {}
    __device__ __forceinline__ void to_image(char*) const {}
};

// GroupBook: the book stays in shared memory, each field a plain array of
// the side's C = 32*K slots.  A side of n orders is stored worst first: the
// order of priority rank r sits at index n-1-r, so the top of the book --
// where adds, cancels and fills mostly happen -- is the end of the array, an
// operation moves only the orders above the one it touches, and consumed
// orders leave by shortening the side.  Adds and removals move whole orders
// by one index, lane-parallel (64 orders per pass, consecutive words); the
// cancel search reads every group of 128 slots at once (lane l: indices
// g*128 + 4*l + (0..3), 128-bit accesses without bank conflicts); a match
// walks those groups from the top in a loop that is not unrolled.  Code that
// reads a grouped side in priority order maps rank r to index n-1-r
// (storage_index<K>).
template <int K>
struct GroupBook : SmemBook<K> {
    static constexpr bool kGrouped = true;
    // the best order sits at index n-1 (see the grouped operations)
    template <int X> __device__ __forceinline__ int32_t best_px(int n) const
    {
        return reinterpret_cast<const int32_t*>(this->template side<X>() + Geo<K>::PX)[n > 0 ? n - 1 : 0];
    }
};

// Books whose two sides fit in registers cheaply (K <= 4: 2 sides x 6 words x
// 4 per lane) stay there for a whole stream; larger capacities work in shared
// memory, group by group.
template <int K>
struct BookPolicy {
    using type = typename std::conditional<(K <= 4), RegBook<K>, GroupBook<K>>::type;
};

// Whether the policy of K stores a side worst first (index = n-1-rank).
template <int K>
__host__ __device__ constexpr bool reversed_layout() { return !(K <= 4); }

// Storage index of priority rank r in a side of n orders.
template <int K>
__host__ __device__ __forceinline__ int storage_index(int r, int n)
{
    return reversed_layout<K>() ? n - 1 - r : r;
}

__device__ __forceinline__ int64_t warp_sum64(int64_t x)
{
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(kFull, x, d);
    return x;
}

// Per-lane counter slot: lane i accumulates counter i of the current book.
struct Counters {
    int64_t v;
    int lane;
    __device__ __forceinline__ void add(int idx, int64_t x) { v += (lane == idx) ? x : 0; }
};

// Book-dependent counters of the current work item, kept warp-uniform (every
// lane holds the same value) and folded into Counters once per item.  Trade
// counts are not tallied: they follow from the trade-log position.
struct Tally {
    int32_t rested = 0, rejected = 0, evicted = 0, cancel_hit = 0;
    int64_t rejected_qty = 0, evicted_qty = 0, cancelled_qty = 0, traded_qty = 0,
            discarded_qty = 0;
};

// ------------------------------------------------------------ book operations

struct TradeSink;
template <int K, int X>
__device__ __forceinline__ void g_add_order(char*, int&, int, int, int32_t, int32_t, int32_t, int32_t, int32_t,
                            int32_t, Tally&);
template <int K, int X>
__device__ __forceinline__ void g_cancel_order(char*, int&, int32_t, int32_t, int32_t, bool,
                                               Tally&);
template <int K, int Y, class Obs>
__device__ __forceinline__ int32_t g_match_order(char*, int&, int32_t, int32_t, int32_t, int32_t, int32_t, int32_t,
                                 TradeSink&, Tally&, Obs&);

// Add the remaining quantity Q as one new order (Sec. 4.1 item 1, Sec. 4.2
// item 1) at the back of its price level on side X, with the full-side rule:
// when the side already holds `cap` orders the worst one is evicted if the new
// order's price is strictly better than its price, else the rest is rejected
// (rule 1: always rejected).
template <int K, int X, class Book>
__device__ __forceinline__ void add_order(Book& bk, int& n, int cap, int rule, int32_t P, int32_t Q,
                                          int32_t oid, int32_t tid, int32_t tlo, int32_t thi,
                                          Tally& ctr)
{
    if constexpr (Book::kGrouped) {
        g_add_order<K, X>(bk.template side<X>(), n, cap, rule, P, Q, oid, tid, tlo, thi, ctr);
        return;
    }
    static_assert(Book::kInRegisters || Book::kGrouped, "add_order: register or grouped books");
    const int l = lane_id();
    SideVec<K> tmp;
    SideVec<K>& v = bk.template acquire<X>(tmp);
    // the shift's cross-lane values (the left neighbour's last slot) do not
    // depend on where the new order goes: fetch them first, so that their
    // latency overlaps the full-side test; the price also decides the place
    const int32_t pv_px = __shfl_up_sync(kFull, v.px[K - 1], 1);
    const int32_t pv_q = __shfl_up_sync(kFull, v.q[K - 1], 1);
    const int32_t pv_oid = __shfl_up_sync(kFull, v.oid[K - 1], 1);
    const int32_t pv_tid = __shfl_up_sync(kFull, v.tid[K - 1], 1);
    const int32_t pv_tlo = __shfl_up_sync(kFull, v.tlo[K - 1], 1);
    const int32_t pv_thi = __shfl_up_sync(kFull, v.thi[K - 1], 1);
    const bool full = n >= cap;
    if (full) {
        // the worst order (slot cap-1) is evicted if its price is strictly
        // worse than P, else the new order is rejected
        const int32_t worst = slot_value<K>(v.px, cap - 1);
        if (rule != 0 || at_least<X>(worst, P)) {
            ctr.rejected += 1;
            ctr.rejected_qty += Q;
            return;
        }
        ctr.evicted += 1;
        ctr.evicted_qty += slot_value<K>(v.q, cap - 1);
    }
    // The side is in priority order, so the resting orders priced at least as
    // well as P are a prefix of the slots, and the new order goes where that
    // prefix ends.  Each slot decides from its own price and its left
    // neighbour's: it keeps its order inside the prefix, takes the new order
    // right after it, and takes its left neighbour's order further on (slots
    // past the new count take whatever the shift brings).  Slot -1 counts as
    // inside the prefix.
    bool in[K + 1];
    in[0] = l == 0 || (l * K - 1 < n && at_least<X>(pv_px, P));
#pragma unroll
    for (int j = 0; j < K; ++j) in[j + 1] = l * K + j < n && at_least<X>(v.px[j], P);
    const bool top = n == 0 || !at_least<X>(bk.template best_px<X>(n), P);
    const int n_after = full ? cap : n + 1;
    shift_in_pred<K>(v.px, in, P, pv_px);
    shift_in_pred<K>(v.q, in, Q, pv_q);
    shift_in_pred<K>(v.oid, in, oid, pv_oid);
    shift_in_pred<K>(v.tid, in, tid, pv_tid);
    shift_in_pred<K>(v.tlo, in, tlo, pv_tlo);
    shift_in_pred<K>(v.thi, in, thi, pv_thi);
    if (top) bk.template set_best<X>(P);
    n = n_after;
    ctr.rested += 1;
}

// Cancellation (Sec. 4.1 item 2): locate OID on side X and remove Q from it;
// the order leaves the book when its quantity drops to 0 or below.
template <int K, int X, class Book>
__device__ __forceinline__ void cancel_order(Book& bk, int& n, int32_t oid, int32_t Q, int32_t P,
                                             bool snap, Tally& ctr)
{
    if constexpr (Book::kGrouped) {
        g_cancel_order<K, X>(bk.template side<X>(), n, oid, Q, P, snap, ctr);
        return;
    }
    const int l = lane_id();
    SideVec<K> tmp;
    SideVec<K>& v = bk.template acquire<X>(tmp);
    int jj = -1;
#pragma unroll
    for (int j = K - 1; j >= 0; --j)
        if (l * K + j < n && v.oid[j] == oid) jj = j;
    unsigned hit = __ballot_sync(kFull, jj >= 0);
    if (hit == 0 && snap) {
        // snapshot rule: the snapshot order resting at the cancel's price
#pragma unroll
        for (int j = K - 1; j >= 0; --j)
            if (l * K + j < n && v.px[j] == P && v.oid[j] <= kSnapshotOidMax) jj = j;
        hit = __ballot_sync(kFull, jj >= 0);
    }
    if (hit == 0) return;  // not live on this side: no-op (counted at the end)
    ctr.cancel_hit += 1;
    const int L = __popc(~hit & (hit - 1u));  // lowest set bit: trailing zeros
    // each lane picks its own candidate, so both values leave lane L at once
    const int32_t q_mine = pick<K>(v.q, jj < 0 ? 0 : jj);
    const int j_hit = __shfl_sync(kFull, jj, L);
    const int32_t q_old = __shfl_sync(kFull, q_mine, L);
    const int p = L * K + j_hit;
    const int32_t q_new = q_old - Q;
    if (q_new > 0) {
        bk.template set_qty<X>(L, j_hit, p, q_new);
        ctr.cancelled_qty += Q;
        return;
    }
    ctr.cancelled_qty += q_old;
    // the removal's cross-lane values (fetched only now: partial cancels and
    // misses, 29 % of the message mix, never need them)
    const int32_t nx_px = __shfl_down_sync(kFull, v.px[0], 1);
    const int32_t nx_q = __shfl_down_sync(kFull, v.q[0], 1);
    const int32_t nx_oid = __shfl_down_sync(kFull, v.oid[0], 1);
    const int32_t nx_tid = __shfl_down_sync(kFull, v.tid[0], 1);
    const int32_t nx_tlo = __shfl_down_sync(kFull, v.tlo[0], 1);
    const int32_t nx_thi = __shfl_down_sync(kFull, v.thi[0], 1);
    shift_out_next<K>(v.px, p, nx_px);
    shift_out_next<K>(v.q, p, nx_q);
    shift_out_next<K>(v.oid, p, nx_oid);
    shift_out_next<K>(v.tid, p, nx_tid);
    shift_out_next<K>(v.tlo, p, nx_tlo);
    shift_out_next<K>(v.thi, p, nx_thi);
    bk.template release<X>(v, lane_touches<K>(p, n - 1));
    bk.template refresh_best<X>();
    n -= 1;
}

// Fill observers: NoObs (plain processing) and VwapObs (execution
// environment: per-lane partial sums of Q*P over all fills and of Q, Q*P over
// the agent's fills -- reduced once per step, Sec. 5.2.4).
struct NoObs {
    template <int K>
    __device__ __forceinline__ void on_fills(const int32_t (&)[K], const int32_t (&)[K],
                                             const int32_t (&)[K], int32_t)
    {
    }
};

struct VwapObs {
    int64_t spq = 0, aq = 0, apq = 0;  // this lane's partial sums
    int32_t agent_tid = 0;
    template <int K>
    __device__ __forceinline__ void on_fills(const int32_t (&fill)[K], const int32_t (&px)[K],
                                             const int32_t (&tid)[K], int32_t tid_a)
    {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int64_t qp = (int64_t)fill[j] * px[j];
            const bool agent = tid_a == agent_tid || tid[j] == agent_tid;
            spq += qp;
            aq += agent ? fill[j] : 0;
            apq += agent ? qp : 0;
        }
    }
};

// Where trades of the current book go and how many are already there.
struct TradeSink {
    Trade* log;      // this book's segment of the trade log
    int64_t count;   // trades executed so far in this log (uniform)
    int32_t cap;     // stored capacity
};

// Matching (Sec. 4.1 item 3 and its while loop) of an aggressor of quantity Q
// with limit price P (0 / max_int for market orders, Sec. 4.2 item 3) against
// opposite side Y.  The method's loop repeatedly takes the best standing
// order, reduces it to max(0, Q_s - Q_a), reduces the aggressor by Q_s and
// logs the trade [P_s, filled quantity, OID_a, OID_s, time_a]; it therefore
// visits the crossing prefix of the priority-sorted side in order: the order at
// slot s therefore receives min(Q_s, max(0, Q - (quantity of slots before s))),
// which one saturating warp prefix scan gives for all slots at once.
// Returns the aggressor's remaining quantity max(0, Q_a).
template <int K, int Y, class Book, class Obs>
__device__ __forceinline__ int32_t match_order(Book& bk, int& n, int32_t P, int32_t Q, int32_t oid_a,
                                               int32_t tid_a, int32_t tlo, int32_t thi,
                                               TradeSink& ts, Tally& ctr, Obs& obs)
{
    if constexpr (Book::kGrouped)
        return g_match_order<K, Y, Obs>(bk.template side<Y>(), n, P, Q, oid_a, tid_a, tlo, thi,
                                        ts, ctr, obs);
    const int l = lane_id();
    SideVec<K> tmp;
    SideVec<K>& v = bk.template acquire<Y>(tmp);

    // Every caller has checked that the side is not empty and that its best
    // order crosses.  When that order alone fills the aggressor (Q <= its
    // quantity) the loop runs once: one trade, written by lane 0, which holds
    // the order, and no scan.
    const int32_t q0 = __shfl_sync(kFull, v.q[0], 0);
    if (Q <= q0) {
        if (l == 0 && ts.count < (int64_t)ts.cap) {
            int4* dst = reinterpret_cast<int4*>(ts.log + ts.count);
            dst[0] = make_int4(v.px[0], Q, oid_a, v.oid[0]);
            dst[1] = make_int4(tid_a, v.tid[0], tlo, thi);
        }
        int32_t fill[K];
#pragma unroll
        for (int j = 0; j < K; ++j) fill[j] = (l == 0 && j == 0) ? Q : 0;
        obs.template on_fills<K>(fill, v.px, v.tid, tid_a);
        ts.count += 1;
        ctr.traded_qty += Q;
        if (Q == q0) {
            drop_front<K>(v.px, 1);
            drop_front<K>(v.q, 1);
            drop_front<K>(v.oid, 1);
            drop_front<K>(v.tid, 1);
            drop_front<K>(v.tlo, 1);
            drop_front<K>(v.thi, 1);
            bk.template release<Y>(v, lane_touches<K>(0, n - 1));
            bk.template refresh_best<Y>();
            n -= 1;
        } else {
            bk.template set_qty<Y>(0, 0, 0, q0 - Q);
        }
        return 0;
    }

    // crossing quantity per slot and lane-local inclusive prefix
    uint32_t cq[K], loc[K];
    uint32_t acc = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const bool c = l * K + j < n && at_least<Y>(v.px[j], P);
        cq[j] = c ? (uint32_t)v.q[j] : 0u;
        acc = sat_add(acc, cq[j]);
        loc[j] = acc;
    }
    // warp inclusive scan of the lane totals (saturating at INT32_MAX: exact
    // wherever the running total is below Q <= INT32_MAX, which is all that
    // the fills depend on)
    uint32_t incl = acc;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, d);
        if (l >= d) incl = sat_add(incl, t);
    }
    uint32_t excl = __shfl_up_sync(kFull, incl, 1);
    if (l == 0) excl = 0;
    const uint32_t total = __shfl_sync(kFull, incl, 31);

    int32_t fill[K];
    unsigned nfull = 0, nfill = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const uint32_t before = sat_add(excl, j == 0 ? 0u : loc[j - 1]);
        const uint32_t room = before < (uint32_t)Q ? (uint32_t)Q - before : 0u;
        fill[j] = (int32_t)min(cq[j], room);
        nfull += (cq[j] != 0u && (uint32_t)fill[j] == cq[j]) ? 1u : 0u;
        nfill += fill[j] > 0 ? 1u : 0u;
    }
    // fully filled orders (they leave the book), trades of this message
    const int m = (int)__reduce_add_sync(kFull, nfull);
    const int nf = (int)__reduce_add_sync(kFull, nfill);
    const int32_t F = (int32_t)min(total, (uint32_t)Q);  // quantity traded

    // trades: the filled slots are the prefix [0, nf), trade k -> slot k
    // slots [0, n_store) still fit in the log
    const int n_store = (int)max(min((int64_t)nf, (int64_t)ts.cap - ts.count), (int64_t)0);
    Trade* const log_at = ts.log + ts.count;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        if (l * K + j < n_store) {
            int4* dst = reinterpret_cast<int4*>(log_at + l * K + j);
            dst[0] = make_int4(v.px[j], fill[j], oid_a, v.oid[j]);
            dst[1] = make_int4(tid_a, v.tid[j], tlo, thi);
        }
    }
    ts.count += nf;
    ctr.traded_qty += F;
    obs.template on_fills<K>(fill, v.px, v.tid, tid_a);

    // standing quantities after the fills (Q_s' per slot), then drop the m
    // fully filled orders at the front (Q <= 0 cleanup)
#pragma unroll
    for (int j = 0; j < K; ++j) v.q[j] -= fill[j];
    if (m > 0) {
        // one general drop for every m: per-m variants execute fewer
        // instructions but enlarge the message loop enough to cost more in
        // instruction fetch than they save
        drop_front<K>(v.px, m);
        drop_front<K>(v.q, m);
        drop_front<K>(v.oid, m);
        drop_front<K>(v.tid, m);
        drop_front<K>(v.tlo, m);
        drop_front<K>(v.thi, m);
        bk.template release<Y>(v, lane_touches<K>(0, n - m));
        bk.template refresh_best<Y>();
        n -= m;
    } else if (nf > 0) {
        // only slot 0 was partly filled
        bk.template set_qty<Y>(0, 0, 0, v.q[0]);
    }
    return Q - F;
}


// ------------------------------------------------------- grouped operations
//
// GroupBook operations.  Where they work on groups, lane l's group g holds
// slots g*128 + 4*l + (0..3).

__device__ __forceinline__ int4 lds4(const int32_t* a) { return *reinterpret_cast<const int4*>(a); }
__device__ __forceinline__ void sts4(int32_t* a, int4 v) { *reinterpret_cast<int4*>(a) = v; }

struct Q64 { int64_t x, y, z, w; };
__device__ __forceinline__ Q64 lds8(const int64_t* a)
{
    const longlong2 u = reinterpret_cast<const longlong2*>(a)[0];
    const longlong2 v = reinterpret_cast<const longlong2*>(a)[1];
    return Q64{u.x, u.y, v.x, v.y};
}
__device__ __forceinline__ void sts8(int64_t* a, Q64 q)
{
    reinterpret_cast<longlong2*>(a)[0] = make_longlong2(q.x, q.y);
    reinterpret_cast<longlong2*>(a)[1] = make_longlong2(q.z, q.w);
}

template <int K>
struct GSide {
    char* b;
    __device__ __forceinline__ int32_t* px() const { return reinterpret_cast<int32_t*>(b + Geo<K>::PX); }
    __device__ __forceinline__ int32_t* qty() const { return reinterpret_cast<int32_t*>(b + Geo<K>::QTY); }
    __device__ __forceinline__ int32_t* oid() const { return reinterpret_cast<int32_t*>(b + Geo<K>::OID); }
    __device__ __forceinline__ int32_t* tid() const { return reinterpret_cast<int32_t*>(b + Geo<K>::TID); }
    __device__ __forceinline__ int64_t* tm() const { return reinterpret_cast<int64_t*>(b + Geo<K>::TM); }
};

// Whole orders (every field) move by one index, lane-parallel: index i of a
// side is element i of each field array, so a pass moves 64 consecutive
// orders (two per lane) with plain 4- and 8-byte accesses (consecutive words:
// no bank conflicts), loading all of them before the warp synchronises and
// stores.

// Orders at [lo, hi) move up one (to lo+1 .. hi).  Passes run from the top
// down, so no pass stores into a range that a later pass still loads.
template <int K>
__device__ __forceinline__ void g_move_up(GSide<K> sd, int lo, int hi)
{
    const int l = lane_id();
#pragma unroll 1
    for (int top = hi; top > lo; top -= 64) {
        const int i0 = top - 1 - l, i1 = top - 33 - l;
        const bool a0 = i0 >= lo, a1 = i1 >= lo;
        const int k0 = a0 ? i0 : lo, k1 = a1 ? i1 : lo;
        const int32_t p0 = sd.px()[k0], q0 = sd.qty()[k0], o0 = sd.oid()[k0], t0 = sd.tid()[k0];
        const int32_t p1 = sd.px()[k1], q1 = sd.qty()[k1], o1 = sd.oid()[k1], t1 = sd.tid()[k1];
        const int64_t e0 = sd.tm()[k0], e1 = sd.tm()[k1];
        __syncwarp();
        if (a0) {
            sd.px()[i0 + 1] = p0;
            sd.qty()[i0 + 1] = q0;
            sd.oid()[i0 + 1] = o0;
            sd.tid()[i0 + 1] = t0;
            sd.tm()[i0 + 1] = e0;
        }
        if (a1) {
            sd.px()[i1 + 1] = p1;
            sd.qty()[i1 + 1] = q1;
            sd.oid()[i1 + 1] = o1;
            sd.tid()[i1 + 1] = t1;
            sd.tm()[i1 + 1] = e1;
        }
    }
}

// Orders at [lo, hi) move down one (to lo-1 .. hi-2); passes run from the
// bottom up.
template <int K>
__device__ __forceinline__ void g_move_down(GSide<K> sd, int lo, int hi)
{
    const int l = lane_id();
#pragma unroll 1
    for (int bot = lo; bot < hi; bot += 64) {
        const int i0 = bot + l, i1 = bot + 32 + l;
        const bool a0 = i0 < hi, a1 = i1 < hi;
        const int k0 = a0 ? i0 : lo, k1 = a1 ? i1 : lo;
        const int32_t p0 = sd.px()[k0], q0 = sd.qty()[k0], o0 = sd.oid()[k0], t0 = sd.tid()[k0];
        const int32_t p1 = sd.px()[k1], q1 = sd.qty()[k1], o1 = sd.oid()[k1], t1 = sd.tid()[k1];
        const int64_t e0 = sd.tm()[k0], e1 = sd.tm()[k1];
        __syncwarp();
        if (a0) {
            sd.px()[i0 - 1] = p0;
            sd.qty()[i0 - 1] = q0;
            sd.oid()[i0 - 1] = o0;
            sd.tid()[i0 - 1] = t0;
            sd.tm()[i0 - 1] = e0;
        }
        if (a1) {
            sd.px()[i1 - 1] = p1;
            sd.qty()[i1 - 1] = q1;
            sd.oid()[i1 - 1] = o1;
            sd.tid()[i1 - 1] = t1;
            sd.tm()[i1 - 1] = e1;
        }
    }
}

template <int K, int X>
__device__ __forceinline__ void g_add_order(char* side, int& n, int cap, int rule, int32_t P,
                                         int32_t Q, int32_t oid, int32_t tid, int32_t tlo,
                                         int32_t thi, Tally& ctr)
{
    const GSide<K> sd{side};
    const int l = lane_id();
    if (n >= cap) {
        // full side: the worst order (index 0) is evicted if its price is
        // strictly worse than P (every other order moves down one), else the
        // new order is rejected
        const int32_t worst = sd.px()[0];
        if (rule != 0 || at_least<X>(worst, P)) {
            ctr.rejected += 1;
            ctr.rejected_qty += Q;
            return;
        }
        ctr.evicted += 1;
        ctr.evicted_qty += sd.qty()[0];
        g_move_down<K>(sd, 1, n);
        n -= 1;
        __syncwarp();
    }
    // The orders at least as good as P are the top p indices n-p .. n-1 (the
    // side is sorted); they move up one and the new order takes index n-p.
    // The 64 best orders (ranks l and l+32, indices n-1-l and n-33-l) are
    // loaded whole; when rank 63 is not among them (p < 64), each of those
    // orders moves from its own comparison, and the last of them (or lane 0
    // for p = 0) places the new order: no count, no second load.
    const int i0 = n - 1 - l, i1 = n - 33 - l;
    const int k0 = i0 >= 0 ? i0 : 0, k1 = i1 >= 0 ? i1 : 0;
    const int32_t p0 = sd.px()[k0], p1 = sd.px()[k1];
    const int32_t q0 = sd.qty()[k0], o0 = sd.oid()[k0], t0 = sd.tid()[k0];
    const int32_t q1 = sd.qty()[k1], o1 = sd.oid()[k1], t1 = sd.tid()[k1];
    const int64_t e0 = sd.tm()[k0], e1 = sd.tm()[k1];
    const bool ok0 = i0 >= 0 && at_least<X>(p0, P);
    const bool ok1 = i1 >= 0 && at_least<X>(p1, P);
    const unsigned b0 = __ballot_sync(kFull, ok0), b1 = __ballot_sync(kFull, ok1);
    const int64_t tnew = (int64_t)(((uint64_t)(uint32_t)thi << 32) | (uint32_t)tlo);
    if ((b1 >> 31) == 0u) {
        // does the next rank (l+1, l+33) stay in place?
        const bool nx0 = l < 31 ? ((b0 >> (l + 1)) & 1u) != 0 : (b1 & 1u) != 0;
        const bool nx1 = l < 31 ? ((b1 >> (l + 1)) & 1u) != 0 : false;
        __syncwarp();
        if (ok0) {
            sd.px()[i0 + 1] = p0;
            sd.qty()[i0 + 1] = q0;
            sd.oid()[i0 + 1] = o0;
            sd.tid()[i0 + 1] = t0;
            sd.tm()[i0 + 1] = e0;
        }
        if (ok1) {
            sd.px()[i1 + 1] = p1;
            sd.qty()[i1 + 1] = q1;
            sd.oid()[i1 + 1] = o1;
            sd.tid()[i1 + 1] = t1;
            sd.tm()[i1 + 1] = e1;
        }
        const bool place0 = ok0 && !nx0, place1 = ok1 && !nx1;
        if (place0 || place1 || (l == 0 && b0 == 0u)) {
            const int at = place1 ? i1 : (place0 ? i0 : n);
            sd.px()[at] = P;
            sd.qty()[at] = Q;
            sd.oid()[at] = oid;
            sd.tid()[at] = tid;
            sd.tm()[at] = tnew;
        }
    } else {
        // a deep insert: count the orders at least as good below the window
        int p = 64;
#pragma unroll 1
        for (int top = n - 64; top > 0; top -= 64) {
            const int j0 = top - 1 - l, j1 = top - 33 - l;
            const bool c0 = j0 >= 0 && at_least<X>(sd.px()[j0 >= 0 ? j0 : 0], P);
            const bool c1 = j1 >= 0 && at_least<X>(sd.px()[j1 >= 0 ? j1 : 0], P);
            const int c = __popc(__ballot_sync(kFull, c0)) + __popc(__ballot_sync(kFull, c1));
            p += c;
            if (c < 64) break;
        }
        __syncwarp();
        const int lo = n - p;
        g_move_up<K>(sd, lo, n);
        if (l == 0) {
            sd.px()[lo] = P;
            sd.qty()[lo] = Q;
            sd.oid()[lo] = oid;
            sd.tid()[lo] = tid;
            sd.tm()[lo] = tnew;
        }
    }
    n += 1;
    ctr.rested += 1;
}

// Snapshot rule (Sec. 5.1.1): index of the earliest (highest-priority, so
// highest-index) order with OID <= -9000 resting at price P, or -1.  Out of
// line: it runs only on a cancel miss.
template <int K>
__device__ __noinline__ int g_find_snapshot(const char* side, int n, int32_t P)
{
    const GSide<K> sd{const_cast<char*>(side)};
    const int l = lane_id();
#pragma unroll 1
    for (int g = (n - 1) >> 7; g >= 0; --g) {
        const int4 v = lds4(sd.oid() + g * 128 + 4 * l);
        const int4 w = lds4(sd.px() + g * 128 + 4 * l);
        const int s = g * 128 + 4 * l;
        int jj = (s < n && w.x == P && v.x <= kSnapshotOidMax) ? 0 : -1;
        jj = (s + 1 < n && w.y == P && v.y <= kSnapshotOidMax) ? 1 : jj;
        jj = (s + 2 < n && w.z == P && v.z <= kSnapshotOidMax) ? 2 : jj;
        jj = (s + 3 < n && w.w == P && v.w <= kSnapshotOidMax) ? 3 : jj;
        const unsigned hit = __ballot_sync(kFull, jj >= 0);
        if (hit) {
            const int L = 31 - __clz(hit);
            return g * 128 + 4 * L + __shfl_sync(kFull, jj, L);
        }
    }
    return -1;
}

template <int K, int X>
__device__ __forceinline__ void g_cancel_order(char* side, int& n, int32_t oid, int32_t Q,
                                               int32_t P, bool snap, Tally& ctr)
{
    const GSide<K> sd{side};
    const int l = lane_id();
    // every group at once (independent loads) and one warp maximum: live ids
    // are unique on a side, so at most one slot matches
    int mine = -1;
#pragma unroll
    for (int g = 0; g < K / 4; ++g) {
        const int s = g * 128 + 4 * l;
        const int4 v = lds4(sd.oid() + s);
        int mg = (s < n && v.x == oid) ? s : -1;
        mg = (s + 1 < n && v.y == oid) ? s + 1 : mg;
        mg = (s + 2 < n && v.z == oid) ? s + 2 : mg;
        mg = (s + 3 < n && v.w == oid) ? s + 3 : mg;
        mine = max(mine, mg);
    }
    int p = __reduce_max_sync(kFull, mine);
    if (p < 0 && snap) p = g_find_snapshot<K>(side, n, P);
    if (p < 0) return;
    ctr.cancel_hit += 1;
    const int32_t q_old = sd.qty()[p];
    const int32_t q_new = q_old - Q;
    if (q_new > 0) {
        __syncwarp();
        if (l == 0) sd.qty()[p] = q_new;
        ctr.cancelled_qty += Q;
        return;
    }
    ctr.cancelled_qty += q_old;
    __syncwarp();
    g_move_down<K>(sd, p + 1, n);  // the orders above move down one
    n -= 1;
}

template <int K, int Y, class Obs>
__device__ __forceinline__ int32_t g_match_order(char* side, int& n, int32_t P, int32_t Q,
                                              int32_t oid_a, int32_t tid_a, int32_t tlo,
                                              int32_t thi, TradeSink& ts, Tally& ctr, Obs& obs)
{
    // The side is stored worst first, so priority order is descending index:
    // groups from the top, lanes from 31 down, and w, z, y, x inside a lane.
    const GSide<K> sd{side};
    const int l = lane_id();
    // Every caller has checked that the side is not empty and that its best
    // order crosses.  When that order alone fills the aggressor (Q <= its
    // quantity) the loop runs once: one trade, written by lane 0, no scan.
    {
        const int top = n - 1;
        const int32_t q_top = sd.qty()[top];
        if (Q <= q_top) {
            const int32_t px_top = sd.px()[top], tid_top = sd.tid()[top];
            if (l == 0) {
                if (ts.count < (int64_t)ts.cap) {
                    int4* dst = reinterpret_cast<int4*>(ts.log + ts.count);
                    dst[0] = make_int4(px_top, Q, oid_a, sd.oid()[top]);
                    dst[1] = make_int4(tid_a, tid_top, tlo, thi);
                }
                if (Q < q_top) sd.qty()[top] = q_top - Q;
            }
            const int32_t fill[4] = {l == 0 ? Q : 0, 0, 0, 0};
            const int32_t pa[4] = {px_top, px_top, px_top, px_top};
            const int32_t ta[4] = {tid_top, tid_top, tid_top, tid_top};
            obs.template on_fills<4>(fill, pa, ta, tid_a);
            ts.count += 1;
            ctr.traded_qty += Q;
            if (Q == q_top) n -= 1;  // used up: it was the top of the side
            __syncwarp();
            return 0;
        }
    }
    const int n0 = n;
    const int g_top = (n0 - 1) >> 7;
    uint32_t consumed = 0;  // quantity filled so far (warp-uniform)
    int m = 0, nf = 0;
    const int64_t count0 = ts.count;
#pragma unroll 1
    for (int g = g_top; g >= 0; --g) {
        const int s = g * 128 + 4 * l;
        const int4 vp = lds4(sd.px() + s);
        const int4 vq = lds4(sd.qty() + s);
        const int32_t pa[4] = {vp.w, vp.z, vp.y, vp.x};
        const int32_t qa[4] = {vq.w, vq.z, vq.y, vq.x};
        uint32_t cq[4], loc[4];
        uint32_t acc = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool c = s + 3 - j < n0 && at_least<Y>(pa[j], P);
            cq[j] = c ? (uint32_t)qa[j] : 0u;
            acc = sat_add(acc, cq[j]);
            loc[j] = acc;
        }
        const uint32_t Qg = (uint32_t)Q - consumed;
        // the group's first lane in priority order; when the fills end inside
        // it (it covers Qg, or the lane after it does not cross) no scan is needed
        const int lt = g == g_top ? ((n0 - 1) & 127) >> 2 : 31;
        const unsigned first_crosses = __ballot_sync(kFull, cq[0] != 0u);
        const uint32_t acct = __shfl_sync(kFull, acc, lt);
        const bool local = acct >= Qg || lt == 0 || !((first_crosses >> (lt - 1)) & 1u);
        uint32_t excl, total;
        if (local) {
            excl = l == lt ? 0u : Qg;
            total = acct;
        } else {
            // saturating scan over the lanes above: incl(l) = sum of lanes >= l
            uint32_t incl = acc;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_down_sync(kFull, incl, d);
                if (l + d < 32) incl = sat_add(incl, t);
            }
            excl = __shfl_down_sync(kFull, incl, 1);
            if (l == 31) excl = 0;
            total = __shfl_sync(kFull, incl, 0);
        }
        int32_t fill[4];
        unsigned nfull = 0, nfill = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t before = sat_add(excl, j == 0 ? 0u : loc[j - 1]);
            const uint32_t room = before < Qg ? Qg - before : 0u;
            fill[j] = (int32_t)min(cq[j], room);
            nfull += (cq[j] != 0u && (uint32_t)fill[j] == cq[j]) ? 1u : 0u;
            nfill += fill[j] > 0 ? 1u : 0u;
        }
        int gm, gnf;
        if (local) {
            const unsigned packed = __shfl_sync(kFull, nfull | (nfill << 16), lt);
            gm = (int)(packed & 0xffffu);
            gnf = (int)(packed >> 16);
        } else {
            gm = (int)__reduce_add_sync(kFull, nfull);
            gnf = (int)__reduce_add_sync(kFull, nfill);
        }
        const uint32_t gF = min(total, Qg);
        if (gnf > 0) {
            const int4 vo = lds4(sd.oid() + s);
            const int4 vt = lds4(sd.tid() + s);
            const int32_t oa[4] = {vo.w, vo.z, vo.y, vo.x};
            const int32_t ta[4] = {vt.w, vt.z, vt.y, vt.x};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                // trade k is the order of priority rank k
                const int64_t idx = count0 + (n0 - 1 - (s + 3 - j));
                if (fill[j] > 0 && idx < ts.cap) {
                    int4* dst = reinterpret_cast<int4*>(ts.log + idx);
                    dst[0] = make_int4(pa[j], fill[j], oid_a, oa[j]);
                    dst[1] = make_int4(tid_a, ta[j], tlo, thi);
                }
            }
            obs.template on_fills<4>(fill, pa, ta, tid_a);
            if (fill[0] | fill[1] | fill[2] | fill[3])
                sts4(sd.qty() + s,
                     make_int4(qa[3] - fill[3], qa[2] - fill[2], qa[1] - fill[1], qa[0] - fill[0]));
        }
        consumed += gF;
        m += gm;
        nf += gnf;
        if (gm < min(128, n0 - g * 128) || consumed >= (uint32_t)Q) break;
    }
    __syncwarp();
    ts.count += nf;
    ctr.traded_qty += consumed;
    n -= m;  // the m fully filled orders were the top of the side
    return Q - (int32_t)consumed;
}

// Dispatch codes written by the chunk pre-pass (Sec. 4.2: eight type x side
// cases, padding and malformed messages folded into one "skip" code).
enum : int32_t {
    OP_SKIP = 0, OP_LIMIT_BID, OP_LIMIT_ASK, OP_CANCEL_BID, OP_CANCEL_ASK, OP_MARKET_BID,
    OP_MARKET_ASK
};

// Classify one message (the part of Sec. 4.2 that does not depend on the book):
// returns the dispatch code; malformed messages (type outside 0..4, side not
// +-1, Q <= 0, limit price <= 0) and type-0 padding map to OP_SKIP.
__device__ __forceinline__ int32_t classify(int32_t T, int32_t S, int32_t P, int32_t Q, int& counter)
{
    if (T == 0) {
        counter = CTR_NOOP;
        return OP_SKIP;
    }
    if (T < 0 || T > 4 || (S != 1 && S != -1) || Q <= 0 || (T == 1 && P <= 0)) {
        counter = CTR_INVALID;
        return OP_SKIP;
    }
    const int bid = S == 1 ? 0 : 1;
    if (T == 1) {
        counter = CTR_LIMIT;
        return OP_LIMIT_BID + bid;
    }
    if (T == 4) {
        counter = CTR_MARKET;
        return OP_MARKET_BID + bid;
    }
    counter = CTR_CANCEL;
    return OP_CANCEL_BID + bid;
}

// Apply one classified message to the book (Sec. 4.2 dispatch; n_bid / n_ask
// are the warp-uniform side counts).  Every branch is warp-uniform.  The full
// form takes one branch per case (fewest branches on the common path); the
// compact form shares the matching code of limit and market orders (half the
// inlined code, for kernels whose instruction cache is the constraint).
template <int K, bool kCompact, class Book, class Obs>
__device__ __forceinline__ void apply_message(Book& bk, int& n_bid, int& n_ask, int cap, int rule,
                                              int32_t op, int32_t P, int32_t Q, int32_t oid,
                                              int32_t tid, int32_t tlo, int32_t thi, TradeSink& ts,
                                              Tally& ctr, Obs& obs, bool snap)
{
    if constexpr (!kCompact) {
        // both best prices before the dispatch (a limit's crossing test needs
        // one): register-resident books keep them in uniform registers,
        // updated only when an operation changes a side's first slot, so
        // they cost nothing here; grouped books read them from shared memory,
        // the load overlapping the dispatch
        const int32_t best_bid = bk.template best_px<0>(n_bid);
        const int32_t best_ask = bk.template best_px<1>(n_ask);
        if (op <= OP_LIMIT_ASK) {
            if (op == OP_LIMIT_BID) {  // buy limit: match the asks, then rest the remainder as a bid
                int32_t rest = Q;
                if (n_ask > 0 && at_least<1>(best_ask, P))
                    rest = match_order<K, 1>(bk, n_ask, P, rest, oid, tid, tlo, thi, ts, ctr, obs);
                if (rest > 0) add_order<K, 0>(bk, n_bid, cap, rule, P, rest, oid, tid, tlo, thi, ctr);
            } else if (op == OP_LIMIT_ASK) {
                int32_t rest = Q;
                if (n_bid > 0 && at_least<0>(best_bid, P))
                    rest = match_order<K, 0>(bk, n_bid, P, rest, oid, tid, tlo, thi, ts, ctr, obs);
                if (rest > 0) add_order<K, 1>(bk, n_ask, cap, rule, P, rest, oid, tid, tlo, thi, ctr);
            }
        } else if (op <= OP_CANCEL_ASK) {  // cancel and delete are treated identically
            if (op == OP_CANCEL_BID)
                cancel_order<K, 0>(bk, n_bid, oid, Q, P, snap, ctr);
            else
                cancel_order<K, 1>(bk, n_ask, oid, Q, P, snap, ctr);
        } else {  // market: price max_int (buy) / 0 (sell), remainder dropped
            int32_t rest = Q;
            if (op == OP_MARKET_BID) {
                if (n_ask > 0) rest = match_order<K, 1>(bk, n_ask, kMaxInt, rest, oid, tid, tlo, thi, ts, ctr, obs);
            } else {
                if (n_bid > 0) rest = match_order<K, 0>(bk, n_bid, 0, rest, oid, tid, tlo, thi, ts, ctr, obs);
            }
            ctr.discarded_qty += rest;
        }
    } else {
        if (op == OP_CANCEL_BID || op == OP_CANCEL_ASK) {  // cancel and delete: identical
            if (op == OP_CANCEL_BID)
                cancel_order<K, 0>(bk, n_bid, oid, Q, P, snap, ctr);
            else
                cancel_order<K, 1>(bk, n_ask, oid, Q, P, snap, ctr);
        } else if (op != OP_SKIP) {
            // limit: match, then rest the remainder; market: match at price max_int
            // (buy) / 0 (sell), then drop the remainder
            const bool market = op >= OP_MARKET_BID;
            int32_t rest = Q;
            if (op == OP_LIMIT_BID || op == OP_MARKET_BID) {
                const int32_t Pm = market ? kMaxInt : P;
                if (n_ask > 0 && at_least<1>(bk.template best_px<1>(n_ask), Pm))
                    rest = match_order<K, 1>(bk, n_ask, Pm, rest, oid, tid, tlo, thi, ts, ctr, obs);
                if (!market && rest > 0)
                    add_order<K, 0>(bk, n_bid, cap, rule, P, rest, oid, tid, tlo, thi, ctr);
            } else {
                const int32_t Pm = market ? 0 : P;
                if (n_bid > 0 && at_least<0>(bk.template best_px<0>(n_bid), Pm))
                    rest = match_order<K, 0>(bk, n_bid, Pm, rest, oid, tid, tlo, thi, ts, ctr, obs);
                if (!market && rest > 0)
                    add_order<K, 1>(bk, n_ask, cap, rule, P, rest, oid, tid, tlo, thi, ctr);
            }
            if (market) ctr.discarded_qty += rest;
        }
    }
    if constexpr (!Book::kInRegisters) __syncwarp();
}

// Invariant check after a message, compiled only into checked builds
// (-DLOB_CHECKS; otherwise it is empty): side counts within 0..cap, both sides
// in priority order, resting quantities > 0, the book not crossed.  A failure
// sets LOB_STATUS_CHECK in the status word; nothing traps.
template <int K, class Book>
__device__ __forceinline__ void check_book(Book& bk, int n_bid, int n_ask, int cap,
                                           int32_t* status)
{
#ifdef LOB_CHECKS
    const int l = lane_id();
    bool bad = n_bid < 0 || n_bid > cap || n_ask < 0 || n_ask > cap;
    if constexpr (Book::kInRegisters) {
        SideVec<K> tmp;
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            const SideVec<K>& v = x == 0 ? bk.template acquire<0>(tmp) : bk.template acquire<1>(tmp);
            const int n = x == 0 ? n_bid : n_ask;
            const int32_t nxt = __shfl_down_sync(kFull, v.px[0], 1);
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const int s = l * K + j;
                const int32_t right = j + 1 < K ? v.px[j + 1] : nxt;
                if (s < n && v.q[j] <= 0) bad = true;
                if (s + 1 < n && (x == 0 ? v.px[j] < right : v.px[j] > right)) bad = true;
            }
        }
    } else {
#pragma unroll 1
        for (int x = 0; x < 2; ++x) {  // stored worst first: index i+1 ranks ahead of i
            const GSide<K> sd{bk.template side<0>() + x * Geo<K>::SIDE_BYTES};
            const int n = x == 0 ? n_bid : n_ask;
            for (int i = l; i < n && i < 32 * K; i += 32) {
                if (sd.qty()[i] <= 0) bad = true;
                if (i + 1 < n && (x == 0 ? sd.px()[i] > sd.px()[i + 1] : sd.px()[i] < sd.px()[i + 1]))
                    bad = true;
            }
        }
    }
    if (n_bid > 0 && n_ask > 0 && n_bid <= cap && n_ask <= cap &&
        bk.template best_px<0>(n_bid) >= bk.template best_px<1>(n_ask))
        bad = true;
    if (__any_sync(kFull, bad) && l == 0) atomicOr(status, LOB_STATUS_CHECK);
#else
    (void)bk;
    (void)n_bid;
    (void)n_ask;
    (void)cap;
    (void)status;
#endif
}

// Top `depth` price levels of one side whose lane vectors are px/q with n
// live slots (Sec. 5.1.1 ten-level state): level k = k-th distinct price in
// priority order with the summed quantity of its orders (saturating at
// INT32_MAX); missing levels are (-1, 0).  The quantity of a level is the
// difference of two prefix sums: its first order stores the exclusive prefix
// (and the price), its last order the inclusive prefix, so no atomics are
// needed.  lq/lp: per-warp shared scratch of `depth` entries (lq holds two
// 64-bit words per level).
template <int K>
__device__ __forceinline__ void emit_levels(const int32_t (&px)[K], const int32_t (&q)[K], int n,
                                            int depth, unsigned long long* lq, int32_t* lp,
                                            int32_t* out_px, int32_t* out_q)
{
    const int l = lane_id();
    const int32_t prev = __shfl_up_sync(kFull, px[K - 1], 1);
    bool start[K];
    int before = 0, levels = 0;
    long long lane_sum = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int s = l * K + j;
        const int32_t left = j == 0 ? prev : px[j - 1];
        start[j] = s < n && (s == 0 || px[j] != left);
        const unsigned bal = __ballot_sync(kFull, start[j]);
        before += __popc(bal & ((1u << l) - 1u));
        levels += __popc(bal);
        lane_sum += s < n ? q[j] : 0;
    }
    // warp exclusive prefix of the lane sums (64-bit: exact for any side)
    long long incl = lane_sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const long long t = __shfl_up_sync(kFull, incl, d);
        if (l >= d) incl += t;
    }
    long long pre = incl - lane_sum;
    // a slot ends its level when the next slot starts one (or it is the last)
    const bool next_lane_start = __shfl_down_sync(kFull, start[0] ? 1 : 0, 1) != 0;
    int lvl = before - 1;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int s = l * K + j;
        lvl += start[j] ? 1 : 0;
        const bool nxt = j + 1 < K ? start[j + 1] : next_lane_start;
        const bool end = s < n && (s == n - 1 || nxt);
        if (start[j] && lvl < depth) {
            lq[2 * lvl] = (unsigned long long)pre;
            lp[lvl] = px[j];
        }
        pre += s < n ? q[j] : 0;
        if (end && lvl < depth) lq[2 * lvl + 1] = (unsigned long long)pre;
    }
    __syncwarp();
    for (int k = l; k < depth; k += 32) {
        const bool have = k < levels;
        out_px[k] = have ? lp[k] : -1;
        out_q[k] = have ? (int32_t)min((long long)(lq[2 * k + 1] - lq[2 * k]), (long long)kMaxInt)
                        : 0;
    }
    __syncwarp();
}

// Prices and quantities of side X in the lane-blocked priority order the
// level code reads (lane l: ranks l*K .. l*K+K-1); ranks >= n are undefined.
template <int K, int X, class Book>
__device__ __forceinline__ void priority_px_q(Book& bk, int n, int32_t (&px)[K], int32_t (&q)[K])
{
    if constexpr (Book::kInRegisters) {
        SideVec<K> tmp;
        const SideVec<K>& v = bk.template acquire<X>(tmp);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            px[j] = v.px[j];
            q[j] = v.q[j];
        }
    } else {
        const GSide<K> sd{bk.template side<X>()};
        const int l = lane_id();
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int r = l * K + j;
            const int i = r < n ? storage_index<K>(r, n) : 0;
            px[j] = sd.px()[i];
            q[j] = sd.qty()[i];
        }
    }
}

// Level-1 state of both sides (Sec. 5.2.1): the best price and the summed
// quantity of the orders at it (the level-0 prefix of each sorted side),
// (-1, 0) for an empty side, quantity saturating at INT32_MAX.  The result is
// valid in lane 0 (the lane that stores it).
template <int K>
__device__ __forceinline__ void level1_scan(const char* side, int n, int32_t& p, int64_t& q)
{
    // grouped side, stored worst first: the best level is the top of the array
    const int32_t* px = reinterpret_cast<const int32_t*>(side + Geo<K>::PX);
    const int32_t* qt = reinterpret_cast<const int32_t*>(side + Geo<K>::QTY);
    p = px[n - 1];
    q = 0;
#pragma unroll 1
    for (int i = n - 1; i >= 0 && px[i] == p; --i) q += qt[i];
}

template <int K, class Book>
__device__ __forceinline__ int4 level1_book(Book& bk, int n_bid, int n_ask)
{
    int32_t pb = -1, pa = -1;
    int64_t qb = 0, qa = 0;
    if constexpr (!Book::kInRegisters) {
        // shared memory: lane 0 walks the best level of each side (a few orders)
        if (lane_id() == 0) {
            if (n_bid > 0) level1_scan<K>(bk.template side<0>(), n_bid, pb, qb);
            if (n_ask > 0) level1_scan<K>(bk.template side<1>(), n_ask, pa, qa);
        }
    } else {
        // registers: every lane sums its slots at the best price, saturated at
        // INT32_MAX (a saturated part means a saturated total), then the 16-bit
        // halves of the parts are summed over the warp: both sums are exact in
        // 32 bits (below 2^21), and the total saturates at INT32_MAX
        const int l = lane_id();
        SideVec<K> tmp;
        SideVec<K>& vb = bk.template acquire<0>(tmp);
        SideVec<K>& va = bk.template acquire<1>(tmp);
        const int32_t bb = bk.template best_px<0>(n_bid);
        const int32_t ba = bk.template best_px<1>(n_ask);
        uint32_t sb = 0, sa = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            sb = sat_add(sb, (l * K + j < n_bid && vb.px[j] == bb) ? (uint32_t)vb.q[j] : 0u);
            sa = sat_add(sa, (l * K + j < n_ask && va.px[j] == ba) ? (uint32_t)va.q[j] : 0u);
        }
        const uint32_t b_lo = __reduce_add_sync(kFull, sb & 0xffffu);
        const uint32_t b_hi = __reduce_add_sync(kFull, sb >> 16);
        const uint32_t a_lo = __reduce_add_sync(kFull, sa & 0xffffu);
        const uint32_t a_hi = __reduce_add_sync(kFull, sa >> 16);
        // hi >= 2^15 means a total of at least 2^31; below, (hi << 16) + lo < 2^32
        const uint32_t tb = b_hi >= 0x8000u ? (uint32_t)kMaxInt : min((b_hi << 16) + b_lo, (uint32_t)kMaxInt);
        const uint32_t ta = a_hi >= 0x8000u ? (uint32_t)kMaxInt : min((a_hi << 16) + a_lo, (uint32_t)kMaxInt);
        pb = n_bid > 0 ? bb : -1;
        pa = n_ask > 0 ? ba : -1;
        return make_int4(pb, (int32_t)tb, pa, (int32_t)ta);
    }
    return make_int4(pb, (int32_t)min(qb, (int64_t)kMaxInt), pa,
                     (int32_t)min(qa, (int64_t)kMaxInt));
}

}  // namespace lob
