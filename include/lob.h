/*
 * lob.h -- C ABI of the batched limit-order-book engine (liblob.so).
 *
 * Thousands of independent limit order books, each with a fixed capacity of N
 * orders per side, process their own message streams in parallel on one GPU
 * (the batching over books of Sec. 4.3).  Within a book messages are applied
 * strictly in order with price-time priority (Sec. 4.1-4.2).
 *
 * Conventions for every entry point below:
 *   - Pointers named d_* are DEVICE pointers owned by the caller (for example
 *     torch CUDA tensors); the library never frees them and keeps no reference
 *     to them after the call returns (the serving executor keeps the buffers
 *     of its descriptor until lob_serve_destroy).  The library owns only what
 *     lob_create / lob_env_create / lob_serve_create allocate (book state,
 *     trade log, counters, work queue; the executor's upload buffers, pinned
 *     ring and events).
 *   - Every call is asynchronous and ordered on `stream` (a cudaStream_t; NULL
 *     means the legacy default stream).  Results are ready once the stream has
 *     reached the call.  The serving executor issues on the two streams of its
 *     descriptor and waits on the host only where its calls say so.
 *   - Return value: LOB_OK (0) or a negative LOB_E_* code; nothing is thrown
 *     across the ABI.  Argument errors are detected on the host before any
 *     launch and leave the context untouched.  lob_last_error() describes the
 *     most recent failure of the calling thread.
 *   - Anomalies found on the device (a book id out of range, a message chunk
 *     that did not arrive in time) never fault: the affected work item is
 *     skipped and a LOB_STATUS_* bit is OR-ed into the context's status word
 *     (lob_get_stats).
 *   - A context must be used from one stream at a time and with the device it
 *     was created on current.
 */
#ifndef LOB_H
#define LOB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- records */

/* Message m = [T, S, Q, P, OID, TID, Ts, Tns] (Sec. 4.2, eq. message), with the
 * two 32-bit time fields joined into one int64 nanosecond stamp.  32 bytes.
 *   type : 0 padding (never processed, cf. the zero-padded steps of Sec. 5.1.1)
 *          1 limit order, 2 cancel, 3 delete, 4 market order
 *   side : +1 bid (buy), -1 ask (sell)
 *   price: integer ticks; ignored for cancels, deletes and market orders
 *   qty  : order size, or the quantity to remove for a cancel/delete
 *   oid  : order id; a cancel/delete names the order it removes from
 *   tid  : trader id, copied into trade records
 *   time_ns: copied into the resting order and into trades it aggresses.
 * Priority between resting orders is arrival order within the book; the time
 * stamp is never compared.  Malformed messages (type outside 0..4, side not
 * +-1, qty <= 0, limit price <= 0) are skipped and counted (LOB_CTR_INVALID).
 * A limit order whose id is already live on its side is a contract violation
 * (behaviour unspecified). */
typedef struct {
    int32_t type, side, price, qty, oid, tid;
    int64_t time_ns;
} lob_msg_t;

/* Trade t = [P_j, Q_j, OID_a, OID_s, Ts, Tns] (Sec. 4.1, eq. trade) plus the
 * two trader ids: price = the standing order's price, qty = the filled
 * quantity, time_ns = the aggressor's time.  32 bytes. */
typedef struct {
    int32_t price, qty, oid_aggr, oid_stand, tid_aggr, tid_stand;
    int64_t time_ns;
} lob_trade_t;

/* ------------------------------------------------------------ configuration */

enum {
    LOB_OVERFLOW_EVICT = 0,  /* full side: evict the worst resting order when the
                                incoming rest has a strictly better price, else
                                reject the rest                                  */
    LOB_OVERFLOW_REJECT = 1  /* full side: always reject the rest               */
};

enum {
    LOB_FLAG_APPEND_TRADES = 1,   /* the trade log of a book keeps growing across
                                     lob_process_batch calls until lob_clear_trades
                                     (default: each call restarts the log of the
                                     books it touches)                            */
    LOB_FLAG_SNAPSHOT_CANCELS = 2 /* books initialised from a level snapshot
                                     (Sec. 5.1.1): snapshot orders carry
                                     OID <= -9000, and a cancel/delete whose OID
                                     is not live on its side applies to the
                                     snapshot order resting at the cancel's price */
};

typedef struct {
    int32_t n_books;         /* independent books, >= 1                           */
    int32_t capacity;        /* N: orders per side, 1..512 (Sec. 4)               */
    int32_t trade_capacity;  /* trades stored per book per call, >= 0; further
                                trades still execute and are counted (eq. trades) */
    int32_t overflow_rule;   /* LOB_OVERFLOW_*                                     */
    int32_t flags;           /* LOB_FLAG_*                                         */
} lob_config_t;

enum {
    LOB_OK = 0,
    LOB_E_INVAL = -1,    /* bad argument (null pointer, size, alignment, range) */
    LOB_E_NOMEM = -2,    /* device or host allocation failed                     */
    LOB_E_CUDA = -3,     /* a CUDA runtime call failed                           */
    LOB_E_TIMEOUT = -4,  /* a bounded device wait gave up (see status word)      */
    LOB_E_STATE = -5     /* call not valid in the context's current state        */
};

/* status word bits (device-side anomalies, sticky until lob_reset) */
enum {
    LOB_STATUS_TIMEOUT = 1,       /* a message chunk did not arrive within the wait bound */
    LOB_STATUS_BAD_BOOK = 2,      /* a book id outside [0, n_books) was skipped            */
    LOB_STATUS_BAD_SEGMENT = 4,   /* a segment with offsets[i+1] < offsets[i] was skipped  */
    LOB_STATUS_BAD_BOOK_LOAD = 8, /* lob_set_book / lob_init_from_levels: a side not in
                                     priority order was loaded empty                      */
    LOB_STATUS_CHECK = 16         /* checked builds only (-DLOB_CHECKS): after some message a
                                     book broke an invariant (side count outside 0..capacity,
                                     a side out of priority order, a resting quantity <= 0,
                                     a crossed book)                                          */
};

/* per-book counters (int64), in this order */
enum {
    LOB_CTR_MSGS = 0,          /* messages examined (padding and invalid included) */
    LOB_CTR_LIMIT,             /* valid limit orders                               */
    LOB_CTR_CANCEL,            /* valid cancels + deletes                          */
    LOB_CTR_MARKET,            /* valid market orders                              */
    LOB_CTR_NOOP,              /* type-0 padding                                   */
    LOB_CTR_INVALID,           /* malformed messages skipped                       */
    LOB_CTR_TRADES,            /* trades executed                                  */
    LOB_CTR_TRADED_QTY,        /* sum of trade quantities                          */
    LOB_CTR_RESTED,            /* limit remainders placed on the book              */
    LOB_CTR_REJECTED,          /* remainders rejected by the full-side rule        */
    LOB_CTR_REJECTED_QTY,
    LOB_CTR_EVICTED,           /* resting orders evicted by the full-side rule     */
    LOB_CTR_EVICTED_QTY,
    LOB_CTR_CANCEL_HIT,        /* cancels/deletes that found their order           */
    LOB_CTR_CANCELLED_QTY,
    LOB_CTR_CANCEL_MISS,       /* cancels/deletes whose id is not live on that side */
    LOB_CTR_MARKET_DISCARDED_QTY, /* unmatched market quantity (dropped)           */
    LOB_CTR_LIMIT_QTY,         /* quantity submitted by valid limit orders         */
    LOB_CTR_MARKET_QTY,        /* quantity submitted by valid market orders        */
    LOB_CTR_TRADES_DROPPED,    /* trades executed but not stored (log full)        */
    LOB_N_COUNTERS
};

typedef struct lob_ctx lob_ctx;

/* ------------------------------------------------------------------ lifecycle */

/* Create a context with `cfg->n_books` empty books (all sides empty, counters
 * zero).  Allocates the book state (48 * roundup(capacity, 32) bytes per
 * book), the trade log (32 * trade_capacity bytes per book) and counters on
 * the current device, and zeroes them on `stream`.  *out is set only on
 * success.  Errors: LOB_E_INVAL (bad config), LOB_E_NOMEM, LOB_E_CUDA. */
int lob_create(lob_ctx** out, const lob_config_t* cfg, void* stream);

/* Release everything the context owns (synchronises its device first).
 * NULL is accepted.  Returns LOB_OK or LOB_E_CUDA. */
int lob_destroy(lob_ctx* ctx);

/* Empty every book, clear the trade logs, counters and status word. */
int lob_reset(lob_ctx* ctx, void* stream);

/* Empty the books d_book_ids[0 .. n) (int32, device) and clear their trade
 * logs and counters; other books are untouched (a serving slot handed to a
 * new episode).  Ids outside [0, n_books) are skipped (LOB_STATUS_BAD_BOOK). */
int lob_reset_books(lob_ctx* ctx, const int32_t* d_book_ids, int32_t n, void* stream);

/* -------------------------------------------------------------- processing */

/* Apply message segments to books (Sec. 4.2 dispatch; Sec. 4.1 add, cancel,
 * match; Sec. 4.3 batching over independent books).
 *   d_msgs     : messages, 16-byte aligned, segment i = d_msgs[d_offsets[i] ..
 *                d_offsets[i+1]) in arrival order
 *   d_offsets  : int64[n_active + 1], non-decreasing
 *   d_book_ids : int32[n_active] target book of each segment, pairwise
 *                distinct; NULL means segment i -> book i (then n_active must
 *                equal n_books)
 *   n_active   : number of segments, 0..n_books (0 is a no-op)
 * Each touched book's trade log restarts (unless LOB_FLAG_APPEND_TRADES) and
 * receives the trades of its segment in execution order.  Books run as
 * independent work items pulled from a device work queue by a persistent
 * grid (one warp per book, book state staged in shared memory, message chunks
 * fetched by bulk asynchronous copies). */
int lob_process_batch(lob_ctx* ctx, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                      const int32_t* d_book_ids, int32_t n_active, void* stream);

/* lob_process_batch that also records the level-1 state after every message
 * (the execution environment's per-message best bid/ask price and volume,
 * Sec. 5.2.1): d_l1 is int32[total messages][4] indexed like d_msgs, entry k =
 * {best bid price, quantity at it, best ask price, quantity at it} after
 * message k; an empty side is (-1, 0); quantities saturate at INT32_MAX.
 * Entries of messages outside every segment are not written. */
int lob_process_batch_l1(lob_ctx* ctx, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                         const int32_t* d_book_ids, int32_t n_active, int32_t* d_l1,
                         void* stream);

/* Same as lob_process_batch, but segment i is d_msgs[d_starts[i] ..
 * d_starts[i] + d_counts[i]) (int64 each, device), so the segments may lie
 * anywhere in d_msgs -- e.g. the current step window of each of many resident
 * episodes whose messages are pre-loaded.  d_book_ids is required. */
int lob_process_segments(lob_ctx* ctx, const lob_msg_t* d_msgs, const int64_t* d_starts,
                         const int64_t* d_counts, const int32_t* d_book_ids, int32_t n_active,
                         void* stream);

/* Same as lob_process_batch, but the trades are appended to the log of the
 * previous call (for orders injected after a replay, Sec. 5.1.3 step 4). */
int lob_inject_orders(lob_ctx* ctx, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                      const int32_t* d_book_ids, int32_t n_active, void* stream);

/* Restart every book's trade log (count 0). */
int lob_clear_trades(lob_ctx* ctx, void* stream);

/* Stream every book's messages from HOST memory through the engine, copy and
 * compute overlapped (message replay, Sec. 4.3, fed from the host): book b's
 * msgs_per_book messages sit at h_msgs[b*msgs_per_book ..] (book-major;
 * page-locked memory, or the copies are not asynchronous).  Chunk k of every
 * book (chunk_msgs messages, the last chunk shorter) is copied by one strided
 * host-to-device copy on a stream of the context while chunk k-1 is being
 * processed; the result equals one lob_process_batch over the same segments
 * (books continue from their current state; the trade logs restart at the
 * call unless LOB_FLAG_APPEND_TRADES).  The context allocates, on first use,
 * three staging chunks of n_books*chunk_msgs*32 bytes (kept until
 * lob_destroy; a larger chunk_msgs later reallocates them after a device
 * synchronisation), a copy stream and events.  h_msgs must stay valid and
 * unchanged until `stream` has passed the call.  Returns once all work is
 * enqueued.  LOB_E_NOMEM when the staging does not fit. */
int lob_process_host(lob_ctx* ctx, const lob_msg_t* h_msgs, int64_t msgs_per_book,
                     int32_t chunk_msgs, void* stream);

/* ----------------------------------------------------------------- outputs */

/* Top `depth` price levels per side (Sec. 5.1.1 ten-level book state): for the
 * k-th best distinct price, the price and the summed quantity of its orders
 * (saturating at INT32_MAX); missing levels are (-1, 0).  Each output is
 * int32[n_books][depth].  depth 1..64. */
int lob_get_levels(lob_ctx* ctx, int32_t depth, int32_t* d_bid_px, int32_t* d_bid_qty,
                   int32_t* d_ask_px, int32_t* d_ask_qty, void* stream);

/* The same levels for the books listed in d_book_ids (int32[n_active],
 * device, caller-owned; e.g. the ids just passed to lob_process_batch), each
 * written to its own row of the int32[n_books][depth] outputs (a book listed
 * twice is written twice with the same values); the rows of books not listed
 * are left as they are.  An id outside 0..n_books-1 sets
 * LOB_STATUS_BAD_BOOK and is skipped.  n_active 0 launches nothing (then
 * d_book_ids may be NULL; otherwise NULL is LOB_E_INVAL).  This is
 * the per-step level output of a batch in which only some books advanced (a
 * serving tick), at the cost of those books alone. */
int lob_get_levels_books(lob_ctx* ctx, const int32_t* d_book_ids, int32_t n_active,
                         int32_t depth, int32_t* d_bid_px, int32_t* d_bid_qty,
                         int32_t* d_ask_px, int32_t* d_ask_qty, void* stream);

/* Trade logs: d_out is lob_trade_t[n_books][trade_capacity] in execution
 * order, entries past the stored count all -1; d_counts int64[n_books] is the
 * number of trades executed (may exceed trade_capacity).  Either pointer may
 * be NULL to skip it. */
int lob_get_trades(lob_ctx* ctx, lob_trade_t* d_out, int64_t* d_counts, void* stream);

/* Canonical book dump: per field [n_books][2][capacity] (side 0 bids, side 1
 * asks), orders in priority order (best price first, then arrival), unused
 * slots -1; d_count int32[n_books][2].  Any pointer may be NULL. */
int lob_get_book(lob_ctx* ctx, int32_t* d_price, int32_t* d_qty, int32_t* d_oid,
                 int32_t* d_tid, int64_t* d_time, int32_t* d_count, void* stream);

/* Load books from the canonical layout above (checkpoint restore, or a book
 * initialised from a level snapshot).  Each side must be in priority order
 * with 0 <= count <= capacity and positive prices and quantities; a side that
 * is not is loaded empty and LOB_STATUS_BAD_BOOK_LOAD is set.  Trade logs,
 * counters and the status word are left as they are. */
int lob_set_book(lob_ctx* ctx, const int32_t* d_price, const int32_t* d_qty,
                 const int32_t* d_oid, const int32_t* d_tid, const int64_t* d_time,
                 const int32_t* d_count, void* stream);

/* Initialise every book from a level snapshot (Sec. 5.1.1: an episode starts
 * from the book's first levels, each known only by its price and total
 * volume, so each level enters the book as ONE order holding that volume,
 * with OIDs from -9000 downward).
 *   d_bid_px, d_bid_qty, d_ask_px, d_ask_qty: int32[n_books][depth] (device),
 *     level k = the k-th best price of the side and its volume -- the layout
 *     lob_get_levels writes.  A side's listed levels are those before its
 *     first level with price <= 0 or volume <= 0 (a shorter side ends there).
 *   depth: 1..capacity.
 *   time_ns: the time stamp every snapshot order carries.
 * Per book, both sides are replaced: listed level k of a side becomes the
 * order [price, volume, OID, TID 0, time_ns] at priority rank k; OIDs are
 * handed out over the listed bid levels best first (-9000, -9001, ...), then
 * over the listed ask levels best first.  A side whose listed levels are not
 * in priority order (a bid level priced above the one before it, an ask level
 * below it) is loaded empty and LOB_STATUS_BAD_BOOK_LOAD is set; its levels
 * still use up their OIDs.  Trade logs and counters are left as they are.
 * Combine with LOB_FLAG_SNAPSHOT_CANCELS so that cancels of orders placed
 * before the snapshot apply to these orders by price.
 * Errors: LOB_E_INVAL (null pointer, depth outside 1..capacity), LOB_E_CUDA. */
int lob_init_from_levels(lob_ctx* ctx, const int32_t* d_bid_px, const int32_t* d_bid_qty,
                         const int32_t* d_ask_px, const int32_t* d_ask_qty, int32_t depth,
                         int64_t time_ns, void* stream);

/* Counters int64[n_books][LOB_N_COUNTERS] (cumulative since create/reset) and
 * the status word (int32, LOB_STATUS_* bits).  Either pointer may be NULL. */
int lob_get_stats(lob_ctx* ctx, int64_t* d_counters, int32_t* d_status, void* stream);

/* ------------------------------------------------- execution environment */

/* One environment per book of a context (Sec. 5, gymnax base and execution
 * environments): each step replays a window of data messages, then submits the
 * agent's orders, then reports the top levels, the agent's fills and the
 * reward R = sum_j Q_j (P_j - P_VWAP) + lambda * sum_j Q_j (P_VWAP - P_init)
 * with P_VWAP = sum_i Q_i P_i / sum_i Q_i (Sec. 5.2.4, eqs. rewardfunc and
 * vwap; i over all trades of the step, j over the agent's trades; R = 0 when
 * the step has no trade or no agent trade; P_init = mid after the first
 * step's data, or the one-sided best price, or p_init_fallback).  The reward
 * is evaluated in IEEE double in that operation order and rounded to float.
 *
 * The agent (a seeded stand-in for the learned policy) sells parent_qty over
 * n_steps steps: at step t < n_steps-1 it splits
 * ceil((parent_qty - submitted) / (n_steps - t)) into the number of child
 * orders its draw gives (equal parts, remainder to the first, empty parts
 * dropped), each a limit sell at last_ask + {-2..+2} ticks (at least 1; last_ask
 * = best ask when the ask side is non-empty) or a market sell; at the last
 * step it cancels its resting orders in priority order and sells
 * parent_qty - executed at market (Sec. 5.2.5).  Agent orders carry
 * oid 2^30 + counter, tid agent_tid and the time of the step's last data
 * message (Sec. 5.1.3).  Draws are uint32: bits 0-1 = child orders - 1,
 * bits 2+3k..4+3k = action of child k (0..4 = -2..+2 ticks, 5 = market).
 *
 * Policy actions (Sec. 5.2.3) replace the stand-in when lob_env_run gets
 * d_actions: four float sizes, placed as limit sells in this order at the far
 * touch (best bid), the mid rounded up to the tick grid (the one best price
 * when a side is empty), the near touch (best ask) and the passive price
 * (best ask + passive_ticks x tick_size), all read from the book after the
 * step's data messages.  A size is the whole part of its component, none
 * below 1 or for NaN, at most parent_qty - submitted (taken in that order);
 * an order whose price needs a missing side is not placed.  The last step
 * ignores the action and closes out as above. */
typedef struct {
    int32_t n_steps;          /* episode length                                 */
    int32_t parent_qty;       /* shares the agent sells over the episode         */
    int32_t agent_tid;        /* trader id of the agent's orders                 */
    int32_t depth;            /* levels per side in the step output, 1..64       */
    int32_t p_init_fallback;  /* initial mid / last_ask when a side is empty     */
    int32_t msgs_per_step;    /* data messages per step, 1..1024                 */
    double lambda;            /* drift weight of eq. rewardfunc                  */
    int32_t passive_ticks;    /* n of P_passive = P_ask + n x ticksize, >= 0     */
    int32_t tick_size;        /* price units per tick, >= 1 (Sec. 5.2.2)         */
} lob_env_config_t;

typedef struct lob_env lob_env;

/* Create the environments of every book of `book` (which must outlive them)
 * and set their agent state to the start of an episode.  Books are not
 * touched (lob_reset empties them). */
int lob_env_create(lob_env** out, lob_ctx* book, const lob_env_config_t* cfg, void* stream);
int lob_env_destroy(lob_env* env);

/* Agent state back to the start of an episode (submitted = executed = 0,
 * counter 0, last_ask = p_init_fallback). */
int lob_env_reset(lob_env* env, void* stream);

/* Run steps step0 .. step0+n_run-1 of every environment in ONE launch (the
 * books stay in on-chip memory across the steps).  n_run = 1 is one step.
 * When there are more environments than resident warps, each environment's
 * steps are split into segments that the persistent grid hands out one after
 * another (a segment resumes from what the previous one wrote back); the
 * results do not depend on it (lob_env_segments).
 *   d_replay : data messages, 16-byte aligned; env b's step t window is
 *              d_replay[b*stride_env + t*msgs_per_step ..][0 .. msgs_per_step)
 *   d_draws  : uint32[n_run][n_books] agent draws of those steps, or NULL
 *              when d_actions is given
 *   d_actions: float[n_run][n_books][4] policy sizes (see above), or NULL
 *   outputs, each [n_run][n_books][...]: d_reward float; d_bid_px, d_bid_qty,
 *   d_ask_px, d_ask_qty int32 [depth]; d_fills int64 [2] = agent quantity and
 *   agent sum of Q*P of the step.
 *   d_l1 (NULL = off): int32 [n_run][n_books][msgs_per_step][4], the level-1
 *              state after every data message of the window (best bid price,
 *              its quantity, best ask price, its quantity; (-1, 0) when empty),
 *              the per-message augmented state of Sec. 5.2.1; 16-byte aligned.
 * After the call the book's trade log holds the trades of the last step run.
 * Errors: LOB_E_INVAL when a step is outside [0, n_steps) or an argument is
 * bad. */
int lob_env_run(lob_env* env, const lob_msg_t* d_replay, int64_t stride_env, int32_t step0,
                int32_t n_run, const uint32_t* d_draws, const float* d_actions, float* d_reward,
                int32_t* d_bid_px, int32_t* d_bid_qty, int32_t* d_ask_px, int32_t* d_ask_qty,
                int64_t* d_fills, int32_t* d_l1, void* stream);

/* No counterpart in the paper (introspection for tests and tuning): how many
 * segments of consecutive steps each environment's run was split into by the
 * most recent lob_env_run (1 = whole runs; the persistent grid hands out
 * segments, not whole episodes, when there are more environments than
 * resident warps), or -1 for a NULL env. */
int32_t lob_env_segments(const lob_env* env);

/* Observation of every environment after its most recent step (Sec. 5.2.2):
 * d_obs float [n_books][6M + 8], M = msgs_per_step, laid out in the order the
 * paper lists: best bid prices [M], best ask prices [M], mid prices [M],
 * passive prices [M], spreads [M], current time [s, ns], elapsed time
 * [s, ns], P_init, drift P_mid - P_init, task size, quantity executed,
 * level-1 imbalances Q_ask - Q_bid [M].  The per-message arrays come from
 * d_l1, that step's level-1 trace (int32 [n_books][M][4] as lob_env_run
 * writes it; for a multi-step run, the last step's slice); a value that needs
 * a missing side is -1.  Current time = the step's last data message; elapsed
 * = current - the time of the episode's first replay record
 * (d_replay[b*stride_env]); the drift uses the mid after the last data
 * message (0 when undefined).  Each value is one IEEE round-to-nearest of an
 * exact integer or half-integer.  d_l1 16-byte aligned. */
int lob_env_observe(lob_env* env, const lob_msg_t* d_replay, int64_t stride_env,
                    const int32_t* d_l1, float* d_obs, void* stream);

/* Agent state: int64[n_books][5] = submitted, executed, id counter, last_ask,
 * last data time; double[n_books] = P_init.  Either pointer may be NULL. */
int lob_env_get_state(lob_env* env, int64_t* d_state, double* d_p_init, void* stream);

/* ------------------------------------------------- paper-literal ablation */

/* The paper's own formulation of the book (Sec. 4, eqs. 1-2; Sec. 4.1), kept
 * as an ablation of this library's sorted-side design: each side an UNSORTED
 * array of `capacity` slots with -1 marking an empty slot; add writes an empty
 * slot, cancel finds the OID by a full scan, matching takes Best(o) by a full
 * arg-max / arg-min (earliest arrival among equal prices) once per fill, and
 * every slot with Q <= 0 is reset to -1 after every fill and operation.  With
 * all_branches = 1 every message also runs all three branches of the dispatch
 * (limit, cancel/delete, market), each on its own copy of the book, and keeps
 * its own one -- what `vmap` does with a branch (Sec. 4.3).
 * Every book starts EMPTY and runs d_msgs[d_offsets[b] .. d_offsets[b+1]);
 * the results equal lob_process_batch's on the same input (same full-side
 * rule, no snapshot rule): d_trades lob_trade_t[n_books][trade_capacity]
 * (-1 past the stored ones), d_trade_counts int64[n_books], and the final
 * books in lob_get_book's canonical layout ([n_books][2][capacity], priority
 * order, -1 padded; d_count int32[n_books][2]).  No counters.  capacity
 * 1..128; d_msgs 16-byte aligned; nothing is allocated.  LOB_E_INVAL on a bad
 * argument. */
int lob_literal_process(const lob_msg_t* d_msgs, const int64_t* d_offsets, int32_t n_books,
                        int32_t capacity, int32_t trade_capacity, int32_t overflow_rule,
                        int32_t all_branches, lob_trade_t* d_trades, int64_t* d_trade_counts,
                        int32_t* d_price, int32_t* d_qty, int32_t* d_oid, int32_t* d_tid,
                        int64_t* d_time, int32_t* d_count, void* stream);

/* ------------------------------------------------------ allocation-free call */

/* No counterpart in the paper: an engineering addition for callers that must
 * not allocate device memory at run time -- for example a service that has
 * reserved the GPU's memory up front for its own pool, or a latency-critical
 * loop in which a cudaMalloc/cudaFree would synchronise the device and stall
 * other streams.  It needs no lob_ctx and allocates nothing: the book state,
 * per-side counts and work-queue counter it needs live in one fixed 32 MiB
 * array inside the library (held on every GPU that loads the library, until
 * the process exits).
 *
 * Every one of n_books books starts EMPTY and processes its segment
 * d_msgs[d_offsets[b] .. d_offsets[b+1]) exactly as lob_process_batch would
 * (same kernel, same results).  Outputs (caller-owned device memory):
 *   d_trades       lob_trade_t[n_books][trade_capacity]: trades in execution
 *                  order; entries past a book's count are left untouched
 *   d_trade_counts int64[n_books]: trades executed per book (zeroed first, so
 *                  a book skipped with LOB_STATUS_BAD_SEGMENT reads 0)
 *   d_counters     int64[n_books][LOB_N_COUNTERS] (overwritten, not accumulated)
 *   d_price .. d_count: final canonical book as in lob_get_book (each may be NULL)
 *   d_status       int32 status word (LOB_STATUS_*), overwritten
 * Limits: capacity 1..512; the scratch must hold n_books books: exactly,
 *   256 + roundup(8 * n_books, 256) + n_books * B <= 32 MiB (33,554,432 B),
 * with B = 48 * S bytes per book and S = capacity rounded up to 32, 64, 128,
 * 256 or 512 slots -- at most 5,454 books at capacity 100 (B = 6,144) and
 * 1,364 at capacity 512 (B = 24,576).  Larger requests return LOB_E_INVAL
 * with the limit in lob_last_error().  The first call on a device resolves the array's device
 * address and sets kernel attributes for that device; make that first call
 * before any stream capture.  Every call reuses the same array: calls whose
 * work overlaps on the GPU (different streams, or several host threads) race
 * and corrupt each other's books; serialise them. */
int lob_process_streams_static(const lob_msg_t* d_msgs, const int64_t* d_offsets,
                               int32_t n_books, int32_t capacity, int32_t trade_capacity,
                               int32_t overflow_rule, lob_trade_t* d_trades,
                               int64_t* d_trade_counts, int64_t* d_counters, int32_t* d_price,
                               int32_t* d_qty, int32_t* d_oid, int32_t* d_tid, int64_t* d_time,
                               int32_t* d_count, int32_t* d_status, void* stream);

/* ------------------------------------------------------------------ tuning */

/* ---------------------------------------------------- serving tick executor */

/* Continuous batching of simulation episodes over the books of one context
 * (no counterpart in the paper; each tick applies one step of every running
 * episode, the replay step of Sec. 5.1.1 / 5.1.3): a book per slot, a running
 * episode per occupied slot, advancing one step per tick.  A tick produces the
 * occupied slots' windows of data messages with the caller's device generator
 * on gen_stream, then, on proc_stream, resets the books of episodes admitted
 * since the last tick, applies the windows (lob_process_batch) and writes the
 * levels of the advanced books (lob_get_levels_books).  The upload of a tick
 * (its offsets, slots and restarts) goes through a ring of `ring` pinned host
 * buffers, so the host may run up to `ring` ticks ahead of the GPU; the windows
 * alternate between two buffers.  Host code; one thread per executor. */

/* The device generator, called on gen_stream: init resets the state of n
 * slots (d_slots int32[n]) to the streams d_stream_ids (uint64[n]); advance
 * writes, for n slots, d_counts[i] messages of slot d_slots[i]'s stream into
 * d_out (lob_msg_t) at d_offsets[i].  Both return 0 on success. */
typedef int (*lob_gen_init_fn)(const void* params, int32_t n, const int32_t* d_slots,
                               const uint64_t* d_stream_ids, void* d_states, void* stream);
typedef int (*lob_gen_advance_fn)(const void* params, const void* d_geo_px,
                                  const void* d_geo_q, int32_t n, const int32_t* d_slots,
                                  void* d_states, void* d_pools, const int64_t* d_counts,
                                  const int64_t* d_offsets, void* d_out, void* stream);

typedef struct {
    lob_ctx* engine;            /* the books: n_books == slots                       */
    const void* gen_params;     /* host, the generator's parameters (caller keeps)   */
    lob_gen_init_fn gen_init;
    lob_gen_advance_fn gen_advance;
    const void* d_geo_px;       /* generator tables and per-slot state (device,      */
    const void* d_geo_q;        /*   caller-owned, passed through to the generator)  */
    void* d_gen_states;
    void* d_gen_pools;
    void* d_win0;               /* two window buffers, lob_msg_t[slots * max_msgs]   */
    void* d_win1;
    int32_t* d_bid_px;          /* levels of the advanced books, int32[slots][depth] */
    int32_t* d_bid_qty;
    int32_t* d_ask_px;
    int32_t* d_ask_qty;
    int64_t* d_trade_counts;    /* int64[slots], written by ticks with `collect`     */
    void* proc_stream;          /* cudaStream_t, caller-owned                        */
    void* gen_stream;
    int32_t slots;
    int32_t max_msgs;           /* messages per step, at most                        */
    int32_t depth;              /* levels 1..64                                      */
    int32_t ring;               /* ticks the host may run ahead, 1..64               */
} lob_serve_desc;

typedef struct lob_serve lob_serve;

/* Allocates the executor (two device upload buffers, the pinned ring, events);
 * every pointer of the descriptor must be non-null.  LOB_E_INVAL on a bad
 * descriptor, LOB_E_NOMEM / LOB_E_CUDA on allocation failure. */
int lob_serve_create(lob_serve** out, const lob_serve_desc* desc);

/* Admit an episode of n_steps steps of msgs_per_step (0..max_msgs) messages
 * from generator stream stream_id into a free slot (*slot_out); its
 * book and generator state are reset at the next tick.  LOB_E_STATE with
 * *slot_out = -1 when every slot is occupied. */
int lob_serve_admit(lob_serve* s, uint64_t stream_id, int64_t n_steps, int32_t msgs_per_step,
                    int32_t* slot_out);

/* One step of every occupied slot, issued asynchronously (waits only for the
 * ring buffer it reuses).  Outputs: *n_active occupied slots advanced (listed
 * in ascending order in h_active, int32[slots], when non-null), *n_finished
 * slots whose episode took its last step (h_finished, int32[slots]; they are
 * free from now on, their books valid until a later admission resets them in
 * stream order), *n_msgs messages.  timing != 0 records the tick's processing
 * and generation times (lob_serve_timings); collect != 0 also writes every
 * book's trade count into d_trade_counts.  No occupied slot: nothing issued. */
int lob_serve_tick(lob_serve* s, int32_t timing, int32_t collect, int32_t* h_active,
                   int32_t* n_active, int32_t* h_finished, int32_t* n_finished,
                   int64_t* n_msgs);

/* 1 when a tick issued now would not wait on the host (the ring buffer it
 * would reuse is free), 0 when it would; never waits.  LOB_E_INVAL for NULL,
 * LOB_E_CUDA when a recorded tick failed. */
int lob_serve_ready(lob_serve* s);

/* Waits for every tick issued so far; *count = timed ticks recorded.  When cap
 * >= *count, copies, oldest first, each tick's processing time (ms, from its
 * windows being ready to its levels written, on proc_stream), generation time
 * (ms, on gen_stream) and slots advanced, and clears the record; otherwise
 * copies nothing. */
int lob_serve_timings(lob_serve* s, float* proc_ms, float* gen_ms, int32_t* n_in_tick,
                      int32_t cap, int32_t* count);

/* Waits for the ticks in flight and frees the executor (not the caller's
 * buffers, streams or context).  NULL is a no-op. */
int lob_serve_destroy(lob_serve* s);

/* Launch shape of the processing kernel: warps (= books in flight) per CTA
 * (1..16; 1..8 for capacity > 128), messages per staged chunk (8..1024,
 * multiple of 8), and CTAs per SM for the persistent grid (0 = as many as
 * fit).  Takes effect for later calls.  Returns LOB_E_INVAL when the shape
 * does not fit in shared memory. */
int lob_set_launch(lob_ctx* ctx, int32_t warps_per_cta, int32_t chunk_msgs,
                   int32_t ctas_per_sm);

/* Number of kernel launches this context has issued since creation. */
int64_t lob_launch_count(const lob_ctx* ctx);

/* Human-readable description of the calling thread's most recent error. */
const char* lob_last_error(void);

/* Failure handling self-test (no counterpart in the paper): run the bounded
 * wait that guards every staged copy on an mbarrier that nothing completes,
 * for limit_ns (1 ns .. 1 s).  The wait gives up as designed, OR-s
 * LOB_STATUS_TIMEOUT into *d_status (int32, device) and, when d_elapsed_ns is
 * non-null, stores the nanoseconds it waited (uint64, device).  No fault, no
 * hang: the device stays usable.  LOB_E_INVAL on a bad argument. */
int lob_selftest_wait(int64_t limit_ns, int32_t* d_status, uint64_t* d_elapsed_ns, void* stream);

/* Library ABI version (incremented on incompatible change). */
int lob_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LOB_H */
