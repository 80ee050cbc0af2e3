// lob_oracle.cpp -- CPU oracle for the limit-order-book engine.
//
// TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
// definition against which the CUDA engine is checked.  Only the test-suite,
// the smoke check and the benchmark's CPU-baseline leg may load it; the
// engine never calls it and shares no code, header or table with it.
//
// What it computes (the paper's Sec. 4, "The JAX-LOB simulator"):
//   * a book has two sides, bids B and asks A, each holding at most N orders
//     o = [P, Q, OID, TID, time] (Sec. 4, eqs. 1-2);
//   * messages m = [T, S, Q, P, OID, TID, time] (Sec. 4.2, eq. message) are
//     processed strictly in order, per book (Sec. 4.3);
//   * limit (T=1): match against the opposite side, then add the remaining
//     quantity as one new order on the own side (Sec. 4.2, step 1);
//   * cancel (T=2) and delete (T=3): identical; locate OID and remove the
//     message quantity from it (Sec. 4.1 item 2, Sec. 4.2 step 2);
//   * market (T=4): match with price 0 (sell) or max_int (buy) and drop the
//     unmatched rest (Sec. 4.2 step 3);
//   * matching repeatedly takes Best(o_s) on the opposite side -- best price,
//     then earliest arrival (Sec. 4.1, eq. best_price, with the bid side read
//     as the maximum) -- while Q_a > 0, the side is non-empty and the prices
//     cross (P_a <= P_s for a sell, P_a >= P_s for a buy); each step applies
//     Q_s' = max(0, Q_s - Q_a), Q_a' = Q_a - Q_s and logs the trade
//     t = [P_s, Q_s - Q_s', OID_a, OID_s, time_a] (Sec. 4.1 item 3, eq. trade);
//   * after each operation orders with Q <= 0 leave the book (Sec. 4.1).
//
// Readings where the paper is silent (all listed in the design notes):
//   priority ties: arrival order within the book; a partially cancelled or
//   partially filled order keeps its place; a cancel looks the id up on side S
//   only and ignores the price; an unknown id is a no-op; a full side evicts
//   its worst order when the incoming residual has a strictly better price and
//   otherwise rejects the residual (or always rejects, rule 1); trades beyond
//   the per-call log capacity are executed but not stored; trade records carry
//   both trader ids; type 0 is padding; malformed messages are counted and
//   skipped.  Execution environment (Sec. 5.2): the seeded stand-in agent, the
//   reward of an empty step, the snapshot OIDs' order and the <= -9000 cancel
//   reading, the action map's rounding (mid up to the tick grid) and sizing
//   (whole shares, task cap), and -1 for observation values of a missing side.
//   Parity unpinned against the paper for these readings: hand-worked
//   examples of the reading pin them.
//
// Data structure: per side an ordered map price -> FIFO queue of orders, and
// a hash map from live OID to its price.
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <deque>
#include <functional>
#include <map>
#include <thread>
#include <unordered_map>
#include <vector>

namespace oracle {

struct Msg {  // 32-byte message record
    int32_t type, side, price, qty, oid, tid;
    int64_t time_ns;
};
struct Trade {  // 32-byte trade record
    int32_t price, qty, oid_aggr, oid_stand, tid_aggr, tid_stand;
    int64_t time_ns;
};
static_assert(sizeof(Msg) == 32, "msg");
static_assert(sizeof(Trade) == 32, "trade");

struct Order {
    int32_t price, qty, oid, tid;
    int64_t time_ns;
};

enum Counter {
    C_MSGS = 0, C_LIMIT, C_CANCEL, C_MARKET, C_NOOP, C_INVALID, C_TRADES, C_TRADED_QTY,
    C_RESTED, C_REJECTED, C_REJECTED_QTY, C_EVICTED, C_EVICTED_QTY, C_CANCEL_HIT,
    C_CANCELLED_QTY, C_CANCEL_MISS, C_MARKET_DISCARDED_QTY, C_LIMIT_QTY, C_MARKET_QTY,
    C_TRADES_DROPPED, N_COUNTERS
};

constexpr int32_t MAX_INT = 2147483647;

// One side of the book.  Levels are kept in an ordered map; priority order is
// descending price for bids and ascending price for asks, FIFO inside a level.
struct Side {
    bool is_bid;
    std::map<int32_t, std::deque<Order>> levels;
    std::unordered_map<int32_t, int32_t> price_of;  // live OID -> its price
    int32_t count = 0;

    explicit Side(bool bid) : is_bid(bid) {}

    bool empty() const { return count == 0; }

    // level holding Best(o) (Sec. 4.1 eq. best_price: min ask, max bid)
    std::deque<Order>& best_level()
    {
        return is_bid ? levels.rbegin()->second : levels.begin()->second;
    }
    std::deque<Order>& worst_level()
    {
        return is_bid ? levels.begin()->second : levels.rbegin()->second;
    }
    Order& best() { return best_level().front(); }
    Order& worst() { return worst_level().back(); }

    bool strictly_better(int32_t a, int32_t b) const { return is_bid ? a > b : a < b; }

    void append(const Order& o)  // rest at the back of its level
    {
        levels[o.price].push_back(o);
        price_of[o.oid] = o.price;
        ++count;
    }
    void remove_level_front(std::deque<Order>& lvl, int32_t price)
    {
        price_of.erase(lvl.front().oid);
        lvl.pop_front();
        --count;
        if (lvl.empty()) levels.erase(price);
    }
    void remove_worst()
    {
        auto& lvl = worst_level();
        int32_t price = lvl.back().price;
        price_of.erase(lvl.back().oid);
        lvl.pop_back();
        --count;
        if (lvl.empty()) levels.erase(price);
    }
    // locate a live order by OID; nullptr when not on this side
    Order* find(int32_t oid, std::deque<Order>** lvl_out)
    {
        auto it = price_of.find(oid);
        if (it == price_of.end()) return nullptr;
        auto& lvl = levels.at(it->second);
        for (auto& o : lvl)
            if (o.oid == oid) {
                *lvl_out = &lvl;
                return &o;
            }
        return nullptr;
    }
    void erase(int32_t oid)
    {
        auto it = price_of.find(oid);
        int32_t price = it->second;
        auto& lvl = levels.at(price);
        for (auto q = lvl.begin(); q != lvl.end(); ++q)
            if (q->oid == oid) {
                lvl.erase(q);
                break;
            }
        price_of.erase(it);
        --count;
        if (lvl.empty()) levels.erase(price);
    }
    // orders in priority order
    void for_each(const std::function<void(const Order&)>& f) const
    {
        if (is_bid) {
            for (auto it = levels.rbegin(); it != levels.rend(); ++it)
                for (const auto& o : it->second) f(o);
        } else {
            for (auto it = levels.begin(); it != levels.end(); ++it)
                for (const auto& o : it->second) f(o);
        }
    }
};

// Per-step trade sums of the execution environment (Sec. 5.2.4): all trades
// of the step, and those of the agent (trader id `agent_tid`).
struct StepSums {
    int64_t sq = 0, spq = 0, aq = 0, apq = 0;
    int32_t agent_tid = 0;
};

struct Book {
    Side bids{true}, asks{false};
    StepSums* sums = nullptr;  // set while an environment step observes trades
    std::vector<Trade> log;   // stored trades of the current call (<= trade capacity)
    int64_t log_count = 0;    // trades executed during the current call
    int64_t counters[N_COUNTERS] = {};
    int32_t error = 0;        // contract violations seen (duplicate live OID)

    Side& side_of(int32_t s) { return s == 1 ? bids : asks; }
};

struct Engine {
    int32_t n_books, capacity, trade_capacity, overflow_rule;
    bool append_trades;
    bool init_price_match = false;  // Sec. 5.1.1 cancels of snapshot orders by price
    std::vector<Book> books;
};

// ---------------------------------------------------------------- operations

static void log_trade(Engine& E, Book& bk, const Trade& t)
{
    if (bk.log_count < E.trade_capacity)
        bk.log.push_back(t);
    else
        bk.counters[C_TRADES_DROPPED] += 1;
    bk.log_count += 1;
    bk.counters[C_TRADES] += 1;
    bk.counters[C_TRADED_QTY] += t.qty;
    if (bk.sums) {
        StepSums& s = *bk.sums;
        s.sq += t.qty;
        s.spq += (int64_t)t.qty * t.price;
        if (t.tid_aggr == s.agent_tid || t.tid_stand == s.agent_tid) {
            s.aq += t.qty;
            s.apq += (int64_t)t.qty * t.price;
        }
    }
}

// Matching (Sec. 4.1 item 3 and the while loop that follows it).
// Returns the aggressor's remaining quantity max(0, Q_a).
static int32_t match(Engine& E, Book& bk, const Msg& m, int32_t P_a)
{
    Side& opp = bk.side_of(-m.side);
    int32_t Q_a = m.qty;
    while (!opp.empty() && Q_a > 0) {
        Order& s = opp.best();
        bool cross = (m.side == -1) ? (P_a <= s.price) : (P_a >= s.price);
        if (!cross) break;
        int32_t Q_s = s.qty;
        int32_t Q_s_new = std::max(0, Q_s - Q_a);  // Q_s' = max(0, Q_s - Q_a)
        int32_t Q_a_new = Q_a - Q_s;               // Q_a' = Q_a - Q_s
        Trade t;
        t.price = s.price;                         // P_j = P_s
        t.qty = Q_s - Q_s_new;                     // Q_j = Q_s - Q_s'
        t.oid_aggr = m.oid;                        // OID_a
        t.oid_stand = s.oid;                       // OID_s
        t.tid_aggr = m.tid;
        t.tid_stand = s.tid;
        t.time_ns = m.time_ns;                     // time of the aggressor
        log_trade(E, bk, t);
        s.qty = Q_s_new;
        Q_a = Q_a_new;
        if (s.qty <= 0) {  // Q <= 0 -> the order leaves the book
            int32_t price = s.price;
            opp.remove_level_front(opp.best_level(), price);
        }
    }
    return std::max(0, Q_a);
}

// Addition of the residual as one new order (Sec. 4.1 item 1), with the
// fixed full-side rule.
static void add(Engine& E, Book& bk, const Msg& m, int32_t Q)
{
    Side& own = bk.side_of(m.side);
    if (own.price_of.count(m.oid)) {
        bk.error += 1;  // duplicate live OID: contract violation
        return;
    }
    if (own.count >= E.capacity) {
        bool evict = (E.overflow_rule == 0) && own.strictly_better(m.price, own.worst().price);
        if (!evict) {
            bk.counters[C_REJECTED] += 1;
            bk.counters[C_REJECTED_QTY] += Q;
            return;
        }
        bk.counters[C_EVICTED] += 1;
        bk.counters[C_EVICTED_QTY] += own.worst().qty;
        own.remove_worst();
    }
    Order o{m.price, Q, m.oid, m.tid, m.time_ns};
    own.append(o);
    bk.counters[C_RESTED] += 1;
}

constexpr int32_t SNAPSHOT_OID_MAX = -9000;  // orders from a level snapshot: OID <= -9000

// Cancellation (Sec. 4.1 item 2): locate OID on side S, remove the quantity.
// With the snapshot rule (Sec. 5.1.1) a cancel whose OID is not live falls back
// to the snapshot order (OID <= -9000) resting at the cancel's price.
static void cancel(Engine& E, Book& bk, const Msg& m)
{
    Side& own = bk.side_of(m.side);
    std::deque<Order>* lvl = nullptr;
    Order* o = own.find(m.oid, &lvl);
    if (!o && E.init_price_match) {
        auto it = own.levels.find(m.price);
        if (it != own.levels.end())
            for (auto& q : it->second)
                if (q.oid <= SNAPSHOT_OID_MAX) {
                    o = &q;
                    break;
                }
    }
    if (!o) {
        bk.counters[C_CANCEL_MISS] += 1;
        return;
    }
    bk.counters[C_CANCEL_HIT] += 1;
    int32_t q_new = o->qty - m.qty;
    if (q_new <= 0) {  // Q <= 0 -> the order leaves the book
        bk.counters[C_CANCELLED_QTY] += o->qty;
        own.erase(o->oid);
    } else {
        bk.counters[C_CANCELLED_QTY] += m.qty;
        o->qty = q_new;
    }
}

// Message dispatch (Sec. 4.2).
static void process(Engine& E, Book& bk, const Msg& m)
{
    bk.counters[C_MSGS] += 1;
    if (m.type == 0) {
        bk.counters[C_NOOP] += 1;
        return;
    }
    bool bad = m.type < 0 || m.type > 4 || (m.side != 1 && m.side != -1) || m.qty <= 0 ||
               (m.type == 1 && m.price <= 0);
    if (bad) {
        bk.counters[C_INVALID] += 1;
        return;
    }
    switch (m.type) {
    case 1: {  // limit: match, then add the remaining quantity
        bk.counters[C_LIMIT] += 1;
        bk.counters[C_LIMIT_QTY] += m.qty;
        int32_t rest = match(E, bk, m, m.price);
        if (rest > 0) add(E, bk, m, rest);
        break;
    }
    case 2:
    case 3:  // cancel and delete are treated identically
        bk.counters[C_CANCEL] += 1;
        cancel(E, bk, m);
        break;
    case 4: {  // market: price 0 for a sell, max_int for a buy; drop the rest
        bk.counters[C_MARKET] += 1;
        bk.counters[C_MARKET_QTY] += m.qty;
        int32_t rest = match(E, bk, m, m.side == -1 ? 0 : MAX_INT);
        bk.counters[C_MARKET_DISCARDED_QTY] += rest;
        break;
    }
    }
}

// Level-1 state of a book (Sec. 5.2.1): best bid price and the quantity at
// that price, best ask price and the quantity at that price; an empty side is
// (-1, 0); quantities saturate at max_int.
static void level1(Book& bk, int32_t* out4)
{
    Side* sides[2] = {&bk.bids, &bk.asks};
    for (int s = 0; s < 2; ++s) {
        Side& sd = *sides[s];
        if (sd.empty()) {
            out4[2 * s] = -1;
            out4[2 * s + 1] = 0;
            continue;
        }
        int64_t vol = 0;
        for (const auto& o : sd.best_level()) vol += o.qty;
        out4[2 * s] = sd.best().price;
        out4[2 * s + 1] = (int32_t)std::min<int64_t>(vol, MAX_INT);
    }
}

template <class F>
static void parallel_for(int32_t n, int32_t n_threads, F&& body)
{
    if (n_threads <= 1 || n <= 1) {
        for (int32_t i = 0; i < n; ++i) body(i);
        return;
    }
    int32_t nt = std::min(n_threads, n);
    std::vector<std::thread> th;
    for (int32_t t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            for (int32_t i = t; i < n; i += nt) body(i);
        });
    for (auto& x : th) x.join();
}

}  // namespace oracle

using namespace oracle;

extern "C" {

int oracle_abi_version(void) { return 1; }
int oracle_n_counters(void) { return N_COUNTERS; }

void* oracle_create(int32_t n_books, int32_t capacity, int32_t trade_capacity,
                    int32_t overflow_rule, int32_t append_trades)
{
    // append_trades bit 1 selects the snapshot cancel rule (Sec. 5.1.1)
    if (n_books < 0 || capacity < 1 || trade_capacity < 0 || overflow_rule < 0 ||
        overflow_rule > 1)
        return nullptr;
    Engine* E = new Engine();
    E->n_books = n_books;
    E->capacity = capacity;
    E->trade_capacity = trade_capacity;
    E->overflow_rule = overflow_rule;
    E->append_trades = (append_trades & 1) != 0;
    E->init_price_match = (append_trades & 2) != 0;
    E->books.resize((size_t)n_books);
    return E;
}

void oracle_destroy(void* h) { delete (Engine*)h; }

// Process segment i (messages [offsets[i], offsets[i+1])) on book
// book_ids[i] (or i).  The trade log of each touched book restarts unless
// the engine appends.  Returns the number of contract violations seen.
int64_t oracle_process(void* h, const Msg* msgs, const int64_t* offsets, const int32_t* book_ids,
                       int32_t n_active, int32_t n_threads)
{
    Engine& E = *(Engine*)h;
    std::vector<int32_t> err((size_t)std::max(n_active, 0), 0);
    parallel_for(n_active, n_threads, [&](int32_t i) {
        int32_t b = book_ids ? book_ids[i] : i;
        Book& bk = E.books[(size_t)b];
        if (!E.append_trades) {
            bk.log.clear();
            bk.log_count = 0;
        }
        int32_t e0 = bk.error;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) process(E, bk, msgs[k]);
        err[(size_t)i] = bk.error - e0;
    });
    int64_t total = 0;
    for (int32_t e : err) total += e;
    return total;
}

// As oracle_process, and writes the level-1 state after every message:
// l1[k][4] = {bid price, bid qty, ask price, ask qty} for message k of `msgs`.
int64_t oracle_process_l1(void* h, const Msg* msgs, const int64_t* offsets,
                          const int32_t* book_ids, int32_t n_active, int32_t n_threads,
                          int32_t* l1)
{
    Engine& E = *(Engine*)h;
    std::vector<int32_t> err((size_t)std::max(n_active, 0), 0);
    parallel_for(n_active, n_threads, [&](int32_t i) {
        int32_t b = book_ids ? book_ids[i] : i;
        Book& bk = E.books[(size_t)b];
        if (!E.append_trades) {
            bk.log.clear();
            bk.log_count = 0;
        }
        int32_t e0 = bk.error;
        for (int64_t k = offsets[i]; k < offsets[i + 1]; ++k) {
            process(E, bk, msgs[k]);
            level1(bk, l1 + 4 * k);
        }
        err[(size_t)i] = bk.error - e0;
    });
    int64_t total = 0;
    for (int32_t e : err) total += e;
    return total;
}

void oracle_clear_trades(void* h)
{
    Engine& E = *(Engine*)h;
    for (auto& bk : E.books) {
        bk.log.clear();
        bk.log_count = 0;
    }
}

// Trades: out[b][trade_capacity], entries beyond the stored count are all -1.
void oracle_get_trades(void* h, Trade* out, int64_t* counts)
{
    Engine& E = *(Engine*)h;
    for (int32_t b = 0; b < E.n_books; ++b) {
        Book& bk = E.books[(size_t)b];
        Trade* o = out + (int64_t)b * E.trade_capacity;
        memset(o, 0xff, sizeof(Trade) * (size_t)E.trade_capacity);
        for (size_t j = 0; j < bk.log.size(); ++j) o[j] = bk.log[j];
        counts[b] = bk.log_count;
    }
}

// Canonical book: [n_books][2][capacity] per field (side 0 = bids, 1 = asks),
// orders in priority order, empty slots all -1; count[n_books][2].
void oracle_get_book(void* h, int32_t* px, int32_t* qty, int32_t* oid, int32_t* tid,
                     int64_t* tm, int32_t* count)
{
    Engine& E = *(Engine*)h;
    const int64_t C = E.capacity;
    for (int32_t b = 0; b < E.n_books; ++b) {
        Book& bk = E.books[(size_t)b];
        for (int s = 0; s < 2; ++s) {
            Side& sd = s == 0 ? bk.bids : bk.asks;
            int64_t base = ((int64_t)b * 2 + s) * C;
            for (int64_t j = 0; j < C; ++j) {
                px[base + j] = qty[base + j] = oid[base + j] = tid[base + j] = -1;
                tm[base + j] = -1;
            }
            int64_t j = 0;
            sd.for_each([&](const Order& o) {
                px[base + j] = o.price;
                qty[base + j] = o.qty;
                oid[base + j] = o.oid;
                tid[base + j] = o.tid;
                tm[base + j] = o.time_ns;
                ++j;
            });
            count[b * 2 + s] = sd.count;
        }
    }
}

// Load books from the canonical layout (orders given in priority order).
// Returns 0, or -1 when a side is not in priority order or over capacity.
int oracle_set_book(void* h, const int32_t* px, const int32_t* qty, const int32_t* oid,
                    const int32_t* tid, const int64_t* tm, const int32_t* count)
{
    Engine& E = *(Engine*)h;
    const int64_t C = E.capacity;
    for (int32_t b = 0; b < E.n_books; ++b) {
        Book& bk = E.books[(size_t)b];
        bk.bids = Side(true);
        bk.asks = Side(false);
        for (int s = 0; s < 2; ++s) {
            Side& sd = s == 0 ? bk.bids : bk.asks;
            int32_t n = count[b * 2 + s];
            if (n < 0 || n > C) return -1;
            int64_t base = ((int64_t)b * 2 + s) * C;
            for (int32_t j = 0; j < n; ++j) {
                if (j > 0 && sd.strictly_better(px[base + j], px[base + j - 1])) return -1;
                if (qty[base + j] <= 0 || px[base + j] <= 0) return -1;
                sd.append(Order{px[base + j], qty[base + j], oid[base + j], tid[base + j],
                                tm[base + j]});
            }
        }
    }
    return 0;
}

// Initialise every book from a level snapshot (Sec. 5.1.1: the environment
// starts from the limit order book's snapshot of its first levels; a snapshot
// knows only each level's price and total volume, so every level enters the
// book as ONE order holding that volume, with OIDs counting down from -9000).
// Inputs are [n_books][depth] per array, level k = k-th best price of a side.
// Per book:
//   1. the book is emptied;
//   2. the listed levels of a side are the levels before the first one whose
//      price or volume is <= 0 (a shorter snapshot ends there);
//   3. OIDs are handed out in this order: the listed bid levels best first
//      (-9000, -9001, ...), then the listed ask levels best first;
//   4. each listed level becomes an order [P = price, Q = volume, OID, TID 0,
//      time = time_ns], appended in listed order (so equal prices keep the
//      listing as their arrival order);
//   5. a side whose listed levels are not in priority order (a bid level above
//      the one before it, an ask level below it), or that lists more levels
//      than the capacity, is left empty.
// Trade logs and counters are not touched.  Returns the number of sides left
// empty by rule 5.
int32_t oracle_init_from_levels(void* h, const int32_t* bid_px, const int32_t* bid_qty,
                                const int32_t* ask_px, const int32_t* ask_qty, int32_t depth,
                                int64_t time_ns)
{
    Engine& E = *(Engine*)h;
    int32_t rejected = 0;
    for (int32_t b = 0; b < E.n_books; ++b) {
        Book& bk = E.books[(size_t)b];
        bk.bids = Side(true);
        bk.asks = Side(false);
        int32_t next_oid = -9000;
        for (int s = 0; s < 2; ++s) {
            const int32_t* px = (s == 0 ? bid_px : ask_px) + (int64_t)b * depth;
            const int32_t* qty = (s == 0 ? bid_qty : ask_qty) + (int64_t)b * depth;
            Side& sd = s == 0 ? bk.bids : bk.asks;
            int32_t listed = 0;
            while (listed < depth && px[listed] > 0 && qty[listed] > 0) ++listed;
            std::vector<Order> orders;
            for (int32_t k = 0; k < listed; ++k) orders.push_back(Order{px[k], qty[k], next_oid--, 0, time_ns});
            bool ok = listed <= E.capacity;
            for (int32_t k = 1; k < listed; ++k)
                if (sd.strictly_better(px[k], px[k - 1])) ok = false;
            if (!ok) {
                ++rejected;
                continue;
            }
            for (const Order& o : orders) sd.append(o);
        }
    }
    return rejected;
}

// Top `depth` price levels per side: aggregated quantity per distinct price,
// best first; empty levels are (-1, 0).  Quantities saturate at max_int.
static void book_levels(Book& bk, int32_t b, int32_t depth, int32_t* bid_px, int32_t* bid_qty,
                        int32_t* ask_px, int32_t* ask_qty);

void oracle_get_levels(void* h, int32_t depth, int32_t* bid_px, int32_t* bid_qty, int32_t* ask_px,
                       int32_t* ask_qty)
{
    Engine& E = *(Engine*)h;
    for (int32_t b = 0; b < E.n_books; ++b)
        book_levels(E.books[(size_t)b], b, depth, bid_px, bid_qty, ask_px, ask_qty);
}

static void book_levels(Book& bk, int32_t b, int32_t depth, int32_t* bid_px, int32_t* bid_qty,
                        int32_t* ask_px, int32_t* ask_qty)
{
    {
        for (int s = 0; s < 2; ++s) {
            Side& sd = s == 0 ? bk.bids : bk.asks;
            int32_t* opx = (s == 0 ? bid_px : ask_px) + (int64_t)b * depth;
            int32_t* oq = (s == 0 ? bid_qty : ask_qty) + (int64_t)b * depth;
            for (int32_t k = 0; k < depth; ++k) {
                opx[k] = -1;
                oq[k] = 0;
            }
            int32_t k = 0;
            auto emit = [&](int32_t price, const std::deque<Order>& lvl) {
                if (k >= depth) return;
                int64_t sum = 0;
                for (const auto& o : lvl) sum += o.qty;
                opx[k] = price;
                oq[k] = (int32_t)std::min<int64_t>(sum, MAX_INT);
                ++k;
            };
            if (sd.is_bid)
                for (auto it = sd.levels.rbegin(); it != sd.levels.rend(); ++it)
                    emit(it->first, it->second);
            else
                for (auto it = sd.levels.begin(); it != sd.levels.end(); ++it)
                    emit(it->first, it->second);
        }
    }
}

void oracle_get_counters(void* h, int64_t* out)
{
    Engine& E = *(Engine*)h;
    for (int32_t b = 0; b < E.n_books; ++b)
        memcpy(out + (int64_t)b * N_COUNTERS, E.books[(size_t)b].counters,
               sizeof(int64_t) * N_COUNTERS);
}

// Resting quantity per book (sum over both sides), for conservation checks.
void oracle_get_resting_qty(void* h, int64_t* out)
{
    Engine& E = *(Engine*)h;
    for (int32_t b = 0; b < E.n_books; ++b) {
        int64_t sum = 0;
        for (int s = 0; s < 2; ++s) {
            Side& sd = s == 0 ? E.books[(size_t)b].bids : E.books[(size_t)b].asks;
            sd.for_each([&](const Order& o) { sum += o.qty; });
        }
        out[b] = sum;
    }
}

}  // extern "C"

// ------------------------------------------------------------------------
// Execution environment (Sec. 5): each book is one environment whose step
// replays a window of data messages, then submits the agent's orders, then
// reports the top levels, the agent's fills and the reward
//   R = sum_j Q_j (P_j - P_VWAP) + lambda * sum_j Q_j (P_VWAP - P_init),
//   P_VWAP = sum_i Q_i P_i / sum_i Q_i                  (eqs. rewardfunc, vwap)
// with i over every trade of the step and j over the agent's trades.
// The agent (not specified by the paper; a seeded stand-in for the learned
// policy) sells a parent order of `parent_qty` over `n_steps` steps: at step
// t < n_steps-1 it splits ceil((parent - submitted) / (n_steps - t)) into
// n in {1..4} child sell orders (equal parts, remainder to the first, empty
// parts dropped), each a limit at last_ask + {-2..+2} ticks (at least 1) or a
// market order, as drawn; at the last step it cancels its resting orders and
// sends a market sell for parent - executed (Sec. 5.2.5).
// Agent orders carry oid 2^30 + counter (the ID counter of Sec. 5.1.2) and the
// time of the step's last data message (Sec. 5.1.3 step 3).
namespace oracle {

struct EnvCfg {
    int32_t n_steps, parent_qty, agent_tid, depth, p_init_fallback;
    int32_t passive_ticks, tick_size;  // P_passive = P_ask + n x ticksize (Sec. 5.2.2)
    double lambda;
};

struct EnvState {
    int64_t submitted = 0, executed = 0;
    int32_t id_counter = 0, last_ask = 0;
    int64_t last_time = 0;
    double p_init = 0.0;
};

struct EnvEngine {
    Engine E;
    EnvCfg cfg;
    std::vector<EnvState> st;
};

static int32_t best_price(Side& sd)
{
    return sd.best().price;
}

// Order size from one continuous action component (Sec. 5.2.3): the whole
// part of the component, nothing for a component below one share (or NaN),
// at most what is left of the task.
static int64_t action_qty(float a, int64_t remaining)
{
    const double x = (double)a;
    if (!(x >= 1.0) || remaining <= 0) return 0;
    const double w = std::floor(x);
    return w >= (double)remaining ? remaining : (int64_t)w;
}

// The four prices of the action space for a sell task (Sec. 5.2.3): far touch
// = best bid, mid (rounded up to the tick grid for a sell), near touch = best
// ask, passive = best ask + n ticks.  A price whose side is missing is -1.
static void action_prices(Book& bk, int32_t passive_ticks, int32_t tick, int32_t out[4])
{
    const bool hb = !bk.bids.empty(), ha = !bk.asks.empty();
    const int64_t pb = hb ? best_price(bk.bids) : -1, pa = ha ? best_price(bk.asks) : -1;
    out[0] = (int32_t)pb;
    if (hb && ha) {
        const int64_t two_t = 2 * (int64_t)tick;
        out[1] = (int32_t)((pb + pa + two_t - 1) / two_t * tick);  // smallest grid price >= mid
    } else {
        out[1] = (int32_t)(hb ? pb : pa);
    }
    out[2] = (int32_t)pa;
    const int64_t pp = pa + (int64_t)passive_ticks * tick;
    out[3] = (ha && pp <= INT32_MAX) ? (int32_t)pp : -1;
}

static void env_step_one(EnvEngine& V, int32_t b, const Msg* msgs, int64_t n_msgs, uint32_t draw,
                         const float* action, int32_t t, float* reward, int32_t* bid_px,
                         int32_t* bid_qty, int32_t* ask_px, int32_t* ask_qty, int64_t* fills,
                         int32_t* l1)
{
    Engine& E = V.E;
    const EnvCfg& cfg = V.cfg;
    EnvState& es = V.st[(size_t)b];
    Book& bk = E.books[(size_t)b];
    bk.log.clear();
    bk.log_count = 0;
    StepSums sums;
    sums.agent_tid = cfg.agent_tid;
    bk.sums = &sums;

    // 1. replay the step's data messages (level-1 state after each, Sec. 5.2.1)
    for (int64_t k = 0; k < n_msgs; ++k) {
        process(E, bk, msgs[k]);
        if (l1) level1(bk, l1 + 4 * k);
    }
    if (n_msgs > 0) es.last_time = msgs[n_msgs - 1].time_ns;

    // 2. initial mid-price of the episode (after the first data window)
    if (t == 0) {
        const bool hb = !bk.bids.empty(), ha = !bk.asks.empty();
        if (hb && ha)
            es.p_init = ((double)best_price(bk.bids) + (double)best_price(bk.asks)) / 2.0;
        else if (hb)
            es.p_init = (double)best_price(bk.bids);
        else if (ha)
            es.p_init = (double)best_price(bk.asks);
        else
            es.p_init = (double)cfg.p_init_fallback;
    }

    // 3. the agent's orders
    auto send = [&](int32_t type, int32_t price, int32_t qty) {
        Msg m;
        m.type = type;
        m.side = -1;
        m.price = price;
        m.qty = qty;
        m.oid = (int32_t)((1u << 30) + (uint32_t)es.id_counter);
        m.tid = cfg.agent_tid;
        m.time_ns = es.last_time;
        es.id_counter += 1;
        es.submitted += qty;
        process(E, bk, m);
    };
    if (t < cfg.n_steps - 1 && action) {
        // the policy's sizes at the four prices, in the order listed (Sec. 5.2.3)
        if (!bk.asks.empty()) es.last_ask = best_price(bk.asks);
        int32_t px[4];
        action_prices(bk, cfg.passive_ticks, cfg.tick_size, px);
        int64_t remaining = cfg.parent_qty - es.submitted;
        for (int k = 0; k < 4; ++k) {
            const int64_t q = action_qty(action[k], remaining);
            if (px[k] <= 0 || q <= 0) continue;
            send(1, px[k], (int32_t)q);
            remaining -= q;
        }
    } else if (t < cfg.n_steps - 1) {
        if (!bk.asks.empty()) es.last_ask = best_price(bk.asks);
        const int64_t remaining = cfg.parent_qty - es.submitted;
        const int64_t steps_left = cfg.n_steps - t;
        const int64_t target = remaining > 0 ? (remaining + steps_left - 1) / steps_left : 0;
        const int32_t n = (int32_t)(draw & 3u) + 1;
        const int64_t base = target / n, extra = target % n;
        for (int32_t k = 0; k < n; ++k) {
            const int32_t q = (int32_t)(base + (k == 0 ? extra : 0));
            if (q <= 0) continue;
            const int32_t a = (int32_t)((draw >> (2 + 3 * k)) & 7u);
            if (a == 5)
                send(4, 0, q);
            else
                send(1, std::max(1, es.last_ask + a - 2), q);
        }
    } else {
        // cancel the agent's resting orders (priority order), then sell the rest
        std::vector<Order> mine;
        bk.asks.for_each([&](const Order& o) {
            if (o.tid == cfg.agent_tid) mine.push_back(o);
        });
        for (const Order& o : mine) {
            Msg m;
            m.type = 2;
            m.side = -1;
            m.price = o.price;
            m.qty = o.qty;
            m.oid = o.oid;
            m.tid = cfg.agent_tid;
            m.time_ns = es.last_time;
            process(E, bk, m);
        }
        const int64_t left = cfg.parent_qty - (es.executed + sums.aq);
        if (left > 0) send(4, 0, (int32_t)left);
    }
    bk.sums = nullptr;
    es.executed += sums.aq;

    // 4. reward (eqs. rewardfunc, vwap), IEEE double, fixed operation order
    double r = 0.0;
    if (sums.sq > 0 && sums.aq > 0) {
        const double vwap = (double)sums.spq / (double)sums.sq;
        const double adv = (double)sums.apq - (double)sums.aq * vwap;
        const double drift = cfg.lambda * ((double)sums.aq * (vwap - es.p_init));
        r = adv + drift;
    }
    reward[b] = (float)r;
    fills[2 * (int64_t)b] = sums.aq;
    fills[2 * (int64_t)b + 1] = sums.apq;
    book_levels(bk, b, cfg.depth, bid_px, bid_qty, ask_px, ask_qty);
}

}  // namespace oracle

extern "C" {

void* oracle_env_create(int32_t n_envs, int32_t capacity, int32_t trade_capacity, int32_t n_steps,
                        int32_t parent_qty, int32_t agent_tid, int32_t depth,
                        int32_t p_init_fallback, int32_t passive_ticks, int32_t tick_size,
                        double lambda)
{
    if (n_envs < 1 || capacity < 1 || trade_capacity < 0 || n_steps < 1 || parent_qty < 0 ||
        depth < 1 || passive_ticks < 0 || tick_size < 1)
        return nullptr;
    EnvEngine* V = new EnvEngine();
    V->E.n_books = n_envs;
    V->E.capacity = capacity;
    V->E.trade_capacity = trade_capacity;
    V->E.overflow_rule = 0;
    V->E.append_trades = false;
    V->E.books.resize((size_t)n_envs);
    V->cfg = EnvCfg{n_steps, parent_qty, agent_tid, depth, p_init_fallback, passive_ticks,
                    tick_size, lambda};
    V->st.assign((size_t)n_envs, EnvState());
    for (auto& s : V->st) s.last_ask = p_init_fallback;
    return V;
}

void oracle_env_destroy(void* h) { delete (EnvEngine*)h; }

// The books of the environments, usable with every oracle_get_* accessor.
void* oracle_env_books(void* h) { return &((EnvEngine*)h)->E; }

// One step for every environment: env b replays replay[offsets[b] .. offsets[b+1]).
// The agent acts from draws[b] (the seeded stand-in), or, when `actions` is
// given, from the four sizes actions[4b .. 4b+4).
// l1 (nullable): level-1 state after every data message, [message][4] indexed
// like `replay`.
void oracle_env_step(void* h, const Msg* replay, const int64_t* offsets, const uint32_t* draws,
                     const float* actions, int32_t step, float* reward, int32_t* bid_px,
                     int32_t* bid_qty, int32_t* ask_px, int32_t* ask_qty, int64_t* fills,
                     int32_t n_threads, int32_t* l1)
{
    EnvEngine& V = *(EnvEngine*)h;
    parallel_for(V.E.n_books, n_threads, [&](int32_t b) {
        env_step_one(V, b, replay + offsets[b], offsets[b + 1] - offsets[b],
                     draws ? draws[b] : 0u, actions ? actions + 4 * (int64_t)b : nullptr, step,
                     reward, bid_px, bid_qty, ask_px, ask_qty, fills,
                     l1 ? l1 + 4 * offsets[b] : nullptr);
    });
}

// Observation of every environment after its most recent step (Sec. 5.2.2),
// float32 [n_envs][6M + 8], M = messages per step, in the order the paper
// lists: best bid prices [M], best ask prices [M], mid prices [M], passive
// prices [M], spreads [M], current time [s, ns], elapsed time [s, ns], P_init,
// drift P_mid - P_init, task size, quantity executed, level-1 imbalances
// Q_ask - Q_bid [M].  l1: that step's level-1 trace, [n_envs][M][4];
// t_init: each episode's initial time (its first replay record's time).
// A per-message value that needs a missing side is -1; the drift uses the mid
// after the step's last data message (0 when it is undefined).
void oracle_env_observe(void* h, const int32_t* l1, int32_t M, const int64_t* t_init, float* obs)
{
    EnvEngine& V = *(EnvEngine*)h;
    const EnvCfg& cfg = V.cfg;
    const int64_t row = 6 * (int64_t)M + 8;
    const int64_t kSec = 1000000000;
    for (size_t b = 0; b < V.st.size(); ++b) {
        const EnvState& es = V.st[b];
        float* o = obs + (int64_t)b * row;
        double mid_last = -1.0;
        for (int32_t k = 0; k < M; ++k) {
            const int32_t* r = l1 + ((int64_t)b * M + k) * 4;
            const int32_t pb = r[0], qb = r[1], pa = r[2], qa = r[3];
            const bool hb = pb > 0, ha = pa > 0;
            double mid = -1.0;
            if (hb && ha)
                mid = ((double)pb + (double)pa) / 2.0;
            else if (hb)
                mid = (double)pb;
            else if (ha)
                mid = (double)pa;
            const int64_t passive = ha ? (int64_t)pa + (int64_t)cfg.passive_ticks * cfg.tick_size
                                       : -1;
            o[k] = (float)pb;
            o[M + k] = (float)pa;
            o[2 * M + k] = (float)mid;
            o[3 * M + k] = (float)passive;
            o[4 * M + k] = (float)(hb && ha ? (int64_t)pa - pb : -1);
            o[5 * M + 8 + k] = (float)((int64_t)qa - qb);
            mid_last = mid;
        }
        float* sc = o + 5 * M;
        const int64_t tc = es.last_time, te = es.last_time - t_init[b];
        sc[0] = (float)(tc / kSec);
        sc[1] = (float)(tc % kSec);
        sc[2] = (float)(te / kSec);
        sc[3] = (float)(te % kSec);
        sc[4] = (float)es.p_init;
        sc[5] = (float)(mid_last >= 0.0 ? mid_last - es.p_init : 0.0);
        sc[6] = (float)cfg.parent_qty;
        sc[7] = (float)es.executed;
    }
}

// Turn the snapshot cancel rule (Sec. 5.1.1) on or off for the environments' books.
void oracle_env_set_snapshot_cancels(void* h, int32_t on)
{
    ((EnvEngine*)h)->E.init_price_match = on != 0;
}

// per env: submitted, executed, id_counter, last_ask, last_time; and p_init
void oracle_env_state(void* h, int64_t* out, double* p_init)
{
    EnvEngine& V = *(EnvEngine*)h;
    for (size_t b = 0; b < V.st.size(); ++b) {
        const EnvState& s = V.st[b];
        out[5 * b + 0] = s.submitted;
        out[5 * b + 1] = s.executed;
        out[5 * b + 2] = s.id_counter;
        out[5 * b + 3] = s.last_ask;
        out[5 * b + 4] = s.last_time;
        p_init[b] = s.p_init;
    }
}

}  // extern "C"
