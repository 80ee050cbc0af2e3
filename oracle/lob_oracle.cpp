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
//   skipped.
//
// Data structure: per side an ordered map price -> FIFO queue of orders, and
// a hash map from live OID to its price.
#include <stdint.h>
#include <string.h>

#include <algorithm>
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

struct Book {
    Side bids{true}, asks{false};
    std::vector<Trade> log;   // stored trades of the current call (<= trade capacity)
    int64_t log_count = 0;    // trades executed during the current call
    int64_t counters[N_COUNTERS] = {};
    int32_t error = 0;        // contract violations seen (duplicate live OID)

    Side& side_of(int32_t s) { return s == 1 ? bids : asks; }
};

struct Engine {
    int32_t n_books, capacity, trade_capacity, overflow_rule;
    bool append_trades;
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

// Cancellation (Sec. 4.1 item 2): locate OID on side S, remove the quantity.
static void cancel(Book& bk, const Msg& m)
{
    Side& own = bk.side_of(m.side);
    std::deque<Order>* lvl = nullptr;
    Order* o = own.find(m.oid, &lvl);
    if (!o) {
        bk.counters[C_CANCEL_MISS] += 1;
        return;
    }
    bk.counters[C_CANCEL_HIT] += 1;
    int32_t q_new = o->qty - m.qty;
    if (q_new <= 0) {  // Q <= 0 -> the order leaves the book
        bk.counters[C_CANCELLED_QTY] += o->qty;
        own.erase(m.oid);
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
        cancel(bk, m);
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
    if (n_books < 0 || capacity < 1 || trade_capacity < 0 || overflow_rule < 0 ||
        overflow_rule > 1)
        return nullptr;
    Engine* E = new Engine();
    E->n_books = n_books;
    E->capacity = capacity;
    E->trade_capacity = trade_capacity;
    E->overflow_rule = overflow_rule;
    E->append_trades = append_trades != 0;
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

// Top `depth` price levels per side: aggregated quantity per distinct price,
// best first; empty levels are (-1, 0).  Quantities saturate at max_int.
void oracle_get_levels(void* h, int32_t depth, int32_t* bid_px, int32_t* bid_qty, int32_t* ask_px,
                       int32_t* ask_qty)
{
    Engine& E = *(Engine*)h;
    for (int32_t b = 0; b < E.n_books; ++b) {
        Book& bk = E.books[(size_t)b];
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
