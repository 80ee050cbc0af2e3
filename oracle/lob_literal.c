/*
 * lob_literal.c -- paper-literal array formulation (second CPU implementation).
 *
 * TEST INFRASTRUCTURE ONLY.  An independent restatement of the same method in
 * the form the paper itself describes, used to cross-check the ordered-map
 * oracle (lob_oracle.cpp) by brute force on tiny books.  It shares no code with
 * that oracle or with the CUDA engine.
 *
 *   Sec. 4, eqs. 1-2: each side is an UNSORTED array of N slots
 *       o_i = [P_i, Q_i, OID_i, TID_i, time_i]; an empty slot has every
 *       feature set to -1.
 *   Sec. 4.1 item 1 (add): find an empty slot (o_i = -1) and write the order.
 *   Sec. 4.1 item 2 (cancel): scan for OID and subtract the quantity.
 *   Sec. 4.1 item 3 (match): repeatedly pick Best(o_s) by a full scan --
 *       lowest ask / highest bid price, earliest arrival among equal prices --
 *       while Q_a > 0, the side is non-empty and the prices cross; apply
 *       Q_s' = max(0, Q_s - Q_a), Q_a' = Q_a - Q_s; log
 *       t = [P_s, Q_s - Q_s', OID_a, OID_s, time_a].
 *   Sec. 4.1 (cleanup): after every operation every slot with Q <= 0 is
 *       reset to all -1.
 *   Sec. 4.2: limit = match then add the rest; cancel = delete; market =
 *       match at price 0 (sell) / max_int (buy), rest dropped.
 *
 * Where the paper is silent this file takes the same readings as the oracle:
 * "earliest arrival" is arrival order (a hidden arrival counter, never the
 * time stamp); a full side evicts its worst order (worst price, latest
 * arrival) when the residual's price is strictly better, else rejects
 * (rule 0), or always rejects (rule 1); type 0 is padding; malformed
 * messages are skipped.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t type, side, price, qty, oid, tid;
    int64_t time_ns;
} lit_msg;

typedef struct {
    int32_t price, qty, oid_aggr, oid_stand, tid_aggr, tid_stand;
    int64_t time_ns;
} lit_trade;

typedef struct {
    int32_t P, Q, OID, TID;
    int64_t T;
    int64_t arrival; /* hidden: arrival counter used for time priority */
} lit_order;

enum { L_MSGS = 0, L_LIMIT, L_CANCEL, L_MARKET, L_NOOP, L_INVALID, L_TRADES, L_TRADED_QTY,
       L_RESTED, L_REJECTED, L_REJECTED_QTY, L_EVICTED, L_EVICTED_QTY, L_CANCEL_HIT,
       L_CANCELLED_QTY, L_CANCEL_MISS, L_MARKET_DISCARDED_QTY, L_LIMIT_QTY, L_MARKET_QTY,
       L_TRADES_DROPPED, L_N };

typedef struct {
    int32_t N, trade_cap, rule;
    lit_order* A; /* asks */
    lit_order* B; /* bids */
    lit_trade* trades;
    int64_t n_trades;
    int64_t arrival;
    int64_t* c; /* counters */
} lit_book;

static int is_empty(const lit_order* o) { return o->OID == -1 && o->Q == -1 && o->P == -1; }

static void set_empty(lit_order* o)
{
    o->P = -1; o->Q = -1; o->OID = -1; o->TID = -1; o->T = -1; o->arrival = -1;
}

/* Best(o): lowest price on the ask array, highest on the bid array; among
 * equal prices the earliest arrival.  Returns the slot or -1 when empty. */
static int best_slot(const lit_order* S, int32_t N, int is_bid)
{
    int best = -1;
    for (int i = 0; i < N; ++i) {
        if (is_empty(&S[i])) continue;
        if (best < 0) { best = i; continue; }
        int better = is_bid ? S[i].P > S[best].P : S[i].P < S[best].P;
        int same = S[i].P == S[best].P;
        if (better || (same && S[i].arrival < S[best].arrival)) best = i;
    }
    return best;
}

/* worst order: worst price, latest arrival among equal prices */
static int worst_slot(const lit_order* S, int32_t N, int is_bid)
{
    int w = -1;
    for (int i = 0; i < N; ++i) {
        if (is_empty(&S[i])) continue;
        if (w < 0) { w = i; continue; }
        int worse = is_bid ? S[i].P < S[w].P : S[i].P > S[w].P;
        int same = S[i].P == S[w].P;
        if (worse || (same && S[i].arrival > S[w].arrival)) w = i;
    }
    return w;
}

static void cleanup(lit_book* bk)
{
    for (int i = 0; i < bk->N; ++i) {
        if (!is_empty(&bk->A[i]) && bk->A[i].Q <= 0) set_empty(&bk->A[i]);
        if (!is_empty(&bk->B[i]) && bk->B[i].Q <= 0) set_empty(&bk->B[i]);
    }
}

static void log_trade(lit_book* bk, lit_trade t)
{
    if (bk->n_trades < bk->trade_cap) bk->trades[bk->n_trades] = t;
    else bk->c[L_TRADES_DROPPED] += 1;
    bk->n_trades += 1;
    bk->c[L_TRADES] += 1;
    bk->c[L_TRADED_QTY] += t.qty;
}

/* matching loop; returns max(0, Q_a) */
static int32_t match(lit_book* bk, const lit_msg* m, int32_t P_a)
{
    lit_order* S = m->side == 1 ? bk->A : bk->B; /* standing side */
    int is_bid = m->side == 1 ? 0 : 1;
    int32_t Q_a = m->qty;
    for (;;) {
        int s = best_slot(S, bk->N, is_bid);
        if (s < 0 || Q_a <= 0) break;
        int cross = m->side == -1 ? (P_a <= S[s].P) : (P_a >= S[s].P);
        if (!cross) break;
        int32_t Q_s = S[s].Q;
        int32_t Q_s_new = Q_s - Q_a > 0 ? Q_s - Q_a : 0;
        int32_t Q_a_new = Q_a - Q_s;
        lit_trade t;
        t.price = S[s].P;
        t.qty = Q_s - Q_s_new;
        t.oid_aggr = m->oid;
        t.oid_stand = S[s].OID;
        t.tid_aggr = m->tid;
        t.tid_stand = S[s].TID;
        t.time_ns = m->time_ns;
        log_trade(bk, t);
        S[s].Q = Q_s_new;
        Q_a = Q_a_new;
        cleanup(bk);
    }
    return Q_a > 0 ? Q_a : 0;
}

static void add(lit_book* bk, const lit_msg* m, int32_t Q)
{
    lit_order* S = m->side == 1 ? bk->B : bk->A;
    int is_bid = m->side == 1;
    int slot = -1;
    for (int i = 0; i < bk->N; ++i)
        if (is_empty(&S[i])) { slot = i; break; }
    if (slot < 0) {
        int w = worst_slot(S, bk->N, is_bid);
        int better = is_bid ? m->price > S[w].P : m->price < S[w].P;
        if (bk->rule == 0 && better) {
            bk->c[L_EVICTED] += 1;
            bk->c[L_EVICTED_QTY] += S[w].Q;
            set_empty(&S[w]);
            slot = w;
        } else {
            bk->c[L_REJECTED] += 1;
            bk->c[L_REJECTED_QTY] += Q;
            return;
        }
    }
    S[slot].P = m->price;
    S[slot].Q = Q;
    S[slot].OID = m->oid;
    S[slot].TID = m->tid;
    S[slot].T = m->time_ns;
    S[slot].arrival = bk->arrival++;
    bk->c[L_RESTED] += 1;
}

static void cancel(lit_book* bk, const lit_msg* m)
{
    lit_order* S = m->side == 1 ? bk->B : bk->A;
    for (int i = 0; i < bk->N; ++i) {
        if (!is_empty(&S[i]) && S[i].OID == m->oid) {
            bk->c[L_CANCEL_HIT] += 1;
            bk->c[L_CANCELLED_QTY] += S[i].Q < m->qty ? S[i].Q : m->qty;
            S[i].Q -= m->qty;
            cleanup(bk);
            return;
        }
    }
    bk->c[L_CANCEL_MISS] += 1;
}

static void process(lit_book* bk, const lit_msg* m)
{
    bk->c[L_MSGS] += 1;
    if (m->type == 0) { bk->c[L_NOOP] += 1; return; }
    if (m->type < 0 || m->type > 4 || (m->side != 1 && m->side != -1) || m->qty <= 0 ||
        (m->type == 1 && m->price <= 0)) {
        bk->c[L_INVALID] += 1;
        return;
    }
    if (m->type == 1) {
        bk->c[L_LIMIT] += 1;
        bk->c[L_LIMIT_QTY] += m->qty;
        int32_t rest = match(bk, m, m->price);
        if (rest > 0) add(bk, m, rest);
    } else if (m->type == 2 || m->type == 3) {
        bk->c[L_CANCEL] += 1;
        cancel(bk, m);
    } else {
        bk->c[L_MARKET] += 1;
        bk->c[L_MARKET_QTY] += m->qty;
        int32_t rest = match(bk, m, m->side == -1 ? 0 : 2147483647);
        bk->c[L_MARKET_DISCARDED_QTY] += rest;
    }
    cleanup(bk);
}

static int cmp_bid(const void* a, const void* b)
{
    const lit_order *x = a, *y = b;
    if (x->P != y->P) return x->P > y->P ? -1 : 1;
    return x->arrival < y->arrival ? -1 : 1;
}

static int cmp_ask(const void* a, const void* b)
{
    const lit_order *x = a, *y = b;
    if (x->P != y->P) return x->P < y->P ? -1 : 1;
    return x->arrival < y->arrival ? -1 : 1;
}

int literal_n_counters(void) { return L_N; }

/* Run every book from empty over its whole stream.
 * book outputs: [n_books][2][N] (side 0 bids, 1 asks) in priority order, -1
 * padded; count[n_books][2]; trades[n_books][trade_cap] (-1 padded);
 * n_trades[n_books]; counters[n_books][L_N]. */
int literal_run(const lit_msg* msgs, const int64_t* offsets, int32_t n_books, int32_t N,
                int32_t trade_cap, int32_t rule, int32_t* px, int32_t* qty, int32_t* oid,
                int32_t* tid, int64_t* tm, int32_t* count, lit_trade* trades, int64_t* n_trades,
                int64_t* counters)
{
    if (N < 1 || trade_cap < 0 || n_books < 0) return -1;
    lit_order* A = malloc(sizeof(lit_order) * (size_t)N);
    lit_order* B = malloc(sizeof(lit_order) * (size_t)N);
    lit_order* tmp = malloc(sizeof(lit_order) * (size_t)N);
    if (!A || !B || !tmp) { free(A); free(B); free(tmp); return -2; }
    for (int32_t b = 0; b < n_books; ++b) {
        lit_book bk;
        bk.N = N; bk.trade_cap = trade_cap; bk.rule = rule; bk.A = A; bk.B = B;
        bk.trades = trades + (int64_t)b * trade_cap;
        bk.n_trades = 0;
        bk.arrival = 0;
        bk.c = counters + (int64_t)b * L_N;
        memset(bk.c, 0, sizeof(int64_t) * L_N);
        memset(bk.trades, 0xff, sizeof(lit_trade) * (size_t)trade_cap);
        for (int i = 0; i < N; ++i) { set_empty(&A[i]); set_empty(&B[i]); }
        for (int64_t k = offsets[b]; k < offsets[b + 1]; ++k) process(&bk, &msgs[k]);
        n_trades[b] = bk.n_trades;
        for (int s = 0; s < 2; ++s) {
            lit_order* S = s == 0 ? B : A;
            int n = 0;
            for (int i = 0; i < N; ++i)
                if (!is_empty(&S[i])) tmp[n++] = S[i];
            qsort(tmp, (size_t)n, sizeof(lit_order), s == 0 ? cmp_bid : cmp_ask);
            int64_t base = ((int64_t)b * 2 + s) * N;
            for (int i = 0; i < N; ++i) {
                int live = i < n;
                px[base + i] = live ? tmp[i].P : -1;
                qty[base + i] = live ? tmp[i].Q : -1;
                oid[base + i] = live ? tmp[i].OID : -1;
                tid[base + i] = live ? tmp[i].TID : -1;
                tm[base + i] = live ? tmp[i].T : -1;
            }
            count[b * 2 + s] = n;
        }
    }
    free(A); free(B); free(tmp);
    return 0;
}
