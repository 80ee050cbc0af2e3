"""Reader for the hand-worked example files in tests/golden/*.lob."""
import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

MSG_DTYPE = np.dtype([("type", "<i4"), ("side", "<i4"), ("price", "<i4"), ("qty", "<i4"),
                      ("oid", "<i4"), ("tid", "<i4"), ("time_ns", "<i8")])


class Case:
    def __init__(self, path):
        self.name = os.path.basename(path)
        self.capacity = None
        self.rule = 0
        self.trade_capacity = 16
        self.cite = ""
        self.msgs = []
        self.bids, self.asks, self.trades = [], [], []
        self.trades_total = None
        self.counters = {}
        self.depth = None
        self.lbid, self.lask = {}, {}
        for raw in open(path):
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            key, *rest = line.split()
            if key == "cite":
                self.cite = line[5:]
                continue
            if key == "counter":
                self.counters[rest[0]] = int(rest[1])
                continue
            vals = [int(v) for v in rest]
            if key == "capacity":
                self.capacity = vals[0]
            elif key == "rule":
                self.rule = vals[0]
            elif key == "trade_capacity":
                self.trade_capacity = vals[0]
            elif key == "msg":
                # file order: T S P Q OID TID TIME -> record order type side price qty oid tid time
                t, s, p, q, oid, tid, tm = vals
                self.msgs.append((t, s, p, q, oid, tid, tm))
            elif key == "bid":
                self.bids.append(tuple(vals))
            elif key == "ask":
                self.asks.append(tuple(vals))
            elif key == "trade":
                self.trades.append(tuple(vals))
            elif key == "trades_total":
                self.trades_total = vals[0]
            elif key == "levels":
                self.depth = vals[0]
            elif key == "lbid":
                self.lbid[vals[0]] = (vals[1], vals[2])
            elif key == "lask":
                self.lask[vals[0]] = (vals[1], vals[2])
            else:
                raise ValueError("%s: unknown record %r" % (path, key))
        assert self.capacity is not None and self.cite, path
        if self.trades_total is None:
            self.trades_total = len(self.trades)

    def message_array(self):
        return np.array(self.msgs, dtype=MSG_DTYPE)


def cases():
    return [Case(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.lob")))]


def side_rows(book, b, side):
    """Live orders of book b, side 0 bids / 1 asks as (P, Q, OID, TID, TIME) tuples."""
    n = int(book["count"][b, side])
    return [(int(book["price"][b, side, j]), int(book["qty"][b, side, j]),
             int(book["oid"][b, side, j]), int(book["tid"][b, side, j]),
             int(book["time_ns"][b, side, j])) for j in range(n)]


def trade_rows(trades, counts, b, cap):
    n = min(int(counts[b]), cap)
    t = trades[b]
    return [(int(t["price"][j]), int(t["qty"][j]), int(t["oid_aggr"][j]), int(t["oid_stand"][j]),
             int(t["tid_aggr"][j]), int(t["tid_stand"][j]), int(t["time_ns"][j]))
            for j in range(n)]
