"""Seeded synthetic order-flow generator (the shared input source).

Stands in for the LOBSTER message files that the paper replays (Sec. 5.1.1,
TSLA 2015-01-02 for Table 6, AMZN April 2021 for the training runs); those
files are not available here.  The generator draws messages
m = [T, S, Q, P, OID, TID, time] (Sec. 4.2, eq. message) and nothing else: it
holds no order-book arithmetic.  Both the CPU checker and the CUDA engine
consume its streams; the host library (C++) and the device library (CUDA)
compile the same ``lobgen_core.h`` so their streams are bit-identical.

Workload recipes (the stated input recipe, see the workload table below):
type mix 55 % limit add / 25 % partial cancel / 12 % delete / 8 % market;
side +-1 with probability 1/2; an exogenous mid walk from 10,000 ticks;
passive limit prices mid -+ (1 + G), G ~ geometric(0.3); 10 % of limits
aggressive at mid +- G; quantity 1 + geometric(0.02); trader id U{1..1000};
time steps 1 + U{0..999} ns; cancels and deletes target an id drawn uniformly
from a bounded pool of remembered limit ids (random replacement once full).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from fractions import Fraction

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
HOST_SO = os.path.join(HERE, "liblobgen_host.so")
CUDA_SO = os.path.join(HERE, "liblobgen_cuda.so")

MSG_DTYPE = np.dtype([("type", "<i4"), ("side", "<i4"), ("price", "<i4"), ("qty", "<i4"),
                      ("oid", "<i4"), ("tid", "<i4"), ("time_ns", "<i8")])
assert MSG_DTYPE.itemsize == 32

T_LIMIT, T_CANCEL, T_DELETE, T_MARKET = 1, 2, 3, 4
BID, ASK = 1, -1

GEO_PX_KMAX = 64
GEO_Q_KMAX = 2000
DEFAULT_POOL = 64
T0_NS = 34_200 * 1_000_000_000  # 09:30:00 in ns after midnight


class Params(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64),
                ("cut_add", ctypes.c_uint32), ("cut_cancel", ctypes.c_uint32),
                ("cut_delete", ctypes.c_uint32), ("cut_mid_down", ctypes.c_uint32),
                ("cut_mid_up", ctypes.c_uint32), ("cut_marketable", ctypes.c_uint32),
                ("start_mid", ctypes.c_int32), ("tid_max", ctypes.c_int32),
                ("dt_max", ctypes.c_int32), ("pool_cap", ctypes.c_int32),
                ("geo_px_kmax", ctypes.c_int32), ("geo_q_kmax", ctypes.c_int32),
                ("t0_ns", ctypes.c_int64), ("first_oid", ctypes.c_int32),
                ("pad_", ctypes.c_int32)]


assert ctypes.sizeof(Params) == 72

STATE_BYTES = 40
POOL_ENTRY_BYTES = 16


def _cut(prob: Fraction) -> int:
    """uint32 cut point floor(prob * 2^32), clamped to the uint32 range."""
    v = math.floor(prob * (1 << 32))
    return max(0, min(v, (1 << 32) - 1))


def geometric_thresholds(p: Fraction, kmax: int) -> np.ndarray:
    """thr[k] = floor(F(k) * 2^64), F(k) = 1 - (1-p)^(k+1): exact rational arithmetic."""
    q = 1 - Fraction(p)
    out = np.empty(kmax, dtype=np.uint64)
    num, den = q.numerator, q.denominator
    pn, pd = num, den  # q^(k+1)
    top = 1 << 64
    for k in range(kmax):
        # floor(2^64 * (1 - pn/pd)) = 2^64 - ceil(2^64*pn/pd)
        c = -((-top * pn) // pd)
        v = top - c
        out[k] = min(v, top - 1)
        pn *= num
        pd *= den
    return out


GEO_PX = geometric_thresholds(Fraction(3, 10), GEO_PX_KMAX)
GEO_Q = geometric_thresholds(Fraction(2, 100), GEO_Q_KMAX)


def make_params(seed: int, mid_walk: str = "pm1", pool_cap: int = DEFAULT_POOL) -> Params:
    """Stream parameters.  mid_walk 'pm1': +-1 tick with 1/2 each;
    'three': {-1, 0, +1} with (0.2, 0.6, 0.2)."""
    p = Params()
    p.seed = seed & ((1 << 64) - 1)
    p.cut_add = _cut(Fraction(55, 100))
    p.cut_cancel = _cut(Fraction(80, 100))
    p.cut_delete = _cut(Fraction(92, 100))
    if mid_walk == "pm1":
        p.cut_mid_down = _cut(Fraction(1, 2))
        p.cut_mid_up = _cut(Fraction(1, 2))
    elif mid_walk == "three":
        p.cut_mid_down = _cut(Fraction(2, 10))
        p.cut_mid_up = _cut(Fraction(8, 10))
    elif mid_walk == "none":
        p.cut_mid_down = 0
        p.cut_mid_up = (1 << 32) - 1
    else:
        raise ValueError(mid_walk)
    p.cut_marketable = _cut(Fraction(1, 10))
    p.start_mid = 10_000
    p.tid_max = 1000
    p.dt_max = 1000
    p.pool_cap = pool_cap
    p.geo_px_kmax = GEO_PX_KMAX
    p.geo_q_kmax = GEO_Q_KMAX
    p.t0_ns = T0_NS
    p.first_oid = 1
    return p


# Workloads (sizes of the paper-style experiments; seeds fixed per workload).
WORKLOADS = {
    # 16 books x 10^4 messages, capacity 100, mid +-1
    "small_16x10k": dict(n_books=16, msgs=10_000, capacity=100, mid_walk="pm1", seed=20230825),
    # 1,024 books x 10^5 messages, capacity 100, mid {-1,0,+1} (0.2,0.6,0.2); plain form
    # launches once per 100-message chunk
    "replay_1024x100k": dict(n_books=1024, msgs=100_000, capacity=100, mid_walk="three",
                             seed=20230826, chunk=100),
    # profiling case: the same books and generator with 10^4 messages per book
    # (328 MB of messages, still larger than L2)
    "replay_1024x10k": dict(n_books=1024, msgs=10_000, capacity=100, mid_walk="three",
                            seed=20230826, chunk=100),
    # 4,096 books, lognormal(ln 1e4, 1.0) counts clipped to [1e3, 2e5], capacity 100
    "uneven_4096_lognormal": dict(n_books=4096, msgs=None, capacity=100, mid_walk="pm1",
                                  seed=20230827),
    # 8,192 RL envs x 400 steps x 100 replay messages (+ 1..4 agent orders), capacity 100
    "rl_exec_8192x400": dict(n_books=8192, steps=400, msgs_per_step=100, capacity=100,
                             mid_walk="pm1", seed=20230828),
    # profiling case: the RL workload cut to 40 steps
    "rl_exec_8192x40": dict(n_books=8192, steps=40, msgs_per_step=100, capacity=100,
                            mid_walk="pm1", seed=20230828),
    # serving mix: Poisson 2,000 episodes/s, capacity {100,250,500}, 200..2,000 steps,
    # 100..500 messages per step
    "serving_mix": dict(rate=2000.0, capacities=(100, 250, 500), steps=(200, 2000),
                        msgs_per_step=(100, 500), mid_walk="pm1", seed=20230829),
}


def lognormal_counts(n_books: int, seed: int, mu: float = math.log(1e4), sigma: float = 1.0,
                     lo: int = 1_000, hi: int = 200_000) -> np.ndarray:
    """Per-book message counts round(exp(mu + sigma*Z)) clipped to [lo, hi];
    Z by Box-Muller from a seeded numpy PCG64 stream (host only)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u1 = rng.random(n_books)
    u2 = rng.random(n_books)
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    c = np.rint(np.exp(mu + sigma * z)).astype(np.int64)
    return np.clip(c, lo, hi)


# --------------------------------------------------------------------------- build / load

def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))


def build(cuda: bool = True, force: bool = False) -> None:
    """Compile the host library (g++) and, when asked, the device library (nvcc, sm_103a)."""
    src_h = os.path.join(HERE, "lobgen_host.cpp")
    core = os.path.join(HERE, "lobgen_core.h")
    newest = max(os.path.getmtime(src_h), os.path.getmtime(core))
    if force or not os.path.exists(HOST_SO) or os.path.getmtime(HOST_SO) < newest:
        _run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
              "-o", HOST_SO, src_h])
    if cuda:
        src_d = os.path.join(HERE, "lobgen_dev.cu")
        newest_d = max(os.path.getmtime(src_d), os.path.getmtime(core))
        if force or not os.path.exists(CUDA_SO) or os.path.getmtime(CUDA_SO) < newest_d:
            _run(["nvcc", "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
                  "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
                  "-o", CUDA_SO, src_d])


_host = None
_cuda = None


def host_lib():
    global _host
    if _host is None:
        if not os.path.exists(HOST_SO):
            build(cuda=False)
        lib = ctypes.CDLL(HOST_SO)
        vp = ctypes.c_void_p
        lib.lobgen_init.argtypes = [vp, ctypes.c_int32, vp, vp]
        lib.lobgen_advance.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp, vp, vp, vp,
                                       ctypes.c_int32]
        lib.lobgen_generate.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp, vp, ctypes.c_int32]
        lib.lobgen_agent_draws.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, vp]
        _host = lib
    return _host


def cuda_lib():
    global _cuda
    if _cuda is None:
        if not os.path.exists(CUDA_SO):
            raise RuntimeError("liblobgen_cuda.so is not built (run lobgen.build())")
        lib = ctypes.CDLL(CUDA_SO)
        vp = ctypes.c_void_p
        lib.lobgen_dev_init.argtypes = [vp, ctypes.c_int32, vp, vp, vp]
        lib.lobgen_dev_advance.argtypes = [vp, vp, vp, ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp]
        lib.lobgen_dev_init_ids.argtypes = [vp, ctypes.c_int32, vp, vp, vp, vp]
        lib.lobgen_dev_agent_draws.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.c_int32, vp, vp]
        _cuda = lib
    return _cuda


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def offsets_from_counts(counts) -> np.ndarray:
    counts = np.asarray(counts, dtype=np.int64)
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return off


def generate(params: Params, counts, stream_ids=None, threads: int | None = None) -> tuple:
    """Fresh streams: book b gets counts[b] messages.  Returns (msgs, offsets)."""
    lib = host_lib()
    counts = np.asarray(counts, dtype=np.int64)
    n = len(counts)
    off = offsets_from_counts(counts)
    out = np.empty(int(off[-1]), dtype=MSG_DTYPE)
    sid = None
    if stream_ids is not None:
        sid = np.ascontiguousarray(stream_ids, dtype=np.uint64)
    rc = lib.lobgen_generate(ctypes.byref(params), _ptr(GEO_PX), _ptr(GEO_Q), n,
                             _ptr(sid) if sid is not None else None, _ptr(off),
                             _ptr(out) if len(out) else None,
                             threads or default_threads())
    if rc != 0:
        raise RuntimeError("lobgen_generate failed (%d)" % rc)
    return out, off


class HostStreams:
    """Resumable host streams (e.g. one RL step or one serving step at a time)."""

    def __init__(self, params: Params, n_books: int, stream_ids=None):
        self.params = params
        self.n = n_books
        self.states = np.zeros(n_books * STATE_BYTES, dtype=np.uint8)
        self.pools = np.zeros(n_books * params.pool_cap * POOL_ENTRY_BYTES, dtype=np.uint8)
        self.sid = (np.ascontiguousarray(stream_ids, dtype=np.uint64)
                    if stream_ids is not None else None)
        rc = host_lib().lobgen_init(ctypes.byref(params), n_books,
                                    _ptr(self.sid) if self.sid is not None else None,
                                    _ptr(self.states))
        if rc != 0:
            raise RuntimeError("lobgen_init failed")

    def advance(self, counts, threads: int | None = None):
        counts = np.ascontiguousarray(counts, dtype=np.int64)
        off = offsets_from_counts(counts)
        out = np.empty(int(off[-1]), dtype=MSG_DTYPE)
        rc = host_lib().lobgen_advance(ctypes.byref(self.params), _ptr(GEO_PX), _ptr(GEO_Q),
                                       self.n, _ptr(self.states), _ptr(self.pools),
                                       _ptr(counts), _ptr(off),
                                       _ptr(out) if len(out) else _ptr(np.empty(1, MSG_DTYPE)),
                                       threads or default_threads())
        if rc != 0:
            raise RuntimeError("lobgen_advance failed")
        return out, off


def agent_draws(seed: int, n_envs: int, n_steps: int) -> np.ndarray:
    """[n_steps, n_envs] uint32 packed agent draws (see lobgen_core.h)."""
    out = np.empty((n_steps, n_envs), dtype=np.uint32)
    rc = host_lib().lobgen_agent_draws(seed & ((1 << 64) - 1), n_envs, n_steps, _ptr(out))
    if rc != 0:
        raise RuntimeError("lobgen_agent_draws failed")
    return out


def decode_agent_draw(w: int):
    """(n_orders, [action codes]) from one packed agent draw."""
    n = (w & 3) + 1
    return n, [(w >> (2 + 3 * k)) & 7 for k in range(4)]


class DeviceStreams:
    """Resumable streams generated on the GPU (same definition as the host
    side, bit for bit).  Memory is torch-allocated on the current device."""

    def __init__(self, params: Params, n_books: int, stream_ids=None):
        import torch
        self.torch = torch
        self.params = params
        self.n = n_books
        lib = cuda_lib()
        self.lib = lib
        dev = "cuda"
        self.states = torch.zeros(n_books * STATE_BYTES, dtype=torch.uint8, device=dev)
        self.pools = torch.zeros(n_books * params.pool_cap * POOL_ENTRY_BYTES, dtype=torch.uint8,
                                 device=dev)
        self.geo_px = torch.from_numpy(GEO_PX.view(np.int64)).to(dev)
        self.geo_q = torch.from_numpy(GEO_Q.view(np.int64)).to(dev)
        self.sid = None
        if stream_ids is not None:
            self.sid = torch.from_numpy(np.ascontiguousarray(stream_ids, dtype=np.uint64)
                                        .view(np.int64)).to(dev)
        rc = lib.lobgen_dev_init(ctypes.byref(params), n_books,
                                 ctypes.c_void_p(self.sid.data_ptr()) if self.sid is not None
                                 else None, ctypes.c_void_p(self.states.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            raise RuntimeError("lobgen_dev_init failed (%d)" % rc)

    def restart(self, ids, stream_ids):
        """Books ids[i] restart as streams stream_ids[i] (device tensors or arrays)."""
        torch = self.torch
        idt = torch.as_tensor(np.asarray(ids, dtype=np.int32)).cuda()
        sid = torch.as_tensor(np.asarray(stream_ids, dtype=np.uint64).view(np.int64)).cuda()
        rc = self.lib.lobgen_dev_init_ids(ctypes.byref(self.params), idt.numel(),
                                          ctypes.c_void_p(idt.data_ptr()),
                                          ctypes.c_void_p(sid.data_ptr()),
                                          ctypes.c_void_p(self.states.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            raise RuntimeError("lobgen_dev_init_ids failed (%d)" % rc)

    def advance(self, counts, ids=None, out=None):
        """Draw counts[i] messages for book ids[i] (or i); returns (int32 [N, 8]
        CUDA tensor, int64 CUDA offsets)."""
        torch = self.torch
        counts = torch.as_tensor(counts, dtype=torch.int64).cuda()
        off = torch.zeros(counts.numel() + 1, dtype=torch.int64, device="cuda")
        torch.cumsum(counts, 0, out=off[1:])
        total = int(off[-1].item())
        if out is None:
            out = torch.empty((max(total, 1), 8), dtype=torch.int32, device="cuda")
        idt = None if ids is None else torch.as_tensor(ids, dtype=torch.int32).cuda()
        p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        rc = self.lib.lobgen_dev_advance(ctypes.byref(self.params), p(self.geo_px), p(self.geo_q),
                                         counts.numel(), p(idt), p(self.states), p(self.pools),
                                         p(counts), p(off), p(out),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc != 0:
            raise RuntimeError("lobgen_dev_advance failed (%d)" % rc)
        return out[:total], off


def agent_draws_device(seed: int, n_envs: int, n_steps: int, step0: int = 0):
    """[n_steps, n_envs] agent draws generated on the GPU (int32 view of uint32)."""
    import torch
    out = torch.empty((n_steps, n_envs), dtype=torch.int32, device="cuda")
    rc = cuda_lib().lobgen_dev_agent_draws(seed & ((1 << 64) - 1), n_envs, step0, n_steps,
                                           ctypes.c_void_p(out.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if rc != 0:
        raise RuntimeError("lobgen_dev_agent_draws failed (%d)" % rc)
    return out
