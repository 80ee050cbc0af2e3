// lob_engine.cu -- C ABI of the batched order-book engine and its small
// kernels (levels, book dump and load, snapshot initialisation, resets, trade
// log copy).  The processing kernel itself is in lob_process.cuh.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <new>
#include <string>

#include "../../include/lob.h"
#include "lob_core.cuh"
#include "lob_engine.h"
#include "lob_process.cuh"

using namespace lob;

static_assert(sizeof(lob_msg_t) == sizeof(Msg), "lob_msg_t layout");
static_assert(sizeof(lob_trade_t) == sizeof(Trade), "lob_trade_t layout");
static_assert(LOB_N_COUNTERS == kNumCtr, "counter count");

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

void lob_set_error(const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

int lob_cuda_fail(cudaError_t e, const char* where)
{
    lob_set_error("%s: %s", where, cudaGetErrorString(e));
    return LOB_E_CUDA;
}

// The dynamic shared-memory limit is an attribute of the kernel function, shared
// by every context in the process: only ever raise it, so that configuring one
// context never invalidates the launch shape of another.
cudaError_t lob_raise_smem_limit(const void* fn, int bytes)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> current;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int& cur = current[std::make_pair(dev, fn)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

// ------------------------------------------------------------------ kernels

namespace {

// Top `depth` levels (warp per book, both sides) of every book, or of the
// `n_items` books listed in `book_ids` (an id outside 0..n_books-1 sets
// LOB_STATUS_BAD_BOOK and is skipped).
template <int K>
__global__ void k_levels(const char* __restrict__ state, const int32_t* __restrict__ counts,
                         int32_t n_books, const int32_t* __restrict__ book_ids, int32_t n_items,
                         int32_t* status, int32_t depth, int32_t* bid_px, int32_t* bid_qty,
                         int32_t* ask_px, int32_t* ask_qty)
{
    __shared__ unsigned long long lq[8][128];
    __shared__ int32_t lp[8][64];
    const int l = lane_id(), w = threadIdx.x >> 5;
    const int item = blockIdx.x * (blockDim.x >> 5) + w;
    if (item >= n_items) return;
    const int b = book_ids ? book_ids[item] : item;
    if (b < 0 || b >= n_books) {
        if (l == 0) atomicOr(status, LOB_STATUS_BAD_BOOK);
        return;
    }
    for (int x = 0; x < 2; ++x) {
        const char* side = state + (int64_t)b * Geo<K>::BOOK_BYTES + x * Geo<K>::SIDE_BYTES;
        const int32_t* px = reinterpret_cast<const int32_t*>(side + Geo<K>::PX);
        const int32_t* q = reinterpret_cast<const int32_t*>(side + Geo<K>::QTY);
        const int n = counts[2 * b + x];
        int32_t vpx[K], vq[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {  // priority rank l*K + j
            const int r = l * K + j;
            const int i = r < n ? storage_index<K>(r, n) : 0;
            vpx[j] = px[i];
            vq[j] = q[i];
        }
        emit_levels<K>(vpx, vq, n, depth, lq[w], lp[w],
                       (x == 0 ? bid_px : ask_px) + (int64_t)b * depth,
                       (x == 0 ? bid_qty : ask_qty) + (int64_t)b * depth);
    }
}

// Canonical dump: thread per (book, side, slot < cap).
template <int K>
__global__ void k_get_book(const char* __restrict__ state, const int32_t* __restrict__ counts,
                           int32_t n_books, int32_t cap, int32_t* px, int32_t* qty, int32_t* oid,
                           int32_t* tid, int64_t* tm, int32_t* count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)n_books * 2 * cap;
    if (i >= total) return;
    const int s = (int)(i % cap);
    const int64_t bx = i / cap;  // book*2 + side
    const int x = (int)(bx & 1);
    const int64_t b = bx >> 1;
    const char* side = state + b * Geo<K>::BOOK_BYTES + x * Geo<K>::SIDE_BYTES;
    const int n = counts[bx];
    const bool live = s < n;
    const int k = live ? storage_index<K>(s, n) : 0;  // priority rank s
    if (px) px[i] = live ? reinterpret_cast<const int32_t*>(side + Geo<K>::PX)[k] : -1;
    if (qty) qty[i] = live ? reinterpret_cast<const int32_t*>(side + Geo<K>::QTY)[k] : -1;
    if (oid) oid[i] = live ? reinterpret_cast<const int32_t*>(side + Geo<K>::OID)[k] : -1;
    if (tid) tid[i] = live ? reinterpret_cast<const int32_t*>(side + Geo<K>::TID)[k] : -1;
    if (tm) tm[i] = live ? reinterpret_cast<const int64_t*>(side + Geo<K>::TM)[k] : -1;
    if (count && s == 0) count[bx] = counts[bx];
}

// Load books from the canonical layout; warp per (book, side).
template <int K>
__global__ void k_set_book(char* state, int32_t* counts, int32_t n_books, int32_t cap,
                           const int32_t* __restrict__ px, const int32_t* __restrict__ qty,
                           const int32_t* __restrict__ oid, const int32_t* __restrict__ tid,
                           const int64_t* __restrict__ tm, const int32_t* __restrict__ count,
                           int32_t* status)
{
    const int l = lane_id();
    const int64_t bx = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (bx >= (int64_t)n_books * 2) return;
    const int x = (int)(bx & 1);
    const int64_t b = bx >> 1;
    int n = count[bx];
    const int64_t base = bx * cap;
    bool bad = n < 0 || n > cap;
    if (!bad) {
        for (int s = l; s < n; s += 32) {
            const int32_t p = px[base + s];
            bool ok = p > 0 && qty[base + s] > 0;
            if (s > 0) {
                const int32_t pp = px[base + s - 1];
                ok = ok && (x == 0 ? p <= pp : p >= pp);
            }
            if (!ok) bad = true;
        }
    }
    bad = __any_sync(kFull, bad);
    if (bad) {
        n = 0;
        if (l == 0) atomicOr(status, LOB_STATUS_BAD_BOOK_LOAD);
    }
    char* side = state + b * Geo<K>::BOOK_BYTES + x * Geo<K>::SIDE_BYTES;
    for (int s = l; s < n; s += 32) {  // priority rank s
        const int k = storage_index<K>(s, n);
        reinterpret_cast<int32_t*>(side + Geo<K>::PX)[k] = px[base + s];
        reinterpret_cast<int32_t*>(side + Geo<K>::QTY)[k] = qty[base + s];
        reinterpret_cast<int32_t*>(side + Geo<K>::OID)[k] = oid[base + s];
        reinterpret_cast<int32_t*>(side + Geo<K>::TID)[k] = tid[base + s];
        reinterpret_cast<int64_t*>(side + Geo<K>::TM)[k] = tm[base + s];
    }
    if (l == 0) counts[bx] = n;
}

// Books from a level snapshot (Sec. 5.1.1), warp per book: each side's listed
// levels (those before the first with price or volume <= 0) become one order
// each, in listed order, OIDs -9000 downward over the bid levels then the ask
// levels, TID 0, time `time_ns`.  A side listed out of priority order is
// loaded empty (LOB_STATUS_BAD_BOOK_LOAD).  depth <= capacity (host check).
template <int K>
__global__ void k_init_from_levels(char* state, int32_t* counts, int32_t n_books, int32_t depth,
                                   const int32_t* __restrict__ bid_px,
                                   const int32_t* __restrict__ bid_qty,
                                   const int32_t* __restrict__ ask_px,
                                   const int32_t* __restrict__ ask_qty, int64_t time_ns,
                                   int32_t* status)
{
    const int l = lane_id();
    const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (b >= n_books) return;
    int32_t oid_next = kSnapshotOidMax;  // first snapshot OID, -9000
    for (int x = 0; x < 2; ++x) {
        const int32_t* px = (x == 0 ? bid_px : ask_px) + b * depth;
        const int32_t* qt = (x == 0 ? bid_qty : ask_qty) + b * depth;
        // listed levels: the prefix before the first level with P <= 0 or Q <= 0
        int n = 0;
        for (int k0 = 0; k0 < depth; k0 += 32) {
            const int k = k0 + l;
            const bool ok = k < depth && px[k] > 0 && qt[k] > 0;
            const unsigned gap = ~__ballot_sync(kFull, ok);
            const int m = gap ? __ffs(gap) - 1 : 32;
            n += m;
            if (m < 32) break;
        }
        // priority order: bids non-increasing, asks non-decreasing
        bool bad = false;
        for (int k = 1 + l; k < n; k += 32)
            bad = bad || (x == 0 ? px[k] > px[k - 1] : px[k] < px[k - 1]);
        bad = __any_sync(kFull, bad);
        char* side = state + b * Geo<K>::BOOK_BYTES + x * Geo<K>::SIDE_BYTES;
        const int n_load = bad ? 0 : n;
        for (int r = l; r < n_load; r += 32) {  // priority rank r = listed level r
            const int i = storage_index<K>(r, n_load);
            reinterpret_cast<int32_t*>(side + Geo<K>::PX)[i] = px[r];
            reinterpret_cast<int32_t*>(side + Geo<K>::QTY)[i] = qt[r];
            reinterpret_cast<int32_t*>(side + Geo<K>::OID)[i] = oid_next - r;
            reinterpret_cast<int32_t*>(side + Geo<K>::TID)[i] = 0;
            reinterpret_cast<int64_t*>(side + Geo<K>::TM)[i] = time_ns;
        }
        oid_next -= n;  // the OIDs count every listed level, loaded or not
        if (l == 0) {
            counts[2 * b + x] = n_load;
            if (bad) atomicOr(status, LOB_STATUS_BAD_BOOK_LOAD);
        }
    }
}

__global__ void k_reset_books(const int32_t* __restrict__ ids, int32_t n, int32_t n_books,
                              int32_t* counts, int64_t* tcounts, int64_t* stats, int32_t* status)
{
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t b = ids[i];
    if (b < 0 || b >= n_books) {
        atomicOr(status, LOB_STATUS_BAD_BOOK);
        return;
    }
    counts[2 * b] = 0;
    counts[2 * b + 1] = 0;
    tcounts[b] = 0;
    for (int k = 0; k < kNumCtr; ++k) stats[(int64_t)b * kNumCtr + k] = 0;
}

__global__ void k_get_trades(const Trade* __restrict__ log, const int64_t* __restrict__ tcounts,
                             int32_t n_books, int32_t cap, Trade* out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_books * cap) return;
    const int64_t b = i / cap, j = i % cap;
    const int4* src = reinterpret_cast<const int4*>(log + i);
    int4* dst = reinterpret_cast<int4*>(out + i);
    if (j < tcounts[b]) {
        dst[0] = src[0];
        dst[1] = src[1];
    } else {
        dst[0] = make_int4(-1, -1, -1, -1);
        dst[1] = make_int4(-1, -1, -1, -1);
    }
}

// ---------------------------------------------------------- dispatch by K

int k_of(int capacity)
{
    if (capacity <= 32) return 1;
    if (capacity <= 64) return 2;
    if (capacity <= 128) return 4;
    if (capacity <= 256) return 8;
    return 16;
}

const void* process_kernel(int K, bool trace = false, bool snap = false)
{
#define LOB_PROC_K(k)                                                                  \
    return trace ? (snap ? reinterpret_cast<const void*>(&k_process<k, true, true>)     \
                         : reinterpret_cast<const void*>(&k_process<k, true, false>))   \
                 : (snap ? reinterpret_cast<const void*>(&k_process<k, false, true>)    \
                         : reinterpret_cast<const void*>(&k_process<k, false, false>))
    switch (K) {
    case 1: LOB_PROC_K(1);
    case 2: LOB_PROC_K(2);
    case 4: LOB_PROC_K(4);
    case 8: LOB_PROC_K(8);
    default: LOB_PROC_K(16);
    }
#undef LOB_PROC_K
}

int smem_per_warp(int K, int chunk)
{
    switch (K) {
    case 1: return warp_smem_bytes<1>(chunk);
    case 2: return warp_smem_bytes<2>(chunk);
    case 4: return warp_smem_bytes<4>(chunk);
    case 8: return warp_smem_bytes<8>(chunk);
    default: return warp_smem_bytes<16>(chunk);
    }
}

int max_warps(int K) { return K >= 4 ? 8 : 16; }

}  // namespace

int lob_book_bytes(int K) { return 48 * 32 * K; }

// ---------------------------------------------------------- internal API

int lob_launch_process(lob_ctx* c, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                       const int32_t* d_book_ids, int32_t n_active, int append,
                       cudaStream_t stream, const int64_t* d_counts, int32_t* d_l1)
{
    if (n_active == 0) return LOB_OK;
    ProcArgs a;
    a.msgs = reinterpret_cast<const Msg*>(d_msgs);
    a.offsets = d_offsets;
    a.counts_in = d_counts;
    a.book_ids = d_book_ids;
    a.n_items = n_active;
    a.n_books = c->cfg.n_books;
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
    a.append = append;
    a.chunk = c->chunk;
    a.pad_ = 0;
    a.wait_ns = kWaitNs;
    a.l1 = d_l1;
    const bool snap = (c->cfg.flags & LOB_FLAG_SNAPSHOT_CANCELS) != 0;
    const int W = c->warps_per_cta;
    int grid = (n_active + W - 1) / W;
    const int resident = c->num_sms * c->ctas_per_sm_eff;
    if (grid > resident) grid = resident;
    if (grid < 1) grid = 1;
    void* args[] = {&a};
    const void* fn = process_kernel(c->K, d_l1 != nullptr, snap);
    if (d_l1 || snap) {  // the default instantiation was set up by configure_launch
        cudaError_t ea = lob_raise_smem_limit(fn, c->smem_per_cta);
        if (ea != cudaSuccess) return lob_cuda_fail(ea, "cudaFuncSetAttribute");
    }
    cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(32 * W), args,
                                     (size_t)c->smem_per_cta, stream);
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_process_batch launch");
    c->launches += 1;
    return LOB_OK;
}

static int configure_launch(lob_ctx* c, int W, int chunk, int ctas_per_sm)
{
    if (W > max_warps(c->K)) {
        lob_set_error("at capacity %d at most %d warps per CTA", c->cfg.capacity, max_warps(c->K));
        return LOB_E_INVAL;
    }
    const int smem = smem_per_warp(c->K, chunk) * W;
    int max_optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                           c->device);
    if (e != cudaSuccess) return lob_cuda_fail(e, "cudaDeviceGetAttribute");
    if (smem > max_optin) {
        lob_set_error("launch shape needs %d B of shared memory per CTA (max %d)", smem, max_optin);
        return LOB_E_INVAL;
    }
    const void* fn = process_kernel(c->K);
    e = lob_raise_smem_limit(fn, smem);
    if (e != cudaSuccess) return lob_cuda_fail(e, "cudaFuncSetAttribute");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * W, smem);
    if (e != cudaSuccess) return lob_cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
    if (per_sm < 1) {
        lob_set_error("launch shape does not fit on an SM");
        return LOB_E_INVAL;
    }
    c->warps_per_cta = W;
    c->chunk = chunk;
    c->ctas_per_sm = ctas_per_sm;
    c->ctas_per_sm_eff = ctas_per_sm > 0 ? (ctas_per_sm < per_sm ? ctas_per_sm : per_sm) : per_sm;
    c->smem_per_cta = smem;
    return LOB_OK;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

namespace {

// Self-test of the bounded wait that guards every staged copy: an mbarrier
// that nothing will ever complete, waited on for limit_ns; running out of
// time sets LOB_STATUS_TIMEOUT, as a late copy does in the processing kernels.
__global__ void k_wait_selftest(uint64_t limit_ns, int32_t* status, uint64_t* elapsed_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncwarp();
    const uint64_t t0 = global_ns();
    const bool done = mbar_wait_bounded(&bar, 0, limit_ns);
    if (threadIdx.x == 0) {
        if (!done) atomicOr(status, LOB_STATUS_TIMEOUT);
        if (elapsed_ns) *elapsed_ns = global_ns() - t0;
    }
}

}  // namespace

int lob_selftest_wait(int64_t limit_ns, int32_t* d_status, uint64_t* d_elapsed_ns, void* stream)
{
    if (limit_ns < 1 || limit_ns > 1000000000LL || !d_status) {
        lob_set_error("lob_selftest_wait: limit must be 1 ns .. 1 s and d_status non-null");
        return LOB_E_INVAL;
    }
    k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>((uint64_t)limit_ns, d_status,
                                                        d_elapsed_ns);
    const cudaError_t err = cudaGetLastError();
    return err == cudaSuccess ? LOB_OK : lob_cuda_fail(err, "lob_selftest_wait");
}

int lob_abi_version(void) { return 2; }

const char* lob_last_error(void) { return g_err.c_str(); }

int64_t lob_launch_count(const lob_ctx* c) { return c ? c->launches : -1; }

int lob_create(lob_ctx** out, const lob_config_t* cfg, void* stream)
{
    if (!out || !cfg) {
        lob_set_error("lob_create: null argument");
        return LOB_E_INVAL;
    }
    if (cfg->n_books < 1 || cfg->capacity < 1 || cfg->capacity > 32 * kMaxK ||
        cfg->trade_capacity < 0 || (cfg->overflow_rule != 0 && cfg->overflow_rule != 1) ||
        (cfg->flags & ~(LOB_FLAG_APPEND_TRADES | LOB_FLAG_SNAPSHOT_CANCELS))) {
        lob_set_error("lob_create: invalid configuration (n_books=%d capacity=%d "
                      "trade_capacity=%d overflow_rule=%d flags=%d)",
                      cfg->n_books, cfg->capacity, cfg->trade_capacity, cfg->overflow_rule,
                      cfg->flags);
        return LOB_E_INVAL;
    }
    lob_ctx* c = new (std::nothrow) lob_ctx();
    if (!c) {
        lob_set_error("lob_create: host allocation failed");
        return LOB_E_NOMEM;
    }
    c->cfg = *cfg;
    c->K = k_of(cfg->capacity);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        delete c;
        return lob_cuda_fail(e, "lob_create");
    }
    const int64_t nb = cfg->n_books;
    const size_t state_b = (size_t)nb * lob_book_bytes(c->K);
    const size_t trade_b = (size_t)nb * (size_t)cfg->trade_capacity * sizeof(lob_trade_t);
    struct {
        void** p;
        size_t bytes;
    } allocs[] = {{(void**)&c->d_state, state_b},
                  {(void**)&c->d_counts, (size_t)nb * 2 * sizeof(int32_t)},
                  {(void**)&c->d_trades, trade_b > 0 ? trade_b : 32},
                  {(void**)&c->d_tcounts, (size_t)nb * sizeof(int64_t)},
                  {(void**)&c->d_stats, (size_t)nb * kNumCtr * sizeof(int64_t)},
                  {(void**)&c->d_status, 64},
                  {(void**)&c->d_queue, 64}};
    for (auto& al : allocs) {
        e = cudaMalloc(al.p, al.bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            lob_destroy(c);
            lob_set_error("lob_create: cudaMalloc of %zu bytes failed", al.bytes);
            return LOB_E_NOMEM;
        }
    }
    e = cudaMemsetAsync(c->d_state, 0, state_b, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_counts, 0, (size_t)nb * 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_tcounts, 0, (size_t)nb * sizeof(int64_t), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_stats, 0, (size_t)nb * kNumCtr * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_queue, 0, 64, s);
    if (e != cudaSuccess) {
        lob_destroy(c);
        return lob_cuda_fail(e, "lob_create memset");
    }
    int rc = configure_launch(c, 4, 64, 0);
    if (rc != LOB_OK) {
        lob_destroy(c);
        return rc;
    }
    *out = c;
    return LOB_OK;
}

int lob_destroy(lob_ctx* c)
{
    if (!c) return LOB_OK;
    cudaError_t first = cudaSuccess;
    if (c->d_state || c->d_trades) first = cudaDeviceSynchronize();
    if (c->copy_stream && first == cudaSuccess) first = cudaStreamSynchronize(c->copy_stream);
    void* ptrs[] = {c->d_state, c->d_counts, c->d_trades, c->d_tcounts,
                    c->d_stats, c->d_status, c->d_queue, c->d_stage, c->d_stage_off};
    for (void* p : ptrs)
        if (p) {
            cudaError_t e = cudaFree(p);
            if (first == cudaSuccess) first = e;
        }
    for (int i = 0; i < lob_ctx::kStages; ++i) {
        if (c->ev_copied[i]) cudaEventDestroy(c->ev_copied[i]);
        if (c->ev_consumed[i]) cudaEventDestroy(c->ev_consumed[i]);
    }
    if (c->ev_start) cudaEventDestroy(c->ev_start);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    delete c;
    if (first != cudaSuccess) return lob_cuda_fail(first, "lob_destroy");
    return LOB_OK;
}

int lob_reset(lob_ctx* c, void* stream)
{
    if (!c) {
        lob_set_error("lob_reset: null context");
        return LOB_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nb = c->cfg.n_books;
    cudaError_t e = cudaMemsetAsync(c->d_counts, 0, (size_t)nb * 2 * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_tcounts, 0, (size_t)nb * sizeof(int64_t), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_stats, 0, (size_t)nb * kNumCtr * sizeof(int64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, 64, s);
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_reset");
    return LOB_OK;
}

int lob_reset_books(lob_ctx* c, const int32_t* d_book_ids, int32_t n, void* stream)
{
    if (!c || n < 0 || (n > 0 && !d_book_ids)) {
        lob_set_error("lob_reset_books: invalid argument");
        return LOB_E_INVAL;
    }
    if (n == 0) return LOB_OK;
    k_reset_books<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(
        d_book_ids, n, c->cfg.n_books, c->d_counts, c->d_tcounts, c->d_stats, c->d_status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_reset_books");
    c->launches += 1;
    return LOB_OK;
}

static int check_batch(lob_ctx* c, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                       const int32_t* d_book_ids, int32_t n_active, const char* who)
{
    if (!c) {
        lob_set_error("%s: null context", who);
        return LOB_E_INVAL;
    }
    if (n_active < 0 || n_active > c->cfg.n_books) {
        lob_set_error("%s: n_active=%d outside [0, %d]", who, n_active, c->cfg.n_books);
        return LOB_E_INVAL;
    }
    if (n_active == 0) return LOB_OK;
    if (!d_book_ids && n_active != c->cfg.n_books) {
        lob_set_error("%s: without book ids every book needs a segment (n_active=%d, n_books=%d)",
                      who, n_active, c->cfg.n_books);
        return LOB_E_INVAL;
    }
    if (!d_msgs || !d_offsets) {
        lob_set_error("%s: null message or offset pointer", who);
        return LOB_E_INVAL;
    }
    if (((uintptr_t)d_msgs & 15u) != 0) {
        lob_set_error("%s: messages must be 16-byte aligned", who);
        return LOB_E_INVAL;
    }
    return LOB_OK;
}

int lob_process_batch(lob_ctx* c, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                      const int32_t* d_book_ids, int32_t n_active, void* stream)
{
    int rc = check_batch(c, d_msgs, d_offsets, d_book_ids, n_active, "lob_process_batch");
    if (rc != LOB_OK) return rc;
    const int append = (c->cfg.flags & LOB_FLAG_APPEND_TRADES) ? 1 : 0;
    return lob_launch_process(c, d_msgs, d_offsets, d_book_ids, n_active, append,
                              (cudaStream_t)stream, nullptr, nullptr);
}

namespace {

// uniform offsets 0, L, 2L, ..., n*L
__global__ void k_uniform_offsets(int64_t* off, int32_t n, int64_t len)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        off[i] = i * len;
}

// staging buffers, streams and events of the host-streamed ingest
int setup_host_stream(lob_ctx* c, int64_t chunk)
{
    if (c->d_stage && c->stage_msgs >= chunk) return LOB_OK;
    cudaError_t err = cudaSuccess;
    if (c->d_stage) {
        err = cudaStreamSynchronize(c->copy_stream);
        if (err == cudaSuccess) err = cudaDeviceSynchronize();
        if (err != cudaSuccess) return lob_cuda_fail(err, "lob_process_host");
        cudaFree(c->d_stage);
        c->d_stage = nullptr;
    }
    const size_t bytes = (size_t)lob_ctx::kStages * c->cfg.n_books * (size_t)chunk * 32;
    err = cudaMalloc(&c->d_stage, bytes);
    if (err != cudaSuccess) {
        c->d_stage = nullptr;
        lob_set_error("lob_process_host: staging (%zu bytes) does not fit on the device", bytes);
        return LOB_E_NOMEM;
    }
    c->stage_msgs = chunk;
    if (!c->d_stage_off) {
        err = cudaMalloc(&c->d_stage_off, sizeof(int64_t) * 2 * ((size_t)c->cfg.n_books + 1));
        if (err != cudaSuccess) {
            c->d_stage_off = nullptr;
            return lob_cuda_fail(err, "lob_process_host offsets");
        }
    }
    if (!c->copy_stream) {
        err = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
        for (int i = 0; i < lob_ctx::kStages && err == cudaSuccess; ++i) {
            err = cudaEventCreateWithFlags(&c->ev_copied[i], cudaEventDisableTiming);
            if (err == cudaSuccess)
                err = cudaEventCreateWithFlags(&c->ev_consumed[i], cudaEventDisableTiming);
        }
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming);
        if (err != cudaSuccess) return lob_cuda_fail(err, "lob_process_host streams");
    }
    return LOB_OK;
}

}  // namespace

int lob_process_host(lob_ctx* c, const lob_msg_t* h_msgs, int64_t msgs_per_book,
                     int32_t chunk_msgs, void* stream)
{
    if (!c || (!h_msgs && msgs_per_book > 0) || msgs_per_book < 0 || chunk_msgs < 1) {
        lob_set_error("lob_process_host: invalid argument");
        return LOB_E_INVAL;
    }
    if (msgs_per_book == 0) return LOB_OK;
    const int64_t chunk = chunk_msgs < msgs_per_book ? chunk_msgs : msgs_per_book;
    int rc = setup_host_stream(c, chunk);
    if (rc != LOB_OK) return rc;
    const int n = c->cfg.n_books;
    const cudaStream_t s = (cudaStream_t)stream;
    const int64_t n_chunks = (msgs_per_book + chunk - 1) / chunk;
    const int64_t tail = msgs_per_book - (n_chunks - 1) * chunk;
    // offsets of a full chunk and of the (possibly shorter) last chunk
    int64_t* off_full = c->d_stage_off;
    int64_t* off_tail = c->d_stage_off + (n + 1);
    const int blocks = (n + 256) / 256;
    k_uniform_offsets<<<blocks, 256, 0, s>>>(off_full, n, chunk);
    k_uniform_offsets<<<blocks, 256, 0, s>>>(off_tail, n, tail);
    cudaError_t err = cudaGetLastError();
    // the copy stream starts after everything already queued on `stream`
    if (err == cudaSuccess) err = cudaEventRecord(c->ev_start, s);
    if (err == cudaSuccess) err = cudaStreamWaitEvent(c->copy_stream, c->ev_start, 0);
    if (err != cudaSuccess) return lob_cuda_fail(err, "lob_process_host");
    const size_t slot_bytes = (size_t)n * (size_t)c->stage_msgs * 32;
    int append = (c->cfg.flags & LOB_FLAG_APPEND_TRADES) ? 1 : 0;
    for (int64_t k = 0; k < n_chunks; ++k) {
        const int st = (int)(k % lob_ctx::kStages);
        const int64_t len = k + 1 < n_chunks ? chunk : tail;
        char* slot = c->d_stage + st * slot_bytes;
        // chunk k of every book: a strided copy (row b = book b's messages
        // [k*chunk, k*chunk + len)), into the slot in book-major order
        if (k >= lob_ctx::kStages) err = cudaStreamWaitEvent(c->copy_stream, c->ev_consumed[st], 0);
        if (err == cudaSuccess)
            err = cudaMemcpy2DAsync(slot, (size_t)len * 32, h_msgs + k * chunk,
                                    (size_t)msgs_per_book * 32, (size_t)len * 32, (size_t)n,
                                    cudaMemcpyHostToDevice, c->copy_stream);
        if (err == cudaSuccess) err = cudaEventRecord(c->ev_copied[st], c->copy_stream);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(s, c->ev_copied[st], 0);
        if (err != cudaSuccess) return lob_cuda_fail(err, "lob_process_host copy");
        rc = lob_launch_process(c, reinterpret_cast<const lob_msg_t*>(slot),
                                k + 1 < n_chunks ? off_full : off_tail, nullptr, n, append, s,
                                nullptr, nullptr);
        if (rc != LOB_OK) return rc;
        append = 1;  // later chunks continue the logs the first one began
        err = cudaEventRecord(c->ev_consumed[st], s);
        if (err != cudaSuccess) return lob_cuda_fail(err, "lob_process_host");
    }
    return LOB_OK;
}

int lob_process_batch_l1(lob_ctx* c, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                         const int32_t* d_book_ids, int32_t n_active, int32_t* d_l1,
                         void* stream)
{
    int rc = check_batch(c, d_msgs, d_offsets, d_book_ids, n_active, "lob_process_batch_l1");
    if (rc != LOB_OK) return rc;
    if (n_active > 0 && (!d_l1 || ((uintptr_t)d_l1 & 15u) != 0)) {
        lob_set_error("lob_process_batch_l1: the trace must be a 16-byte aligned buffer");
        return LOB_E_INVAL;
    }
    const int append = (c->cfg.flags & LOB_FLAG_APPEND_TRADES) ? 1 : 0;
    return lob_launch_process(c, d_msgs, d_offsets, d_book_ids, n_active, append,
                              (cudaStream_t)stream, nullptr, d_l1);
}

int lob_process_segments(lob_ctx* c, const lob_msg_t* d_msgs, const int64_t* d_starts,
                         const int64_t* d_counts, const int32_t* d_book_ids, int32_t n_active,
                         void* stream)
{
    int rc = check_batch(c, d_msgs, d_starts, d_book_ids, n_active, "lob_process_segments");
    if (rc != LOB_OK) return rc;
    if (n_active > 0 && (!d_counts || !d_book_ids)) {
        lob_set_error("lob_process_segments: null counts or book ids");
        return LOB_E_INVAL;
    }
    const int append = (c->cfg.flags & LOB_FLAG_APPEND_TRADES) ? 1 : 0;
    return lob_launch_process(c, d_msgs, d_starts, d_book_ids, n_active, append,
                              (cudaStream_t)stream, d_counts, nullptr);
}

int lob_inject_orders(lob_ctx* c, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                      const int32_t* d_book_ids, int32_t n_active, void* stream)
{
    int rc = check_batch(c, d_msgs, d_offsets, d_book_ids, n_active, "lob_inject_orders");
    if (rc != LOB_OK) return rc;
    return lob_launch_process(c, d_msgs, d_offsets, d_book_ids, n_active, 1,
                              (cudaStream_t)stream, nullptr, nullptr);
}

int lob_clear_trades(lob_ctx* c, void* stream)
{
    if (!c) {
        lob_set_error("lob_clear_trades: null context");
        return LOB_E_INVAL;
    }
    cudaError_t e = cudaMemsetAsync(c->d_tcounts, 0, (size_t)c->cfg.n_books * sizeof(int64_t),
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_clear_trades");
    return LOB_OK;
}

#define LOB_DISPATCH_K(KV, CALL)                      \
    switch (KV) {                                     \
    case 1: { constexpr int KK = 1; CALL; } break;    \
    case 2: { constexpr int KK = 2; CALL; } break;    \
    case 4: { constexpr int KK = 4; CALL; } break;    \
    case 8: { constexpr int KK = 8; CALL; } break;    \
    default: { constexpr int KK = 16; CALL; } break;  \
    }

static int launch_levels(lob_ctx* c, const int32_t* d_book_ids, int32_t n_items, int32_t depth,
                         int32_t* d_bid_px, int32_t* d_bid_qty, int32_t* d_ask_px,
                         int32_t* d_ask_qty, void* stream, const char* who)
{
    if (!c || depth < 1 || depth > 64 || !d_bid_px || !d_bid_qty || !d_ask_px || !d_ask_qty ||
        n_items < 0 || (n_items > 0 && d_book_ids == nullptr && n_items != c->cfg.n_books)) {
        lob_set_error("%s: invalid argument (depth=%d, n_active=%d)", who, depth, n_items);
        return LOB_E_INVAL;
    }
    if (n_items == 0) return LOB_OK;
    const int wpb = 8;
    dim3 grid((n_items + wpb - 1) / wpb), block(32 * wpb);
    cudaStream_t s = (cudaStream_t)stream;
    LOB_DISPATCH_K(c->K, (k_levels<KK><<<grid, block, 0, s>>>(
                             c->d_state, c->d_counts, c->cfg.n_books, d_book_ids, n_items,
                             c->d_status, depth, d_bid_px, d_bid_qty, d_ask_px, d_ask_qty)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lob_cuda_fail(e, who);
    c->launches += 1;
    return LOB_OK;
}

int lob_get_levels(lob_ctx* c, int32_t depth, int32_t* d_bid_px, int32_t* d_bid_qty,
                   int32_t* d_ask_px, int32_t* d_ask_qty, void* stream)
{
    return launch_levels(c, nullptr, c ? c->cfg.n_books : 0, depth, d_bid_px, d_bid_qty,
                         d_ask_px, d_ask_qty, stream, "lob_get_levels");
}

int lob_get_levels_books(lob_ctx* c, const int32_t* d_book_ids, int32_t n_active, int32_t depth,
                         int32_t* d_bid_px, int32_t* d_bid_qty, int32_t* d_ask_px,
                         int32_t* d_ask_qty, void* stream)
{
    if (!d_book_ids && n_active != 0) {
        lob_set_error("lob_get_levels_books: d_book_ids is NULL");
        return LOB_E_INVAL;
    }
    return launch_levels(c, d_book_ids, n_active, depth, d_bid_px, d_bid_qty, d_ask_px,
                         d_ask_qty, stream, "lob_get_levels_books");
}

int lob_get_trades(lob_ctx* c, lob_trade_t* d_out, int64_t* d_counts, void* stream)
{
    if (!c) {
        lob_set_error("lob_get_trades: null context");
        return LOB_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (d_out && c->cfg.trade_capacity > 0) {
        const int64_t n = (int64_t)c->cfg.n_books * c->cfg.trade_capacity;
        k_get_trades<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<const Trade*>(c->d_trades), c->d_tcounts, c->cfg.n_books,
            c->cfg.trade_capacity, reinterpret_cast<Trade*>(d_out));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return lob_cuda_fail(e, "lob_get_trades");
        c->launches += 1;
    }
    if (d_counts) {
        cudaError_t e = cudaMemcpyAsync(d_counts, c->d_tcounts,
                                        (size_t)c->cfg.n_books * sizeof(int64_t),
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return lob_cuda_fail(e, "lob_get_trades counts");
    }
    return LOB_OK;
}

int lob_get_book(lob_ctx* c, int32_t* px, int32_t* qty, int32_t* oid, int32_t* tid, int64_t* tm,
                 int32_t* count, void* stream)
{
    if (!c) {
        lob_set_error("lob_get_book: null context");
        return LOB_E_INVAL;
    }
    const int64_t n = (int64_t)c->cfg.n_books * 2 * c->cfg.capacity;
    dim3 grid((unsigned)((n + 255) / 256)), block(256);
    cudaStream_t s = (cudaStream_t)stream;
    const int cap = c->cfg.capacity, nb = c->cfg.n_books;
    LOB_DISPATCH_K(c->K, (k_get_book<KK><<<grid, block, 0, s>>>(c->d_state, c->d_counts, nb, cap,
                                                                px, qty, oid, tid, tm, count)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_get_book");
    c->launches += 1;
    return LOB_OK;
}

int lob_set_book(lob_ctx* c, const int32_t* px, const int32_t* qty, const int32_t* oid,
                 const int32_t* tid, const int64_t* tm, const int32_t* count, void* stream)
{
    if (!c || !px || !qty || !oid || !tid || !tm || !count) {
        lob_set_error("lob_set_book: null argument");
        return LOB_E_INVAL;
    }
    const int wpb = 8;
    const int64_t nw = (int64_t)c->cfg.n_books * 2;
    dim3 grid((unsigned)((nw + wpb - 1) / wpb)), block(32 * wpb);
    cudaStream_t s = (cudaStream_t)stream;
    const int cap = c->cfg.capacity, nb = c->cfg.n_books;
    LOB_DISPATCH_K(c->K, (k_set_book<KK><<<grid, block, 0, s>>>(c->d_state, c->d_counts, nb, cap,
                                                                px, qty, oid, tid, tm, count,
                                                                c->d_status)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_set_book");
    c->launches += 1;
    return LOB_OK;
}

int lob_init_from_levels(lob_ctx* c, const int32_t* d_bid_px, const int32_t* d_bid_qty,
                         const int32_t* d_ask_px, const int32_t* d_ask_qty, int32_t depth,
                         int64_t time_ns, void* stream)
{
    if (!c || !d_bid_px || !d_bid_qty || !d_ask_px || !d_ask_qty) {
        lob_set_error("lob_init_from_levels: null argument");
        return LOB_E_INVAL;
    }
    if (depth < 1 || depth > c->cfg.capacity) {
        lob_set_error("lob_init_from_levels: depth %d outside 1..capacity (%d)", depth,
                      c->cfg.capacity);
        return LOB_E_INVAL;
    }
    const int wpb = 8;
    dim3 grid((unsigned)((c->cfg.n_books + wpb - 1) / wpb)), block(32 * wpb);
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = c->cfg.n_books;
    LOB_DISPATCH_K(c->K, (k_init_from_levels<KK><<<grid, block, 0, s>>>(
                             c->d_state, c->d_counts, nb, depth, d_bid_px, d_bid_qty, d_ask_px,
                             d_ask_qty, time_ns, c->d_status)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_init_from_levels");
    c->launches += 1;
    return LOB_OK;
}

int lob_get_stats(lob_ctx* c, int64_t* d_counters, int32_t* d_status, void* stream)
{
    if (!c) {
        lob_set_error("lob_get_stats: null context");
        return LOB_E_INVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (d_counters)
        e = cudaMemcpyAsync(d_counters, c->d_stats,
                            (size_t)c->cfg.n_books * kNumCtr * sizeof(int64_t),
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d_status)
        e = cudaMemcpyAsync(d_status, c->d_status, sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_get_stats");
    return LOB_OK;
}

int lob_set_launch(lob_ctx* c, int32_t warps_per_cta, int32_t chunk_msgs, int32_t ctas_per_sm)
{
    if (!c || warps_per_cta < 1 || warps_per_cta > 16 || chunk_msgs < 8 || chunk_msgs > 1024 ||
        (chunk_msgs % 8) != 0 || ctas_per_sm < 0) {
        lob_set_error("lob_set_launch: invalid shape (warps=%d chunk=%d ctas_per_sm=%d)",
                      warps_per_cta, chunk_msgs, ctas_per_sm);
        return LOB_E_INVAL;
    }
    return configure_launch(c, warps_per_cta, chunk_msgs, ctas_per_sm);
}

}  // extern "C"

// ------------------------------------------------ allocation-free entry point
//
// lob_process_streams_static runs the same processing kernel as
// lob_process_batch, but takes no context: every book starts empty, and the
// only device memory it needs besides the caller's inputs and outputs -- the
// work-queue counter, the per-side order counts and the staged book state --
// lives in the file-scope array below.  It exists for callers that must not
// allocate device memory at run time, for example a service that reserved the
// GPU's memory up front for its own pool, or a latency-critical loop where a
// cudaMalloc/cudaFree would synchronise the device and stall other streams.

namespace {

constexpr size_t kStaticScratchBytes = 32u << 20;  // 32 MiB per GPU that loads the library
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
struct StaticSetup {
    bool done = false;
    unsigned char* scratch = nullptr;  // device address of g_static_scratch
    int num_sms = 0;
    int per_sm[5] = {0, 0, 0, 0, 0};  // resident CTAs of k_process<K>, K = 1,2,4,8,16
};
StaticSetup g_static[kMaxDevices];
std::mutex g_static_mu;

// scratch layout: [queue: 256 B][counts: n_books*2 int32, padded to 256 B][book state]
size_t static_state_offset(int64_t n_books)
{
    return 256 + (((size_t)n_books * 8 + 255) / 256) * 256;
}

size_t static_scratch_bytes(int64_t n_books, int K)
{
    return static_state_offset(n_books) + (size_t)n_books * (size_t)lob_book_bytes(K);
}

// the largest n_books whose scratch fits (exact)
int static_max_books(int K)
{
    int64_t n = (int64_t)(kStaticScratchBytes - 256) / ((int64_t)lob_book_bytes(K) + 8);
    while (n > 0 && static_scratch_bytes(n, K) > kStaticScratchBytes) --n;
    while (static_scratch_bytes(n + 1, K) <= kStaticScratchBytes) ++n;
    return (int)n;
}

constexpr int kStaticChunk = 64;
int static_warps(int K) { return K >= 8 ? 4 : 8; }
int k_index(int K) { return K == 1 ? 0 : K == 2 ? 1 : K == 4 ? 2 : K == 8 ? 3 : 4; }

// Once per device, with that device current: resolve the array's device
// address and prepare the kernel launch attributes.  Allocates nothing.
int static_setup(int dev, StaticSetup** out)
{
    std::lock_guard<std::mutex> lock(g_static_mu);
    StaticSetup& s = g_static[dev];
    if (!s.done) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return lob_cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        e = cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return lob_cuda_fail(e, "cudaDeviceGetAttribute");
        const int ks[5] = {1, 2, 4, 8, 16};
        for (int i = 0; i < 5; ++i) {
            const int K = ks[i], W = static_warps(K);
            const int smem = smem_per_warp(K, kStaticChunk) * W;
            const void* fn = process_kernel(K);
            e = lob_raise_smem_limit(fn, smem);
            if (e != cudaSuccess) return lob_cuda_fail(e, "cudaFuncSetAttribute");
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&s.per_sm[i], fn, 32 * W, smem);
            if (e != cudaSuccess) return lob_cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
            if (s.per_sm[i] < 1) s.per_sm[i] = 1;
        }
        s.scratch = static_cast<unsigned char*>(p);
        s.done = true;
    }
    *out = &s;
    return LOB_OK;
}

}  // namespace

extern "C" int lob_process_streams_static(const lob_msg_t* d_msgs, const int64_t* d_offsets,
                                          int32_t n_books, int32_t capacity,
                                          int32_t trade_capacity, int32_t overflow_rule,
                                          lob_trade_t* d_trades, int64_t* d_trade_counts,
                                          int64_t* d_counters, int32_t* d_price, int32_t* d_qty,
                                          int32_t* d_oid, int32_t* d_tid, int64_t* d_time,
                                          int32_t* d_count, int32_t* d_status, void* stream)
{
    if (n_books < 1 || capacity < 1 || capacity > 32 * kMaxK || trade_capacity < 0 ||
        (overflow_rule != 0 && overflow_rule != 1)) {
        lob_set_error("lob_process_streams_static: invalid sizes (n_books=%d capacity=%d "
                      "trade_capacity=%d overflow_rule=%d)",
                      n_books, capacity, trade_capacity, overflow_rule);
        return LOB_E_INVAL;
    }
    if (!d_msgs || !d_offsets || !d_trade_counts || !d_counters || !d_status ||
        (trade_capacity > 0 && !d_trades)) {
        lob_set_error("lob_process_streams_static: null input or output pointer");
        return LOB_E_INVAL;
    }
    if (((uintptr_t)d_msgs & 15u) != 0) {
        lob_set_error("lob_process_streams_static: messages must be 16-byte aligned");
        return LOB_E_INVAL;
    }
    const int K = k_of(capacity);
    const size_t counts_off = 256;
    const size_t state_off = static_state_offset(n_books);
    const size_t need = static_scratch_bytes(n_books, K);
    if (need > kStaticScratchBytes) {
        lob_set_error("lob_process_streams_static: %d books of capacity %d need %zu bytes of "
                      "scratch, more than the library's fixed %zu bytes (at most %d books at "
                      "this capacity)",
                      n_books, capacity, need, kStaticScratchBytes, static_max_books(K));
        return LOB_E_INVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return lob_cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        lob_set_error("lob_process_streams_static: device index %d not supported", dev);
        return LOB_E_INVAL;
    }
    StaticSetup* s = nullptr;
    int rc = static_setup(dev, &s);
    if (rc != LOB_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* scratch = s->scratch;
    int32_t* queue = reinterpret_cast<int32_t*>(scratch);
    int32_t* counts = reinterpret_cast<int32_t*>(scratch + counts_off);
    char* state = reinterpret_cast<char*>(scratch + state_off);
    // the array keeps the previous call's contents: clear what must start at zero
    e = cudaMemsetAsync(queue, 0, 256, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, (size_t)n_books * 8, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_counters, 0, (size_t)n_books * kNumCtr * sizeof(int64_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int32_t), st);
    // every book's count is defined, also for one that is skipped (bad segment)
    if (e == cudaSuccess) e = cudaMemsetAsync(d_trade_counts, 0, (size_t)n_books * 8, st);
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_process_streams_static memset");

    ProcArgs a;
    a.msgs = reinterpret_cast<const Msg*>(d_msgs);
    a.offsets = d_offsets;
    a.counts_in = nullptr;
    a.book_ids = nullptr;
    a.n_items = n_books;
    a.n_books = n_books;
    a.state = state;
    a.counts = counts;
    a.trades = reinterpret_cast<Trade*>(d_trades);
    a.tcounts = d_trade_counts;
    a.stats = d_counters;
    a.status = d_status;
    a.queue = queue;
    a.cap = capacity;
    a.rule = overflow_rule;
    a.trade_cap = trade_capacity;
    a.append = 0;
    a.chunk = kStaticChunk;
    a.pad_ = 0;
    a.wait_ns = kWaitNs;
    a.l1 = nullptr;
    const int W = static_warps(K);
    int grid = (n_books + W - 1) / W;
    const int resident = s->num_sms * s->per_sm[k_index(K)];
    if (grid > resident) grid = resident;
    void* args[] = {&a};
    e = cudaLaunchKernel(process_kernel(K), dim3(grid), dim3(32 * W), args,
                         (size_t)(smem_per_warp(K, kStaticChunk) * W), st);
    if (e != cudaSuccess) return lob_cuda_fail(e, "lob_process_streams_static launch");
    if (d_price || d_qty || d_oid || d_tid || d_time || d_count) {
        const int64_t n = (int64_t)n_books * 2 * capacity;
        dim3 g2((unsigned)((n + 255) / 256)), b2(256);
        LOB_DISPATCH_K(K, (k_get_book<KK><<<g2, b2, 0, st>>>(state, counts, n_books, capacity,
                                                             d_price, d_qty, d_oid, d_tid,
                                                             d_time, d_count)));
        e = cudaGetLastError();
        if (e != cudaSuccess) return lob_cuda_fail(e, "lob_process_streams_static dump");
    }
    return LOB_OK;
}
