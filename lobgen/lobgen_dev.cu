// lobgen_dev.cu -- device (CUDA) side of the seeded order-flow generator.
//
// Same stream definition as the host side (lobgen_core.h is compiled for
// both): a warp per book for the usual pool sizes, a thread per book above.
// Used where streams are too large to stage from the host (long RL episodes,
// the serving mix).  C ABI, device pointers, asynchronous on the given stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lobgen_core.h"

namespace {

__global__ void k_init(lobgen_params_t p, int32_t n_books, const uint64_t* stream_ids,
                       lobgen_state_t* states)
{
    int32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_books) return;
    lobgen_state_t s;
    lg_init_state(&p, stream_ids ? stream_ids[b] : (uint64_t)b, &s);
    states[b] = s;
}

// State of book ids[i] restarts as stream stream_ids[i].
__global__ void k_init_ids(lobgen_params_t p, int32_t n, const int32_t* ids,
                           const uint64_t* stream_ids, lobgen_state_t* states)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    lobgen_state_t s;
    lg_init_state(&p, stream_ids[i], &s);
    states[ids[i]] = s;
}

// Book b (= ids[i] when ids is given) appends counts[i] messages at
// out + out_offsets[i].
__global__ void k_advance(lobgen_params_t p, const uint64_t* __restrict__ geo_px,
                          const uint64_t* __restrict__ geo_q, int32_t n,
                          const int32_t* __restrict__ ids, lobgen_state_t* states,
                          lobgen_pool_entry_t* pools, const int64_t* __restrict__ counts,
                          const int64_t* __restrict__ out_offsets, lobgen_msg_t* out)
{
    int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t b = ids ? ids[i] : i;
    lobgen_state_t s = states[b];
    lobgen_pool_entry_t* pool = pools + (int64_t)b * p.pool_cap;
    lobgen_msg_t* o = out + out_offsets[i];
    int64_t c = counts[i];
    for (int64_t k = 0; k < c; ++k) o[k] = lg_next(&p, geo_px, geo_q, &s, pool);
    states[b] = s;
}

// Warp per book: the same stream as lg_next, 32 messages at a time.  Every
// random draw of a message is a keyed hash of (stream, message index, draw
// slot), so the lanes compute the draws of 32 consecutive messages at once; the
// mid walk (clamped at 1) and the time stamps are prefix scans over the lanes;
// only the order-id counter and the pool of remembered ids -- which decide a
// cancel's target and turn a cancel on an empty pool into an add -- are
// stepped message by message, by lane 0 in shared memory.
constexpr int kWarpPoolMax = 128;  // pools up to this size use the warp kernel
constexpr int kGenWarps = 4;       // warps per block

struct WarpStage {
    lobgen_pool_entry_t pool[kWarpPoolMax];
    int32_t type[32], side[32], price[32], qty[32], oid[32];
    uint32_t r5[32], r7[32];  // high words of draws 5 and 7
};

__device__ __forceinline__ uint32_t lg_uniform_hi(uint32_t hi, uint32_t n)
{
    return (uint32_t)(((uint64_t)hi * (uint64_t)n) >> 32);
}

__global__ void __launch_bounds__(32 * kGenWarps)
k_advance_warp(lobgen_params_t p, const uint64_t* __restrict__ geo_px,
               const uint64_t* __restrict__ geo_q, int32_t n, const int32_t* __restrict__ ids,
               lobgen_state_t* states, lobgen_pool_entry_t* pools,
               const int64_t* __restrict__ counts, const int64_t* __restrict__ out_offsets,
               lobgen_msg_t* out)
{
    __shared__ WarpStage stage[kGenWarps];
    const int l = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int32_t i = blockIdx.x * kGenWarps + w;
    if (i >= n) return;  // uniform over the warp
    const int32_t b = ids ? ids[i] : i;
    WarpStage& S = stage[w];
    lobgen_state_t s = states[b];
    lobgen_pool_entry_t* gpool = pools + (int64_t)b * p.pool_cap;
    int32_t pc = s.pool_count;  // only [0, pool_count) is ever read
    for (int j = l; j < pc; j += 32) S.pool[j] = gpool[j];
    __syncwarp();
    const int64_t c = counts[i];
    lobgen_msg_t* o = out + out_offsets[i];
    const uint64_t key = s.key;
    int32_t mid = s.mid, next_oid = s.next_oid;
    int64_t time = s.time_ns;
    for (int64_t base = 0; base < c; base += 32) {
        const int64_t k = base + l;
        const bool live = k < c;
        const uint64_t ix = s.index + (uint64_t)k;
        // the message's draws (slots as in lg_next)
        const uint32_t rm = lg_hi32(lg_draw(key, ix, 0));
        const int32_t dmid = rm < p.cut_mid_down ? -1 : (rm >= p.cut_mid_up ? 1 : 0);
        const uint32_t rt = lg_hi32(lg_draw(key, ix, 1));
        const int32_t type = rt < p.cut_add ? 1 : rt < p.cut_cancel ? 2 : rt < p.cut_delete ? 3 : 4;
        const int32_t side = (lg_draw(key, ix, 2) >> 63) ? 1 : -1;
        const int32_t g = lg_geometric(lg_draw(key, ix, 3), geo_px, p.geo_px_kmax);
        const bool aggressive = lg_hi32(lg_draw(key, ix, 4)) < p.cut_marketable;
        const uint64_t r5 = lg_draw(key, ix, 5);
        const int32_t q_geo = 1 + lg_geometric(r5, geo_q, p.geo_q_kmax);
        const int32_t tid = 1 + (int32_t)lg_uniform(lg_draw(key, ix, 6), (uint32_t)p.tid_max);
        const uint32_t r7 = lg_hi32(lg_draw(key, ix, 7));
        const int64_t dt = 1 + (int64_t)lg_uniform(lg_draw(key, ix, 8), (uint32_t)p.dt_max);
        // mid after message k: m_k = max(1, m_{k-1} + d_k), the composition of
        // the maps x -> max(a, x + d) (a = 1 per message; identity for lanes
        // past the end): (a1, d1) then (a2, d2) = (max(a2, a1 + d2), d1 + d2)
        int32_t ma = live ? 1 : -(1 << 29), md = live ? dmid : 0;
        int64_t tsum = live ? dt : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t pa = __shfl_up_sync(0xffffffffu, ma, d);
            const int32_t pd = __shfl_up_sync(0xffffffffu, md, d);
            const int64_t pt = __shfl_up_sync(0xffffffffu, tsum, d);
            if (l >= d) {
                ma = max(ma, pa + md);
                md = pd + md;
                tsum += pt;
            }
        }
        const int32_t mid_k = max(ma, mid + md);
        const int64_t time_k = time + tsum;
        int32_t price = aggressive ? (side == 1 ? mid_k + g : mid_k - g)
                                   : (side == 1 ? mid_k - 1 - g : mid_k + 1 + g);
        if (price < 1) price = 1;
        S.type[l] = type;
        S.side[l] = side;
        S.price[l] = price;
        S.qty[l] = q_geo;
        S.r5[l] = lg_hi32(r5);
        S.r7[l] = r7;
        __syncwarp();
        const int nb = (int)(c - base < 32 ? c - base : 32);
        if (l == 0) {
            for (int j = 0; j < nb; ++j) {
                int32_t t = S.type[j];
                if ((t == 2 || t == 3) && pc == 0) t = 1;
                if (t == 1) {
                    const int32_t oid = next_oid++;
                    lobgen_pool_entry_t e;
                    e.oid = oid; e.qty = S.qty[j]; e.price = S.price[j]; e.side = S.side[j];
                    if (pc < p.pool_cap) S.pool[pc++] = e;
                    else S.pool[lg_uniform_hi(S.r7[j], (uint32_t)p.pool_cap)] = e;
                    S.oid[j] = oid;
                } else if (t == 2 || t == 3) {
                    const uint32_t jj = lg_uniform_hi(S.r7[j], (uint32_t)pc);
                    const lobgen_pool_entry_t e = S.pool[jj];
                    S.side[j] = e.side; S.price[j] = e.price; S.oid[j] = e.oid;
                    if (t == 2) {
                        S.qty[j] = e.qty >= 2 ? 1 + (int32_t)lg_uniform_hi(S.r5[j], (uint32_t)(e.qty - 1)) : 1;
                    } else {
                        S.qty[j] = e.qty;
                        S.pool[jj] = S.pool[pc - 1];
                        pc -= 1;
                    }
                } else {
                    S.oid[j] = next_oid++;
                    S.price[j] = 0;
                }
                S.type[j] = t;
            }
        }
        __syncwarp();
        pc = __shfl_sync(0xffffffffu, pc, 0);
        next_oid = __shfl_sync(0xffffffffu, next_oid, 0);
        if (live) {
            lobgen_msg_t m;
            m.type = S.type[l]; m.side = S.side[l]; m.price = S.price[l]; m.qty = S.qty[l];
            m.oid = S.oid[l]; m.tid = tid; m.time_ns = time_k;
            o[k] = m;
        }
        mid = __shfl_sync(0xffffffffu, mid_k, nb - 1);
        time = __shfl_sync(0xffffffffu, time_k, nb - 1);
        __syncwarp();
    }
    for (int j = l; j < pc; j += 32) gpool[j] = S.pool[j];
    if (l == 0) {
        s.time_ns = time;
        s.index += (uint64_t)c;
        s.mid = mid;
        s.next_oid = next_oid;
        s.pool_count = pc;
        states[b] = s;
    }
}

__global__ void k_agent(uint64_t seed, int32_t n_envs, int32_t step0, int32_t n_steps,
                        uint32_t* out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n_envs * n_steps) return;
    int32_t t = (int32_t)(i / n_envs), e = (int32_t)(i % n_envs);
    out[i] = lg_agent_draw(seed, (uint64_t)e, (uint64_t)(step0 + t));
}

}  // namespace

extern "C" {

int lobgen_dev_init(const lobgen_params_t* p, int32_t n_books, const uint64_t* d_stream_ids,
                    lobgen_state_t* d_states, void* stream)
{
    if (!p || !d_states || n_books < 0 || p->pool_cap < 1 || p->pool_cap > 4096) return -1;
    if (n_books == 0) return 0;
    k_init<<<(n_books + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*p, n_books, d_stream_ids,
                                                                     d_states);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lobgen_dev_init_ids(const lobgen_params_t* p, int32_t n, const int32_t* d_ids,
                        const uint64_t* d_stream_ids, lobgen_state_t* d_states, void* stream)
{
    if (!p || !d_ids || !d_stream_ids || !d_states || n < 0) return -1;
    if (n == 0) return 0;
    k_init_ids<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(*p, n, d_ids, d_stream_ids,
                                                                 d_states);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lobgen_dev_advance(const lobgen_params_t* p, const uint64_t* d_geo_px,
                       const uint64_t* d_geo_q, int32_t n, const int32_t* d_ids,
                       lobgen_state_t* d_states, lobgen_pool_entry_t* d_pools,
                       const int64_t* d_counts, const int64_t* d_out_offsets,
                       lobgen_msg_t* d_out, void* stream)
{
    if (!p || !d_geo_px || !d_geo_q || !d_states || !d_pools || !d_counts || !d_out_offsets ||
        !d_out || n < 0)
        return -1;
    if (n == 0) return 0;
    if (p->pool_cap <= kWarpPoolMax)
        k_advance_warp<<<(n + kGenWarps - 1) / kGenWarps, 32 * kGenWarps, 0, (cudaStream_t)stream>>>(
            *p, d_geo_px, d_geo_q, n, d_ids, d_states, d_pools, d_counts, d_out_offsets, d_out);
    else
        k_advance<<<(n + 63) / 64, 64, 0, (cudaStream_t)stream>>>(
            *p, d_geo_px, d_geo_q, n, d_ids, d_states, d_pools, d_counts, d_out_offsets, d_out);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

int lobgen_dev_agent_draws(uint64_t seed, int32_t n_envs, int32_t step0, int32_t n_steps,
                           uint32_t* d_out, void* stream)
{
    if (!d_out || n_envs < 0 || n_steps < 0) return -1;
    int64_t n = (int64_t)n_envs * n_steps;
    if (n == 0) return 0;
    k_agent<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(seed, n_envs, step0,
                                                                          n_steps, d_out);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // extern "C"
