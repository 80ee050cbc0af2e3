// lobgen_dev.cu -- device (CUDA) side of the seeded order-flow generator.
//
// Same stream definition as the host side (lobgen_core.h is compiled for
// both), one thread per book.  Used where streams are too large to stage from
// the host (long RL episodes, the serving mix).  C ABI, device pointers,
// asynchronous on the given stream.
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
