// lob_engine.h -- context layout shared by the engine's translation units
// (book engine and execution environment).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lob.h"

struct lob_ctx {
    lob_config_t cfg;
    int device = 0;
    int num_sms = 0;
    int K = 4;                        // slots per lane: capacity rounded up to 32*K
    char* d_state = nullptr;          // [n_books][48*32*K] book state (priority-sorted sides)
    int32_t* d_counts = nullptr;      // [n_books][2] orders per side
    lob_trade_t* d_trades = nullptr;  // [n_books][trade_capacity]
    int64_t* d_tcounts = nullptr;     // [n_books] trades in the current log
    int64_t* d_stats = nullptr;       // [n_books][LOB_N_COUNTERS]
    int32_t* d_status = nullptr;      // status word (LOB_STATUS_*)
    int32_t* d_queue = nullptr;       // work queue: [0] next item, [1] warps finished
    int warps_per_cta = 8;
    int chunk = 64;
    int ctas_per_sm = 0;
    int ctas_per_sm_eff = 1;
    int smem_per_cta = 0;
    int64_t launches = 0;
    // host-streamed ingest (lob_process_host), set up on first use
    static constexpr int kStages = 3;
    char* d_stage = nullptr;          // kStages x [n_books][stage_msgs] message slots
    int64_t* d_stage_off = nullptr;   // uniform offsets 0, L, 2L, ... for every L <= stage_msgs
    int64_t stage_msgs = 0;           // messages per book per staged chunk
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_copied[kStages] = {};
    cudaEvent_t ev_consumed[kStages] = {};
    cudaEvent_t ev_start = nullptr;
};

void lob_set_error(const char* fmt, ...);
int lob_cuda_fail(cudaError_t e, const char* where);
int lob_book_bytes(int K);
cudaError_t lob_raise_smem_limit(const void* fn, int bytes);
int lob_launch_process(lob_ctx* c, const lob_msg_t* d_msgs, const int64_t* d_offsets,
                       const int32_t* d_book_ids, int32_t n_active, int append,
                       cudaStream_t stream, const int64_t* d_counts, int32_t* d_l1);
