// Host-side helpers shared by the C-ABI translation units: error reporting,
// plan layout, table construction and argument checks.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/dctgb.h"
#include "kernels.cuh"

namespace dctgb {

// thread-local last error
void set_error(const std::string& msg);
dct_status fail(dct_status st, const std::string& msg);
dct_status cuda_fail(cudaError_t e, const char* what);

// Allocations of the plan workspaces (batch work lists, rate-control state,
// autotuner events and flush buffer) go through these, which count every
// attempt and fail the one that dct_debug_fail_alloc armed with
// cudaErrorMemoryAllocation, without calling CUDA.
cudaError_t ws_malloc(void** p, size_t bytes);
cudaError_t ws_malloc_host(void** p, size_t bytes);
cudaError_t ws_stream_create(cudaStream_t* s);
cudaError_t ws_event_create(cudaEvent_t* e);

// Builds Q, M, W for one plane.  quality 1..100 scales the T.81 Annex K
// table (chroma selects K.2); quality 0 takes qtab (64 or 128 entries).
dct_status build_tables(int quality, const uint16_t* qtab, int qtab_entries, int chroma, QuantSet& out);

// Batch and rate-control state live in batch.cu / ratecontrol.cu; the plan
// only holds pointers to them.
struct BatchState;
struct RcState;

}  // namespace dctgb

struct dct_plan_s {
    dct_plan_desc desc;
    int device;
    int num_sms;
    dct_launch_shape shape;        // batch launch shape (tuned or default)
    dctgb::BatchState* batch;      // batch workspace and graph
    dctgb::RcState* rc;            // rate-control workspace
};

namespace dctgb {

// Launch shape of the batched kernels until dct_autotune picks one: 256
// threads, a grid of 8 CTAs per SM (more than fit at once), two lanes per
// block for the operations that have a two-lane form.
inline dct_launch_shape default_shape() { return dct_launch_shape{256, 8, kTileBlocks, 2}; }

// Checks one plane against the plan limits; `what` names it in errors.
dct_status check_plane(const dct_plan_s* plan, const dct_plane& p, const char* what);

// Fills the PlaneArg geometry fields and the running tile/coef offsets.
void fill_plane(PlaneArg& a, const dct_plane& p, int& tile_cursor);

// Frees the plan's batch workspace and graph (batch.cu).
void batch_release(dct_plan_t plan);

// Launches the batched persistent kernel of `mode` over a device work list
// (no graph), with the plan's launch shape (batch.cu).  With tile_counter (a
// device word the caller has zeroed on `s` before the launch) a two-lane
// kernel claims its tiles from it; without, warps take fixed ranges.
cudaError_t batch_launch(unsigned mode, const PlaneArg* items, const int32_t* tile_begin, const QuantSet* tabs,
                         int nitems, int ntiles, const dct_plan_s* plan, cudaStream_t s,
                         unsigned int* tile_counter = nullptr);

// Frees the plan's rate-control workspace (ratecontrol.cu).
void rc_release(dct_plan_t plan);

// Network kernels (mlp.cu).
cudaError_t launch_features(const unsigned long long* stats, const int* w, const int* h, const float* t, int n,
                            float* out, cudaStream_t s);
cudaError_t launch_mlp_forward(const dct_mlp* net, const float* feats, int n, float* y, int* q, cudaStream_t s);

}  // namespace dctgb
