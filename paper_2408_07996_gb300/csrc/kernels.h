// kernels.h -- host-callable launchers of the renderer's kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace mcev {

enum { MODE_REFERENCE = 0, MODE_DETECT = 1, MODE_MEAN = 2 };
enum { VAR_ONE_TAILED = 0, VAR_TWO_TAILED = 1, VAR_MEAN_ONLY = 2, VAR_UNIFORM = 3 };
enum { SE_PAPER = 0, SE_WELCH = 1 };

struct StatsArgs {
    PixStats cur, ref;
    const float* tcrit;   // critical t per test round r, n = spp_min + r * spp_batch
    int8_t* events;
    int32_t* spp_out;
    float* mean_out;
    float eps, C;
    int32_t spp_r;        // samples per pixel traced this round
    int32_t sub;          // batch size: the round's samples are merged and tested in batches of `sub`
    int64_t k_base;       // samples taken before this round
    int32_t spp_min, spp_batch, spp_max;
    int32_t mode, variant, se_mode;
    int64_t n_total;      // per-pixel array length, checked only by the allocation-free entry point
};

// State of the device-resident round loop of one call (device memory): the
// round's pixel queue and sizes, the current chunk, and what was done.  The
// control kernel advances it after every chunk; raygen and the statistics
// kernel read their sizes from it instead of from launch arguments.
struct RoundCtl {
    int32_t* queue[2];        // ping-pong pixel queues; queue[qi] is this round's
    int64_t Q;                // pixels queued this round
    int64_t n_done;           // samples every queued pixel already has (k_base)
    int64_t j0, nj;           // current chunk: first queue entry, pixels
    int64_t per_chunk;        // pixels per chunk this round
    int64_t paths;            // samples traced by finished rounds
    int64_t stats_pix;        // pixel visits of the statistics kernel
    int32_t spp_r, sub;       // samples per pixel this round; batch size of its tests
    int32_t qi, rounds, iters;
    int32_t status;           // RC_OK, RC_TIMEOUT (a bound ran out), RC_CAP (undecided at spp_max)
    unsigned long long t_start;  // %globaltimer (ns) when the loop started
};
enum { RC_OK = 0, RC_TIMEOUT = 1, RC_CAP = 2 };

// Bounds and schedule of a device-resident round loop.
struct RoundPlan {
    int64_t cap;              // wavefront paths per chunk
    int64_t Q0;               // pixels queued in the first round
    int32_t spp_min, spp_batch, spp_max, window_max;
    int32_t max_iters;        // chunks after which the loop gives up (RC_TIMEOUT)
    int32_t pad;
    unsigned long long timeout_ns;  // wall-clock bound of the loop (RC_TIMEOUT)
};

// `jobs`: device job table of a batched render, or nullptr for a single
// context (then the frame / settings / state arguments are used).  `rc`:
// sizes from the device-resident round loop instead of the arguments.
cudaError_t launch_raygen(const DevFrame& fr, const DevParams& P, const Wave& w, const int32_t* queue, int64_t j0,
                          int32_t spp_r, int64_t k_base, int64_t n_paths, int cur, int sms, cudaStream_t st,
                          const Job* jobs, const RoundCtl* rc = nullptr);
// `wide`: the scenes' BLAS use the compressed 8-wide layout (Node8)
// Traversal kernel variant (the `trav` argument of the launchers): the BLAS
// layout, and whether the frame has two or more moving instances under a
// TLAS (frames with at most one run kernels without the TLAS loop).
enum { TRAV_WIDE = 1, TRAV_TLAS = 2 };

cudaError_t launch_extend(const DevScene& sc, const DevFrame& fr, float t_min, const Wave& w, int cur, int64_t max_n,
                          int32_t* err, int sms, cudaStream_t st, const Job* jobs, int trav);
cudaError_t launch_shade(const DevScene& sc, const DevFrame& fr, const DevParams& P, const Wave& w, int cur,
                         int64_t max_n, int sms, cudaStream_t st, const Job* jobs);
cudaError_t launch_shadow(const DevScene& sc, const DevFrame& fr, const DevParams& P, const Wave& w, int cur,
                          int64_t max_n, int32_t* err, int sms, cudaStream_t st, const Job* jobs, int trav);
// shadow rays of the bounce with queue `cur` and closest hits of queue 1 - cur, in one launch
cudaError_t launch_shadow_extend(const DevScene& sc, const DevFrame& fr, const DevParams& P, const Wave& w, int cur,
                                 int64_t max_n, int32_t* err, int sms, cudaStream_t st, const Job* jobs, int trav);
cudaError_t launch_stats(const Wave& w, const StatsArgs& A, const int32_t* queue, int64_t j0, int64_t n_pix,
                         int32_t* next_queue, int sms, cudaStream_t st, const Job* jobs, const RoundCtl* rc = nullptr);
// device-resident round loop: start state (and, with iota, queue 0 = 0..Q0-1)
cudaError_t launch_round_init(RoundCtl* rc, const Wave& w, const RoundPlan& plan, int32_t* q0, int32_t* q1,
                              bool iota, int sms, cudaStream_t st);
// after a chunk: next chunk or round, or the end of the loop (condition 0)
cudaError_t launch_round_next(RoundCtl* rc, const Wave& w, const RoundPlan& plan, cudaGraphConditionalHandle h,
                              cudaStream_t st);
// out[i] += (float)acc[i] for i < n (the adjoint's FP64 emission accumulator)
cudaError_t launch_add_f64(float* out, const double* acc, int n, cudaStream_t st);
cudaError_t launch_fill_entries(int32_t* q, int64_t n, int job, int sms, cudaStream_t st);
cudaError_t launch_write_samples(const Wave& w, int64_t out0, int64_t n_paths, float* L_out, uint32_t* sig_out,
                                 int sms, cudaStream_t st);
cudaError_t launch_iota(int32_t* q, int64_t n, int sms, cudaStream_t st);

}  // namespace mcev
