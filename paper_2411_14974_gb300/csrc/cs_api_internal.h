// Host-side objects behind the C-ABI handles.
#pragma once

#include <cuda_runtime.h>

#include <condition_variable>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cs_common.cuh"

struct cs_context {
    int device = 0;
    int sm_count = 0;
    cudaMemPool_t pool = nullptr;             // stream-ordered pool for every transient buffer
    unsigned long long *host_total = nullptr; // pinned readback slots (8 words): the forward's totals
    unsigned long long *host_total_dev = nullptr;  // the same slots in the device's address space
    cudaEvent_t totals_ready = nullptr;       // recorded after the readback of the forward's totals
    // stage profiling: events recorded on the launching stream around every stage
    bool profiling = false;
    struct StageRec {
        int stage;
        cudaEvent_t a, b;
    };
    std::mutex prof_mu;
    std::vector<StageRec> prof;
    std::vector<cudaEvent_t> free_events;
    // pipelined host-buffer steps (cs_step_host_submit): HOST_SLOTS slots of device buffers
    // (scene, cotangent, image, gradients).  The caller's thread copies a step's inputs into its
    // slot on the upload stream and queues the step; the context's worker thread enqueues the
    // step's forward and backward on the compute stream (waiting there for the forward's pair
    // count) and the copies of its outputs on the download stream.  Uploads of later steps, the
    // compute of one step and downloads of earlier ones thus run at the same time.
    static constexpr int HOST_SLOTS = 3;
    struct HostSlot {
        void *buf = nullptr;  // the slot's twelve arrays, 256-byte aligned
        size_t cap = 0;
        cudaEvent_t uploaded = nullptr, computed = nullptr, done = nullptr;
        uint64_t ticket = 0;  // the last step submitted into this slot (0: none)
    };
    struct HostJob {          // one queued step, its inputs already on the upload stream
        uint64_t ticket = 0;
        int slot = 0;
        bool bwd = false;
        bool has_settings = false;
        cs_scene scene{};     // the slot's device copies of the scene
        cs_camera cam{};
        cs_settings settings{};
        float *image_host = nullptr;
        float *outs_host[5] = {};
        void *d[12] = {};
        size_t sizes[12] = {};
    };
    HostSlot host_slots[HOST_SLOTS];
    cudaStream_t upload_stream = nullptr, compute_stream = nullptr, download_stream = nullptr;
    uint64_t host_tickets = 0;
    std::mutex host_mu;                 // one submit or wait at a time
    std::thread host_worker;
    std::mutex job_mu;                  // guards the queue and the fields below
    std::condition_variable job_cv;
    std::deque<HostJob> jobs;
    bool worker_stop = false;
    uint64_t jobs_enqueued = 0;         // every step up to this ticket has its GPU work enqueued
    cs_status host_code = CS_OK;        // first failure of a queued step since the last report
    std::string host_msg;
};

struct cs_fwd_state {
    cs_context *ctx = nullptr;
    cudaStream_t stream = nullptr;  // stream of the forward; buffers are freed on it
    cs_scene scene{};
    int k = 0;
    cs_settings settings{};
    cs::Settings st{};
    std::vector<cs::ViewDesc> views;  // host copy (with device pointers filled in)
    cs::ViewDesc *views_dev = nullptr;
    int64_t n_records = 0, n_pairs = 0;
    uint32_t n_tiles = 0;
    int local_bits = 0;  // pair key = view << local_bits | tile index within the view
    int mask_shift = 0;  // block masks above the view bits (0: none)
    float4 *records = nullptr;
    uint32_t *depth_keys = nullptr;
    uint2 *rects = nullptr;
    uint32_t *counts = nullptr;
    float4 *bboxes = nullptr;
    uint32_t *pair_keys = nullptr, *pair_vals = nullptr;
    uint2 *ranges = nullptr;
    uint32_t *n_last = nullptr;
    float *t_final_own = nullptr;          // [pixels of all views], read by the backward
    std::vector<float *> user_t_final;     // caller's T_final buffers (copied to after the blend)
    // when not empty (one event per view): the forward blends view by view, in view order, and
    // records view_done[v] on the stream once view v's image is written
    std::vector<cudaEvent_t> view_done;
    // when not NULL (set by the serving loop, with view_done, at most 32 views, no tile split):
    // the views are blended by one persistent launch, which stores flag_value into view_flags[v]
    // (mapped host memory, device address) once view v's image is written
    uint32_t *view_flags = nullptr;
    uint32_t flag_value = 0;
    // tile split (settings.tile_split > 0): work items, heavy tiles, slots and chunk states, kept
    // for the backward
    uint32_t *tile_order = nullptr;  // blend launch order of the tiles (longest lists first)
    uint2 *split_items = nullptr, *split_heavy = nullptr;
    uint32_t *split_slot = nullptr;
    float *chunk_state = nullptr;
    uint32_t n_items = 0, n_heavy = 0;
};

namespace cs {
cs_status fail(cs_status st, const char *fmt, ...);
cs_status fail_cuda(cudaError_t e, const char *what);
cudaError_t pool_alloc(cs_context *ctx, void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);
cs_status check_settings(const cs_settings *st);
cs_status check_camera(const cs_camera *c);
cs_status check_scene(const cs_scene *s);
void fill_view(ViewDesc &vd, const cs_camera &c);
Settings to_settings(const cs_settings &s);
cs_status run_forward(cs_context *ctx, cs_fwd_state *s, cudaStream_t stream);
// checked builds: after the work enqueued on s, the kernels' failed index tests as CS_ERR_DEVICE
// (synchronises s); production builds: CS_OK without synchronising
cs_status take_device_status(cudaStream_t s, const char *what);
void state_free(cs_fwd_state *s);

// makes ctx's device current for the lifetime of the guard
struct DeviceGuard {
    int prev = 0;
    explicit DeviceGuard(int d) {
        cudaGetDevice(&prev);
        cudaSetDevice(d);
    }
    ~DeviceGuard() { cudaSetDevice(prev); }
};

// brackets a stage with events when the context is profiling
class StageTimer {
  public:
    StageTimer(cs_context *ctx, int stage, cudaStream_t s);
    ~StageTimer();

  private:
    cs_context *ctx_;
    int stage_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr;
};
}  // namespace cs
