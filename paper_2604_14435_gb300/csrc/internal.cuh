// Internal helpers of the D-VQLS CUDA library: the context, its device
// workspace arena, pinned staging of host arguments, and error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <unordered_set>
#include <vector>

#include "../../include/dvqls.h"

namespace dvqls {

// Status word the kernels write (first error wins); read by dvqls_sync and
// by the synchronous entry points.
enum DeviceStatus : int {
    DEV_OK = 0,
    DEV_BAD_MASK = 1,
    DEV_NONFINITE_INPUT = 2,
    DEV_BAD_NORM = 3,
    DEV_BAD_DENOMINATOR = 4,
    DEV_TIMEOUT = 5,
};

struct GraphCacheEntry;  // defined in terms.cu

}  // namespace dvqls

namespace dvqls {
// An NVTX range over a scope: names the library's API phases on a profiler's
// timeline (Nsight Systems and the like); without a profiler attached the
// calls return at once.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};
}  // namespace dvqls
#define DVQLS_NVTX(name) ::dvqls::NvtxScope dvqls_nvtx_scope_(name)

struct dvqls_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;  // the caller's stream (nullptr: default stream)
    int num_sms = 0;
    size_t smem_optin = 0;
    std::string err;

    // Device workspace: one allocation, carved per call.
    char* ws = nullptr;
    size_t ws_cap = 0;
    // Pinned host staging for host arguments and results.
    char* pin = nullptr;
    size_t pin_cap = 0;
    // Device status word + queue counters (separate small allocation so the
    // workspace can grow without invalidating it).
    int* d_status = nullptr;
    unsigned long long* d_queue = nullptr;
    // Pinned word the status is read into (an asynchronous copy, then one
    // stream synchronisation).
    int* h_status = nullptr;

    // Pinned staging is reused by every call: pin_event marks the last
    // host-to-device copy out of it; it is waited on before the next write.
    cudaEvent_t pin_event = nullptr;
    bool pin_event_live = false;
    // Last instance table uploaded by the batched call (skipped when equal).
    std::vector<char> last_table;

    // Kernel timing (dvqls_profile_*): event pairs not yet read, a pool of
    // reusable events, and per-phase totals.
    bool profiling = false;
    struct Mark { int phase; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    long long prof_launches[5] = {0, 0, 0, 0, 0};
    double prof_ms[5] = {0, 0, 0, 0, 0};

    // Time each bounded device wait of the tensor-core term kernel allows
    // before it gives up, in microseconds (dvqls_set_wait_budget).
    long long wait_budget_us = 1000000;

    // dvqls_set_tuning: a fixed amplitude split (0: tune) and state layout (-1: tune).
    int fixed_split = 0, fixed_layout = -1;

    // Addresses already found to be host memory (not device memory of this
    // device, not managed): a later call skips their pointer-kind query.  A
    // host address stays outside the range the driver reserves for device
    // allocations, so the answer cannot turn into "device"; at worst memory
    // that became managed there is staged through the pinned buffer.
    std::unordered_set<const void*> host_ptrs;

    // Cached batched-call state (see terms.cu): the last captured graph of a
    // cost pass, the private stream graphs are captured on, and the
    // autotuned amplitude split per problem signature.
    dvqls::GraphCacheEntry* graph = nullptr;
    cudaStream_t cap_stream = nullptr;
    std::map<std::string, int> tune;
    // Deferred staging (stage_in / enqueue_out between begin_staging and
    // flush_in / flush_out): copies are recorded and issued merged.
    struct CopySeg {
        size_t pin_off, dev_off, bytes;
    };
    bool defer = false;
    std::vector<CopySeg> seg_in, seg_out;
};

namespace dvqls {

int set_error(dvqls_ctx* ctx, int code, const char* fmt, ...);

// Drop the captured cost-pass graph (terms.cu).
void release_graph_cache(dvqls_ctx* ctx);

#define DVQLS_CUDA_TRY(ctx, call)                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::dvqls::set_error((ctx), DVQLS_ERR_CUDA, "%s: %s (%s:%d)", #call,        \
                                      cudaGetErrorString(e_), __FILE__, __LINE__);          \
    } while (0)

// True when p is memory the context's device can dereference (device or
// managed memory of that device).
bool is_device_ptr(const dvqls_ctx* ctx, const void* p);

// A per-call plan of device workspace and pinned staging regions.  Sizes
// are added first (reserve), the memory is then made available (commit) and
// the regions are handed out in the same order (take).
class Arena {
   public:
    size_t reserve(size_t bytes) {
        size_t off = total_;
        total_ += (bytes + 255) & ~size_t(255);
        return off;
    }
    size_t total() const { return total_; }

   private:
    size_t total_ = 0;
};

int ensure_workspace(dvqls_ctx* ctx, size_t bytes);
// Wait until no copy out of the pinned staging is pending, so it can be
// written again; pin_release records the end of the copies just enqueued.
int pin_acquire(dvqls_ctx* ctx);
int pin_release(dvqls_ctx* ctx);
int ensure_pinned(dvqls_ctx* ctx, size_t bytes);

// Stage a caller buffer for device use: device pointers pass through; host
// data is copied to pinned memory at pin_off and then to the device region
// at ws_off.  Returns the device pointer.
const void* stage_in(dvqls_ctx* ctx, const void* p, size_t bytes, size_t pin_off, size_t ws_off);

// Deferred staging: after begin_staging, stage_in and enqueue_out record
// their host <-> device copies; flush_in / flush_out issue them, merging
// segments that follow each other in both the pinned and the device arena
// (consecutive Arena reservations, so only alignment padding is copied
// along) into one cudaMemcpyAsync each.  end_staging returns to immediate
// copies.
void begin_staging(dvqls_ctx* ctx);
int flush_in(dvqls_ctx* ctx);
int flush_out(dvqls_ctx* ctx);
void end_staging(dvqls_ctx* ctx);

// Copy a device result to the caller's buffer (device or host).  Host
// destinations go through pinned memory at pin_off; the copy to the caller
// happens in finish_out after the stream is synchronised.
struct PendingOut {
    void* dst;
    size_t pin_off;
    size_t bytes;
};
int enqueue_out(dvqls_ctx* ctx, void* dst, const void* dev_src, size_t bytes, size_t pin_off,
                std::vector<PendingOut>& pending);
int finish_out(dvqls_ctx* ctx, const std::vector<PendingOut>& pending);

// Kernel timing: prof_begin before a launch, prof_end after it (no-ops when
// profiling is off).
void prof_begin(dvqls_ctx* ctx, int phase);
void prof_end(dvqls_ctx* ctx);

// Synchronise, then turn the device status word into a status code.
int sync_and_check(dvqls_ctx* ctx);

// Raises the dynamic shared-memory limit of kernel `fn` on the current device
// to everything the device allows (its opt-in maximum less the kernel's
// static shared memory).  Every caller sets the same value, so one caller
// cannot lower the limit between another caller's set-up and its launch (two
// contexts on two threads, or a context and the allocation-free entry point).
cudaError_t allow_dynamic_smem(const void* fn);

inline int ceil_div(long long a, long long b) { return int((a + b - 1) / b); }

// A cost pass over the shifts s0 .. s1 - 1 of one instance that writes the
// per-shift sums (4 doubles per shift of the instance, zeros outside the
// range) to `partials` instead of forming the cost (terms.cu).
struct ShiftRange {
    int s0, s1;
    double* partials;
};

// F = |<xhat|psi(alpha)>|^2 / ||xhat||^2 with psi built in HBM (terms.cu), for
// n above the shared-memory size.
int fidelity_hbm(dvqls_ctx* ctx, int n, int d, const double* alpha, const double* xhat, double* F);

// The batched cost pass (terms.cu): cost and gradient (or, with a shift range,
// per-shift sums) of `count` instances.
int run_batch(dvqls_ctx* ctx, int count, const dvqls_instance* inst, int precision, bool want_grad, double* costs,
              double* grads, double* beta_out, double* delta_out, bool local, const ShiftRange* range = nullptr);

}  // namespace dvqls
