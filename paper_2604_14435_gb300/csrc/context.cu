// Context life cycle, workspace and staging for the D-VQLS C-ABI.
#include <algorithm>

#include "internal.cuh"

namespace dvqls {

int set_error(dvqls_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return code;
}

bool is_device_ptr(const dvqls_ctx* ctx, const void* p) {
    if (!p) return false;
    auto& seen = const_cast<dvqls_ctx*>(ctx)->host_ptrs;
    if (seen.count(p)) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const bool dev = a.type == cudaMemoryTypeDevice ? a.device == ctx->device : a.type == cudaMemoryTypeManaged;
    if (!dev && a.type != cudaMemoryTypeDevice) {  // host memory (device memory of another GPU is not cached)
        if (seen.size() >= 4096) seen.clear();
        seen.insert(p);
    }
    return dev;
}

cudaError_t allow_dynamic_smem(const void* fn) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, fn);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(fa.sharedSizeBytes));
    return e;
}

int ensure_workspace(dvqls_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->ws_cap) return DVQLS_OK;
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->last_table.clear();
    release_graph_cache(ctx);
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
    size_t cap = bytes + bytes / 4 + (1 << 20);
    if (cudaMalloc(&ctx->ws, cap) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, DVQLS_ERR_ALLOC, "device workspace of %zu bytes", cap);
    }
    ctx->ws_cap = cap;
    return DVQLS_OK;
}

int pin_acquire(dvqls_ctx* ctx) {
    if (ctx->pin_event_live) {
        DVQLS_CUDA_TRY(ctx, cudaEventSynchronize(ctx->pin_event));
        ctx->pin_event_live = false;
    }
    return DVQLS_OK;
}

int pin_release(dvqls_ctx* ctx) {
    DVQLS_CUDA_TRY(ctx, cudaEventRecord(ctx->pin_event, ctx->stream));
    ctx->pin_event_live = true;
    return DVQLS_OK;
}

int ensure_pinned(dvqls_ctx* ctx, size_t bytes) {
    if (bytes <= ctx->pin_cap) return DVQLS_OK;
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->pin) cudaFreeHost(ctx->pin);
    ctx->pin = nullptr;
    ctx->pin_cap = 0;
    size_t cap = bytes + bytes / 4 + (1 << 16);
    if (cudaMallocHost(&ctx->pin, cap) != cudaSuccess) {
        cudaGetLastError();
        return set_error(ctx, DVQLS_ERR_ALLOC, "pinned staging of %zu bytes", cap);
    }
    ctx->pin_cap = cap;
    return DVQLS_OK;
}

const void* stage_in(dvqls_ctx* ctx, const void* p, size_t bytes, size_t pin_off, size_t ws_off) {
    if (!p || bytes == 0) return p;
    if (is_device_ptr(ctx, p)) return p;
    memcpy(ctx->pin + pin_off, p, bytes);
    void* dst = ctx->ws + ws_off;
    if (ctx->defer) ctx->seg_in.push_back({pin_off, ws_off, bytes});
    else cudaMemcpyAsync(dst, ctx->pin + pin_off, bytes, cudaMemcpyHostToDevice, ctx->stream);
    return dst;
}

int enqueue_out(dvqls_ctx* ctx, void* dst, const void* dev_src, size_t bytes, size_t pin_off,
                std::vector<PendingOut>& pending) {
    if (!dst || bytes == 0) return DVQLS_OK;
    if (is_device_ptr(ctx, dst)) {
        if (dst != dev_src)
            DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(dst, dev_src, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        return DVQLS_OK;
    }
    const char* src = static_cast<const char*>(dev_src);
    if (ctx->defer && src >= ctx->ws && src + bytes <= ctx->ws + ctx->ws_cap)
        ctx->seg_out.push_back({pin_off, size_t(src - ctx->ws), bytes});
    else
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pin + pin_off, dev_src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    pending.push_back({dst, pin_off, bytes});
    return DVQLS_OK;
}

void begin_staging(dvqls_ctx* ctx) {
    ctx->defer = true;
    ctx->seg_in.clear();
    ctx->seg_out.clear();
}

void end_staging(dvqls_ctx* ctx) {
    ctx->defer = false;
    ctx->seg_in.clear();
    ctx->seg_out.clear();
}

// Issues the recorded segments in order, one copy per run of segments that
// follow each other (next offset = previous offset + bytes rounded up to the
// 256-byte Arena granule) in both arenas.
static int flush_segs(dvqls_ctx* ctx, std::vector<dvqls_ctx::CopySeg>& segs, bool to_device) {
    size_t i = 0;
    while (i < segs.size()) {
        const size_t p0 = segs[i].pin_off, d0 = segs[i].dev_off;
        size_t end = segs[i].bytes, j = i + 1;
        while (j < segs.size()) {
            const size_t gap = (end + 255) & ~size_t(255);
            if (segs[j].pin_off != p0 + gap || segs[j].dev_off != d0 + gap) break;
            end = gap + segs[j].bytes;
            ++j;
        }
        if (to_device)
            DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + d0, ctx->pin + p0, end, cudaMemcpyHostToDevice, ctx->stream));
        else
            DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pin + p0, ctx->ws + d0, end, cudaMemcpyDeviceToHost, ctx->stream));
        i = j;
    }
    segs.clear();
    return DVQLS_OK;
}

int flush_in(dvqls_ctx* ctx) { return flush_segs(ctx, ctx->seg_in, true); }
int flush_out(dvqls_ctx* ctx) { return flush_segs(ctx, ctx->seg_out, false); }

int finish_out(dvqls_ctx* ctx, const std::vector<PendingOut>& pending) {
    for (const auto& p : pending) memcpy(p.dst, ctx->pin + p.pin_off, p.bytes);
    return DVQLS_OK;
}

int sync_and_check(dvqls_ctx* ctx) {
    DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    const int st = *ctx->h_status;
    if (st == DEV_OK) return DVQLS_OK;
    DVQLS_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int), ctx->stream));
    switch (st) {
        case DEV_BAD_MASK:
            return set_error(ctx, DVQLS_ERR_INVALID_ARG, "a Pauli mask is >= 2^n");
        case DEV_NONFINITE_INPUT:
            return set_error(ctx, DVQLS_ERR_INVALID_ARG, "non-finite angle, coefficient or b entry");
        case DEV_BAD_NORM:
            return set_error(ctx, DVQLS_ERR_INVALID_ARG, "||b|| is zero or not finite");
        case DEV_BAD_DENOMINATOR:
            return set_error(ctx, DVQLS_ERR_NUMERIC, "denominator <x|A^dag A|x> <= 0 or not finite");
        case DEV_TIMEOUT:
            return set_error(ctx, DVQLS_ERR_TIMEOUT, "a bounded device wait gave up");
        default:
            return set_error(ctx, DVQLS_ERR_NUMERIC, "device status %d", st);
    }
}

static cudaEvent_t take_event(dvqls_ctx* ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(dvqls_ctx* ctx, int phase) {
    if (!ctx->profiling) return;
    dvqls_ctx::Mark m{phase, take_event(ctx), take_event(ctx)};
    cudaEventRecord(m.a, ctx->stream);
    ctx->marks.push_back(m);
}

void prof_end(dvqls_ctx* ctx) {
    if (!ctx->profiling || ctx->marks.empty()) return;
    cudaEventRecord(ctx->marks.back().b, ctx->stream);
}

static int prof_drain(dvqls_ctx* ctx) {
    if (ctx->marks.empty()) return DVQLS_OK;
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& m : ctx->marks) {
        float ms = 0.f;
        DVQLS_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, m.a, m.b));
        ctx->prof_launches[m.phase] += 1;
        ctx->prof_ms[m.phase] += ms;
        ctx->event_pool.push_back(m.a);
        ctx->event_pool.push_back(m.b);
    }
    ctx->marks.clear();
    return DVQLS_OK;
}

}  // namespace dvqls

using namespace dvqls;

extern "C" int dvqls_profile_enable(dvqls_ctx* ctx, int enable) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    int rc = prof_drain(ctx);
    if (rc) return rc;
    if (enable) {
        for (int k = 0; k < 5; ++k) {
            ctx->prof_launches[k] = 0;
            ctx->prof_ms[k] = 0.0;
        }
    }
    ctx->profiling = enable != 0;
    return DVQLS_OK;
}

extern "C" int dvqls_profile_read(dvqls_ctx* ctx, int phase, long long* launches, double* ms) {
    if (!ctx || phase < 0 || phase > 4 || !launches || !ms) return DVQLS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    int rc = prof_drain(ctx);
    if (rc) return rc;
    *launches = ctx->prof_launches[phase];
    *ms = ctx->prof_ms[phase];
    return DVQLS_OK;
}

extern "C" int dvqls_create(dvqls_ctx** out, int device, void* stream) {
    if (!out) return DVQLS_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return DVQLS_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return DVQLS_ERR_INVALID_ARG;
    dvqls_ctx* ctx = new dvqls_ctx();
    ctx->device = device;
    int rc = DVQLS_OK;
    do {
        if (cudaSetDevice(device) != cudaSuccess) { rc = DVQLS_ERR_CUDA; break; }
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { rc = DVQLS_ERR_CUDA; break; }
        ctx->num_sms = prop.multiProcessorCount;
        ctx->smem_optin = prop.sharedMemPerBlockOptin;
        ctx->stream = (cudaStream_t)stream;
        if (cudaEventCreateWithFlags(&ctx->pin_event, cudaEventDisableTiming) != cudaSuccess) {
            rc = DVQLS_ERR_CUDA;
            break;
        }
        if (cudaMalloc(&ctx->d_status, 256) != cudaSuccess) { rc = DVQLS_ERR_ALLOC; break; }
        if (cudaMallocHost(&ctx->h_status, 64) != cudaSuccess) { rc = DVQLS_ERR_ALLOC; break; }
        ctx->d_queue = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctx->d_status) + 64);
        if (cudaMemsetAsync(ctx->d_status, 0, 256, ctx->stream) != cudaSuccess) { rc = DVQLS_ERR_CUDA; break; }
        if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) { rc = DVQLS_ERR_CUDA; break; }
    } while (0);
    if (rc != DVQLS_OK) {
        cudaGetLastError();
        dvqls_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return DVQLS_OK;
}

extern "C" void dvqls_destroy(dvqls_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    dvqls::release_graph_cache(ctx);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->pin_event) cudaEventDestroy(ctx->pin_event);
    for (auto& m : ctx->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    cudaGetLastError();
    delete ctx;
}

extern "C" int dvqls_set_wait_budget(dvqls_ctx* ctx, long long microseconds) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->wait_budget_us = microseconds > 0 ? std::min(microseconds, 3600LL * 1000000LL) : 1000000LL;
    return DVQLS_OK;
}

extern "C" int dvqls_set_tuning(dvqls_ctx* ctx, int split, int layout) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    if (split != 0 && split != 1 && split != 2 && split != 4 && split != 8)
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "split %d is not 0, 1, 2, 4 or 8", split);
    if (layout < -1 || layout > 2) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "layout %d is not -1 .. 2", layout);
    ctx->fixed_split = split;
    ctx->fixed_layout = layout;
    return DVQLS_OK;
}

extern "C" const char* dvqls_last_error(const dvqls_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int dvqls_sync(dvqls_ctx* ctx) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    return sync_and_check(ctx);
}
