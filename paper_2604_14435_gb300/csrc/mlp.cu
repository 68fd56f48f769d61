// Learned warm start: a small MLP that maps a problem description to initial
// ansatz angles, trained and run on the GPU by the kernels below (FP32).
//
//   h1 = GELU(W1 x + b1), h2 = GELU(W2 h1 + b2), y = W3 h2 + b3,
//   GELU(z) = z (1 + erf(z / sqrt 2)) / 2,
//   loss = sum M (y - t)^2 / sum M  (masked mean squared error),
//
// with back-propagation and Adam.  Every product is a tiled GEMM whose
// output element is reduced by one thread in a fixed order, so gradients are
// deterministic.  Parameters are one flat FP32 vector: W1 [H x I], b1 [H],
// W2 [H x H], b2 [H], W3 [O x H], b3 [O] (row-major).
#include <algorithm>
#include <cstdio>

#include "internal.cuh"

struct dvqls_ws {
    dvqls_ctx* ctx;
    int I, H, O;
    long long np;
    float* params;  // np
    float* grad;    // np
    float* m;       // np
    float* v;       // np
    long long step;
    int cap;        // batch capacity of the activations
    float* act;     // X, z1, h1, z2, h2, y, dy, dz2, dz1, T, M (batch-major)
    float* lossbuf; // 2 floats: sum M (y-t)^2, sum M
    char* pin;      // small pinned buffer for the loss
};

namespace dvqls {
namespace {

constexpr int TG = 16;

// C[m, n] = sum_k A(m, k) B(k, n) (+ bias[n]); A(m, k) = A[m*sam + k*sak],
// B(k, n) = B[k*sbk + n*sbn].  epi: 0 none, 1 bias, 2 bias + GELU (z kept in
// Z, GELU(z) in C).
__global__ void k_gemm(int M, int N, int K, const float* __restrict__ A, long long sam, long long sak,
                       const float* __restrict__ B, long long sbk, long long sbn, float* C, const float* bias,
                       float* Z, int epi) {
    __shared__ float As[TG][TG + 1], Bs[TG][TG + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int m = blockIdx.y * TG + ty, n = blockIdx.x * TG + tx;
    float acc = 0.f;
    for (int k0 = 0; k0 < K; k0 += TG) {
        const int ka = k0 + tx, kb = k0 + ty;
        As[ty][tx] = (m < M && ka < K) ? A[m * sam + ka * sak] : 0.f;
        Bs[ty][tx] = (kb < K && n < N) ? B[kb * sbk + n * sbn] : 0.f;
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TG; ++k) acc = fmaf(As[ty][k], Bs[k][tx], acc);
        __syncthreads();
    }
    if (m < M && n < N) {
        if (epi >= 1) acc += bias[n];
        if (epi == 2) {
            Z[(long long)m * N + n] = acc;
            acc = 0.5f * acc * (1.f + erff(acc * 0.70710678118654752f));
        }
        C[(long long)m * N + n] = acc;
    }
}

// dz = da * GELU'(z), in place on da.
__global__ void k_gelu_back(long long count, const float* __restrict__ z, float* da) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float x = z[i];
    const float d = 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.3989422804014327f;
    da[i] *= d;
}

// Column sums (bias gradients): out[n] = sum_b D[b, n], fixed order.
__global__ void k_colsum(int B, int N, const float* __restrict__ D, float* out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float s = 0.f;
    for (int b = 0; b < B; ++b) s += D[(long long)b * N + n];
    out[n] = s;
}

// dy = 2 M (y - t) / sum M; loss numerator and sum M to lossbuf (one CTA).
__global__ void k_loss(long long count, const float* __restrict__ y, const float* __restrict__ t,
                       const float* __restrict__ Mk, float* dy, float* lossbuf) {
    __shared__ float r1[32], r2[32];
    float a = 0.f, c = 0.f;
    for (long long i = threadIdx.x; i < count; i += blockDim.x) {
        const float e = y[i] - t[i];
        a += Mk[i] * e * e;
        c += Mk[i];
    }
    for (int o = 16; o; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = a;
        r2[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    a = c = 0.f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        a += r1[k];
        c += r2[k];
    }
    const float inv = c > 0.f ? 2.f / c : 0.f;
    for (long long i = threadIdx.x; i < count; i += blockDim.x) dy[i] = inv * Mk[i] * (y[i] - t[i]);
    if (threadIdx.x == 0) {
        lossbuf[0] = a;
        lossbuf[1] = c;
    }
}

__global__ void k_adam32(long long np, const float* __restrict__ g, float* p, float* m, float* v, float lr, float b1,
                         float b2, float eps, float c1, float c2) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

struct Views {
    float *X, *z1, *h1, *z2, *h2, *y, *dy, *d2, *d1, *T, *M;
};

Views views(dvqls_ws* w, int Bc) {
    Views a;
    float* p = w->act;
    auto take = [&](long long n) {
        float* r = p;
        p += n;
        return r;
    };
    a.X = take((long long)Bc * w->I);
    a.z1 = take((long long)Bc * w->H);
    a.h1 = take((long long)Bc * w->H);
    a.z2 = take((long long)Bc * w->H);
    a.h2 = take((long long)Bc * w->H);
    a.y = take((long long)Bc * w->O);
    a.dy = take((long long)Bc * w->O);
    a.d2 = take((long long)Bc * w->H);
    a.d1 = take((long long)Bc * w->H);
    a.T = take((long long)Bc * w->O);
    a.M = take((long long)Bc * w->O);
    return a;
}

long long act_floats(const dvqls_ws* w, int Bc) {
    return (long long)Bc * (w->I + 6LL * w->H + 4LL * w->O);
}

int ensure_batch(dvqls_ws* w, int batch) {
    if (batch <= w->cap) return DVQLS_OK;
    dvqls_ctx* ctx = w->ctx;
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    if (w->act) cudaFree(w->act);
    w->act = nullptr;
    int cap = std::max(batch, 64);
    if (cudaMalloc(&w->act, act_floats(w, cap) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        w->cap = 0;
        return set_error(ctx, DVQLS_ERR_ALLOC, "warm-start activations for batch %d", cap);
    }
    w->cap = cap;
    return DVQLS_OK;
}

void gemm(dvqls_ctx* ctx, int M, int N, int K, const float* A, long long sam, long long sak, const float* B,
          long long sbk, long long sbn, float* C, const float* bias, float* Z, int epi) {
    dim3 blk(TG, TG), grd(ceil_div(N, TG), ceil_div(M, TG));
    k_gemm<<<grd, blk, 0, ctx->stream>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, bias, Z, epi);
}

void forward(dvqls_ws* w, const Views& a, int B) {
    const float* W1 = w->params;
    const float* b1 = W1 + (long long)w->H * w->I;
    const float* W2 = b1 + w->H;
    const float* b2 = W2 + (long long)w->H * w->H;
    const float* W3 = b2 + w->H;
    const float* b3 = W3 + (long long)w->O * w->H;
    // z1[b, h] = sum_i X[b, i] W1[h, i]: B(k=i, n=h) = W1[h*I + i]
    gemm(w->ctx, B, w->H, w->I, a.X, w->I, 1, W1, 1, w->I, a.h1, b1, a.z1, 2);
    gemm(w->ctx, B, w->H, w->H, a.h1, w->H, 1, W2, 1, w->H, a.h2, b2, a.z2, 2);
    gemm(w->ctx, B, w->O, w->H, a.h2, w->H, 1, W3, 1, w->H, a.y, b3, nullptr, 1);
}

// Gradient of the masked loss into w->grad; loss parts into w->lossbuf.
void backward(dvqls_ws* w, const Views& a, int B) {
    dvqls_ctx* ctx = w->ctx;
    const int I = w->I, H = w->H, O = w->O;
    const float* W2 = w->params + (long long)H * I + H;
    const float* W3 = W2 + (long long)H * H + H;
    float* gW1 = w->grad;
    float* gb1 = gW1 + (long long)H * I;
    float* gW2 = gb1 + H;
    float* gb2 = gW2 + (long long)H * H;
    float* gW3 = gb2 + H;
    float* gb3 = gW3 + (long long)O * H;
    k_loss<<<1, 1024, 0, ctx->stream>>>((long long)B * O, a.y, a.T, a.M, a.dy, w->lossbuf);
    // gW3[o, h] = sum_b dy[b, o] h2[b, h]: A(m=o, k=b) = dy[b*O + o], B(k=b, n=h) = h2[b*H + h]
    gemm(ctx, O, H, B, a.dy, 1, O, a.h2, H, 1, gW3, nullptr, nullptr, 0);
    k_colsum<<<ceil_div(O, 128), 128, 0, ctx->stream>>>(B, O, a.dy, gb3);
    // d2[b, h] = sum_o dy[b, o] W3[o, h], then * GELU'(z2)
    gemm(ctx, B, H, O, a.dy, O, 1, W3, H, 1, a.d2, nullptr, nullptr, 0);
    k_gelu_back<<<ceil_div((long long)B * H, 256), 256, 0, ctx->stream>>>((long long)B * H, a.z2, a.d2);
    gemm(ctx, H, H, B, a.d2, 1, H, a.h1, H, 1, gW2, nullptr, nullptr, 0);
    k_colsum<<<ceil_div(H, 128), 128, 0, ctx->stream>>>(B, H, a.d2, gb2);
    gemm(ctx, B, H, H, a.d2, H, 1, W2, H, 1, a.d1, nullptr, nullptr, 0);
    k_gelu_back<<<ceil_div((long long)B * H, 256), 256, 0, ctx->stream>>>((long long)B * H, a.z1, a.d1);
    gemm(ctx, H, I, B, a.d1, 1, H, a.X, I, 1, gW1, nullptr, nullptr, 0);
    k_colsum<<<ceil_div(H, 128), 128, 0, ctx->stream>>>(B, H, a.d1, gb1);
}

int copy_in(dvqls_ws* w, float* dst, const float* src, long long n) {
    if (!src) return set_error(w->ctx, DVQLS_ERR_INVALID_ARG, "NULL input");
    DVQLS_CUDA_TRY(w->ctx, cudaMemcpyAsync(dst, src, size_t(n) * 4, cudaMemcpyDefault, w->ctx->stream));
    return DVQLS_OK;
}

int read_loss(dvqls_ws* w, float* loss) {
    if (!loss) return DVQLS_OK;
    float* hb = reinterpret_cast<float*>(w->pin);
    DVQLS_CUDA_TRY(w->ctx, cudaMemcpyAsync(hb, w->lossbuf, 8, cudaMemcpyDeviceToHost, w->ctx->stream));
    DVQLS_CUDA_TRY(w->ctx, cudaStreamSynchronize(w->ctx->stream));
    *loss = hb[1] > 0.f ? hb[0] / hb[1] : 0.f;
    return DVQLS_OK;
}

}  // namespace
}  // namespace dvqls

using namespace dvqls;

extern "C" long long dvqls_ws_param_count(int I, int H, int O) {
    if (I < 1 || H < 1 || O < 1) return -1;
    return (long long)H * I + H + (long long)H * H + H + (long long)O * H + O;
}

extern "C" void dvqls_ws_destroy(dvqls_ws* w) {
    if (!w) return;
    cudaSetDevice(w->ctx->device);
    cudaStreamSynchronize(w->ctx->stream);
    if (w->params) cudaFree(w->params);
    if (w->act) cudaFree(w->act);
    if (w->pin) cudaFreeHost(w->pin);
    cudaGetLastError();
    delete w;
}

extern "C" int dvqls_ws_create(dvqls_ctx* ctx, int I, int H, int O, const float* params, dvqls_ws** out) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!out || !params) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    const long long np = dvqls_ws_param_count(I, H, O);
    if (np < 1 || I > 4096 || H > 4096 || O > 4096) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "bad dimensions");
    cudaSetDevice(ctx->device);
    dvqls_ws* w = new dvqls_ws();
    w->ctx = ctx;
    w->I = I;
    w->H = H;
    w->O = O;
    w->np = np;
    // params, grad, m, v in one allocation, then the loss buffer.
    if (cudaMalloc(&w->params, size_t(4 * np + 64) * sizeof(float)) != cudaSuccess ||
        cudaMallocHost(&w->pin, 64) != cudaSuccess) {
        cudaGetLastError();
        dvqls_ws_destroy(w);
        return set_error(ctx, DVQLS_ERR_ALLOC, "warm-start parameters");
    }
    w->grad = w->params + np;
    w->m = w->grad + np;
    w->v = w->m + np;
    w->lossbuf = w->v + np;
    int rc = copy_in(w, w->params, params, np);
    if (!rc && cudaMemsetAsync(w->m, 0, size_t(2 * np) * 4, ctx->stream) != cudaSuccess) rc = DVQLS_ERR_CUDA;
    if (!rc && cudaStreamSynchronize(ctx->stream) != cudaSuccess) rc = DVQLS_ERR_CUDA;
    if (rc) {
        cudaGetLastError();
        dvqls_ws_destroy(w);
        return set_error(ctx, rc, "warm-start initialisation");
    }
    *out = w;
    return DVQLS_OK;
}

extern "C" int dvqls_ws_infer(dvqls_ws* w, int batch, const float* feats, float* out) {
    DVQLS_NVTX("dvqls_ws_infer");
    if (!w) return DVQLS_ERR_INVALID_ARG;
    dvqls_ctx* ctx = w->ctx;
    ctx->err.clear();
    if (batch < 1 || !feats || !out) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "batch < 1 or NULL");
    cudaSetDevice(ctx->device);
    int rc = ensure_batch(w, batch);
    if (rc) return rc;
    Views a = views(w, w->cap);
    rc = copy_in(w, a.X, feats, (long long)batch * w->I);
    if (rc) return rc;
    forward(w, a, batch);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(out, a.y, size_t(batch) * w->O * 4, cudaMemcpyDefault, ctx->stream));
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    return DVQLS_OK;
}

static int grad_common(dvqls_ws* w, int batch, const float* feats, const float* target, const float* mask) {
    dvqls_ctx* ctx = w->ctx;
    if (batch < 1 || !feats || !target || !mask) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "batch < 1 or NULL");
    cudaSetDevice(ctx->device);
    int rc = ensure_batch(w, batch);
    if (rc) return rc;
    Views a = views(w, w->cap);
    rc = copy_in(w, a.X, feats, (long long)batch * w->I);
    if (!rc) rc = copy_in(w, a.T, target, (long long)batch * w->O);
    if (!rc) rc = copy_in(w, a.M, mask, (long long)batch * w->O);
    if (rc) return rc;
    forward(w, a, batch);
    backward(w, a, batch);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    return DVQLS_OK;
}

extern "C" int dvqls_ws_grad(dvqls_ws* w, int batch, const float* feats, const float* target, const float* mask,
                             float* loss, float* grad) {
    if (!w) return DVQLS_ERR_INVALID_ARG;
    w->ctx->err.clear();
    if (!grad) return set_error(w->ctx, DVQLS_ERR_INVALID_ARG, "grad is NULL");
    int rc = grad_common(w, batch, feats, target, mask);
    if (rc) return rc;
    DVQLS_CUDA_TRY(w->ctx, cudaMemcpyAsync(grad, w->grad, size_t(w->np) * 4, cudaMemcpyDefault, w->ctx->stream));
    rc = read_loss(w, loss);
    if (rc) return rc;
    DVQLS_CUDA_TRY(w->ctx, cudaStreamSynchronize(w->ctx->stream));
    return DVQLS_OK;
}

extern "C" int dvqls_ws_train_step(dvqls_ws* w, int batch, const float* feats, const float* target, const float* mask,
                                   float lr, float* loss) {
    DVQLS_NVTX("dvqls_ws_train_step");
    if (!w) return DVQLS_ERR_INVALID_ARG;
    w->ctx->err.clear();
    if (!(lr > 0.f)) return set_error(w->ctx, DVQLS_ERR_INVALID_ARG, "lr must be > 0");
    int rc = grad_common(w, batch, feats, target, mask);
    if (rc) return rc;
    w->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, float(w->step)), c2 = 1.f - powf(b2, float(w->step));
    k_adam32<<<ceil_div(w->np, 256), 256, 0, w->ctx->stream>>>(w->np, w->grad, w->params, w->m, w->v, lr, b1, b2, eps,
                                                               c1, c2);
    DVQLS_CUDA_TRY(w->ctx, cudaGetLastError());
    return read_loss(w, loss);
}

extern "C" int dvqls_ws_get_params(dvqls_ws* w, float* params) {
    if (!w) return DVQLS_ERR_INVALID_ARG;
    if (!params) return set_error(w->ctx, DVQLS_ERR_INVALID_ARG, "NULL params");
    cudaSetDevice(w->ctx->device);
    DVQLS_CUDA_TRY(w->ctx, cudaMemcpyAsync(params, w->params, size_t(w->np) * 4, cudaMemcpyDefault, w->ctx->stream));
    DVQLS_CUDA_TRY(w->ctx, cudaStreamSynchronize(w->ctx->stream));
    return DVQLS_OK;
}

// File: "DVQLSWS1", int32 I, H, O, int64 Adam step, then params, m, v (FP32).
extern "C" int dvqls_ws_save(dvqls_ws* w, const char* path) {
    if (!w) return DVQLS_ERR_INVALID_ARG;
    if (!path) return set_error(w->ctx, DVQLS_ERR_INVALID_ARG, "NULL path");
    cudaSetDevice(w->ctx->device);
    std::vector<float> buf(size_t(3 * w->np));
    DVQLS_CUDA_TRY(w->ctx, cudaStreamSynchronize(w->ctx->stream));
    DVQLS_CUDA_TRY(w->ctx, cudaMemcpy(buf.data(), w->params, size_t(w->np) * 4, cudaMemcpyDeviceToHost));
    DVQLS_CUDA_TRY(w->ctx, cudaMemcpy(buf.data() + w->np, w->m, size_t(2 * w->np) * 4, cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) return set_error(w->ctx, DVQLS_ERR_INVALID_ARG, "cannot open %s", path);
    const int dims[3] = {w->I, w->H, w->O};
    bool ok = fwrite("DVQLSWS1", 1, 8, f) == 8 && fwrite(dims, 4, 3, f) == 3 && fwrite(&w->step, 8, 1, f) == 1 &&
              fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? DVQLS_OK : set_error(w->ctx, DVQLS_ERR_INVALID_ARG, "write failed: %s", path);
}

extern "C" int dvqls_ws_load(dvqls_ctx* ctx, const char* path, dvqls_ws** out) {
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    if (!path || !out) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL argument");
    FILE* f = fopen(path, "rb");
    if (!f) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "cannot open %s", path);
    char magic[8];
    int dims[3];
    long long step = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "DVQLSWS1", 8) == 0 && fread(dims, 4, 3, f) == 3 &&
              fread(&step, 8, 1, f) == 1;
    const long long np = ok ? dvqls_ws_param_count(dims[0], dims[1], dims[2]) : -1;
    std::vector<float> buf(np > 0 ? size_t(3 * np) : 0);
    ok = ok && np > 0 && fread(buf.data(), 4, buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "not a warm-start file: %s", path);
    int rc = dvqls_ws_create(ctx, dims[0], dims[1], dims[2], buf.data(), out);
    if (rc) return rc;
    (*out)->step = step;
    DVQLS_CUDA_TRY(ctx, cudaMemcpy((*out)->m, buf.data() + np, size_t(2 * np) * 4, cudaMemcpyHostToDevice));
    return DVQLS_OK;
}
