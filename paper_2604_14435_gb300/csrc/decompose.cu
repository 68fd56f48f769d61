// FWHT-based Pauli decomposition with tau pruning and top-L selection
// (Sec. 2.2, Eq. 5; Algorithm 1, Steps 1-2).
//
// Pipeline (all on the device; the host only reads three counts back):
//   1. X-mask scan: every nonzero A[r, c] marks mask r ^ c;  compaction gives
//      the present masks in ascending order.
//   2. Per mask x: gather d_x(i) = A[i ^ x, i], Walsh-Hadamard transform with
//      the radix-2 butterfly at strides 1, 2, ..., N/2 (u, v) -> (u+v, u-v),
//      then c(x,z) = (-i)^popc(x&z) W_x(z) / N and key = re*re + im*im.
//      n <= 12: one CTA per mask, the whole diagonal in shared memory.
//      n > 12: strides < 4096 in shared-memory chunks, the remaining strides
//      in a second pass over column tiles; the butterfly graph (and so every
//      rounding) is the same as a stride-by-stride transform.
//   3. max key, the counts L_pre (key > 0) and L_post (key > thr) with
//      thr = (tau*tau) * max key, and the top-L_max select ordered by key
//      descending then (x << n) | z ascending: rounds of block-local bitonic
//      sorts that keep each block's best L_max until one block remains.
//
// Add/sub, power-of-two scaling and the phase are exact or correctly
// rounded, and the key is formed with explicit _rn intrinsics (no fused
// multiply-add), so coefficients, masks, order and counts are bit-identical to
// any implementation that follows the same butterfly order.
#include "internal.cuh"

namespace {

constexpr int SEL_CHUNK = 4096;
constexpr int SEL_THREADS = 1024;
constexpr int MAX_BANDS = 64;

struct Band {
    int nbands;
    int off[MAX_BANDS];
};

__device__ __forceinline__ double band_entry(const Band& bd, const double* vals, int n, long long row,
                                             long long col) {
    const long long o = col - row;
    for (int k = 0; k < bd.nbands; ++k)
        if (bd.off[k] == o) return vals[(long long)k << n | row];
    return 0.0;
}

__device__ __forceinline__ double entry(const double* A, const Band& bd, const double* vals, int n,
                                        long long row, long long col) {
    return A ? A[(row << n) | col] : band_entry(bd, vals, n, row, col);
}

__global__ void k_flags_dense(const double* __restrict__ A, int n, unsigned char* flags, int* status) {
    const long long N = 1LL << n, NN = N * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < NN;
         e += (long long)gridDim.x * blockDim.x) {
        const double v = A[e];
        if (!isfinite(v)) atomicCAS(status, 0, dvqls::DEV_NONFINITE_INPUT);
        if (v != 0.0) flags[(e >> n) ^ (e & (N - 1))] = 1;
    }
}

__global__ void k_flags_banded(int n, Band bd, const double* __restrict__ vals, unsigned char* flags,
                               int* status) {
    const long long N = 1LL << n, tot = (long long)bd.nbands * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = int(e >> n);
        const long long r = e & (N - 1), c = r + bd.off[k];
        if (c < 0 || c >= N) continue;
        const double v = vals[e];
        if (!isfinite(v)) atomicCAS(status, 0, dvqls::DEV_NONFINITE_INPUT);
        if (v != 0.0) flags[r ^ c] = 1;
    }
}

// Single CTA: masks in ascending order, count to *count.
__global__ void k_compact(const unsigned char* __restrict__ flags, long long N, uint32_t* masks, int* count) {
    __shared__ int part[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const long long seg = (N + T - 1) / T, beg = t * seg, end = beg + seg < N ? beg + seg : N;
    int c = 0;
    for (long long i = beg; i < end; ++i) c += flags[i] != 0;
    part[t] = c;
    __syncthreads();
    for (int s = 1; s < T; s <<= 1) {  // inclusive scan
        int v = t >= s ? part[t - s] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int o = part[t] - c;
    for (long long i = beg; i < end; ++i)
        if (flags[i]) masks[o++] = uint32_t(i);
    if (t == T - 1) *count = part[t];
}

__device__ __forceinline__ void emit(int n, uint32_t x, long long z, double w, double scale, double2* coef,
                                     double* key, long long pos) {
    const double v = w * scale;
    const int k = __popcll((long long)x & z) & 3;
    double re = 0.0, im = 0.0;
    if (k == 0) re = v;
    else if (k == 1) im = -v;
    else if (k == 2) re = -v;
    else im = v;
    coef[pos] = make_double2(re, im);
    key[pos] = __dadd_rn(__dmul_rn(re, re), __dmul_rn(im, im));
}

// n <= 12: one CTA per mask, the whole transform in shared memory.
__global__ void k_fwht_smem(const double* __restrict__ A, Band bd, const double* __restrict__ vals, int n,
                            const uint32_t* __restrict__ masks, double2* coef, double* key) {
    extern __shared__ double w[];
    const int r = blockIdx.x;
    const long long N = 1LL << n;
    const uint32_t x = masks[r];
    for (long long i = threadIdx.x; i < N; i += blockDim.x) w[i] = entry(A, bd, vals, n, i ^ x, i);
    __syncthreads();
    for (long long h = 1; h < N; h <<= 1) {
        for (long long p = threadIdx.x; p < N / 2; p += blockDim.x) {
            const long long i0 = (p / h) * 2 * h + (p % h), i1 = i0 + h;
            const double u = w[i0], v = w[i1];
            w[i0] = __dadd_rn(u, v);
            w[i1] = __dsub_rn(u, v);
        }
        __syncthreads();
    }
    const double scale = ldexp(1.0, -n);
    for (long long z = threadIdx.x; z < N; z += blockDim.x) emit(n, x, z, w[z], scale, coef, key, r * N + z);
}

constexpr int LO_BITS = 12, LO = 1 << LO_BITS, HI_TILE = 16;

// n > 12, pass 1: gather and strides 1 .. 2048 inside 4096-element chunks.
__global__ void k_fwht_lo(const double* __restrict__ A, Band bd, const double* __restrict__ vals, int n,
                          const uint32_t* __restrict__ masks, double* work) {
    __shared__ double w[LO];
    const long long N = 1LL << n;
    const int chunks = int(N >> LO_BITS);
    const int r = blockIdx.x / chunks, ch = blockIdx.x % chunks;
    const uint32_t x = masks[r];
    const long long base = (long long)ch << LO_BITS;
    for (int i = threadIdx.x; i < LO; i += blockDim.x) w[i] = entry(A, bd, vals, n, (base + i) ^ x, base + i);
    __syncthreads();
    for (int h = 1; h < LO; h <<= 1) {
        for (int p = threadIdx.x; p < LO / 2; p += blockDim.x) {
            const int i0 = (p / h) * 2 * h + (p % h), i1 = i0 + h;
            const double u = w[i0], v = w[i1];
            w[i0] = __dadd_rn(u, v);
            w[i1] = __dsub_rn(u, v);
        }
        __syncthreads();
    }
    double* out = work + ((long long)r << n) + base;
    for (int i = threadIdx.x; i < LO; i += blockDim.x) out[i] = w[i];
}

// n > 12, pass 2: strides 4096 .. N/2 on tiles of HI_TILE consecutive low
// indices, then phase, scale and key.
__global__ void k_fwht_hi(int n, const uint32_t* __restrict__ masks, const double* __restrict__ work,
                          double2* coef, double* key) {
    extern __shared__ double w[];  // [H][HI_TILE]
    const long long N = 1LL << n;
    const int H = int(N >> LO_BITS);
    const int tiles = LO / HI_TILE;
    const int r = blockIdx.x / tiles, lo0 = (blockIdx.x % tiles) * HI_TILE;
    const uint32_t x = masks[r];
    const double* src = work + ((long long)r << n);
    for (int e = threadIdx.x; e < H * HI_TILE; e += blockDim.x) {
        const int hi = e / HI_TILE, lo = e % HI_TILE;
        w[e] = src[((long long)hi << LO_BITS) + lo0 + lo];
    }
    __syncthreads();
    for (int h = 1; h < H; h <<= 1) {
        for (int p = threadIdx.x; p < (H / 2) * HI_TILE; p += blockDim.x) {
            const int q = p / HI_TILE, lo = p % HI_TILE;
            const int i0 = (q / h) * 2 * h + (q % h), i1 = i0 + h;
            const double u = w[i0 * HI_TILE + lo], v = w[i1 * HI_TILE + lo];
            w[i0 * HI_TILE + lo] = __dadd_rn(u, v);
            w[i1 * HI_TILE + lo] = __dsub_rn(u, v);
        }
        __syncthreads();
    }
    const double scale = ldexp(1.0, -n);
    for (int e = threadIdx.x; e < H * HI_TILE; e += blockDim.x) {
        const int hi = e / HI_TILE, lo = e % HI_TILE;
        const long long z = ((long long)hi << LO_BITS) + lo0 + lo;
        emit(n, x, z, w[e], scale, coef, key, ((long long)r << n) + z);
    }
}

// max key (as ordered bit patterns of non-negative doubles) and L_pre.
__global__ void k_key_stats(const double* __restrict__ key, long long E, unsigned long long* kmax, int* lpre) {
    unsigned long long m = 0;
    int c = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x) {
        const double k = key[e];
        const unsigned long long b = (unsigned long long)__double_as_longlong(k);
        m = b > m ? b : m;
        c += k > 0.0;
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, m, o);
        m = m2 > m ? m2 : m;
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(kmax, m);
        atomicAdd(lpre, c);
    }
}

__device__ __forceinline__ double threshold(double tau, const unsigned long long* kmax) {
    const double smax = __longlong_as_double((long long)*kmax);
    return tau > 0.0 ? __dmul_rn(__dmul_rn(tau, tau), smax) : 0.0;
}

__global__ void k_count_post(const double* __restrict__ key, long long E, double tau,
                             const unsigned long long* kmax, int* lpost) {
    const double thr = threshold(tau, kmax);
    int c = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < E; e += (long long)gridDim.x * blockDim.x)
        c += key[e] > thr;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(lpost, c);
}

struct Cand {
    unsigned long long k;  // ~bits(key) for passing keys, ~0 for the rest
    unsigned long long p;  // flat position r * N + z (monotone in (x << n) | z)
};

__device__ __forceinline__ bool cand_less(const Cand& a, const Cand& b) {
    return a.k < b.k || (a.k == b.k && a.p < b.p);
}

// One selection round: each CTA sorts SEL_CHUNK candidates and keeps its
// best `keep`.  Round 0 reads keys directly (src_key != nullptr).
__global__ void k_select_round(const double* __restrict__ src_key, const Cand* __restrict__ src, long long E,
                               double tau, const unsigned long long* kmax, int keep, Cand* dst) {
    extern __shared__ Cand s[];
    const long long base = (long long)blockIdx.x * SEL_CHUNK;
    const double thr = src_key ? threshold(tau, kmax) : 0.0;
    for (int i = threadIdx.x; i < SEL_CHUNK; i += blockDim.x) {
        const long long e = base + i;
        Cand c{~0ull, ~0ull};
        if (e < E) {
            if (src_key) {
                const double k = src_key[e];
                c.p = (unsigned long long)e;
                c.k = k > thr ? ~(unsigned long long)__double_as_longlong(k) : ~0ull;
            } else {
                c = src[e];
            }
        }
        s[i] = c;
    }
    __syncthreads();
    for (int k = 2; k <= SEL_CHUNK; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < SEL_CHUNK; i += blockDim.x) {
                const int ixj = i ^ j;
                if (ixj > i) {
                    const bool up = (i & k) == 0;
                    const Cand a = s[i], b = s[ixj];
                    if (cand_less(b, a) == up) {
                        s[i] = b;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < keep; i += blockDim.x) dst[(long long)blockIdx.x * keep + i] = s[i];
}

__global__ void k_emit_terms(const Cand* __restrict__ best, int n, const uint32_t* __restrict__ masks,
                             const double2* __restrict__ coef, const int* lpost, int L_max, double2* out_c,
                             uint32_t* out_x, uint32_t* out_z, int* lout) {
    const int L = min(*lpost, L_max);
    if (blockIdx.x == 0 && threadIdx.x == 0) *lout = L;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L; i += gridDim.x * blockDim.x) {
        const unsigned long long p = best[i].p;
        out_c[i] = coef[p];
        out_x[i] = masks[p >> n];
        out_z[i] = uint32_t(p & ((1ull << n) - 1));
    }
}

int decompose_common(dvqls_ctx* ctx, const double* A_in, int n, int nbands, const int* offsets,
                     const double* bands_in, double tau, int L_max, double* coef_out, uint32_t* x_out,
                     uint32_t* z_out, int* L_out, int* L_pre, int* L_post) {
    using namespace dvqls;
    if (!ctx) return DVQLS_ERR_INVALID_ARG;
    ctx->err.clear();
    const bool dense = A_in != nullptr;
    if (n < 1 || n > (dense ? DVQLS_MAX_DENSE_QUBITS : DVQLS_MAX_QUBITS))
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "n = %d out of range", n);
    if (L_max < 1) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "L_max must be >= 1");
    if (L_max > SEL_CHUNK / 2)
        return set_error(ctx, DVQLS_ERR_UNSUPPORTED, "L_max = %d above the supported %d", L_max, SEL_CHUNK / 2);
    if (tau != tau || tau == -INFINITY) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "tau is NaN");
    if (!coef_out || !x_out || !z_out || !L_out || !L_pre || !L_post)
        return set_error(ctx, DVQLS_ERR_INVALID_ARG, "NULL output");
    Band bd{};
    const long long N = 1LL << n;
    if (!dense) {
        if (nbands < 1 || nbands > MAX_BANDS || !offsets || !bands_in)
            return set_error(ctx, DVQLS_ERR_INVALID_ARG, "need 1..%d bands", MAX_BANDS);
        if (is_device_ptr(ctx, offsets)) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "offsets must be host memory");
        bd.nbands = nbands;
        for (int k = 0; k < nbands; ++k) {
            if (offsets[k] <= -N || offsets[k] >= N)
                return set_error(ctx, DVQLS_ERR_INVALID_ARG, "band offset %d out of range", offsets[k]);
            for (int j = 0; j < k; ++j)
                if (offsets[j] == offsets[k]) return set_error(ctx, DVQLS_ERR_INVALID_ARG, "repeated band offset");
            bd.off[k] = offsets[k];
        }
    }
    cudaSetDevice(ctx->device);

    // Plan: the input, flags, masks, coefficient and key arrays for up to
    // N masks (the count is only known after the scan), selection buffers.
    const size_t in_bytes = dense ? size_t(N) * N * 8 : size_t(nbands) * N * 8;
    const long long maxE = N * N;  // masks x N upper bound
    Arena ar;
    const size_t o_in = ar.reserve(in_bytes);
    const size_t o_flags = ar.reserve(N);
    const size_t o_masks = ar.reserve(N * 4);
    const size_t o_misc = ar.reserve(64);
    ar.reserve(0);
    // Coefficients/keys are reserved after the count is known (second plan).
    int rc = ensure_workspace(ctx, ar.total());
    if (rc) return rc;
    rc = ensure_pinned(ctx, in_bytes + 4096 + size_t(L_max) * 24);
    if (!rc) rc = pin_acquire(ctx);
    if (rc) return rc;
    char* ws = ctx->ws;
    const double* dA = (const double*)stage_in(ctx, dense ? A_in : bands_in, in_bytes, 0, o_in);
    unsigned char* flags = (unsigned char*)(ws + o_flags);
    uint32_t* masks = (uint32_t*)(ws + o_masks);
    int* misc = (int*)(ws + o_misc);  // [0] mask count [1] L_pre [2] L_post [3] L_out, [4..5] kmax
    unsigned long long* kmax = (unsigned long long*)(misc + 4);
    DVQLS_CUDA_TRY(ctx, cudaMemsetAsync(flags, 0, N, ctx->stream));
    DVQLS_CUDA_TRY(ctx, cudaMemsetAsync(misc, 0, 64, ctx->stream));
    const int grid = ctx->num_sms * 8;
    if (dense) k_flags_dense<<<grid, 256, 0, ctx->stream>>>(dA, n, flags, ctx->d_status);
    else k_flags_banded<<<grid, 256, 0, ctx->stream>>>(n, bd, dA, flags, ctx->d_status);
    k_compact<<<1, 1024, 0, ctx->stream>>>(flags, N, masks, misc);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    int M = 0;
    DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(&M, misc, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    rc = sync_and_check(ctx);
    if (rc) return rc;
    if (M == 0) {
        *L_out = *L_pre = *L_post = 0;
        return DVQLS_OK;
    }

    // Second plan: everything above stays in place (same offsets), append
    // the M x N coefficient and key arrays and the selection buffers.
    const long long E = (long long)M * N;
    (void)maxE;
    const size_t o_coef = ar.reserve(size_t(E) * 16);
    const size_t o_key = ar.reserve(size_t(E) * 8);
    const size_t o_work = n > LO_BITS ? ar.reserve(size_t(E) * 8) : 0;
    long long blocks0 = (E + SEL_CHUNK - 1) / SEL_CHUNK;
    const size_t o_candA = ar.reserve(size_t(blocks0) * L_max * sizeof(Cand));
    const size_t o_candB = ar.reserve(size_t((blocks0 * L_max + SEL_CHUNK - 1) / SEL_CHUNK + 1) * L_max * sizeof(Cand));
    const size_t o_out = ar.reserve(size_t(L_max) * 24);
    if (ar.total() > ctx->ws_cap) {
        // Growing reallocates: the staged input, flags and masks must be
        // rebuilt, so copy the small mask list out and back.
        std::vector<uint32_t> hm(M);
        DVQLS_CUDA_TRY(ctx, cudaMemcpy(hm.data(), masks, size_t(M) * 4, cudaMemcpyDeviceToHost));
        rc = ensure_workspace(ctx, ar.total());
        if (rc) return rc;
        ws = ctx->ws;
        masks = (uint32_t*)(ws + o_masks);
        misc = (int*)(ws + o_misc);
        kmax = (unsigned long long*)(misc + 4);
        dA = (const double*)stage_in(ctx, dense ? A_in : bands_in, in_bytes, 0, o_in);
        DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(masks, hm.data(), size_t(M) * 4, cudaMemcpyHostToDevice, ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
        DVQLS_CUDA_TRY(ctx, cudaMemsetAsync(misc, 0, 64, ctx->stream));
    }
    double2* coef = (double2*)(ws + o_coef);
    double* key = (double*)(ws + o_key);
    if (n <= LO_BITS) {
        const size_t smem = size_t(N) * 8;
        DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_fwht_smem));
        k_fwht_smem<<<M, 512, smem, ctx->stream>>>(dense ? dA : nullptr, bd, dense ? nullptr : dA, n, masks, coef, key);
    } else {
        double* work = (double*)(ws + o_work);
        k_fwht_lo<<<M * int(N >> LO_BITS), 512, 0, ctx->stream>>>(dense ? dA : nullptr, bd, dense ? nullptr : dA, n,
                                                                  masks, work);
        const size_t smem = size_t(N >> LO_BITS) * HI_TILE * 8;
        DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_fwht_hi));
        k_fwht_hi<<<M * (LO / HI_TILE), 512, smem, ctx->stream>>>(n, masks, work, coef, key);
    }
    k_key_stats<<<grid, 256, 0, ctx->stream>>>(key, E, kmax, misc + 1);
    k_count_post<<<grid, 256, 0, ctx->stream>>>(key, E, tau, kmax, misc + 2);
    const size_t sel_smem = SEL_CHUNK * sizeof(Cand);
    DVQLS_CUDA_TRY(ctx, allow_dynamic_smem((const void*)k_select_round));
    Cand* bufA = (Cand*)(ws + o_candA);
    Cand* bufB = (Cand*)(ws + o_candB);
    long long cur = E;
    long long blocks = blocks0;
    k_select_round<<<int(blocks), SEL_THREADS, sel_smem, ctx->stream>>>(key, nullptr, cur, tau, kmax, L_max, bufA);
    cur = blocks * L_max;
    Cand* src = bufA;
    Cand* dst = bufB;
    while (blocks > 1) {
        blocks = (cur + SEL_CHUNK - 1) / SEL_CHUNK;
        k_select_round<<<int(blocks), SEL_THREADS, sel_smem, ctx->stream>>>(nullptr, src, cur, tau, kmax, L_max, dst);
        cur = blocks * L_max;
        Cand* t = src;
        src = dst;
        dst = t;
    }
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    char* out = ws + o_out;
    double2* oc = (double2*)out;
    uint32_t* ox = (uint32_t*)(out + size_t(L_max) * 16);
    uint32_t* oz = ox + L_max;
    k_emit_terms<<<ceil_div(L_max, 256), 256, 0, ctx->stream>>>(src, n, masks, coef, misc + 2, L_max, oc, ox, oz,
                                                                 misc + 3);
    DVQLS_CUDA_TRY(ctx, cudaGetLastError());
    int counts[4];
    DVQLS_CUDA_TRY(ctx, cudaMemcpyAsync(counts, misc, sizeof counts, cudaMemcpyDeviceToHost, ctx->stream));
    rc = sync_and_check(ctx);
    if (rc) return rc;
    const int L = counts[3];
    std::vector<PendingOut> pend;
    const size_t pin0 = 0;
    rc = enqueue_out(ctx, coef_out, oc, size_t(L) * 16, pin0, pend);
    if (!rc) rc = enqueue_out(ctx, x_out, ox, size_t(L) * 4, pin0 + size_t(L_max) * 16, pend);
    if (!rc) rc = enqueue_out(ctx, z_out, oz, size_t(L) * 4, pin0 + size_t(L_max) * 20, pend);
    if (rc) return rc;
    DVQLS_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    finish_out(ctx, pend);
    *L_out = L;
    *L_pre = counts[1];
    *L_post = counts[2];
    return DVQLS_OK;
}

}  // namespace

extern "C" int dvqls_pauli_decompose(dvqls_ctx* ctx, const double* A, int n, double tau, int L_max, double* coef,
                                     uint32_t* xmask, uint32_t* zmask, int* L_out, int* L_pre, int* L_post) {
    DVQLS_NVTX("dvqls_pauli_decompose");
    if (!A) return ctx ? dvqls::set_error(ctx, DVQLS_ERR_INVALID_ARG, "A is NULL") : DVQLS_ERR_INVALID_ARG;
    return decompose_common(ctx, A, n, 0, nullptr, nullptr, tau, L_max, coef, xmask, zmask, L_out, L_pre, L_post);
}

extern "C" int dvqls_pauli_decompose_banded(dvqls_ctx* ctx, int n, int nbands, const int* offsets,
                                            const double* band_values, double tau, int L_max, double* coef,
                                            uint32_t* xmask, uint32_t* zmask, int* L_out, int* L_pre, int* L_post) {
    DVQLS_NVTX("dvqls_pauli_decompose_banded");
    return decompose_common(ctx, nullptr, n, nbands, offsets, band_values, tau, L_max, coef, xmask, zmask, L_out,
                            L_pre, L_post);
}
