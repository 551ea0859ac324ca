// gq_probe.cu -- FMA-throughput probe used as the measured FP64 / FP32 peak
// of the ALU roofline (the measured peaks cover HBM and BF16 only).
#include "gq_internal.cuh"
#include "gq_dfl.cuh"
#include "gq_math.cuh"
#include "gq_tc.cuh"

namespace {

constexpr int kChains = 8;     // independent FMA chains per thread
constexpr int kIters = 4096;

template <class T>
__global__ void k_fma_loop(T *out, T a, T b) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < kIters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) out[0] = s;   // keeps the loop alive; never true for these inputs
}

template <class T>
double run(gq_ctx *ctx) {
    int dev = ctx->device, sms = 0;
    GQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    dbuf<T> out;
    out.alloc(1);
    const int threads = 256;
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    GQ_CUDA(cudaEventCreate(&e0));
    GQ_CUDA(cudaEventCreate(&e1));
    GQ_LAUNCH(ctx, k_fma_loop<T>, blocks, threads, 0, out.p, (T)0.999999, (T)1e-7);  // warm-up
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        GQ_CUDA(cudaEventRecord(e0, ctx->stream));
        GQ_LAUNCH(ctx, k_fma_loop<T>, blocks, threads, 0, out.p, (T)0.999999, (T)1e-7);
        GQ_CUDA(cudaEventRecord(e1, ctx->stream));
        GQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        GQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        double flops = 2.0 * kChains * (double)kIters * threads * blocks;
        double tf = flops / (ms * 1e-3) / 1e12;
        if (tf > best) best = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// FP64 tensor-core rate: warp-wide mma.sync m8n8k4 (D = A B + C, 8x8x4, FP64),
// kMma independent accumulators per warp so that the latency is hidden.
constexpr int kMma = 4;
constexpr int kMmaIters = 2048;

__global__ void k_dmma_loop(double *out, double a0, double b0) {
    double a = a0 * (double)(threadIdx.x + 1), b = b0;
    double c[kMma][2];
#pragma unroll
    for (int j = 0; j < kMma; ++j) c[j][0] = c[j][1] = 0.0;
    for (int i = 0; i < kMmaIters; ++i) {
#pragma unroll
        for (int j = 0; j < kMma; ++j)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                         : "+d"(c[j][0]), "+d"(c[j][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < kMma; ++j) s += c[j][0] + c[j][1];
    if (s == -1.2345) out[0] = s;   // keeps the loop alive; never true for these inputs
}

double run_dmma(gq_ctx *ctx) {
    int dev = ctx->device, sms = 0;
    GQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    dbuf<double> out;
    out.alloc(1);
    const int threads = 256;
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    GQ_CUDA(cudaEventCreate(&e0));
    GQ_CUDA(cudaEventCreate(&e1));
    GQ_LAUNCH(ctx, k_dmma_loop, blocks, threads, 0, out.p, 1e-3, 1e-7);  // warm-up
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        GQ_CUDA(cudaEventRecord(e0, ctx->stream));
        GQ_LAUNCH(ctx, k_dmma_loop, blocks, threads, 0, out.p, 1e-3, 1e-7);
        GQ_CUDA(cudaEventRecord(e1, ctx->stream));
        GQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        GQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        double flops = 2.0 * 8 * 8 * 4 * (double)kMma * kMmaIters * (threads / 32) * blocks;
        double tf = flops / (ms * 1e-3) / 1e12;
        if (tf > best) best = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

// Both FP64 paths at once: even warps run the FP64 FMA loop, odd warps the FP64
// MMA loop, each sized to the same flop count (kChains * kIters * 32 FMAs
// against kMma * kMmaIters MMAs of 256 multiply-adds).  The combined rate is
// about the larger single rate if the two share one pipe and about their sum
// if they issue to separate units.
constexpr int kMixIters = kMma * kMmaIters * 256 / (kChains * 32);

__global__ void k_fma_dmma_loop(double *out, double a, double b) {
    const int warp = threadIdx.x >> 5;
    double s = 0.0;
    if ((warp & 1) == 0) {
        double x[kChains];
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
        for (int i = 0; i < kMixIters; ++i) {
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
        }
#pragma unroll
        for (int c = 0; c < kChains; ++c) s += x[c];
    } else {
        double aa = 1e-3 * (double)(threadIdx.x + 1), bb = 1e-7;
        double c[kMma][2];
#pragma unroll
        for (int j = 0; j < kMma; ++j) c[j][0] = c[j][1] = 0.0;
        for (int i = 0; i < kMmaIters; ++i) {
#pragma unroll
            for (int j = 0; j < kMma; ++j)
                asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                             : "+d"(c[j][0]), "+d"(c[j][1])
                             : "d"(aa), "d"(bb));
        }
#pragma unroll
        for (int j = 0; j < kMma; ++j) s += c[j][0] + c[j][1];
    }
    if (s == -1.2345) out[0] = s;   // keeps the loops alive; never true for these inputs
}

double run_fma_dmma(gq_ctx *ctx) {
    int dev = ctx->device, sms = 0;
    GQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    dbuf<double> out;
    out.alloc(1);
    const int threads = 256;
    const int blocks = sms * 8;
    cudaEvent_t e0, e1;
    GQ_CUDA(cudaEventCreate(&e0));
    GQ_CUDA(cudaEventCreate(&e1));
    GQ_LAUNCH(ctx, k_fma_dmma_loop, blocks, threads, 0, out.p, 0.999999, 1e-7);  // warm-up
    double best = 0;
    for (int rep = 0; rep < 3; ++rep) {
        GQ_CUDA(cudaEventRecord(e0, ctx->stream));
        GQ_LAUNCH(ctx, k_fma_dmma_loop, blocks, threads, 0, out.p, 0.999999, 1e-7);
        GQ_CUDA(cudaEventRecord(e1, ctx->stream));
        GQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0;
        GQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        const double warps = (threads / 32) * (double)blocks;
        double flops = warps / 2 * (2.0 * kChains * kMixIters * 32) + warps / 2 * (2.0 * 256 * kMma * kMmaIters);
        double tf = flops / (ms * 1e-3) / 1e12;
        if (tf > best) best = tf;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}


// ---------------------------------------------------------------- tensor-core check
// One CTA of 128 threads: D[128][32] = A[128][K] * B[32][K]^T with BF16 A and
// B (given as raw bit patterns) and FP32 accumulation in tensor memory, by
// K/16 chained tcgen05.mma of shape 128 x 32 x 16.  Used to check the
// descriptor encodings and that integer-valued products accumulate exactly
// (the precondition of the split-digit FP64 emulation).  lbo_sbo_swap = 1
// exchanges the two byte offsets of the shared-memory descriptors (both
// choices address only inside the staged tiles).  *err = 1 if the
// completion wait gave up.
__global__ void __launch_bounds__(128) k_umma_probe(const uint16_t *__restrict__ A, const uint16_t *__restrict__ B,
                                                    int K, int lbo_sbo_swap, float *__restrict__ D,
                                                    int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    unsigned char *sa = sm;                         // 128 x K
    unsigned char *sb = sm + (size_t)128 * K * 2;   // 32 x K
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) gqtc::tmem_alloc(&tslot, 32);
    if (tid == 0) gqtc::mbar_init(&bar, 1);
    for (int i = tid; i < 128 * K; i += 128)
        *(uint16_t *)(sa + gqtc::tile_offset(i / K, i % K, K)) = A[i];
    for (int i = tid; i < 32 * K; i += 128)
        *(uint16_t *)(sb + gqtc::tile_offset(i / K, i % K, K)) = B[i];
    gqtc::fence_smem_to_async();
    gqtc::fence_before_sync();
    __syncthreads();
    gqtc::fence_after_sync();
    const uint32_t tmem = tslot;
    if (tid == 0) {
        const uint32_t idesc = gqtc::idesc_bf16_f32(128, 32);
        const uint32_t kstride = (uint32_t)(K / 8) * 128;
        const uint32_t lbo = lbo_sbo_swap ? kstride : 128u, sbo = lbo_sbo_swap ? 128u : kstride;
        for (int ks = 0; ks < K / 16; ++ks) {
            uint64_t ad = gqtc::smem_desc(gqtc::smem_u32(sa) + ks * 256, lbo, sbo);
            uint64_t bd = gqtc::smem_desc(gqtc::smem_u32(sb) + ks * 256, lbo, sbo);
            gqtc::mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        gqtc::mma_commit(&bar);
    }
    bool ok = gqtc::mbar_wait(&bar, 0, 2000000000ull);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok && (tid & 31) == 0) atomicExch(err, 1);
    gqtc::fence_after_sync();
    if (ok) {
        uint32_t v[32];
        gqtc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16), v);
        gqtc::tmem_ld_wait();
        const int row = warp * 32 + (tid & 31);
        for (int j = 0; j < 32; ++j) D[row * 32 + j] = __uint_as_float(v[j]);
    }
    gqtc::fence_before_sync();
    __syncthreads();
    if (warp == 0) gqtc::tmem_free(tmem, 32);
}

}  // namespace

double gq_probe_fma(gq_ctx *ctx, int what) {
    return what == 0 ? run<double>(ctx) : what == 1 ? run<float>(ctx) : what == 2 ? run_dmma(ctx) : run_fma_dmma(ctx);
}

namespace {
__global__ void k_probe_math(int fn, int n, const double *__restrict__ x, const double *__restrict__ tab,
                             const float *__restrict__ ftab, double *__restrict__ y) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double v = x[i];
    if (fn == 4) y[i] = dfl_to_double(dfl_log(dfl_from_double(v), ftab, ftab + 128, ftab + 256));
    else if (fn == 5) y[i] = dfl_to_double(dfl_rcp(dfl_from_double(v)));
    else y[i] = fn == 0 ? gq_log(v, tab) : fn == 1 ? log(v) : fn == 2 ? gq_rcp(v) : 1.0 / v;
}
}  // namespace

void gq_probe_math_impl(gq_ctx *ctx, int fn, int n, const double *x_dev, double *y_dev) {
    GqLogTable T;
    gq_log_table_host(&T);
    dbuf<double> tab;
    tab.alloc(kGqLogN);
    GQ_CUDA(cudaMemcpyAsync(tab.p, &T, sizeof(T), cudaMemcpyHostToDevice, ctx->stream));
    GqDflLogTable F;
    gq_dfl_log_table_host(&F);
    dbuf<float> ftab;
    ftab.alloc(384);
    GQ_CUDA(cudaMemcpyAsync(ftab.p, &F, sizeof(F), cudaMemcpyHostToDevice, ctx->stream));
    if (n > 0) GQ_LAUNCH(ctx, k_probe_math, gq_blocks(n, 256), 256, 0, fn, n, x_dev, (const double *)tab.p,
                         (const float *)ftab.p, y_dev);
    GQ_CUDA(cudaStreamSynchronize(ctx->stream));
}


void gq_probe_umma_impl(gq_ctx *ctx, int K, const uint16_t *A_host, const uint16_t *B_host, int swap, float *D_host) {
    GQ_REQUIRE(K >= 16 && K <= 256 && K % 16 == 0, GQ_ERR_INVALID, "gq_probe_umma: K must be a multiple of 16 in [16, 256]");
    dbuf<uint16_t> a, b;
    dbuf<float> d;
    dbuf<int> err;
    a.alloc((size_t)128 * K);
    b.alloc((size_t)32 * K);
    d.alloc(128 * 32);
    err.alloc(1);
    cudaStream_t st = ctx->stream;
    GQ_CUDA(cudaMemcpyAsync(a.p, A_host, sizeof(uint16_t) * 128 * K, cudaMemcpyHostToDevice, st));
    GQ_CUDA(cudaMemcpyAsync(b.p, B_host, sizeof(uint16_t) * 32 * K, cudaMemcpyHostToDevice, st));
    GQ_CUDA(cudaMemsetAsync(d.p, 0, sizeof(float) * 128 * 32, st));
    GQ_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), st));
    size_t smem = (size_t)160 * K * 2;
    GQ_CUDA(cudaFuncSetAttribute(k_umma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    GQ_LAUNCH(ctx, k_umma_probe, 1, 128, smem, (const uint16_t *)a.p, (const uint16_t *)b.p, K, swap, d.p, err.p);
    int herr = 0;
    GQ_CUDA(cudaMemcpyAsync(D_host, d.p, sizeof(float) * 128 * 32, cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaStreamSynchronize(st));
    GQ_REQUIRE(herr == 0, GQ_ERR_TIMEOUT, "gq_probe_umma: tensor-core completion wait gave up");
}
