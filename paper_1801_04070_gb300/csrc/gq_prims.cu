// gq_prims.cu -- device-wide exclusive scan and stable LSD radix sort used by
// the quadtree and list construction (tree build by sorting and scanning).
#include "gq_internal.cuh"
#include "gq_tc.cuh"

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// exclusive scan of one value per thread across the block; returns the
// thread's exclusive prefix and the block total
__device__ int block_exclusive_scan(int v, int &total) {
    __shared__ int warp_tot[32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    int nw = blockDim.x >> 5;
    if (wid == 0) {
        int t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive
    }
    __syncthreads();
    int warp_excl = wid ? warp_tot[wid - 1] : 0;
    total = warp_tot[nw - 1];
    __syncthreads();
    return warp_excl + x - v;
}

// Single-pass exclusive scan with decoupled look-back: a block takes the next
// tile number from a counter, publishes its tile's sum, then walks back over
// its predecessors' published words (32 at a time, one lane each) until it
// meets one that carries an inclusive prefix; it publishes its own inclusive
// prefix and writes its outputs.  A word is (flag << 32) | value, flag 1 = the
// tile's sum, 2 = the inclusive prefix, written with one 64-bit atomic.  A
// block waits only for tiles taken before its own, by blocks already running
// that wait only for earlier tiles, so every wait ends; the spin is bounded
// all the same (about 1 s), after which the error word is set and the block
// goes on with what it has.
__device__ int g_scan_err;

__device__ __forceinline__ unsigned long long scan_word_load(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}

// the scanned values: an array, or the flags vals[i] > thresh
struct ScanArray {
    const int *p;
    __device__ __forceinline__ int operator()(long long i) const { return p[i]; }
};
struct ScanAbove {
    const int *p;
    int thresh;
    __device__ __forceinline__ int operator()(long long i) const { return p[i] > thresh ? 1 : 0; }
};

template <class Ld>
__global__ void __launch_bounds__(kScanThreads) k_scan_single(Ld in, long long n, int *__restrict__ out,
                                                               unsigned int *counter, unsigned long long *status) {
    __shared__ int stile, sprefix;
    if (threadIdx.x == 0) stile = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int tile = stile;
    const long long nb = (n + kScanTile - 1) / kScanTile;
    const long long base = (long long)tile * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long idx = base + i;
        v[i] = idx < n ? in(idx) : 0;
        s += v[i];
    }
    int tot;
    const int pre = block_exclusive_scan(s, tot);
    if (threadIdx.x < 32) {
        int prefix = 0;
        if (tile == 0) {
            if (threadIdx.x == 0) atomicExch(&status[0], (2ull << 32) | (unsigned)tot);
        } else {
            if (threadIdx.x == 0) atomicExch(&status[tile], (1ull << 32) | (unsigned)tot);
            const int lane = threadIdx.x;
            const unsigned long long t0 = gqtc::globaltimer_ns();
            int look = tile - 1;   // the newest predecessor not yet added
            bool timed_out = false;
            while (look >= 0) {
                const int j = look - lane;
                unsigned long long w = 0;
                if (j >= 0) {
                    for (;;) {   // bounded: waits for a tile taken earlier
                        w = scan_word_load(&status[j]);
                        if ((w >> 32) != 0ull || timed_out) break;
                        if (gqtc::globaltimer_ns() - t0 > 1000000000ull) {
                            timed_out = true;
                            atomicExch(&g_scan_err, 1);
                        }
                    }
                }
                timed_out = __any_sync(0xffffffffu, timed_out);
                const unsigned flag = (unsigned)(w >> 32);
                // the nearest predecessor (lowest lane) with an inclusive prefix
                const unsigned incl = __ballot_sync(0xffffffffu, j >= 0 && flag == 2u);
                const int stop = incl ? __ffs(incl) - 1 : 31;
                int val = (lane <= stop && j >= 0) ? (int)(unsigned)(w & 0xffffffffull) : 0;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                prefix += val;
                if (incl || timed_out) break;
                look -= 32;
            }
            if (lane == 0) atomicExch(&status[tile], (2ull << 32) | (unsigned)(prefix + tot));
        }
        if (threadIdx.x == 0) sprefix = prefix;
    }
    __syncthreads();
    int run = sprefix + pre;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const long long idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (tile == nb - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;   // the total
    if (nb == 0 && threadIdx.x == 0) out[0] = 0;
}

}  // namespace

size_t gq_scan_tmp_size(long long n) {
    const long long nb = (n + kScanTile - 1) / kScanTile;
    return (size_t)(2 * (nb + 2) + 4);   // 8-byte aligned counter + status words, in ints
}

template <class Ld>
static void scan_launch(gq_ctx *ctx, Ld in, int *out, long long n, int *tmp) {
    const long long nb = (n + kScanTile - 1) / kScanTile;
    unsigned long long *w = (unsigned long long *)(((uintptr_t)tmp + 7) & ~(uintptr_t)7);
    GQ_CUDA(cudaMemsetAsync(w, 0, sizeof(unsigned long long) * (nb + 1), ctx->stream));
    auto k = k_scan_single<Ld>;
    GQ_LAUNCH(ctx, k, (int)(nb > 0 ? nb : 1), kScanThreads, 0, in, n, out, (unsigned int *)w, w + 1);
}

void gq_exclusive_scan(gq_ctx *ctx, const int *in, int *out, long long n, int *tmp) {
    scan_launch(ctx, ScanArray{in}, out, n, tmp);
}

void gq_exclusive_scan_above(gq_ctx *ctx, const int *vals, int thresh, int *out, long long n, int *tmp) {
    scan_launch(ctx, ScanAbove{vals, thresh}, out, n, tmp);
}

int gq_scan_error_take() {
    int h = 0, z = 0;
    GQ_CUDA(cudaMemcpyFromSymbol(&h, g_scan_err, sizeof(int)));
    if (h) GQ_CUDA(cudaMemcpyToSymbol(g_scan_err, &z, sizeof(int)));
    return h;
}

// ------------------------------------------------------------------ radix sort
namespace {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsChunks = 8;                       // 32-element chunks per warp
constexpr int kRsTile = kRsThreads * kRsChunks;    // 2048 elements per block
constexpr int kRsBits = 8;
constexpr int kRsDigits = 1 << kRsBits;
static_assert(kRsDigits <= kRsThreads, "one thread per digit in the histogram and prefix steps");

template <class K>
__global__ void k_rs_hist(const K *__restrict__ keys, long long n, int shift, int nblk, int *__restrict__ hist) {
    __shared__ int cnt[kRsDigits];
    if (threadIdx.x < kRsDigits) cnt[threadIdx.x] = 0;
    __syncthreads();
    long long base = (long long)blockIdx.x * kRsTile;
    for (int i = threadIdx.x; i < kRsTile; i += kRsThreads) {
        long long idx = base + i;
        if (idx < n) atomicAdd(&cnt[(int)((keys[idx] >> shift) & (kRsDigits - 1))], 1);
    }
    __syncthreads();
    if (threadIdx.x < kRsDigits) hist[threadIdx.x * nblk + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: element order within a block is warp-major, chunk-major,
// lane-minor, and ranks among equal digits follow that order.
template <class K>
__global__ void k_rs_scatter(const K *__restrict__ keys, const int *__restrict__ vals, long long n, int shift,
                             int nblk, const int *__restrict__ offs, K *__restrict__ keys_out,
                             int *__restrict__ vals_out) {
    __shared__ int wrun[kRsWarps][kRsDigits];
    __shared__ int wpre[kRsWarps][kRsDigits];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = lane; i < kRsDigits; i += 32) wrun[w][i] = 0;
    __syncwarp();
    long long base = (long long)blockIdx.x * kRsTile + (long long)w * (32 * kRsChunks);
    int rank[kRsChunks], dig[kRsChunks];
    unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int c = 0; c < kRsChunks; ++c) {
        long long idx = base + c * 32 + lane;
        bool valid = idx < n;
        int d = valid ? (int)((keys[idx] >> shift) & (kRsDigits - 1)) : kRsDigits;
        unsigned m = __match_any_sync(0xffffffffu, d);
        int r0 = valid ? wrun[w][d] : 0;
        __syncwarp();
        int r = r0 + __popc(m & lt);
        if (valid && lane == __ffs(m) - 1) wrun[w][d] = r0 + __popc(m);
        __syncwarp();
        rank[c] = r;
        dig[c] = d;
    }
    __syncthreads();
    if (threadIdx.x < kRsDigits) {
        int acc = 0;
        for (int ww = 0; ww < kRsWarps; ++ww) {
            wpre[ww][threadIdx.x] = acc;
            acc += wrun[ww][threadIdx.x];
        }
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < kRsChunks; ++c) {
        long long idx = base + c * 32 + lane;
        if (idx < n) {
            int d = dig[c];
            long long pos = (long long)offs[d * nblk + blockIdx.x] + wpre[w][d] + rank[c];
            keys_out[pos] = keys[idx];
            vals_out[pos] = vals[idx];
        }
    }
}

template <class K>
void radix_sort_impl(gq_ctx *ctx, K *keys, int *vals, long long n, int bits) {
    if (n <= 1 || bits <= 0) return;
    int nblk = (int)((n + kRsTile - 1) / kRsTile);
    dbuf<K> k2;
    dbuf<int> v2, hist, offs, tmp;
    k2.alloc(n);
    v2.alloc(n);
    long long nh = (long long)kRsDigits * nblk;
    hist.alloc(nh);
    offs.alloc(nh + 1);
    tmp.alloc(gq_scan_tmp_size(nh));
    K *ka = keys, *kb = k2.p;
    int *va = vals, *vb = v2.p;
    int passes = (bits + kRsBits - 1) / kRsBits;
    for (int ps = 0; ps < passes; ++ps) {
        int shift = ps * kRsBits;
        GQ_LAUNCH(ctx, k_rs_hist<K>, nblk, kRsThreads, 0, (const K *)ka, n, shift, nblk, hist.p);
        gq_exclusive_scan(ctx, hist.p, offs.p, nh, tmp.p);
        GQ_LAUNCH(ctx, k_rs_scatter<K>, nblk, kRsThreads, 0, (const K *)ka, (const int *)va, n, shift, nblk,
                  (const int *)offs.p, kb, vb);
        K *tk = ka; ka = kb; kb = tk;
        int *tv = va; va = vb; vb = tv;
    }
    if (ka != keys) {
        GQ_CUDA(cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        GQ_CUDA(cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    // temporaries are freed by their destructors; make sure the stream is done with them
    GQ_CUDA(cudaStreamSynchronize(ctx->stream));
}

}  // namespace

void gq_radix_sort_pairs(gq_ctx *ctx, uint64_t *keys, int *vals, long long n, int bits) {
    radix_sort_impl<uint64_t>(ctx, keys, vals, n, bits);
}
void gq_radix_sort_pairs32(gq_ctx *ctx, uint32_t *keys, int *vals, long long n, int bits) {
    radix_sort_impl<uint32_t>(ctx, keys, vals, n, bits);
}
