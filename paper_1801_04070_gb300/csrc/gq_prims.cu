// gq_prims.cu -- device-wide exclusive scan and stable LSD radix sort used by
// the quadtree and list construction (tree build by sorting and scanning).
#include "gq_internal.cuh"

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

__global__ void k_scan_reduce(const int *__restrict__ in, long long n, int *__restrict__ part) {
    long long base = (long long)blockIdx.x * kScanTile;
    int s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + (long long)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    int tot;
    block_exclusive_scan(s, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// offs == nullptr: single tile, also writes out[n] = total
__global__ void k_scan_tiles(const int *__restrict__ in, long long n, const int *__restrict__ offs,
                             int *__restrict__ out) {
    long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    int tot;
    int pre = block_exclusive_scan(s, tot);
    int off = offs ? offs[blockIdx.x] : 0;
    int run = off + pre;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        long long idx = base + i;
        if (idx < n) out[idx] = run;
        run += v[i];
    }
    if (!offs && threadIdx.x == 0) out[n] = tot;
}

__global__ void k_set_total(const int *offs_scanned, long long nblk, int *out, long long n) {
    out[n] = offs_scanned[nblk];
}

}  // namespace

size_t gq_scan_tmp_size(long long n) {
    size_t s = 0;
    while (n > kScanTile) {
        long long nb = (n + kScanTile - 1) / kScanTile;
        s += 2 * nb + 1;
        n = nb;
    }
    return s + 16;
}

void gq_exclusive_scan(gq_ctx *ctx, const int *in, int *out, long long n, int *tmp) {
    if (n <= kScanTile) {
        GQ_LAUNCH(ctx, k_scan_tiles, 1, kScanThreads, 0, in, n, (const int *)nullptr, out);
        return;
    }
    long long nb = (n + kScanTile - 1) / kScanTile;
    int *part = tmp, *part_scan = tmp + nb;
    GQ_LAUNCH(ctx, k_scan_reduce, (int)nb, kScanThreads, 0, in, n, part);
    gq_exclusive_scan(ctx, part, part_scan, nb, tmp + 2 * nb + 1);
    GQ_LAUNCH(ctx, k_scan_tiles, (int)nb, kScanThreads, 0, in, n, (const int *)part_scan, out);
    GQ_LAUNCH(ctx, k_set_total, 1, 1, 0, (const int *)part_scan, nb, out, n);
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
