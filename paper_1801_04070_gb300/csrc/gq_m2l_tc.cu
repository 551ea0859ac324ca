// gq_m2l_tc.cu -- Stage 4 (M2L over List 2, Sec. 3.1 eq. m2l, Sec. 4.4) on
// the BF16 tensor cores with FP64 accuracy, by exact digit splitting.
//
// With box-scaled coefficients (M_k = a_k / rho^k, L_m = beta_m rho^m) a List 2
// translation between same-level boxes depends only on their offset
// delta = (z_b - z_d) / rho = 2 (tx - sx) + 2i (ty - sy) (index differences):
//     L_m += sum_k T_delta[m][k] M_k,
//     T[0][0] = log|delta|, T[0][k] = delta^-k,
//     T[m][0] = -(-1)^m delta^-m / m, T[m][k] = (-1)^m C(m+k-1, k-1) delta^-(m+k),
// plus M_0 log rho for m = 0 (added in FP64).  In real form T is a 32 x 32
// matrix per offset (p_fmm <= 15).  A target box b in quadrant (bx & 1, by & 1)
// of its parent has its List 2 boxes among 75 offsets of a 10 x 10 window, so
// for 128 target boxes of one quadrant
//     L[128 x 32] = sum over window slots s of  Mg_s[128 x 32] * T_s^T,
// Mg_s holding row b's List 2 multipole at slot s (or zeros): one GEMM with
// K = 100 slots x 32, accumulated across slots in tensor memory.
//
// FP64 accuracy: every multipole entry is a 54-bit fixed-point integer at the
// largest exponent of its tree level, every T entry one at the largest
// exponent of its output column (over all offsets), both written as 11
// balanced base-32 digits in [-16, 16] -- exact in BF16.  Digit products
// (|.| <= 256) summed over at most 100 x 32 terms and 11 digit pairs stay
// below 2^24, so the FP32 accumulators hold exact integers; the sums for
// digit levels w = i + j <= 11 (i, j the digit indices) go to 12 accumulators
// and are recombined in 64-bit integers, converted to FP64 once.  Emulated on
// random multipoles this gives about 4e-15 of max|L| (the FP64 sum itself
// carries about 1e-16 per term).
//
// One CTA (128 threads) per SM walks tiles of 128 target boxes; per occupied
// slot, all threads stage the 11 multipole digit tiles (cp.async, 16 bytes)
// and the 11 translation digit tiles into one of two shared-memory stages,
// and thread 0 issues the MMAs (128 x N x 16, N up to 256: the 11 translation
// digits are stacked along N so that digit pair (i, j) lands in the
// accumulator columns of level i + j) and commits them to the stage's
// mbarrier; the next slot is staged while they run.  Thread r then reads row
// r's 12 x 32 accumulators (tcgen05.ld), recombines them and adds L_m.
#include <math.h>

#include <mutex>
#include <vector>

#include "gq_internal.cuh"
#include "gq_tc.cuh"

namespace {

constexpr int kTcND = 11;          // digits per operand
constexpr int kTcLev = 12;         // accumulated digit levels w = 0 .. 11
constexpr int kTcBits = 54;        // fixed-point bits
constexpr int kTcSlots = 100;      // 10 x 10 window of List 2 offsets
constexpr int kTcRows = 128;       // target boxes per tile (MMA M)
constexpr int kTcK = 32;           // real multipole terms per box (16 complex)
constexpr int kTcN = 32;           // real outputs per box
constexpr uint32_t kTileA = kTcRows * kTcK * 2;          // bytes per multipole digit tile (8 KiB)
constexpr uint32_t kTileB = kTcN * kTcK * 2;             // bytes per translation digit tile (2 KiB)
constexpr uint32_t kStage = kTcND * (kTileA + kTileB);   // 112,640 bytes
constexpr uint64_t kWaitNs = 2000000000ull;              // bounded waits: 2 s

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void st_shared_zero16(uint32_t dst) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0) : "memory");
}

// balanced base-32 digits of |X| <= 2^54, most significant first
__host__ __device__ inline void tc_digits(long long X, int (&d)[kTcND]) {
    for (int j = kTcND - 1; j >= 1; --j) {
        int r = (int)(X & 31);
        if (r >= 16) r -= 32;
        d[j] = r;
        X = (X - r) / 32;
    }
    d[0] = (int)X;
}

__host__ __device__ inline uint16_t bf16_of_small_int(int v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

// ---------------------------------------------------------------- per-eval: multipole digits
// largest biased exponent of the 32 real multipole terms of every box of a
// level (a warp per box, then an atomic maximum per level; lexp zeroed first)
__global__ void k_tc_levexp(int nbox, int P, const int *__restrict__ blev, const double2 *__restrict__ M,
                            int *__restrict__ lexp) {
    int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, kk = threadIdx.x & 31;
    if (b >= nbox) return;
    int k = kk >> 1;
    double x = 0.0;
    if (k <= P) {
        double2 v = M[(size_t)b * (P + 1) + k];
        x = (kk & 1) ? v.y : v.x;
    }
    unsigned e = (unsigned)(((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff);
    e = __reduce_max_sync(0xffffffffu, e);
    if (kk == 0 && e) atomicMax(&lexp[blev[b]], (int)e);
}

// 11 BF16 digits of every real multipole term at its level's exponent:
// mdig[b][i][kk], term kk = 2k + (0 re, 1 im)
__global__ void k_tc_digits(int nbox, int P, const int *__restrict__ blev, const int *__restrict__ lexp,
                            const double2 *__restrict__ M, uint16_t *__restrict__ mdig) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int b = (int)(t >> 5), kk = (int)(t & 31);
    if (b >= nbox) return;
    int k = kk >> 1;
    double x = 0.0;
    if (k <= P) {
        double2 v = M[(size_t)b * (P + 1) + k];
        x = (kk & 1) ? v.y : v.x;
    }
    int le = lexp[blev[b]];
    int d[kTcND];
    if (le == 0) {
        for (int i = 0; i < kTcND; ++i) d[i] = 0;
    } else {
        // |x| < 2^(le - 1022): X = round(x 2^(54 - (le - 1022))), |X| <= 2^54
        long long X = __double2ll_rn(ldexp(x, kTcBits - (le - 1022)));
        tc_digits(X, d);
    }
    uint16_t *dst = mdig + (size_t)b * kTcND * kTcK + kk;
#pragma unroll
    for (int i = 0; i < kTcND; ++i) dst[i * kTcK] = bf16_of_small_int(d[i]);
}

// ---------------------------------------------------------------- per-build: tiles
// window slot of List 2 box d seen from b (quadrant q), or -1 outside the window
__device__ __forceinline__ int tc_slot(int q, int bx, int by, int dx_, int dy_) {
    int sx = dx_ - bx + 4 + (q & 1), sy = dy_ - by + 4 + (q >> 1);
    return (sx < 0 || sx > 9 || sy < 0 || sy > 9) ? -1 : sy * 10 + sx;
}

constexpr uint32_t kNoTile = 0xffffffffu;

// Sort key of every box: quadrant in bits 30-31, then which of the quadrant's
// first 29 List 2 window slots (row-major, the 5 x 5 block of the box's
// 2-colleagues skipped) it uses; boxes without List 2 get kNoTile (sorted
// last).  Boxes with similar keys share slots, so sorted tiles touch fewer.
__global__ void k_tc_keys(int nbox, const int *__restrict__ voff, const int *__restrict__ vidx,
                          const int *__restrict__ bix, const int *__restrict__ biy, uint32_t *__restrict__ key,
                          int *__restrict__ val, int *__restrict__ cnt, int *__restrict__ err) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    val[b] = b;
    if (voff[b + 1] == voff[b]) {
        key[b] = kNoTile;
        return;
    }
    const int q = (bix[b] & 1) | ((biy[b] & 1) << 1), qx = q & 1, qy = q >> 1;
    uint32_t k = 0;
    for (int e = voff[b]; e < voff[b + 1]; ++e) {
        int d = vidx[e];
        int s = tc_slot(q, bix[b], biy[b], bix[d], biy[d]);
        if (s < 0) {
            atomicExch(err, 2);
            continue;
        }
        int sx = s % 10, sy = s / 10;
        int rows_inner = min(max(sy - (2 + qy), 0), 5);
        int in_row = (sy >= 2 + qy && sy <= 6 + qy) ? min(max(sx - (2 + qx), 0), 5) : 0;
        int c = s - 5 * rows_inner - in_row;   // index among the quadrant's valid slots
        if (c < 29) k |= 1u << (28 - c);   // bit 29 stays clear: no key equals kNoTile
    }
    key[b] = ((uint32_t)q << 30) | k;
    atomicAdd(&cnt[q], 1);
}

// Rows in sorted order; each quadrant starts a new tile (padded to 128 rows).
__global__ void k_tc_fill(int nbox, const uint32_t *__restrict__ key, const int *__restrict__ sorted_box,
                          const int *__restrict__ cnt, const int *__restrict__ voff, const int *__restrict__ vidx,
                          const int *__restrict__ bix, const int *__restrict__ biy, int *__restrict__ tile_box,
                          int *__restrict__ tile_q, int *__restrict__ slot_src, unsigned *__restrict__ tile_mask,
                          int *__restrict__ ntiles) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int start[4], row0[4], rows = 0, seen = 0;
    for (int q = 0; q < 4; ++q) {
        start[q] = seen;
        row0[q] = rows;
        seen += cnt[q];
        rows += (cnt[q] + kTcRows - 1) / kTcRows * kTcRows;
    }
    if (i == 0) *ntiles = rows / kTcRows;
    if (i >= nbox || key[i] == kNoTile) return;
    const int q = (int)(key[i] >> 30);
    const int b = sorted_box[i];
    const int row = row0[q] + (i - start[q]), tile = row / kTcRows;
    tile_box[row] = b;
    tile_q[tile] = q;
    for (int e = voff[b]; e < voff[b + 1]; ++e) {
        int d = vidx[e];
        int s = tc_slot(q, bix[b], biy[b], bix[d], biy[d]);
        if (s < 0) continue;   // reported by k_tc_keys
        slot_src[((size_t)tile * kTcSlots + s) * kTcRows + (row % kTcRows)] = d;
        atomicOr(&tile_mask[tile * 4 + (s >> 5)], 1u << (s & 31));
    }
}

// ---------------------------------------------------------------- the tensor-core M2L
struct TcArgs {
    const int *ntiles;   // device: number of tiles of the current build
    int P;
    const int *tile_box, *tile_q, *slot_src;
    const unsigned *tile_mask;
    const uint16_t *mdig, *tdig;
    const int *fexp;     // [32] column exponents (|T[n][.]| < 2^fexp[n])
    const int *lexp;     // per level: largest biased exponent of the multipoles
    const int *blev, *voff, *vidx;
    const double2 *M;
    double2 *L;
    double logH, ln2;    // log rho_l = logH - l log 2
    int *err;
    int *next_tile;      // dynamic tile counter (zero at launch)
};

constexpr int kTcThreads = 160;   // warps 0-3: staging and epilogue (row = thread), warp 4: MMA issue

__device__ __forceinline__ int next_slot(const unsigned *mask, int s) {
    for (++s; s < kTcSlots; ++s)
        if ((mask[s >> 5] >> (s & 31)) & 1u) return s;
    return kTcSlots;
}

__global__ void __launch_bounds__(kTcThreads, 1) k_m2l_tc(TcArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[2], empty[2], accfull, accfree;
    __shared__ uint32_t tslot;
    __shared__ unsigned smask[2][4];
    __shared__ int sq[2];
    __shared__ int stile[2];
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) gqtc::tmem_alloc(&tslot, 512);
    if (tid == 0) {
        gqtc::mbar_init(&full[0], 2 * kTcRows);   // per staging thread: one arrive + one cp.async arrive
        gqtc::mbar_init(&full[1], 2 * kTcRows);
        gqtc::mbar_init(&empty[0], 1);
        gqtc::mbar_init(&empty[1], 1);
        gqtc::mbar_init(&accfull, 1);
        gqtc::mbar_init(&accfree, kTcRows);
        abort_flag = 0;
    }
    gqtc::fence_before_sync();
    __syncthreads();
    gqtc::fence_after_sync();
    const uint32_t tmem = tslot;
    const uint32_t sbase = gqtc::smem_u32(sm);
    int it = 0;       // tiles done by this CTA
    uint32_t g = 0;   // slots staged / consumed so far (both roles count the same slots)
    bool zero_row[2] = {false, false};   // staging: this thread's row of stage s holds zeros
    for (;; ++it) {
        // tiles are taken from a shared counter (their slot counts differ), one
        // per CTA at a time; every thread passes the barrier below once per
        // tile, and a wait that gave up (abort_flag) ends the loop for all
        if (tid == 0) stile[it & 1] = atomicAdd(a.next_tile, 1);
        __syncthreads();
        const int tile = stile[it & 1];
        if (tile >= *a.ntiles) break;
        if (tid < 4) smask[it & 1][tid] = a.tile_mask[tile * 4 + tid];
        if (tid == 4) sq[it & 1] = a.tile_q[tile];
        if (__syncthreads_or(abort_flag)) break;
        const unsigned *mask = smask[it & 1];
        if (warp == 4) {
            // ---------------- MMA issue (one thread)
            if ((tid & 31) == 0) {
                bool ok = it == 0 || gqtc::mbar_wait_abortable(&accfree, (uint32_t)((it - 1) & 1), kWaitNs, &abort_flag);
                gqtc::fence_after_sync();
                bool first = true;
                for (int s = next_slot(mask, -1); s < kTcSlots; s = next_slot(mask, s), ++g) {
                    const int st = g & 1;
                    if (ok) ok = gqtc::mbar_wait_abortable(&full[st], (g >> 1) & 1, kWaitNs, &abort_flag);
                    if (!ok) continue;   // count the remaining slots only
                    gqtc::fence_smem_to_async();
                    gqtc::fence_after_sync();
                    const uint32_t sA = sbase + st * kStage, sB = sA + kTcND * kTileA;
#pragma unroll 1
                    for (int ks = 0; ks < 2; ++ks) {
                        const bool init = first && ks == 0;
#pragma unroll 1
                        for (int i = 0; i < kTcND; ++i) {
                            const int jmax = min(kTcND - 1, kTcLev - 1 - i);
                            const uint64_t ad = gqtc::smem_desc(sA + i * kTileA + ks * 256, 128, 512);
                            // digit groups [j0, j1] stacked along N; the first MMAs of a tile
                            // overwrite the levels not written yet (i = 0: 0..10; i = 1: 11)
                            int gj[3][3], ng = 0;
                            gj[ng][0] = 0; gj[ng][1] = min(jmax, 7); gj[ng][2] = (init && i == 0) ? 0 : 1; ++ng;
                            if (jmax >= 8) {
                                if (init && i == 1) {
                                    gj[ng][0] = 8; gj[ng][1] = 9; gj[ng][2] = 1; ++ng;
                                    gj[ng][0] = 10; gj[ng][1] = 10; gj[ng][2] = 0; ++ng;
                                } else {
                                    gj[ng][0] = 8; gj[ng][1] = jmax; gj[ng][2] = (init && i == 0) ? 0 : 1; ++ng;
                                }
                            }
                            for (int x = 0; x < ng; ++x) {
                                const int j0 = gj[x][0], j1 = gj[x][1];
                                const uint64_t bd = gqtc::smem_desc(sB + j0 * kTileB + ks * 256, 128, 512);
                                gqtc::mma_bf16(tmem + (uint32_t)((i + j0) * 32), ad, bd,
                                               gqtc::idesc_bf16_f32(128, 32 * (j1 - j0 + 1)), (uint32_t)gj[x][2]);
                            }
                        }
                    }
                    gqtc::mma_commit(&empty[st]);
                    first = false;
                }
                if (ok) gqtc::mma_commit(&accfull);
            } else {
                for (int s = next_slot(mask, -1); s < kTcSlots; s = next_slot(mask, s)) ++g;
            }
        } else {
            // ---------------- staging (row = tid) and epilogue
            const size_t row = (size_t)tile * kTcRows + tid;
            const uint32_t rowoff = (uint32_t)(((tid >> 3) * 4) << 7) + (uint32_t)((tid & 7) << 4);
            const int qx = sq[it & 1] & 1, qy = sq[it & 1] >> 1;
            bool ok = true;
            // slot sources of this tile, [slot][row]: a warp's loads are contiguous;
            // prefetched two slots ahead
            const int *ssrc = a.slot_src + (size_t)tile * kTcSlots * kTcRows + tid;
            int s = next_slot(mask, -1);
            int s1 = next_slot(mask, s);
            int d = s < kTcSlots ? ssrc[s * kTcRows] : -1;
            int d1 = s1 < kTcSlots ? ssrc[s1 * kTcRows] : -1;
            for (; s < kTcSlots; ++g) {
                const int s2 = next_slot(mask, s1);
                const int d2 = s2 < kTcSlots ? ssrc[s2 * kTcRows] : -1;
                const int st = g & 1;
                if (ok && g >= 2) ok = gqtc::mbar_wait_abortable(&empty[st], ((g >> 1) - 1) & 1, kWaitNs, &abort_flag);
                if (ok) {
                    const uint32_t sA = sbase + st * kStage, sB = sA + kTcND * kTileA;
                    if (d >= 0 || !zero_row[st]) {   // a row already zero in this stage stays zero
#pragma unroll
                        for (int i = 0; i < kTcND; ++i)
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                const uint32_t dst = sA + i * kTileA + rowoff + (c << 7);
                                if (d >= 0) cp_async16(dst, a.mdig + ((size_t)d * kTcND + i) * kTcK + c * 8);
                                else st_shared_zero16(dst);
                            }
                        zero_row[st] = d < 0;
                    }
                    const int dx = (s % 10) - 4 - qx, dy = (s / 10) - 4 - qy;
                    const uint16_t *tsrc = a.tdig + (size_t)((-dy + 5) * 11 + (-dx + 5)) * kTcND * (kTileB / 2);
                    for (int c = tid; c < (int)(kTcND * kTileB / 16); c += kTcRows) cp_async16(sB + c * 16, tsrc + c * 8);
                    gqtc::mbar_arrive(&full[st]);            // orders the zero stores
                    gqtc::mbar_arrive_cp_async(&full[st]);   // fires when this thread's copies have landed
                }
                s = s1;
                s1 = s2;
                d = d1;
                d1 = d2;
            }
            if (ok) ok = gqtc::mbar_wait_abortable(&accfull, (uint32_t)(it & 1), kWaitNs, &abort_flag);
            // tcgen05.ld is warp-collective: the warp decides together
            if (__all_sync(0xffffffffu, ok)) {
                gqtc::fence_after_sync();
                long long shi[kTcN], slo[kTcN];
#pragma unroll
                for (int n = 0; n < kTcN; ++n) shi[n] = slo[n] = 0;
                const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
                for (int w = 0; w < kTcLev; ++w) {
                    uint32_t v[32];
                    gqtc::tmem_ld32(lane_base + (uint32_t)(w * 32), v);
                    gqtc::tmem_ld_wait();
                    if (w <= 5) {
                        const int sh = 5 * (5 - w);
#pragma unroll
                        for (int n = 0; n < kTcN; ++n) shi[n] += (long long)__float2int_rn(__uint_as_float(v[n])) << sh;
                    } else {
                        const int sh = 5 * (11 - w);
#pragma unroll
                        for (int n = 0; n < kTcN; ++n) slo[n] += (long long)__float2int_rn(__uint_as_float(v[n])) << sh;
                    }
                }
                gqtc::fence_before_sync();
                gqtc::mbar_arrive(&accfree);   // the accumulators may be overwritten now
                const int b = a.tile_box[row];
                if (b >= 0) {
                    const int l = a.blev[b];
                    const int E = a.lexp[l] - 1022;   // |M| < 2^E at this level
                    const int P1 = a.P + 1;
                    double2 *Lb = a.L + (size_t)b * P1;
                    double m0 = 0.0;                   // sum of M_0 over the List 2 boxes (the log rho term)
                    for (int e = a.voff[b]; e < a.voff[b + 1]; ++e) m0 += a.M[(size_t)a.vidx[e] * P1].x;
                    const double logrho = a.logH - l * a.ln2;
#pragma unroll
                    for (int n = 0; n < kTcN; ++n) {
                        const int m = n >> 1;
                        if (m > a.P) continue;
                        const int F = a.fexp[n];
                        // value = 2^(E+F-108) sum_w acc_w 2^(5 (20 - w)) = 2^(E+F-33) shi + 2^(E+F-63) slo
                        double v = fma((double)shi[n], ldexp(1.0, E + F - 33), (double)slo[n] * ldexp(1.0, E + F - 63));
                        if (n == 0) v += m0 * logrho;
                        if (n & 1) Lb[m].y += v;
                        else Lb[m].x += v;
                    }
                }
            } else if (!ok) {
                abort_flag = 1;
            }
        }
    }
    // a role that gave up has set abort_flag; wait for this thread's copies before leaving
    cp_async_wait_all();
    if (abort_flag && tid == 0) atomicExch(a.err, 1);
    gqtc::fence_before_sync();
    __syncthreads();
    if (warp == 0) gqtc::tmem_free(tmem, 512);
}

// ---------------------------------------------------------------- constant tables
struct TcConst {
    uint16_t *tdig = nullptr;   // [121 offsets][11 digits][32 x 32 tile order]
    int *fexp = nullptr;        // [32]
};

void host_tc_tables(std::vector<uint16_t> &tdig, std::vector<int> &fexp) {
    const int P1 = 16;
    std::vector<long double> C(64 * 64, 0.0L);
    for (int n = 0; n < 64; ++n) {
        C[n * 64] = 1.0L;
        for (int k = 1; k <= n; ++k) C[n * 64 + k] = C[(n - 1) * 64 + k - 1] + (k <= n - 1 ? C[(n - 1) * 64 + k] : 0.0L);
    }
    // real-form matrices B[off][n][kk]: n = 2m + c', kk = 2k + c
    std::vector<long double> B((size_t)121 * 32 * 32, 0.0L);
    for (int ty = -5; ty <= 5; ++ty)
        for (int tx = -5; tx <= 5; ++tx) {
            const int off = (ty + 5) * 11 + (tx + 5);
            if (tx >= -2 && tx <= 2 && ty >= -2 && ty <= 2) continue;   // never a List 2 offset
            long double dr = 2.0L * tx, di = 2.0L * ty, n2 = dr * dr + di * di;
            long double ir = dr / n2, ii = -di / n2;   // 1 / delta
            std::vector<long double> pr(2 * P1 + 1), pi(2 * P1 + 1);   // delta^-j
            pr[0] = 1.0L;
            pi[0] = 0.0L;
            for (int j = 1; j <= 2 * P1; ++j) {
                pr[j] = pr[j - 1] * ir - pi[j - 1] * ii;
                pi[j] = pr[j - 1] * ii + pi[j - 1] * ir;
            }
            for (int m = 0; m < P1; ++m)
                for (int k = 0; k < P1; ++k) {
                    long double tr, ti;
                    if (m == 0 && k == 0) {
                        tr = 0.5L * logl(n2);
                        ti = 0.0L;
                    } else if (m == 0) {
                        tr = pr[k];
                        ti = pi[k];
                    } else if (k == 0) {
                        long double s = ((m & 1) ? 1.0L : -1.0L) / m;   // -(-1)^m / m
                        tr = s * pr[m];
                        ti = s * pi[m];
                    } else {
                        long double s = ((m & 1) ? -1.0L : 1.0L) * C[(m + k - 1) * 64 + (k - 1)];
                        tr = s * pr[m + k];
                        ti = s * pi[m + k];
                    }
                    long double *Bo = &B[(size_t)off * 1024];
                    Bo[(2 * m) * 32 + 2 * k] = tr;
                    Bo[(2 * m) * 32 + 2 * k + 1] = -ti;
                    Bo[(2 * m + 1) * 32 + 2 * k] = ti;
                    Bo[(2 * m + 1) * 32 + 2 * k + 1] = tr;
                }
        }
    fexp.assign(32, -1074);
    for (int n = 0; n < 32; ++n) {
        long double mx = 0.0L;
        for (int off = 0; off < 121; ++off)
            for (int kk = 0; kk < 32; ++kk) mx = fmaxl(mx, fabsl(B[(size_t)off * 1024 + n * 32 + kk]));
        int e = 0;
        frexpl(mx, &e);   // mx < 2^e
        fexp[n] = e;
    }
    tdig.assign((size_t)121 * kTcND * 1024, 0);
    for (int off = 0; off < 121; ++off)
        for (int n = 0; n < 32; ++n)
            for (int kk = 0; kk < 32; ++kk) {
                long double v = B[(size_t)off * 1024 + n * 32 + kk];
                long long X = llroundl(ldexpl(v, kTcBits - fexp[n]));
                int d[kTcND];
                tc_digits(X, d);
                GQ_REQUIRE(d[0] >= -16 && d[0] <= 16, GQ_ERR_CUDA, "tensor-core M2L: translation digit out of range");
                const uint32_t o = gqtc::tile_offset(n, kk, 32) / 2;
                for (int j = 0; j < kTcND; ++j) tdig[((size_t)off * kTcND + j) * 1024 + o] = bf16_of_small_int(d[j]);
            }
}

const TcConst &tc_const(int dev) {
    static std::mutex mu;
    static TcConst per_dev[64];
    static bool ready[64] = {};
    GQ_REQUIRE(dev >= 0 && dev < 64, GQ_ERR_UNSUPPORTED, "device index >= 64");
    std::lock_guard<std::mutex> lk(mu);
    if (ready[dev]) return per_dev[dev];
    std::vector<uint16_t> tdig;
    std::vector<int> fexp;
    host_tc_tables(tdig, fexp);
    int cur = 0;
    GQ_CUDA(cudaGetDevice(&cur));
    GQ_CUDA(cudaSetDevice(dev));
    TcConst T;
    GQ_CUDA(cudaMalloc(&T.tdig, sizeof(uint16_t) * tdig.size()));
    GQ_CUDA(cudaMalloc(&T.fexp, sizeof(int) * fexp.size()));
    GQ_CUDA(cudaMemcpy(T.tdig, tdig.data(), sizeof(uint16_t) * tdig.size(), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaMemcpy(T.fexp, fexp.data(), sizeof(int) * fexp.size(), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaSetDevice(cur));
    per_dev[dev] = T;
    ready[dev] = true;
    return per_dev[dev];
}

}  // namespace

bool gq_m2l_tc_supported(const gq_geom *g) { return g->prm.p_fmm <= 15 && g->prm.m2l == GQ_M2L_AUTO; }

// Tiles of the current build: the target boxes with a nonempty List 2,
// grouped by quadrant and sorted by slot pattern, 128 per tile.  Device work
// only (no host read); the tile count stays on the device.
void gq_m2l_tc_build(gq_geom *g) {
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    const int nbox = g->nbox;
    const size_t max_tiles = ((size_t)nbox + kTcRows - 1) / kTcRows + 4, max_rows = max_tiles * kTcRows;
    g->tc_tile_box.alloc(max_rows);
    g->tc_slot_src.alloc(max_rows * kTcSlots);
    g->tc_tile_mask.alloc(max_tiles * 4);
    g->tc_tile_q.alloc(max_tiles);
    g->tc_err.alloc(1);
    g->tc_ntiles_dev.alloc(1);
    g->tc_cnt.alloc(4);
    dbuf<uint32_t> key;
    dbuf<int> val;
    key.alloc(nbox);
    val.alloc(nbox);
    GQ_CUDA(cudaMemsetAsync(g->tc_tile_box.p, 0xff, sizeof(int) * max_rows, st));
    GQ_CUDA(cudaMemsetAsync(g->tc_slot_src.p, 0xff, sizeof(int) * max_rows * kTcSlots, st));
    GQ_CUDA(cudaMemsetAsync(g->tc_tile_mask.p, 0, sizeof(unsigned) * max_tiles * 4, st));
    GQ_CUDA(cudaMemsetAsync(g->tc_err.p, 0, sizeof(int), st));
    GQ_CUDA(cudaMemsetAsync(g->tc_cnt.p, 0, sizeof(int) * 4, st));
    GQ_LAUNCH(ctx, k_tc_keys, gq_blocks(nbox, 256), 256, 0, nbox, (const int *)g->list_off[1].p,
              (const int *)g->list_idx[1].p, (const int *)g->bix.p, (const int *)g->biy.p, key.p, val.p, g->tc_cnt.p,
              g->tc_err.p);
    gq_radix_sort_pairs32(ctx, key.p, val.p, nbox, 32);
    GQ_LAUNCH(ctx, k_tc_fill, gq_blocks(nbox, 256), 256, 0, nbox, (const uint32_t *)key.p, (const int *)val.p,
              (const int *)g->tc_cnt.p, (const int *)g->list_off[1].p, (const int *)g->list_idx[1].p,
              (const int *)g->bix.p, (const int *)g->biy.p, g->tc_tile_box.p, g->tc_tile_q.p, g->tc_slot_src.p,
              g->tc_tile_mask.p, g->tc_ntiles_dev.p);
    g->tc_ready = true;
}

// M2L of the current multipoles M into L (added) on the tensor cores.
void gq_m2l_tc(gq_geom *g, const double2 *M, double2 *L) {
    gq_ctx *ctx = g->ctx;
    if (!g->tc_ready) gq_m2l_tc_build(g);
    const TcConst &T = tc_const(ctx->device);
    const int nbox = g->nbox, P = g->prm.p_fmm;
    g->tc_lexp.alloc(g->nlev);
    g->tc_mdig.alloc((size_t)nbox * kTcND * kTcK);
    GQ_CUDA(cudaMemsetAsync(g->tc_lexp.p, 0, sizeof(int) * g->nlev, ctx->stream));
    GQ_LAUNCH(ctx, k_tc_levexp, gq_blocks((long long)nbox * 32, 256), 256, 0, nbox, P, (const int *)g->blev.p, M,
              g->tc_lexp.p);
    GQ_LAUNCH(ctx, k_tc_digits, gq_blocks((long long)nbox * 32, 256), 256, 0, nbox, P, (const int *)g->blev.p,
              (const int *)g->tc_lexp.p, M, g->tc_mdig.p);
    TcArgs a;
    a.ntiles = g->tc_ntiles_dev;
    a.P = P;
    a.tile_box = g->tc_tile_box;
    a.tile_q = g->tc_tile_q;
    a.slot_src = g->tc_slot_src;
    a.tile_mask = g->tc_tile_mask;
    a.mdig = g->tc_mdig;
    a.tdig = T.tdig;
    a.fexp = T.fexp;
    a.lexp = g->tc_lexp;
    a.blev = g->blev;
    a.voff = g->list_off[1];
    a.vidx = g->list_idx[1];
    a.M = M;
    a.L = L;
    a.logH = log(g->root.H);
    a.ln2 = log(2.0);
    a.err = g->tc_err;
    g->tc_counter.alloc(1);
    GQ_CUDA(cudaMemsetAsync(g->tc_counter.p, 0, sizeof(int), ctx->stream));
    a.next_tile = g->tc_counter;
    static bool attr_set[64] = {};
    int dev = ctx->device;
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        GQ_CUDA(cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * kStage)));
        attr_set[dev] = true;
    }
    int sms = 0;
    GQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int grid = sms;   // persistent: each CTA takes tiles from the counter until none is left
    GQ_LAUNCH(ctx, k_m2l_tc, grid, kTcThreads, 2 * kStage, a);
}

// the device error flag of the tensor-core M2L (synchronises): 0 none, 1 a
// bounded wait gave up, 2 a List 2 entry outside the offset window
int gq_m2l_tc_error(gq_geom *g) {
    if (!g->tc_err.p) return 0;
    int h = 0;
    GQ_CUDA(cudaMemcpyAsync(&h, g->tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, g->ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(g->ctx->stream));
    return h;
}
