// gq_w_tc.cu -- Stage 5b (List 3 far multipoles to the QBX centres, M2QBXL,
// Sec. 4.4 Algorithm; the translation of Sec. 3.1 from a multipole to a local
// expansion about the centre) on the BF16 tensor cores with FP64 accuracy.
//
// Per pair (centre c of radius r, far box d of half-width rho and box-scaled
// multipole A), with y = c - z_d, v = rho / y, s = -r / y and At_k = A_k v^k:
//     Q_0 += A_0 log|y| + G_0,   Q_m += s^m (G_m - A_0 / m)   (1 <= m <= q),
//     G_m = sum_{k=1..P} C(m+k-1, k-1) At_k.
// The G_m are the dense part: a constant integer matrix applied to a per-pair
// vector.  In real form, for a tile of 128 pairs,
//     D[128 x 32] = A[128 x 32] * B^T,  A row = [Re At_1..16, Im At_1..16],
//     B[n][k] = C(m+k'-1, k'-1) on the re-re (n < 16) and im-im (n >= 16)
//     blocks (m = n mod 16, k' = k mod 16 + 1), zero elsewhere,
// D row = [Re G_0..15, Im G_0..15].
//
// FP64 accuracy: each row's 32 entries are a 64-bit fixed-point integer at the
// row's largest exponent (|x| < 2^E), written as eight base-256 digits (sign
// carried by every digit, |digit| <= 255: exact in BF16); every B entry
// (< 2^24) is three base-256 digits.  Digit products (< 2^16) summed over
// K = 32 and at most three digit pairs per level stay below 2^24, so the FP32
// accumulators of the ten digit levels w = i + j hold exact integers.  Each
// column is recombined in 64-bit integers after dropping the low bits that its
// bound (sum_k C(m+k-1, k-1) 2^64) does not need, and converted to FP64 once.
// The truncation of the fixed point moves G_m by at most 2^(E-64) sum_k
// C(m+k-1, k-1); after the factor |s|^m < 1 this stays near 1e-15 of the far
// box's leading term.
//
// The FP64 work left per pair: At (2P complex products), the recombination and
// the epilogue (q complex products and powers, one logarithm) -- about 250
// FP64 instructions against about 580 for the direct FP64 kernel.
//
// CTA: warps 0-3, 4-7 and 8-11 are three groups that stage, in turn, tiles
// of 128 pairs (thread = pair: FP64 At, integer digit split into shared
// memory); the group's first thread then issues the tile's 48 MMAs
// (128 x 32 x 16) into ten tensor-memory accumulators, once the previous
// tile has been read out, and commits them.  One accumulator set: a group
// reads it out (tcgen05.ld) and releases it before finishing its epilogue
// from registers, while the next group's tile is multiplied.  Twelve warps
// put three on each SM sub-partition, so a thread may hold 168 registers.
// Per-pair contributions go to a buffer; a second kernel adds each centre's
// contributions in list order (deterministic, no atomics).
#include <math.h>

#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "gq_internal.cuh"
#include "gq_math.cuh"
#include "gq_tc.cuh"

namespace {

constexpr int kWRows = 128;                           // pairs per tile (MMA M)
constexpr int kWK = 32;                               // real inputs per pair
constexpr int kWN = 32;                               // real outputs per pair
constexpr int kWAD = 8;                               // digits of the pair operand (64 bits)
constexpr int kWBD = 3;                               // digits of the constant matrix (24 bits)
constexpr int kWLev = kWAD + kWBD - 1;                // accumulated digit levels (10)
constexpr uint32_t kWTileA = kWRows * kWK * 2;        // bytes per pair digit tile (8 KiB)
constexpr uint32_t kWTileB = kWN * kWK * 2;           // bytes per constant digit tile (2 KiB)
constexpr uint32_t kWStageA = kWAD * kWTileA;         // 64 KiB per group
constexpr int kWGroups = 3;                           // staging/epilogue warp groups (4 warps each)
constexpr uint32_t kWSmem = kWGroups * kWStageA + kWBD * kWTileB;   // 202,752 bytes
constexpr int kWThreads = 32 * 4 * kWGroups;
constexpr uint64_t kWWaitNs = 2000000000ull;          // bounded waits: 2 s

// 2^e from its bits (ldexp outside the normal range)
__device__ __forceinline__ double w_pow2(int e) {
    return (e >= -1022 && e <= 1023) ? __longlong_as_double((long long)(e + 1023) << 52) : ldexp(1.0, e);
}

// x 2^e by adding e to the exponent field (integer operations; a multiply
// where the result would leave the normal range)
__device__ __forceinline__ double w_scale2(double x, int e) {
    const long long bits = __double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0 || ex + e < 1 || ex + e > 2046) return x * w_pow2(e);
    return __longlong_as_double(bits + ((long long)e << 52));
}

__device__ __forceinline__ double2 w_box_centre(const RootInfo &R, int l, int ix, int iy) {
    double h = R.H * w_pow2(-l);
    return make_double2(R.lo_x + (double)(2 * ix + 1) * h, R.lo_y + (double)(2 * iy + 1) * h);
}

__host__ __device__ inline uint16_t w_bf16_int(int v) {
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

// 16-byte store of eight BF16 values to shared memory
__device__ __forceinline__ void st_shared16(uint32_t dst, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

struct WArgs {
    const int *npairs;        // device: pairs of the current build
    const int *pc, *pd;       // pair -> sorted centre, far box
    const double2 *sc_xy;     // sorted centres
    const double *sc_r;
    const int *blev, *bix, *biy;
    const double2 *M;         // box-scaled multipoles [nbox][P + 1]
    RootInfo R;
    int P, q;
    const uint16_t *bdig;     // [3][32 x 32 tile order]
    const int *drop;          // [32] low bits dropped per output column
    const double *logt;
    double2 *contrib;         // [npairs][q + 1]
    int *err;
};

__global__ void __launch_bounds__(kWThreads, 1) k_w_centres_tc(WArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    __shared__ uint64_t full[kWGroups], accfull[kWGroups], tfree[kWGroups];
    __shared__ uint32_t tslot;
    __shared__ int sdrop[kWN];
    __shared__ volatile int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) gqtc::tmem_alloc(&tslot, 512);
    if (tid < kWN) sdrop[tid] = a.drop[tid];
    if (tid == 0) {
        for (int g = 0; g < kWGroups; ++g) {
            gqtc::mbar_init(&full[g], kWRows);
            gqtc::mbar_init(&accfull[g], 1);
            gqtc::mbar_init(&tfree[g], kWRows);   // group g's tile read out
        }
        abort_flag = 0;
    }
    const uint32_t sbase = gqtc::smem_u32(sm);
    const uint32_t sB = sbase + kWGroups * kWStageA;
    // the constant digit tiles, once per CTA
    for (int c = tid; c < (int)(kWBD * kWTileB / 16); c += blockDim.x) {
        const uint4 v = reinterpret_cast<const uint4 *>(a.bdig)[c];
        st_shared16(sB + c * 16, v.x, v.y, v.z, v.w);
    }
    gqtc::fence_smem_to_async();
    gqtc::fence_before_sync();
    __syncthreads();
    gqtc::fence_after_sync();
    const uint32_t tmem = tslot;
    const int npairs = *a.npairs;
    const int ntiles = (npairs + kWRows - 1) / kWRows;
    {
        // ---------------- staging and epilogue: group w, thread r = row of its tiles
        const int w = warp >> 2, r = tid & 127, wq = warp & 3;
        const uint32_t sA = sbase + w * kWStageA;
        const uint32_t rowoff = (uint32_t)(((r >> 3) * (kWK / 8)) << 7) + (uint32_t)((r & 7) << 4);
        const int P = a.P, q = a.q;
        bool ok = true;
        int k = w, pend = -1;   // pend: a tile this thread committed but has not seen complete
        for (int t = blockIdx.x + w * gridDim.x; t < ntiles; t += kWGroups * gridDim.x, k += kWGroups) {
            const int p = t * kWRows + r;
            const bool valid = p < npairs;
            // ---- stage: At_k of this pair, the row exponent, eight digits per entry
            double2 y = make_double2(0.0, 0.0), s = make_double2(0.0, 0.0);
            double n2 = 1.0, A0 = 0.0;
            int c = 0;
            double at[2][16];
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) at[0][kk] = at[1][kk] = 0.0;
            unsigned emax = 0;
            if (valid) {
                c = a.pc[p];
                const int d = a.pd[p], l = a.blev[d];
                const double rho = a.R.H * w_pow2(-l);
                const double2 zd = w_box_centre(a.R, l, a.bix[d], a.biy[d]);
                const double2 cz = a.sc_xy[c];
                y = make_double2(cz.x - zd.x, cz.y - zd.y);
                n2 = y.x * y.x + y.y * y.y;
                const double inv = gq_rcp(n2);
                const double2 yinv = make_double2(y.x * inv, -y.y * inv);
                const double2 v = make_double2(rho * yinv.x, rho * yinv.y);
                const double rc = a.sc_r[c];
                s = make_double2(-rc * yinv.x, -rc * yinv.y);
                const double2 *Ad = a.M + (size_t)d * (P + 1);
                A0 = Ad[0].x;
                double2 vk = v;
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    if (kk < P) {
                        const double2 Ak = Ad[kk + 1];
                        at[0][kk] = Ak.x * vk.x - Ak.y * vk.y;
                        at[1][kk] = Ak.x * vk.y + Ak.y * vk.x;
                        vk = make_double2(vk.x * v.x - vk.y * v.y, vk.x * v.y + vk.y * v.x);
                    }
                }
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) {
                        const unsigned e = (unsigned)(((unsigned long long)__double_as_longlong(at[h][kk]) >> 52) & 0x7ff);
                        emax = e > emax ? e : emax;
                    }
            }
            // group's buffer is free: its previous tile's MMAs completed before that
            // tile's epilogue (accfull was waited), in program order
            // digits: X = |x| 2^(64 - E), E = emax - 1022 (|x| < 2^E), as the mantissa
            // shifted; byte i of X becomes the FP32 value 2^23 + byte (one byte permute
            // into the bits of 2^23), then +-byte by one FMA, and two of those pack
            // into a BF16 pair by taking their upper halves (exact: at most 8
            // significant bits)
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int g8 = 0; g8 < 2; ++g8) {
                    uint32_t pk[kWAD][4];
#pragma unroll
                    for (int e8 = 0; e8 < 8; e8 += 2) {
                        uint32_t wlo[2], whi[2];
                        float sgf[2];
#pragma unroll
                        for (int u = 0; u < 2; ++u) {
                            const double x = at[h][g8 * 8 + e8 + u];
                            const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
                            const int ex = (int)((bits >> 52) & 0x7ff);
                            unsigned long long X = 0;
                            if (ex != 0 && emax != 0) {
                                const unsigned long long m53 = (bits & 0x000fffffffffffffull) | 0x0010000000000000ull;
                                const int sh = ex - (int)emax + 11;   // <= 11
                                X = sh >= 0 ? (m53 << sh) : (sh > -64 ? (m53 >> -sh) : 0ull);
                            }
                            wlo[u] = (uint32_t)X;
                            whi[u] = (uint32_t)(X >> 32);
                            sgf[u] = (bits >> 63) ? -1.0f : 1.0f;
                        }
#pragma unroll
                        for (int i = 0; i < kWAD; ++i) {
                            float f[2];
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const uint32_t m = __byte_perm(i < 4 ? wlo[u] : whi[u], 0x4B000000u, 0x7650u | (uint32_t)(i & 3));
                                f[u] = fmaf(__uint_as_float(m), sgf[u], -8388608.0f * sgf[u]);
                            }
                            pk[i][e8 >> 1] = __byte_perm(__float_as_uint(f[0]), __float_as_uint(f[1]), 0x7632u);
                        }
                    }
                    // column group kk = 16 h + 8 g8 .. + 7: core matrix (16 h + 8 g8) / 8 of this row
                    const uint32_t coff = (uint32_t)((2 * h + g8) << 7);
#pragma unroll
                    for (int i = 0; i < kWAD; ++i)
                        st_shared16(sA + i * kWTileA + rowoff + coff, pk[i][0], pk[i][1], pk[i][2], pk[i][3]);
                }
            gqtc::fence_smem_to_async();
            gqtc::mbar_arrive(&full[w]);
            // ---- issue: the group's first thread, once the whole group has staged
            // and the previous tile (another group's) has left the accumulators
            if (r == 0) {
                if (ok) ok = gqtc::mbar_wait_abortable(&full[w], (uint32_t)((k / kWGroups) & 1), kWWaitNs, &abort_flag);
                // tile k - 1 belongs to group (k - 1) % G; its read-out is that barrier's
                // completion number (k - 1) / G, and the one before (tile k - 1 - G) is
                // complete (this group's tile k - G was issued after it), so the parity
                // wait is never more than one phase behind
                if (ok && k >= 1)
                    ok = gqtc::mbar_wait_abortable(&tfree[(k - 1) % kWGroups], (uint32_t)(((k - 1) / kWGroups) & 1),
                                                   kWWaitNs, &abort_flag);
                if (ok) {
                    gqtc::fence_smem_to_async();
                    gqtc::fence_after_sync();
                    // digit pair (i, j) lands in level i + j (32 columns each); the first
                    // product written to a level overwrites it
#pragma unroll 1
                    for (int j = 0; j < kWBD; ++j)
#pragma unroll 1
                        for (int i = 0; i < kWAD; ++i)
#pragma unroll 1
                            for (int ks = 0; ks < 2; ++ks) {
                                const bool first = ks == 0 && (j == 0 || i == kWAD - 1);
                                const uint64_t ad = gqtc::smem_desc(sA + i * kWTileA + ks * 256, 128, 512);
                                const uint64_t bd = gqtc::smem_desc(sB + j * kWTileB + ks * 256, 128, 512);
                                gqtc::mma_bf16(tmem + (uint32_t)((i + j) * 32), ad, bd, gqtc::idesc_bf16_f32(128, 32),
                                               first ? 0u : 1u);
                            }
                    gqtc::mma_commit(&accfull[w]);
                    pend = k;
                } else {
                    abort_flag = 1;
                }
            }
            // ---- epilogue: the ten levels of this row, recombined per column
            if (ok) ok = gqtc::mbar_wait_abortable(&accfull[w], (uint32_t)((k / kWGroups) & 1), kWWaitNs, &abort_flag);
            if (ok) pend = -1;
            if (!__all_sync(0xffffffffu, ok)) {   // tcgen05.ld is warp-collective
                abort_flag = 1;
                break;
            }
            gqtc::fence_after_sync();
            // per column: levels 0-4 and 5-9 summed with compile-time weights
            // (each part below 2^56), then joined after dropping the column's
            // unneeded low bits; only the columns m <= q are used
            long long vcol[kWN];
            const uint32_t lane_base = tmem + ((uint32_t)(wq * 32) << 16);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                long long vlo[16], vhi[16];
#pragma unroll
                for (int n = 0; n < 16; ++n) vlo[n] = vhi[n] = 0;
#pragma unroll
                for (int lv = 0; lv < kWLev; ++lv) {
                    uint32_t acc[16];
                    gqtc::tmem_ld16(lane_base + (uint32_t)(lv * 32 + hh * 16), acc);
                    gqtc::tmem_ld_wait();
#pragma unroll
                    for (int n = 0; n < 16; ++n) {
                        if (n > q) continue;
                        const long long xv = (long long)__float2int_rn(__uint_as_float(acc[n]));
                        if (lv < 5) vlo[n] += xv * (1LL << (8 * lv));
                        else vhi[n] += xv * (1LL << (8 * (lv - 5)));
                    }
                }
#pragma unroll
                for (int n = 0; n < 16; ++n) {
                    const int d = sdrop[hh * 16 + n];
                    vcol[hh * 16 + n] = n > q ? 0 : (vhi[n] << (40 - d)) + (vlo[n] >> d);
                }
            }
            gqtc::fence_before_sync();
            gqtc::mbar_arrive(&tfree[w]);   // the accumulators may be overwritten now
            if (valid) {
                const int E = (int)emax - 1022;
                double2 *dst = a.contrib + (size_t)p * (q + 1);
                double2 sm_ = make_double2(1.0, 0.0);
#pragma unroll
                for (int m = 0; m < 16; ++m) {
                    if (m > q) break;
                    double2 G = make_double2(emax ? w_scale2((double)vcol[m], E - 64 + sdrop[m]) : 0.0,
                                             emax ? w_scale2((double)vcol[16 + m], E - 64 + sdrop[16 + m]) : 0.0);
                    if (m == 0) {
                        dst[0] = make_double2(A0 * gq_log_half(n2, a.logt) + G.x, G.y);
                    } else {
                        sm_ = make_double2(sm_.x * s.x - sm_.y * s.y, sm_.x * s.y + sm_.y * s.x);   // (-r/y)^m
                        G.x -= A0 * (1.0 / m);
                        dst[m] = make_double2(sm_.x * G.x - sm_.y * G.y, sm_.x * G.y + sm_.y * G.x);
                    }
                }
            }
        }
        if (!ok) abort_flag = 1;
        // leave no MMA in flight (the accumulators are freed below): wait, boundedly,
        // for a commit whose completion this thread has not seen
        if (pend >= 0) gqtc::mbar_wait(&accfull[pend % kWGroups], (uint32_t)((pend / kWGroups) & 1), kWWaitNs);
    }
    if (abort_flag && tid == 0) atomicExch(a.err, 1);
    gqtc::fence_before_sync();
    __syncthreads();
    if (warp == 0) gqtc::tmem_free(tmem, 512);
}

// each centre's contributions in list order, added to its QBX coefficients:
// one thread per (centre, real component), so that the threads of a centre
// read each 16 (q + 1)-byte record together
__global__ void k_w_centres_reduce(int nc, int q, const int *__restrict__ pstart, const double *__restrict__ contrib,
                                   double *__restrict__ Q) {
    const int ncomp = 2 * (q + 1);
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)nc * ncomp) return;
    const int c = (int)(t / ncomp), comp = (int)(t - (long long)c * ncomp);
    const int p0 = pstart[c], p1 = pstart[c + 1];
    if (p0 == p1) return;
    double acc = 0.0;
    for (int p = p0; p < p1; ++p) acc += contrib[(size_t)p * ncomp + comp];
    Q[(size_t)c * ncomp + comp] += acc;
}

// ---------------------------------------------------------------- pairs (per build)
__global__ void k_w_pair_count(int nc, const int *__restrict__ owner, const int *__restrict__ woff,
                               int *__restrict__ cnt) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int b = owner[c];
    cnt[c] = woff[b + 1] - woff[b];
}

__global__ void k_w_pair_fill(int nc, const int *__restrict__ owner, const int *__restrict__ woff,
                              const int *__restrict__ widx, const int *__restrict__ pstart, int *__restrict__ pc,
                              int *__restrict__ pd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int b = owner[c];
    int p = pstart[c];
    for (int e = woff[b]; e < woff[b + 1]; ++e, ++p) {
        pc[p] = c;
        pd[p] = widx[e];
    }
}

// ---------------------------------------------------------------- constant tables (per P, q)
struct WConst {
    uint16_t *bdig = nullptr;   // [3][32 x 32 tile order]
    int *drop = nullptr;        // [32]
};

bool w_binom_fits(int P, int q) {
    // the largest entry C(q+P-1, P-1) below 2^24
    long double c = 1.0L;
    for (int i = 1; i <= P - 1; ++i) c = c * (q + i) / i;
    return c < 16777216.0L;
}

const WConst &w_const(int dev, int P, int q) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, WConst> tabs[64];
    GQ_REQUIRE(dev >= 0 && dev < 64, GQ_ERR_UNSUPPORTED, "device index >= 64");
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(P, q);
    auto it = tabs[dev].find(key);
    if (it != tabs[dev].end()) return it->second;
    std::vector<long long> C(64 * 64, 0);
    for (int n = 0; n < 64; ++n) {
        C[n * 64] = 1;
        for (int k = 1; k <= n && k < 64; ++k) C[n * 64 + k] = C[(n - 1) * 64 + k - 1] + (k <= n - 1 ? C[(n - 1) * 64 + k] : 0);
    }
    std::vector<long long> B(32 * 32, 0);
    std::vector<int> drop(32, 0);
    for (int n = 0; n < 32; ++n) {
        const int m = n & 15;
        long long S = 0;
        for (int kk = 0; kk < 32; ++kk) {
            const int kp = (kk & 15) + 1;
            if ((n >> 4) != (kk >> 4) || m > q || kp > P) continue;
            B[n * 32 + kk] = C[(m + kp - 1) * 64 + (kp - 1)];
            S += B[n * 32 + kk];
        }
        // |sum_k B X_k| < S 2^64: keep it below 2^62 after dropping
        int lg = 0;
        while ((1LL << lg) <= S) ++lg;
        drop[n] = lg + 2;
    }
    std::vector<uint16_t> bdig((size_t)kWBD * 1024, 0);
    for (int n = 0; n < 32; ++n)
        for (int kk = 0; kk < 32; ++kk) {
            long long v = B[n * 32 + kk];
            GQ_REQUIRE(v < (1LL << 24), GQ_ERR_UNSUPPORTED, "M2QBXL on tensor cores: binomial above 2^24");
            const uint32_t o = gqtc::tile_offset(n, kk, 32) / 2;
            for (int j = 0; j < kWBD; ++j) bdig[(size_t)j * 1024 + o] = w_bf16_int((int)((v >> (8 * j)) & 255));
        }
    int cur = 0;
    GQ_CUDA(cudaGetDevice(&cur));
    GQ_CUDA(cudaSetDevice(dev));
    WConst T;
    GQ_CUDA(cudaMalloc(&T.bdig, sizeof(uint16_t) * bdig.size()));
    GQ_CUDA(cudaMalloc(&T.drop, sizeof(int) * drop.size()));
    GQ_CUDA(cudaMemcpy(T.bdig, bdig.data(), sizeof(uint16_t) * bdig.size(), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaMemcpy(T.drop, drop.data(), sizeof(int) * drop.size(), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaSetDevice(cur));
    return tabs[dev][key] = T;
}

// Once per device: the shared-memory attribute, and whether one CTA fits an SM
// (resident blocks per SM from the occupancy calculator).
bool w_tc_launchable(int dev) {
    static std::mutex mu;
    static int state[64] = {};   // 0 unknown, 1 fits, 2 does not
    if (dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lk(mu);
    if (state[dev] == 0) {
        int cur = 0;
        GQ_CUDA(cudaGetDevice(&cur));
        GQ_CUDA(cudaSetDevice(dev));
        GQ_CUDA(cudaFuncSetAttribute(k_w_centres_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWSmem));
        int nb = 0;
        GQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_w_centres_tc, kWThreads, kWSmem));
        GQ_CUDA(cudaSetDevice(cur));
        state[dev] = nb >= 1 ? 1 : 2;
    }
    return state[dev] == 1;
}

}  // namespace

bool gq_w_tc_supported(const gq_geom *g) {
    return g->prm.m2l == GQ_M2L_AUTO && g->prm.p_fmm <= 16 && g->prm.p_qbx <= 15 &&
           w_binom_fits(g->prm.p_fmm, g->prm.p_qbx) && w_tc_launchable(g->ctx->device);
}

// Pairs of the current build: every sorted centre with each box of its owner's
// List 3 far, in list order (one host read: the pair count).
void gq_w_tc_build(gq_geom *g) {
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    const int nc = g->nc;
    g->wtc_pstart.alloc((size_t)nc + 1);
    dbuf<int> cnt, tmp;
    cnt.alloc(nc > 0 ? nc : 1);
    tmp.alloc(gq_scan_tmp_size(nc));
    if (nc)
        GQ_LAUNCH(ctx, k_w_pair_count, gq_blocks(nc, 256), 256, 0, nc, (const int *)g->ctr_owner.p,
                  (const int *)g->list_off[3].p, cnt.p);
    gq_exclusive_scan(ctx, cnt.p, g->wtc_pstart.p, nc, tmp.p);
    int np = 0;
    GQ_CUDA(cudaMemcpyAsync(&np, g->wtc_pstart.p + nc, sizeof(int), cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaStreamSynchronize(st));
    g->wtc_npairs = np;
    g->wtc_pc.alloc(np > 0 ? np : 1);
    g->wtc_pd.alloc(np > 0 ? np : 1);
    if (nc)
        GQ_LAUNCH(ctx, k_w_pair_fill, gq_blocks(nc, 256), 256, 0, nc, (const int *)g->ctr_owner.p,
                  (const int *)g->list_off[3].p, (const int *)g->list_idx[3].p, (const int *)g->wtc_pstart.p,
                  g->wtc_pc.p, g->wtc_pd.p);
    if (!g->tc_err.p) {
        g->tc_err.alloc(1);
        GQ_CUDA(cudaMemsetAsync(g->tc_err.p, 0, sizeof(int), st));
    }
    g->wtc_ready = true;
}

// M2QBXL of the multipoles M into the (sorted-centre) QBX coefficients Q (added).
void gq_w_centres_tc(gq_geom *g, const RootInfo &R, const double2 *M, const double *logt, double2 *Q) {
    gq_ctx *ctx = g->ctx;
    if (!g->wtc_ready) gq_w_tc_build(g);
    const int P = g->prm.p_fmm, q = g->prm.p_qbx;
    const WConst &T = w_const(ctx->device, P, q);
    const int np = g->wtc_npairs;
    if (np == 0) return;
    g->wtc_contrib.alloc((size_t)np * (q + 1));
    WArgs a;
    a.npairs = g->wtc_pstart.p + g->nc;
    a.pc = g->wtc_pc;
    a.pd = g->wtc_pd;
    a.sc_xy = g->sc_xy;
    a.sc_r = g->sc_r;
    a.blev = g->blev;
    a.bix = g->bix;
    a.biy = g->biy;
    a.M = M;
    a.R = R;
    a.P = P;
    a.q = q;
    a.bdig = T.bdig;
    a.drop = T.drop;
    a.logt = logt;
    a.contrib = g->wtc_contrib;
    a.err = g->tc_err;
    const int dev = ctx->device;
    GQ_REQUIRE(w_tc_launchable(dev), GQ_ERR_UNSUPPORTED, "M2QBXL on tensor cores: the kernel does not fit an SM");
    int sms = 0;
    GQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int ntiles = (np + kWRows - 1) / kWRows;
    const int grid = ntiles < sms ? ntiles : sms;
    GQ_LAUNCH(ctx, k_w_centres_tc, grid, kWThreads, kWSmem, a);
    GQ_LAUNCH(ctx, k_w_centres_reduce, gq_blocks((long long)g->nc * 2 * (q + 1), 256), 256, 0, g->nc, q,
              (const int *)g->wtc_pstart.p, (const double *)g->wtc_contrib.p, (double *)Q);
}
