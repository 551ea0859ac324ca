// gq_learned.cu -- learned order selection (an extension; the paper chooses
// orders from its error bounds, Sec. 4.1, and notes those bounds
// overestimate the error by about two orders of magnitude, Sec. 5.1).
//
// A small MLP (32 -> 64 -> 32 -> 32 -> 2, ReLU) maps per-centre geometry
// features to the predicted log10 relative QBX truncation error at p_qbx =
// q_ref and log10 relative FMM error at p_fmm = p_ref.  Training (FP32,
// mean-squared error, Adam) and inference (BF16 weights and activations,
// FP32 sums) are CUDA kernels of this file.  Deployment turns the
// predictions into one QBX order per centre and one FMM order for the tree
// using measured per-order decay rates; the bound-driven orders remain the
// fallback and the cap.
#include <cuda_bf16.h>
#include <math.h>

#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "gq_internal.cuh"

namespace {

constexpr int kT = 256;
constexpr int kNF = 32;                       // features per centre
constexpr int kDims[5] = {32, 64, 32, 32, 2};
constexpr int kLayers = 4;
// parameter offsets: W_l [out][in] then b_l [out]
__host__ __device__ constexpr int woff(int l) {
    return l == 0 ? 0 : woff(l - 1) + (l == 1 ? 32 * 64 + 64 : l == 2 ? 64 * 32 + 32 : l == 3 ? 32 * 32 + 32 : 32 * 2 + 2);
}
constexpr int kNParams = woff(kLayers);
// the same layout for device code (runtime layer index)
__device__ __forceinline__ int ddim(int l) { return l == 0 ? 32 : l == 1 ? 64 : l == 2 ? 32 : l == 3 ? 32 : 2; }
__device__ __forceinline__ int dwoff(int l) {
    int o = 0;
    for (int i = 0; i < l; ++i) o += ddim(i) * ddim(i + 1) + ddim(i + 1);
    return o;
}

// ------------------------------------------------------------------ features
// curvature at base nodes from the turning of the normal between the
// neighbouring nodes of the same panel (one-sided at the panel ends)
__global__ void k_base_curvature(int nbase, int nb, const double *__restrict__ xy, const double *__restrict__ n,
                                 float *__restrict__ kappa) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbase) return;
    int j = i % nb;
    int a = j == 0 ? i : i - 1, b = j == nb - 1 ? i : i + 1;
    double cr = n[2 * a] * n[2 * b + 1] - n[2 * a + 1] * n[2 * b];
    double dt = n[2 * a] * n[2 * b] + n[2 * a + 1] * n[2 * b + 1];
    double ds = hypot(xy[2 * b] - xy[2 * a], xy[2 * b + 1] - xy[2 * a + 1]);
    kappa[i] = ds > 0 ? (float)(atan2(cr, dt) / ds) : 0.f;
}

// Per centre (sorted position j): among the sources of its box's direct lists,
// the 8 nearest distinct panels (distance to their nearest source, over r,
// ascending) and their lengths (over the centre's own panel length); then
// the curvature times r at the base nodes k - 8 .. k + 7 of its own panel
// (k its own node, clamped to the panel), signed so that positive means the
// curve bends towards the centre.
__global__ void k_centre_features(int nc, int nb, int nu, const int *__restrict__ ctr_perm,
                                  const int *__restrict__ ctr_owner, const double2 *__restrict__ sc_xy,
                                  const double *__restrict__ sc_r, const int *__restrict__ loff0,
                                  const int *__restrict__ lidx0, const int *__restrict__ loff2,
                                  const int *__restrict__ lidx2, const int *__restrict__ loff4,
                                  const int *__restrict__ lidx4, const int *__restrict__ src_beg,
                                  const int *__restrict__ src_end, const double2 *__restrict__ s_xy,
                                  const int *__restrict__ src_perm, const double *__restrict__ panel_len,
                                  const float *__restrict__ kappa, float *__restrict__ feat) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nc) return;
    int cid = ctr_perm[j], b = ctr_owner[j];
    int node = cid >> 1, side = cid & 1, panel = node / nb;
    double2 c = sc_xy[j];
    double r = sc_r[j];
    float pd[8];
    int pp[8];
    for (int k = 0; k < 8; ++k) { pd[k] = 3.0e38f; pp[k] = -1; }
    const int *offs[3] = {loff0, loff2, loff4};
    const int *idxs[3] = {lidx0, lidx2, lidx4};
    for (int L = 0; L < 3; ++L)
        for (int e = offs[L][b]; e < offs[L][b + 1]; ++e) {
            int d = idxs[L][e];
            for (int s = src_beg[d]; s < src_end[d]; ++s) {
                int p = src_perm[s] / nu;
                if (p == panel) continue;
                float dist = (float)(hypot(s_xy[s].x - c.x, s_xy[s].y - c.y) / r);
                int at = -1;
                for (int k = 0; k < 8; ++k) if (pp[k] == p) at = k;
                if (at >= 0) {
                    if (dist >= pd[at]) continue;
                    // move the improved entry towards the front
                    while (at > 0 && pd[at - 1] > dist) { pd[at] = pd[at - 1]; pp[at] = pp[at - 1]; --at; }
                    pd[at] = dist; pp[at] = p;
                } else if (dist < pd[7]) {
                    int k = 7;
                    while (k > 0 && pd[k - 1] > dist) { pd[k] = pd[k - 1]; pp[k] = pp[k - 1]; --k; }
                    pd[k] = dist; pp[k] = p;
                }
            }
        }
    float *f = feat + (size_t)cid * kNF;
    double own = panel_len[panel];
    for (int k = 0; k < 8; ++k) {
        f[k] = pp[k] >= 0 ? fminf(pd[k], 64.f) : 64.f;
        f[8 + k] = pp[k] >= 0 ? (float)(panel_len[pp[k]] / own) : 0.f;
    }
    float sg = side ? -1.f : 1.f;   // interior centre (side 0) sits on the concave side when kappa > 0
    int own_k = node - panel * nb;
    for (int k = 0; k < 16; ++k) {
        int kk = own_k + k - 8;     // window centred on the centre's own node, clamped to its panel
        kk = kk < 0 ? 0 : (kk > nb - 1 ? nb - 1 : kk);
        f[16 + k] = sg * kappa[panel * nb + kk] * (float)r;
    }
}

// ------------------------------------------------------------------ MLP kernels
// Z = A_prev W^T + b, A = relu(Z) (or A = Z for the last layer); thread per (sample, neuron)
__global__ void k_dense_fwd(int B, int nin, int nout, const float *__restrict__ Ain, const float *__restrict__ W,
                            const float *__restrict__ bias, float *__restrict__ Z, float *__restrict__ A, int relu) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * nout) return;
    int s = t / nout, o = t % nout;
    const float *a = Ain + (size_t)s * nin, *w = W + (size_t)o * nin;
    float z = bias[o];
    for (int i = 0; i < nin; ++i) z = fmaf(w[i], a[i], z);
    Z[t] = z;
    A[t] = relu ? fmaxf(z, 0.f) : z;
}

// delta = 2 (Yhat - Y) / (B * nout); per-sample squared error into err
__global__ void k_mse_delta(int B, int nout, const float *__restrict__ Yh, const float *__restrict__ Y,
                            float *__restrict__ delta, float *__restrict__ err) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * nout) return;
    float d = Yh[t] - Y[t];
    delta[t] = 2.f * d / (float)(B * nout);
    err[t] = d * d;
}

// dW[o][i] = sum_s delta[s][o] A[s][i], db[o] = sum_s delta[s][o]; thread per parameter
__global__ void k_dense_grad(int B, int nin, int nout, const float *__restrict__ delta, const float *__restrict__ Ain,
                             float *__restrict__ dW, float *__restrict__ db) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nout * (nin + 1)) return;
    if (t < nout * nin) {
        int o = t / nin, i = t % nin;
        float g = 0.f;
        for (int s = 0; s < B; ++s) g = fmaf(delta[(size_t)s * nout + o], Ain[(size_t)s * nin + i], g);
        dW[t] = g;
    } else {
        int o = t - nout * nin;
        float g = 0.f;
        for (int s = 0; s < B; ++s) g += delta[(size_t)s * nout + o];
        db[o] = g;
    }
}

// delta_prev[s][i] = (sum_o delta[s][o] W[o][i]) * relu'(Z_prev[s][i])
__global__ void k_dense_bwd(int B, int nin, int nout, const float *__restrict__ delta, const float *__restrict__ W,
                            const float *__restrict__ Zprev, float *__restrict__ dprev) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * nin) return;
    int s = t / nin, i = t % nin;
    float g = 0.f;
    for (int o = 0; o < nout; ++o) g = fmaf(delta[(size_t)s * nout + o], W[(size_t)o * nin + i], g);
    dprev[t] = Zprev[t] > 0.f ? g : 0.f;
}

__global__ void k_adam(int n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
}

// rows perm[k] of X (n x d) into out (B x d), normalised (x - mu) / sd
__global__ void k_gather_rows(int B, int d, const int *__restrict__ perm, const float *__restrict__ X,
                              const float *__restrict__ mu, const float *__restrict__ sd, float *__restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= B * d) return;
    int s = t / d, c = t % d;
    out[t] = (X[(size_t)perm[s] * d + c] - mu[c]) / sd[c];
}

// BF16 inference on the tensor cores (mma.sync m16n8k16, BF16 inputs, FP32
// accumulators): a warp takes 16 samples through all four layers.  Inputs
// are normalised and rounded to BF16; each layer's accumulators start at its
// BF16 bias, and after ReLU the accumulator fragments of output columns
// 16k ... 16k+15 are, packed to BF16 pairs, exactly the A fragment of the
// next layer's k-block k (row g = lane / 4 and g + 8, columns 2 (lane % 4)
// and + 1, + 8), so activations never leave registers.  The last layer
// (2 outputs) fills the first two columns of one 8-wide tile; its weight
// rows 2 ... 7 read as zero.
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// one dense layer for a warp's 16 rows: NIN inputs as NIN/16 A fragments,
// NOUT outputs as NOUT/8 accumulator tiles; W [nout_real][NIN] BF16 in
// shared memory, rows >= nout_real read as zero
template <int NIN, int NOUT>
__device__ __forceinline__ void mma_layer(const uint32_t (&A)[NIN / 16][4], const __nv_bfloat16 *W,
                                          const __nv_bfloat16 *bias, int nout_real, float (&C)[NOUT / 8][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < NOUT / 8; ++j) {
        const int c0 = 8 * j + 2 * t;
        const float bl = c0 < nout_real ? __bfloat162float(bias[c0]) : 0.f;
        const float bh = c0 + 1 < nout_real ? __bfloat162float(bias[c0 + 1]) : 0.f;
        C[j][0] = bl; C[j][1] = bh; C[j][2] = bl; C[j][3] = bh;
        const int n = 8 * j + g;
#pragma unroll
        for (int kb = 0; kb < NIN / 16; ++kb) {
            uint32_t b0 = 0, b1 = 0;
            if (n < nout_real) {
                const __nv_bfloat16 *wr = W + n * NIN + 16 * kb + 2 * t;
                b0 = *reinterpret_cast<const uint32_t *>(wr);
                b1 = *reinterpret_cast<const uint32_t *>(wr + 8);
            }
            mma_bf16_16816(C[j], A[kb], b0, b1);
        }
    }
}

// accumulators of a hidden layer -> ReLU -> BF16 A fragments of the next layer
template <int NOUT>
__device__ __forceinline__ void relu_to_frags(const float (&C)[NOUT / 8][4], uint32_t (&A)[NOUT / 16][4]) {
#pragma unroll
    for (int kb = 0; kb < NOUT / 16; ++kb) {
        A[kb][0] = pack_bf16x2(fmaxf(C[2 * kb][0], 0.f), fmaxf(C[2 * kb][1], 0.f));
        A[kb][1] = pack_bf16x2(fmaxf(C[2 * kb][2], 0.f), fmaxf(C[2 * kb][3], 0.f));
        A[kb][2] = pack_bf16x2(fmaxf(C[2 * kb + 1][0], 0.f), fmaxf(C[2 * kb + 1][1], 0.f));
        A[kb][3] = pack_bf16x2(fmaxf(C[2 * kb + 1][2], 0.f), fmaxf(C[2 * kb + 1][3], 0.f));
    }
}

static_assert(kDims[0] == 32 && kDims[1] == 64 && kDims[2] == 32 && kDims[3] == 32 && kDims[4] == 2,
              "the tensor-core inference is written for 32-64-32-32-2");

__global__ void __launch_bounds__(128) k_mlp_infer_mma(int n, const float *__restrict__ X,
                                                       const __nv_bfloat16 *__restrict__ Wb,
                                                       const float *__restrict__ xmu, const float *__restrict__ xsd,
                                                       const float *__restrict__ ymu, const float *__restrict__ ysd,
                                                       float *__restrict__ Y) {
    __shared__ __align__(16) __nv_bfloat16 sw[kNParams + 8];
    for (int i = threadIdx.x; i < kNParams; i += blockDim.x) sw[i] = Wb[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int s0 = 16 * (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); s0 < n; s0 += 16 * warps) {
        // input fragments: rows s0 + g, s0 + g + 8; features 16 kb + 2t (+1), + 8
        uint32_t A0[2][4];
#pragma unroll
        for (int kb = 0; kb < 2; ++kb)
#pragma unroll
            for (int h = 0; h < 2; ++h)        // column half: + 0 or + 8
#pragma unroll
                for (int r = 0; r < 2; ++r) {  // row g or g + 8
                    const int s = s0 + g + 8 * r, f = 16 * kb + 8 * h + 2 * t;
                    float lo = 0.f, hi = 0.f;
                    if (s < n) {
                        lo = (X[(size_t)s * kNF + f] - xmu[f]) / xsd[f];
                        hi = (X[(size_t)s * kNF + f + 1] - xmu[f + 1]) / xsd[f + 1];
                    }
                    A0[kb][2 * h + r] = pack_bf16x2(lo, hi);
                }
        float C1[8][4];
        mma_layer<32, 64>(A0, sw + woff(0), sw + woff(0) + 32 * 64, 64, C1);
        uint32_t A1[4][4];
        relu_to_frags<64>(C1, A1);
        float C2[4][4];
        mma_layer<64, 32>(A1, sw + woff(1), sw + woff(1) + 64 * 32, 32, C2);
        uint32_t A2[2][4];
        relu_to_frags<32>(C2, A2);
        float C3[4][4];
        mma_layer<32, 32>(A2, sw + woff(2), sw + woff(2) + 32 * 32, 32, C3);
        uint32_t A3[2][4];
        relu_to_frags<32>(C3, A3);
        float C4[1][4];
        mma_layer<32, 8>(A3, sw + woff(3), sw + woff(3) + 32 * 2, 2, C4);
        if (t == 0) {   // columns 0 and 1 of rows g and g + 8
            const int sa = s0 + g, sb = s0 + g + 8;
            if (sa < n) {
                Y[(size_t)sa * 2] = C4[0][0] * ysd[0] + ymu[0];
                Y[(size_t)sa * 2 + 1] = C4[0][1] * ysd[1] + ymu[1];
            }
            if (sb < n) {
                Y[(size_t)sb * 2] = C4[0][2] * ysd[0] + ymu[0];
                Y[(size_t)sb * 2 + 1] = C4[0][3] * ysd[1] + ymu[1];
            }
        }
    }
}

__global__ void k_to_bf16(int n, const float *__restrict__ in, __nv_bfloat16 *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16(in[i]);
}

// per-centre QBX order from the predicted truncation error at q_ref; the FMM
// prediction is reduced to its maximum (the tree uses one FMM order)
__global__ void k_learned_q(int nc, const int *__restrict__ ctr_perm, const float *__restrict__ pred, double log_tol,
                            double margin, int q_ref, double qbx_slope, int q_cap, int *__restrict__ q_sorted,
                            unsigned int *__restrict__ fmm_max_bits, int *__restrict__ qmax) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nc) return;
    int cid = ctr_perm[j];
    double yq = pred[(size_t)cid * 2], yf = pred[(size_t)cid * 2 + 1];
    int q = q_ref + (int)ceil((yq + margin - log_tol) / qbx_slope);
    q = q < 1 ? 1 : (q > q_cap ? q_cap : q);
    q_sorted[j] = q;
    atomicMax(qmax, q);
    // order-preserving map of a float to unsigned int for atomicMax
    float f = (float)yf;
    unsigned int u = __float_as_uint(f);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    atomicMax(fmm_max_bits, u);
}

}  // namespace

// ====================================================================== host side
struct gq_mlp {
    gq_ctx *ctx = nullptr;
    dbuf<float> w, m, v, g;
    dbuf<__nv_bfloat16> wb;
    dbuf<float> xmu, xsd, ymu, ysd;   // normalisation (identity until trained)
    int adam_t = 0;
    // work buffers for a batch
    int cap = 0;
    dbuf<float> Xb, Yb, Z[kLayers], A[kLayers], D[kLayers], err;
    dbuf<int> perm;
};

namespace {

void ensure_batch(gq_mlp *M, int B) {
    if (B <= M->cap) return;
    M->Xb.alloc((size_t)B * kNF);
    M->Yb.alloc((size_t)B * 2);
    M->err.alloc((size_t)B * 2);
    for (int l = 0; l < kLayers; ++l) {
        M->Z[l].alloc((size_t)B * kDims[l + 1]);
        M->A[l].alloc((size_t)B * kDims[l + 1]);
        M->D[l].alloc((size_t)B * kDims[l + 1]);
    }
    M->perm.alloc(B);
    M->cap = B;
}

// forward + backward on the batch in Xb / Yb (already normalised); gradient into M->g; returns sum of squares
void fwd_bwd(gq_mlp *M, int B, bool want_err, double *sse) {
    gq_ctx *ctx = M->ctx;
    const float *in = M->Xb.p;
    for (int l = 0; l < kLayers; ++l) {
        int nin = kDims[l], nout = kDims[l + 1];
        GQ_LAUNCH(ctx, k_dense_fwd, gq_blocks((long long)B * nout, kT), kT, 0, B, nin, nout, in,
                  (const float *)M->w.p + woff(l), (const float *)M->w.p + woff(l) + nin * nout, M->Z[l].p, M->A[l].p,
                  l < kLayers - 1 ? 1 : 0);
        in = M->A[l].p;
    }
    GQ_LAUNCH(ctx, k_mse_delta, gq_blocks((long long)B * 2, kT), kT, 0, B, 2, (const float *)M->A[kLayers - 1].p,
              (const float *)M->Yb.p, M->D[kLayers - 1].p, M->err.p);
    for (int l = kLayers - 1; l >= 0; --l) {
        int nin = kDims[l], nout = kDims[l + 1];
        const float *Ain = l == 0 ? (const float *)M->Xb.p : (const float *)M->A[l - 1].p;
        GQ_LAUNCH(ctx, k_dense_grad, gq_blocks((long long)nout * (nin + 1), kT), kT, 0, B, nin, nout,
                  (const float *)M->D[l].p, Ain, M->g.p + woff(l), M->g.p + woff(l) + nin * nout);
        if (l > 0)
            GQ_LAUNCH(ctx, k_dense_bwd, gq_blocks((long long)B * nin, kT), kT, 0, B, nin, nout, (const float *)M->D[l].p,
                      (const float *)M->w.p + woff(l), (const float *)M->Z[l - 1].p, M->D[l - 1].p);
    }
    if (want_err) {
        std::vector<float> e((size_t)B * 2);
        GQ_CUDA(cudaMemcpyAsync(e.data(), M->err.p, sizeof(float) * e.size(), cudaMemcpyDeviceToHost, ctx->stream));
        GQ_CUDA(cudaStreamSynchronize(ctx->stream));
        double s = 0;
        for (float x : e) s += x;
        *sse = s;
    }
}

const float *to_device(gq_ctx *ctx, const float *p, size_t n, dbuf<float> &tmp, bool is_dev) {
    if (is_dev) return p;
    tmp.alloc(n);
    GQ_CUDA(cudaMemcpyAsync(tmp.p, p, sizeof(float) * n, cudaMemcpyDefault, ctx->stream));
    return tmp.p;
}

}  // namespace

int gq_mlp_param_count() { return kNParams; }

gq_mlp *gq_mlp_new(gq_ctx *ctx, uint64_t seed) {
    gq_mlp *M = new gq_mlp;
    M->ctx = ctx;
    std::vector<float> w(kNParams, 0.f);
    std::mt19937_64 rng(seed);
    for (int l = 0; l < kLayers; ++l) {
        int nin = kDims[l], nout = kDims[l + 1];
        std::normal_distribution<float> nd(0.f, sqrtf(2.f / nin));   // He initialisation
        for (int i = 0; i < nin * nout; ++i) w[woff(l) + i] = nd(rng);
    }
    M->w.alloc(kNParams);
    M->m.alloc(kNParams);
    M->v.alloc(kNParams);
    M->g.alloc(kNParams);
    M->wb.alloc(kNParams);
    GQ_CUDA(cudaMemcpyAsync(M->w.p, w.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, ctx->stream));
    GQ_CUDA(cudaMemsetAsync(M->m.p, 0, sizeof(float) * kNParams, ctx->stream));
    GQ_CUDA(cudaMemsetAsync(M->v.p, 0, sizeof(float) * kNParams, ctx->stream));
    std::vector<float> zero(kNF, 0.f), one(kNF, 1.f);
    M->xmu.alloc(kNF); M->xsd.alloc(kNF); M->ymu.alloc(2); M->ysd.alloc(2);
    GQ_CUDA(cudaMemcpyAsync(M->xmu.p, zero.data(), sizeof(float) * kNF, cudaMemcpyHostToDevice, ctx->stream));
    GQ_CUDA(cudaMemcpyAsync(M->xsd.p, one.data(), sizeof(float) * kNF, cudaMemcpyHostToDevice, ctx->stream));
    GQ_CUDA(cudaMemcpyAsync(M->ymu.p, zero.data(), sizeof(float) * 2, cudaMemcpyHostToDevice, ctx->stream));
    GQ_CUDA(cudaMemcpyAsync(M->ysd.p, one.data(), sizeof(float) * 2, cudaMemcpyHostToDevice, ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(ctx->stream));
    return M;
}

void gq_mlp_free(gq_mlp *M) { delete M; }
gq_ctx *gq_mlp_ctx(const gq_mlp *M) { return M->ctx; }

void gq_mlp_weights_impl(gq_mlp *M, float *get, const float *set) {
    if (set) GQ_CUDA(cudaMemcpyAsync(M->w.p, set, sizeof(float) * kNParams, cudaMemcpyDefault, M->ctx->stream));
    if (get) GQ_CUDA(cudaMemcpyAsync(get, M->w.p, sizeof(float) * kNParams, cudaMemcpyDefault, M->ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(M->ctx->stream));
}

// loss = mean squared error of the raw network on (X, Y); grad = d loss / d parameters
void gq_mlp_loss_grad_impl(gq_mlp *M, const float *X, const float *Y, int n, bool dev, float *loss, float *grad) {
    ensure_batch(M, n);
    dbuf<float> tx, ty;
    const float *Xd = to_device(M->ctx, X, (size_t)n * kNF, tx, dev), *Yd = to_device(M->ctx, Y, (size_t)n * 2, ty, dev);
    GQ_CUDA(cudaMemcpyAsync(M->Xb.p, Xd, sizeof(float) * n * kNF, cudaMemcpyDeviceToDevice, M->ctx->stream));
    GQ_CUDA(cudaMemcpyAsync(M->Yb.p, Yd, sizeof(float) * n * 2, cudaMemcpyDeviceToDevice, M->ctx->stream));
    double sse = 0;
    fwd_bwd(M, n, true, &sse);
    if (loss) *loss = (float)(sse / (2.0 * n));
    if (grad) GQ_CUDA(cudaMemcpy(grad, M->g.p, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
}

// Adam on normalised features and labels (statistics of this training set)
double gq_mlp_train_impl(gq_mlp *M, const float *X, const float *Y, int n, bool dev, int epochs, int B, float lr,
                         uint64_t seed) {
    gq_ctx *ctx = M->ctx;
    cudaStream_t st = ctx->stream;
    B = B < n ? B : n;
    ensure_batch(M, B);
    dbuf<float> tx, ty;
    const float *Xd = to_device(ctx, X, (size_t)n * kNF, tx, dev), *Yd = to_device(ctx, Y, (size_t)n * 2, ty, dev);
    // normalisation statistics (host, FP64)
    std::vector<float> hx((size_t)n * kNF), hy((size_t)n * 2);
    GQ_CUDA(cudaMemcpyAsync(hx.data(), Xd, sizeof(float) * hx.size(), cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaMemcpyAsync(hy.data(), Yd, sizeof(float) * hy.size(), cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaStreamSynchronize(st));
    std::vector<float> xmu(kNF), xsd(kNF), ymu(2), ysd(2);
    for (int c = 0; c < kNF + 2; ++c) {
        const std::vector<float> &h = c < kNF ? hx : hy;
        int d = c < kNF ? kNF : 2, cc = c < kNF ? c : c - kNF;
        double s = 0, s2 = 0;
        for (int i = 0; i < n; ++i) { double x = h[(size_t)i * d + cc]; s += x; s2 += x * x; }
        double mu = s / n, sd = sqrt(fmax(s2 / n - mu * mu, 0.0));
        if (sd < 1e-6) sd = 1.0;
        (c < kNF ? xmu[cc] : ymu[cc]) = (float)mu;
        (c < kNF ? xsd[cc] : ysd[cc]) = (float)sd;
    }
    GQ_CUDA(cudaMemcpyAsync(M->xmu.p, xmu.data(), sizeof(float) * kNF, cudaMemcpyHostToDevice, st));
    GQ_CUDA(cudaMemcpyAsync(M->xsd.p, xsd.data(), sizeof(float) * kNF, cudaMemcpyHostToDevice, st));
    GQ_CUDA(cudaMemcpyAsync(M->ymu.p, ymu.data(), sizeof(float) * 2, cudaMemcpyHostToDevice, st));
    GQ_CUDA(cudaMemcpyAsync(M->ysd.p, ysd.data(), sizeof(float) * 2, cudaMemcpyHostToDevice, st));
    dbuf<int> permall;
    permall.alloc(n);
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    std::mt19937_64 rng(seed);
    double last = 0;
    const float b1 = 0.9f, b2 = 0.999f;
    for (int ep = 0; ep < epochs; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        GQ_CUDA(cudaMemcpyAsync(permall.p, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        double sse = 0;
        for (int s0 = 0; s0 + B <= n; s0 += B) {
            GQ_LAUNCH(ctx, k_gather_rows, gq_blocks((long long)B * kNF, kT), kT, 0, B, kNF, (const int *)permall.p + s0,
                      Xd, (const float *)M->xmu.p, (const float *)M->xsd.p, M->Xb.p);
            GQ_LAUNCH(ctx, k_gather_rows, gq_blocks((long long)B * 2, kT), kT, 0, B, 2, (const int *)permall.p + s0, Yd,
                      (const float *)M->ymu.p, (const float *)M->ysd.p, M->Yb.p);
            bool last_batch = ep == epochs - 1;
            double e = 0;
            fwd_bwd(M, B, last_batch, &e);
            sse += e;
            ++M->adam_t;
            float c1 = 1.f - powf(b1, (float)M->adam_t), c2 = 1.f - powf(b2, (float)M->adam_t);
            GQ_LAUNCH(ctx, k_adam, gq_blocks(kNParams, kT), kT, 0, kNParams, M->w.p, (const float *)M->g.p, M->m.p,
                      M->v.p, lr, b1, b2, c1, c2);
        }
        last = sse / (2.0 * (n / B) * B);
    }
    GQ_CUDA(cudaStreamSynchronize(st));
    return last;   // mean squared error of the last epoch, in normalised units
}

void gq_mlp_predict_impl(gq_mlp *M, const float *X, int n, bool xdev, float *Y, bool ydev) {
    gq_ctx *ctx = M->ctx;
    dbuf<float> tx, ty;
    const float *Xd = to_device(ctx, X, (size_t)n * kNF, tx, xdev);
    float *Yd = Y;
    if (!ydev) {
        ty.alloc((size_t)n * 2);
        Yd = ty.p;
    }
    GQ_LAUNCH(ctx, k_to_bf16, gq_blocks(kNParams, kT), kT, 0, kNParams, (const float *)M->w.p, M->wb.p);
    if (n > 0) {
        const int blocks = std::min(gq_blocks(n, 64), 152 * 8);
        GQ_LAUNCH(ctx, k_mlp_infer_mma, blocks, 128, 0, n, Xd, (const __nv_bfloat16 *)M->wb.p,
                  (const float *)M->xmu.p, (const float *)M->xsd.p, (const float *)M->ymu.p, (const float *)M->ysd.p, Yd);
    }
    if (!ydev) GQ_CUDA(cudaMemcpyAsync(Y, Yd, sizeof(float) * n * 2, cudaMemcpyDeviceToHost, ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(ctx->stream));
}

void gq_centre_features_impl(gq_geom *g, float *feat_dev) {
    gq_ctx *ctx = g->ctx;
    dbuf<float> kappa;
    kappa.alloc(g->nbase);
    GQ_LAUNCH(ctx, k_base_curvature, gq_blocks(g->nbase, kT), kT, 0, g->nbase, g->nb, (const double *)g->base_xy,
              (const double *)g->base_n, kappa.p);
    if (g->nc)
        GQ_LAUNCH(ctx, k_centre_features, gq_blocks(g->nc, 128), 128, 0, g->nc, g->nb, g->nu, (const int *)g->ctr_perm,
                  (const int *)g->ctr_owner, (const double2 *)g->sc_xy, (const double *)g->sc_r,
                  (const int *)g->list_off[0], (const int *)g->list_idx[0], (const int *)g->list_off[2],
                  (const int *)g->list_idx[2], (const int *)g->list_off[4], (const int *)g->list_idx[4],
                  (const int *)g->src_beg, (const int *)g->src_end, (const double2 *)g->s_xy, (const int *)g->src_perm,
                  (const double *)g->panel_len, (const float *)kappa.p, feat_dev);
    GQ_CUDA(cudaStreamSynchronize(ctx->stream));
}

// Learned orders: per-centre q = q_ref + ceil((yq + margin - log10(eps/2)) / qbx_slope),
// p_fmm = p_ref + ceil((max yf + margin_fmm - log10(eps/2)) / fmm_slope), capped by the
// bound-driven order (its fallback).
void gq_learned_orders_impl(gq_geom *g, gq_mlp *M, double eps, double margin, double margin_fmm, int q_ref,
                            int p_ref, int q_bound, int p_bound, int *p_out, int *q_out) {
    gq_ctx *ctx = g->ctx;
    dbuf<float> feat, pred;
    feat.alloc((size_t)g->nc * kNF);
    pred.alloc((size_t)g->nc * 2);
    gq_centre_features_impl(g, feat.p);
    gq_mlp_predict_impl(M, feat.p, g->nc, true, pred.p, true);
    dbuf<unsigned int> fbits;
    dbuf<int> qmax;
    fbits.alloc(1);
    qmax.alloc(1);
    GQ_CUDA(cudaMemsetAsync(fbits.p, 0, sizeof(unsigned int), ctx->stream));
    GQ_CUDA(cudaMemsetAsync(qmax.p, 0, sizeof(int), ctx->stream));
    const bool per_centre = q_ref > 0;
    g->q_ctr.alloc(g->nc);
    double log_tol = log10(eps / 2.0);
    const double qbx_slope = 1.26, fmm_slope = 0.5;   // decades per order, measured on starfish curves
    if (g->nc)
        GQ_LAUNCH(ctx, k_learned_q, gq_blocks(g->nc, kT), kT, 0, g->nc, (const int *)g->ctr_perm, (const float *)pred.p,
                  log_tol, margin, per_centre ? q_ref : 1, qbx_slope, q_bound, g->q_ctr.p, fbits.p, qmax.p);
    unsigned int ub = 0;
    int qm = 0;
    GQ_CUDA(cudaMemcpyAsync(&ub, fbits.p, sizeof(ub), cudaMemcpyDeviceToHost, ctx->stream));
    GQ_CUDA(cudaMemcpyAsync(&qm, qmax.p, sizeof(qm), cudaMemcpyDeviceToHost, ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(ctx->stream));
    ub = (ub & 0x80000000u) ? (ub & 0x7fffffffu) : ~ub;
    float yf;
    memcpy(&yf, &ub, sizeof(yf));
    int p = p_ref + (int)ceil((yf + margin_fmm - log_tol) / fmm_slope);
    p = p < 1 ? 1 : (p > p_bound ? p_bound : p);
    g->prm.p_fmm = p;
    if (per_centre) {
        g->prm.p_qbx = qm < 1 ? 1 : qm;
        g->has_qc = true;
    }
    g->have_eval = false;
    *p_out = p;
    *q_out = g->prm.p_qbx;
}

__global__ void k_scatter_orders(int nc, const int *__restrict__ ctr_pos, const int *__restrict__ q_by_id,
                                 int *__restrict__ q_sorted, int *__restrict__ qmax) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int q = q_by_id[c];
    q_sorted[ctr_pos[c]] = q;
    atomicMax(qmax, q);
}

void gq_set_centre_orders_impl(gq_geom *g, const int *q_dev) {
    gq_ctx *ctx = g->ctx;
    g->q_ctr.alloc(g->nc);
    dbuf<int> qmax;
    qmax.alloc(1);
    GQ_CUDA(cudaMemsetAsync(qmax.p, 0, sizeof(int), ctx->stream));
    if (g->nc)
        GQ_LAUNCH(ctx, k_scatter_orders, gq_blocks(g->nc, 256), 256, 0, g->nc, (const int *)g->ctr_pos, q_dev,
                  g->q_ctr.p, qmax.p);
    int qm = 0;
    GQ_CUDA(cudaMemcpyAsync(&qm, qmax.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(ctx->stream));
    g->prm.p_qbx = qm < 1 ? 1 : qm;
    g->has_qc = true;
    g->have_eval = false;
}

