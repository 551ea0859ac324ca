// gq_fmm.cu -- Stages 2-8 of the GIGAQBX Algorithm (Sec. 4.4) and the final
// QBX evaluation (eq. qbx), in complex-variable form (Sec. 3.1).
//
// Complex potential Phi: S mu = -(1/2pi) Re Phi_S with Phi_S(z) = sum q log(z - y),
// q = w mu; D mu = -(1/2pi) Re Phi_D with Phi_D(z) = sum d / (y - z), d = w mu n.
//
// Storage is box-scaled so that translations between same-level boxes do not
// depend on the level:  a box b of half-width rho keeps
//   M_b[k] = a_k / rho^k   (multipole about the box centre, eq. multipole)
//   L_b[m] = beta_m rho^m  (local about the box centre, eq. local)
// and a QBX centre c of radius r keeps Q_c[m] = beta_m r^m (eq. qbx).
// Constant terms of S keep their real part (log|.|): imaginary parts of
// constant terms never feed a real part of any later coefficient or value.
//
// Translations used (y = target centre - source centre):
//   M2M  alpha_m = -a_0 t^m/m + sum_{k<=m} C(m-1,k-1) a_k t^(m-k),  t = -y   (eq. m2m)
//   M2L  beta_0  = a_0 log y + sum_k a_k / y^k
//        beta_m  = (-1)^m y^-m [ -a_0/m + sum_k C(m+k-1,k-1) a_k y^-k ]       (eq. m2l,
//        a_0 term with the sign obtained by expanding log z about y)
//   L2L  beta_m  = sum_{k>=m} C(k,m) b_k y^(k-m)                             (eq. l2l)
// M2L is evaluated in that factored form: scale a_k by y^-k, apply the real
// matrix C(m+k-1,k-1) shared by every pair, scale by (-1)^m y^-m.
#include <math.h>
#include <stdlib.h>

#include <map>
#include <mutex>

#include <memory>

#include "gq_internal.cuh"
#include "gq_dfl.cuh"
#include "gq_math.cuh"

namespace {

constexpr double kInv2Pi = 0.15915494309189533576888376337251;

__device__ __forceinline__ unsigned long long gqtc_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// MIXED: FP32 direct sums from this accuracy up.  Their rounding, measured up
// to 3e-7 relative (D on a single starfish, where the double-layer terms
// cancel most), stays below eps/5 = 1e-6 here; smaller eps use FP32 pairs.
constexpr double kF32TierEps = 5e-6;
constexpr int kBinN = 64;   // binomial table C(n, k), n, k < 64

// C(m+k-1, k-1) for m <= GQ_MAX_PQBX, k <= 32: the real matrix of the factored
// M2L applied at QBX order (List 3 far to centres).  Read with warp-uniform
// indices, so constant-cache broadcasts serve it.
__constant__ double c_pascal[GQ_MAX_PQBX + 1][33];

struct EvalView {
    RootInfo R;
    int P, Q, kernel;
    const int *blev, *bix, *biy, *bparent;
    const int4 *bchild;
    const int *src_beg, *src_end;
    const int *ctr_beg, *ctr_end, *pt_beg, *pt_end;
    const int *sub_src, *sub_tgt;
    const double2 *s_xy;
    const double2 *str;
    const double2 *sc_xy;
    const double *sc_r;
    const double2 *sp_xy;
    const int *loff[6];
    const int *lidx[6];
    const double *binom;   // [kBinN][kBinN]
    const int *qc;         // per-centre QBX order (sorted centres) or nullptr: all use Q
    const double *logt;    // GqLogTable
    const unsigned int *qexp;   // largest biased exponent of the S strengths (k_strengths)
    int nwork_ctr;              // boxes owning centres (batched items)
};

__device__ __forceinline__ double box_rho(const RootInfo &R, int l) { return ldexp(R.H, -l); }
__device__ __forceinline__ double2 box_centre(const RootInfo &R, int l, int ix, int iy) {
    double h = ldexp(R.H, -l);
    return make_double2(R.lo_x + (double)(2 * ix + 1) * h, R.lo_y + (double)(2 * iy + 1) * h);
}

__device__ __forceinline__ double2 shfl2(double2 v, int src, int width) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src, width), __shfl_sync(0xffffffffu, v.y, src, width));
}
__device__ __forceinline__ double2 shfl2_up(double2 v, int d, int width) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d, width), __shfl_up_sync(0xffffffffu, v.y, d, width));
}
// lane g of a group of `width` lanes receives u^g
__device__ __forceinline__ double2 lane_powers(double2 u, int g, int width) {
    double2 v = g == 0 ? make_double2(1.0, 0.0) : u;
    for (int o = 1; o < width; o <<= 1) {
        double2 t = shfl2_up(v, o, width);
        if (g >= o) v = cmul(v, t);
    }
    return v;
}

// ------------------------------------------------------------------ A1: upsample + strengths
__global__ void k_strengths(int nsrc, int nu, int nb, const int *__restrict__ src_perm, const double *__restrict__ interp,
                            const double *__restrict__ dens, const double *__restrict__ s_w,
                            const double2 *__restrict__ s_n, int kernel, double2 *__restrict__ str,
                            unsigned int *__restrict__ qexp) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned int ex = 0;
    if (j < nsrc) {
        int id = src_perm[j];
        int panel = id / nu, jj = id - panel * nu;
        const double *row = interp + (size_t)jj * nb;
        const double *mu_b = dens + (size_t)panel * nb;
        double mu = 0.0;
        for (int i = 0; i < nb; ++i) mu += row[i] * mu_b[i];
        double wm = s_w[j] * mu;
        str[j] = kernel == GQ_D ? cscale(s_n[j], wm) : make_double2(wm, 0.0);
        ex = (unsigned int)(((unsigned long long)__double_as_longlong(wm) >> 52) & 0x7ff);
    }
    // the largest exponent of w mu (qexp cleared before the launch): the direct
    // kernels scale their FP32 copies of the strengths by it
    if (qexp) {
        ex = __reduce_max_sync(0xffffffffu, ex);
        if ((threadIdx.x & 31) == 0 && ex) atomicMax(qexp, ex);
    }
}

// ------------------------------------------------------------------ Stage 2: P2M
// A group of kP2MG lanes per source leaf; the lanes stride over its sources
// and keep all p+1 coefficients in registers (PM >= p, guarded unrolled
// loops); a butterfly inside the group sums them.  S: A_0 = sum q,
// A_k = -(1/k) sum q u^k; D: A_k = -(1/rho) sum d u^(k-1), u = (y - z_b)/rho.
constexpr int kP2MG = 4;

template <int PM>
__global__ void k_p2m(EvalView E, int nwork, const int *__restrict__ work, double2 *__restrict__ M) {
    int wid = (blockIdx.x * blockDim.x + threadIdx.x) / kP2MG, lane = threadIdx.x % kP2MG;
    // whole groups leave together; the shuffles below stay inside a group
    if (wid >= nwork) return;
    int b = work[wid];
    int l = E.blev[b], P = E.P;
    double rho = box_rho(E.R, l), irho = 1.0 / rho;
    double2 zc = box_centre(E.R, l, E.bix[b], E.biy[b]);
    double2 acc[PM + 1];
#pragma unroll
    for (int k = 0; k <= PM; ++k) acc[k] = make_double2(0.0, 0.0);
    for (int s = E.src_beg[b] + lane; s < E.src_end[b]; s += kP2MG) {
        double2 y = E.s_xy[s], st = E.str[s];
        double2 u = make_double2((y.x - zc.x) * irho, (y.y - zc.y) * irho);
        if (E.kernel == GQ_D) {
            double2 t = cscale(st, irho);
            acc[1] = cadd(acc[1], t);
#pragma unroll
            for (int k = 2; k <= PM; ++k)
                if (k <= P) {
                    t = cmul(t, u);
                    acc[k] = cadd(acc[k], t);
                }
        } else {
            acc[0].x += st.x;
            double2 t = make_double2(st.x * u.x, st.x * u.y);
            acc[1] = cadd(acc[1], t);
#pragma unroll
            for (int k = 2; k <= PM; ++k)
                if (k <= P) {
                    t = cmul(t, u);
                    acc[k] = cadd(acc[k], t);
                }
        }
    }
    const unsigned gmask = ((1u << kP2MG) - 1u) << (threadIdx.x & 31 & ~(kP2MG - 1));
#pragma unroll
    for (int k = 0; k <= PM; ++k)
        if (k <= P)
            for (int o = kP2MG / 2; o > 0; o >>= 1)
                acc[k] = cadd(acc[k], make_double2(__shfl_xor_sync(gmask, acc[k].x, o), __shfl_xor_sync(gmask, acc[k].y, o)));
#pragma unroll
    for (int k = 0; k <= PM; ++k)
        if (k <= P && k % kP2MG == lane) {
            double2 v = acc[k];
            if (k >= 1) v = E.kernel == GQ_D ? make_double2(-v.x, -v.y) : cscale(v, -1.0 / k);
            M[(size_t)b * (P + 1) + k] = v;
        }
}

// M2M and L2L with the translation matrices tabulated: with box-scaled
// coefficients the child offsets (z_c - z_p)/rho_p are the four numbers
// eta_q = (+-1 +- i)/2 at every level, so each translation is a fixed lower
// (M2M) or upper (L2L) triangular complex matrix per quadrant q:
//   M2M  T_q[m][0] = -eta_q^m / m,  T_q[m][k] = C(m-1, k-1) 2^-k eta_q^(m-k)  (1 <= k <= m)
//   L2L  U_q[m][k] = 2^-m C(k, m) eta_q^(k-m)                                 (k >= m)
// applied as complex multiply-adds (four FMAs each).
constexpr int kTN = GQ_MAX_PFMM + 1;

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}

// M2M and L2L with the quadrant matrices, one level per launch: a block takes
// 128 / (P + 1) boxes, thread (box, order m).  The block first stages the
// boxes' children's multipoles (M2M) or parents' local expansions (L2L) in
// shared memory with one round of independent loads; each output is then
// summed over k in ascending order exactly as one thread per order would.
__device__ __forceinline__ int tab_boxes(int P1) { return 128 / P1; }
__device__ __forceinline__ int child_of(int4 c4, int q) { return q == 0 ? c4.x : q == 1 ? c4.y : q == 2 ? c4.z : c4.w; }

// The boxes are entries [lstart, lend) of `boxes` (one level's non-leaf boxes
// with sources below), or box numbers [lstart, lend) when boxes is null.
__global__ void __launch_bounds__(128) k_m2m_t(EvalView E, const int *__restrict__ boxes, int lstart, int lend,
                                               const double2 *__restrict__ T, double2 *__restrict__ M) {
    __shared__ double2 sA[4 * 128];
    const int P1 = E.P + 1, bpb = tab_boxes(P1);
    const int i0 = lstart + blockIdx.x * bpb;
    for (int i = threadIdx.x; i < bpb * 4 * P1; i += blockDim.x) {
        const int bb = i / (4 * P1), rest = i - bb * 4 * P1, q = rest / P1, k = rest - q * P1;
        const int ib = i0 + bb;
        double2 v = make_double2(0.0, 0.0);
        if (ib < lend) {
            const int c = child_of(E.bchild[boxes ? boxes[ib] : ib], q);
            if (c >= 0) v = M[(size_t)c * P1 + k];
        }
        sA[i] = v;
    }
    __syncthreads();
    const int bl = threadIdx.x / P1, m = threadIdx.x - bl * P1, ib = i0 + bl;
    if (bl >= bpb || ib >= lend) return;
    const int b = boxes ? boxes[ib] : ib;
    int4 c4 = E.bchild[b];
    int ch[4] = {c4.x, c4.y, c4.z, c4.w};
    if (ch[0] < 0 && ch[1] < 0 && ch[2] < 0 && ch[3] < 0) return;  // leaf
    if (E.sub_src[b] == 0) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int q = 0; q < 4; ++q) {
        int c = ch[q];
        if (c < 0 || E.sub_src[c] == 0) continue;
        const double2 *A = sA + (bl * 4 + q) * P1;
        if (m == 0) {
            acc = cadd(acc, A[0]);
            continue;
        }
        const double2 *Tq = T + ((size_t)q * kTN + m) * kTN;
        double2 sacc = cscale(__ldg(&Tq[0]), A[0].x);
        for (int k = 1; k <= m; ++k) sacc = cfma(__ldg(&Tq[k]), A[k], sacc);
        acc = cadd(acc, sacc);
    }
    M[(size_t)b * P1 + m] = acc;
}

__global__ void __launch_bounds__(128) k_l2l_t(EvalView E, int lstart, int lend, const double2 *__restrict__ U,
                                               double2 *__restrict__ L) {
    __shared__ double2 sB[128];
    const int P1 = E.P + 1, bpb = tab_boxes(P1);
    const int c0 = lstart + blockIdx.x * bpb;
    for (int i = threadIdx.x; i < bpb * P1; i += blockDim.x) {
        const int bb = i / P1, k = i - bb * P1, c = c0 + bb;
        double2 v = make_double2(0.0, 0.0);
        if (c < lend) v = L[(size_t)E.bparent[c] * P1 + k];   // levels >= 1: the parent exists
        sB[i] = v;
    }
    __syncthreads();
    const int bl = threadIdx.x / P1, m = threadIdx.x - bl * P1, c = c0 + bl;
    if (bl >= bpb || c >= lend || E.sub_tgt[c] == 0) return;
    int q = (E.bix[c] & 1) | ((E.biy[c] & 1) << 1);
    const double2 *B = sB + bl * P1;
    const double2 *Uq = U + ((size_t)q * kTN + m) * kTN;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = m; k <= E.P; ++k) acc = cfma(__ldg(&Uq[k]), B[k], acc);
    double2 *dst = L + (size_t)c * P1 + m;
    *dst = cadd(*dst, acc);
}

// ------------------------------------------------------------------ Stage 4: M2L over List 2
// Groups of G lanes (G = 16 when p_fmm < 16, two boxes per warp); lane g is
// the order index.  dtab[off][k] = delta^-k for the 11x11 same-level offsets,
// delta = (z_b - z_d)/rho in units of the half-width.
template <int G>
__global__ void k_m2l(EvalView E, int nwork, const int *__restrict__ work, const double2 *__restrict__ M,
                      const double2 *__restrict__ dtab, const double *__restrict__ logtab, double2 *__restrict__ L) {
    extern __shared__ double pasc[];   // [P+1][P+1]: C(m+k-1, k-1)
    int P = E.P, P1 = P + 1;
    for (int i = threadIdx.x; i < P1 * P1; i += blockDim.x) {
        int m = i / P1, k = i % P1;
        pasc[i] = k >= 1 ? E.binom[(m + k - 1) * kBinN + (k - 1)] : 0.0;
    }
    __syncthreads();
    int lane = threadIdx.x & 31, g = lane % G;
    long long grp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    bool act = grp < nwork;
    int b = act ? work[grp] : 0;
    int beg = act ? E.loff[1][b] : 0, end = act ? E.loff[1][b + 1] : 0;
    int n = end - beg, nmax = n;
    for (int o = G; o < 32; o <<= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    int l = E.blev[b], bx = E.bix[b], by = E.biy[b];
    double logrho = log(box_rho(E.R, l));
    const double ig = g >= 1 ? 1.0 / g : 0.0;   // 1/g, once per lane
    double2 acc = make_double2(0.0, 0.0);
    const double *prow = pasc + (g <= P ? g : 0) * P1;
    for (int i = 0; i < nmax; ++i) {
        bool valid = i < n;
        int d = valid ? E.lidx[1][beg + i] : b;
        int off = valid ? (by - E.biy[d] + 5) * 11 + (bx - E.bix[d] + 5) : 0;
        double2 A = (valid && g <= P) ? M[(size_t)d * P1 + g] : make_double2(0.0, 0.0);
        double2 tk = dtab[off * 32 + g];                       // delta^-g
        double2 At = g >= 1 ? cmul(A, tk) : make_double2(0.0, 0.0);
        double A0 = __shfl_sync(0xffffffffu, A.x, 0, G);
        double2 Gm = make_double2(0.0, 0.0);
        for (int k = 1; k <= P; ++k) {
            double2 a = shfl2(At, k, G);
            double c = prow[k];
            Gm.x += c * a.x;
            Gm.y += c * a.y;
        }
        if (!valid) continue;
        if (g == 0) {
            acc.x += A0 * (logrho + logtab[off]) + Gm.x;
            acc.y += Gm.y;
        } else if (g <= P) {
            double2 t = make_double2(Gm.x - A0 * ig, Gm.y);
            double2 s = (g & 1) ? make_double2(-tk.x, -tk.y) : tk;
            acc = cfma(s, t, acc);
        }
    }
    if (act && g <= P) {
        double2 *dst = L + (size_t)b * P1 + g;
        *dst = cadd(*dst, acc);
    }
}

// ------------------------------------------------------------------ Stage 6b: P2L over List 4 far
// Warp per box; a group of G lanes per source, lane m of the group = order m.
// With p_fmm < 16 (G = 16) the two half-warps take alternate sources of each
// List 4 far box, so the per-source reciprocal and powers are formed once per
// 16 orders instead of once per 32 lanes, and add their sums at the end.
__global__ void k_p2l(EvalView E, int nwork, const int *__restrict__ work, double2 *__restrict__ L) {
    int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (wid >= nwork) return;
    const int G = E.P < 16 ? 16 : 32, NS = 32 / G;
    const int m = lane & (G - 1), h = lane / G;
    int b = work[wid];
    int beg = E.loff[5][b], end = E.loff[5][b + 1];
    if (beg == end) return;
    int l = E.blev[b];
    double rho = box_rho(E.R, l);
    double2 zc = box_centre(E.R, l, E.bix[b], E.biy[b]);
    const double im = m >= 1 ? 1.0 / m : 0.0;   // 1/m, once per lane
    double2 acc = make_double2(0.0, 0.0);
    for (int i = beg; i < end; ++i) {
        int d = E.lidx[5][i];
        const int s0 = E.src_beg[d], s1 = E.src_end[d];
        for (int sb = s0; sb < s1; sb += NS) {   // the same trip count in every lane
            const int s = sb + h;
            const bool valid = s < s1;
            double2 y = E.s_xy[valid ? s : sb], st = valid ? E.str[s] : make_double2(0.0, 0.0);
            double2 w = make_double2(y.x - zc.x, y.y - zc.y);
            double n2 = w.x * w.x + w.y * w.y, inv = gq_rcp(n2);
            double2 winv = make_double2(w.x * inv, -w.y * inv);      // 1/w
            double2 um = lane_powers(cscale(winv, rho), m, G);       // (rho/w)^m
            if (E.kernel == GQ_D) {
                acc = cfma(cmul(st, winv), um, acc);
            } else if (m == 0) {
                acc.x += st.x * gq_log_half(n2, E.logt);
            } else {
                acc = csub(acc, cscale(um, st.x * im));
            }
        }
    }
    if (G == 16) {
        acc.x += __shfl_down_sync(0xffffffffu, acc.x, 16);
        acc.y += __shfl_down_sync(0xffffffffu, acc.y, 16);
    }
    if (h == 0 && m <= E.P) {
        double2 *dst = L + (size_t)b * (E.P + 1) + m;
        *dst = cadd(*dst, acc);
    }
}

// ------------------------------------------------------------------ Stages 3, 5a, 6a: direct near field
// One block per target box; the box's List 1, 3 close and 4 close source
// ranges are flattened into shared memory; each warp takes one target and its
// lanes stride over the flattened sources.
constexpr int kNearThreads = 128;
constexpr int kNearRanges = 256;

struct NearRanges {
    int beg[kNearRanges];
    int pre[kNearRanges + 1];
    int n;
};

__device__ int block_excl_scan_128(int v, int *wsum) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    int off = 0;
    for (int i = 0; i < w; ++i) off += wsum[i];
    __syncthreads();
    return off + x - v;
}

// load entries [e0, e0 + kNearRanges) of the concatenated lists U, WC, XC of box b
__device__ void load_ranges(const EvalView &E, int b, int e0, int ne, NearRanges &R, int *wsum) {
    int n0 = E.loff[0][b + 1] - E.loff[0][b], n2 = E.loff[2][b + 1] - E.loff[2][b];
    int cnt = min(kNearRanges, ne - e0);
    int lens[2] = {0, 0};
    for (int r = 0; r < 2; ++r) {
        int i = threadIdx.x * 2 + r;
        if (i < cnt) {
            int e = e0 + i, d;
            if (e < n0) d = E.lidx[0][E.loff[0][b] + e];
            else if (e < n0 + n2) d = E.lidx[2][E.loff[2][b] + e - n0];
            else d = E.lidx[4][E.loff[4][b] + e - n0 - n2];
            R.beg[i] = E.src_beg[d];
            lens[r] = E.src_end[d] - E.src_beg[d];
        }
    }
    int pre = block_excl_scan_128(lens[0] + lens[1], wsum);
    if (threadIdx.x * 2 < kNearRanges) R.pre[threadIdx.x * 2] = pre;
    if (threadIdx.x * 2 + 1 < kNearRanges) R.pre[threadIdx.x * 2 + 1] = pre + lens[0];
    if (threadIdx.x == kNearThreads - 1) R.pre[kNearRanges] = pre + lens[0] + lens[1];
    if (threadIdx.x == 0) R.n = cnt;
    __syncthreads();
}

// Warp reduce-scatter of NV values per lane: at each of the five butterfly
// steps a lane keeps one half of its values, sends the other half to its
// partner and adds what it receives, so a warp spends about NV adds instead of
// 5 NV.  Afterwards lane L holds the warp sums of the original entries
// base .. base + cnt - 1 in v[0 .. cnt) (cnt may be 0; for NV <= 32 it is 0 or 1).
template <int N, int O, class V, class Add, class Shfl>
__device__ __forceinline__ void rs_step(V *v, int lane, V zero, Add add, Shfl shfl, int &base, int &cnt) {
    constexpr int H = (N + 1) / 2;
    const bool up = (lane & O) != 0;
#pragma unroll
    for (int i = 0; i < H; ++i) {
        V x = v[i], y = (i + H < N) ? v[i + H < N ? i + H : 0] : zero;
        V send = up ? x : y, keep = up ? y : x;
        v[i] = add(keep, shfl(send, O));
    }
    if (up) {
        base += H;
        cnt -= H;
    } else if (cnt > H) {
        cnt = H;
    }
}

template <int NV, class V, class Add, class Shfl>
__device__ __forceinline__ void warp_reduce_scatter(V (&v)[NV], V zero, int lane, Add add, Shfl shfl, int &base,
                                                    int &cnt) {
    constexpr int H1 = (NV + 1) / 2, H2 = (H1 + 1) / 2, H3 = (H2 + 1) / 2, H4 = (H3 + 1) / 2;
    base = 0;
    cnt = NV;
    rs_step<NV, 16>(v, lane, zero, add, shfl, base, cnt);
    rs_step<H1, 8>(v, lane, zero, add, shfl, base, cnt);
    rs_step<H2, 4>(v, lane, zero, add, shfl, base, cnt);
    rs_step<H3, 2>(v, lane, zero, add, shfl, base, cnt);
    rs_step<H4, 1>(v, lane, zero, add, shfl, base, cnt);
    if (cnt < 0) cnt = 0;
}

// QBX coefficients at centres: S: Q_0 = sum q log|w|, Q_m = -(1/m) sum q (r/w)^m;
// D: Q_m = sum (d/w) (r/w)^m, with w = y - c.  One warp per centre, lanes
// stride over the sources; the coefficients are summed by a reduce-scatter.
template <int QQ, int KERNEL>
__global__ void __launch_bounds__(kNearThreads) k_near_centres(EvalView E, int nwork, const int *__restrict__ work,
                                                                double2 *__restrict__ Qout) {
    __shared__ NearRanges R;
    __shared__ int wsum[kNearThreads / 32];
    __shared__ double lt[kGqLogN];
    for (int i = threadIdx.x; i < kGqLogN; i += kNearThreads) lt[i] = E.logt[i];
    // FP32 strengths are rebased to the largest one: q = qf * 2^(qe - 1023)
    const int qe = KERNEL == GQ_D ? 1023 : (int)*E.qexp;
    const double qscale = gq_pow2_biased(qe);
    int b = work[blockIdx.x];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ne = (E.loff[0][b + 1] - E.loff[0][b]) + (E.loff[2][b + 1] - E.loff[2][b]) + (E.loff[4][b + 1] - E.loff[4][b]);
    int cb = E.ctr_beg[b], ce = E.ctr_end[b];
    bool single = ne <= kNearRanges;
    if (single) load_ranges(E, b, 0, ne, R, wsum);
    for (int c0 = cb; c0 < ce; c0 += kNearThreads / 32) {
        int c = c0 + w;
        bool valid = c < ce;
        double2 cz = valid ? E.sc_xy[c] : make_double2(0.0, 0.0);
        double rc = valid ? E.sc_r[c] : 1.0;
        const int qc = (valid && E.qc) ? E.qc[c] : QQ;
        double2 acc[QQ + 1];
#pragma unroll
        for (int m = 0; m <= QQ; ++m) acc[m] = make_double2(0.0, 0.0);
        float acc0f = 0.0f;   // S: FP32 tails of the logarithms, strengths rebased by qe
        for (int e0 = 0; e0 < ne; e0 += kNearRanges) {
            if (!single) {
                __syncthreads();
                load_ranges(E, b, e0, ne, R, wsum);
            }
            int T = R.pre[R.n];
            if (valid) {
                int r = 0;
                for (int v = lane; v < T; v += 32) {
                    while (R.pre[r + 1] <= v) ++r;
                    int s = R.beg[r] + (v - R.pre[r]);
                    double2 y = E.s_xy[s], st = E.str[s];
                    double wx = y.x - cz.x, wy = y.y - cz.y;
                    double n2 = wx * wx + wy * wy;
                    double inv = gq_rcp(n2);
                    double2 winv = make_double2(wx * inv, -wy * inv);    // 1/w (D only)
                    double2 u;                                            // r/w
                    if (KERNEL == GQ_D) {
                        u = make_double2(rc * winv.x, rc * winv.y);
                    } else {
                        double ir = rc * inv;
                        u = make_double2(wx * ir, -wy * ir);
                    }
                    if (KERNEL == GQ_D) {
                        double2 t = cmul(st, winv);
                        acc[0] = cadd(acc[0], t);
#pragma unroll
                        for (int m = 1; m < QQ; ++m) {
                            if (m > qc) break;
                            t = cmul(t, u);
                            acc[m] = cadd(acc[m], t);
                        }
                        // last term: a multiply-add into the sum (t is not needed again)
                        if (qc >= QQ) acc[QQ] = cfma(t, u, acc[QQ]);
                    } else {
                        float tail;
                        acc[0].x = fma(st.x, gq_log_half_split(n2, lt, tail), acc[0].x);
                        acc0f = fmaf(gq_f32_rebased(st.x, qe), tail, acc0f);
                        double2 t = make_double2(st.x * u.x, st.x * u.y);
                        acc[1] = cadd(acc[1], t);
#pragma unroll
                        for (int m = 2; m < QQ; ++m) {
                            if (m > qc) break;
                            t = cmul(t, u);
                            acc[m] = cadd(acc[m], t);
                        }
                        if (QQ >= 2 && qc >= QQ) acc[QQ] = cfma(t, u, acc[QQ]);
                    }
                }
            }
        }
        if (KERNEL != GQ_D) acc[0].x = fma((double)acc0f, qscale, acc[0].x);
        double vals[2 * (QQ + 1)];
#pragma unroll
        for (int m = 0; m <= QQ; ++m) {
            vals[2 * m] = acc[m].x;
            vals[2 * m + 1] = acc[m].y;
        }
        int base, cnt;
        warp_reduce_scatter(vals, 0.0, lane, [](double a, double x) { return a + x; },
                            [](double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }, base, cnt);
        if (valid) {
            double *dst = reinterpret_cast<double *>(Qout + (size_t)c * (QQ + 1));
#pragma unroll
            for (int j = 0; j < (2 * (QQ + 1) + 31) / 32; ++j)
                if (j < cnt) {
                    int i = base + j, m = i >> 1;
                    double x = vals[j];
                    if (KERNEL != GQ_D && m >= 1) x *= -1.0 / m;
                    dst[i] = x;
                }
        }
    }
}

// potential at point targets: S: sum q log|t - y| (coincident sources skipped), D: Re sum d/(y - t)
// Body for target box b (a block of kNearThreads); lt holds the log table
// (S) in shared memory, loaded by the caller.
template <int KERNEL>
__device__ void near_points_box(const EvalView &E, int b, const double2 *__restrict__ str, double *__restrict__ pot,
                                NearRanges &R, int *wsum, const double *lt) {
    const int qe = KERNEL == GQ_D ? 1023 : (int)*E.qexp;
    const double qscale = gq_pow2_biased(qe);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ne = (E.loff[0][b + 1] - E.loff[0][b]) + (E.loff[2][b + 1] - E.loff[2][b]) + (E.loff[4][b + 1] - E.loff[4][b]);
    int tb = E.pt_beg[b], te = E.pt_end[b];
    bool single = ne <= kNearRanges;
    if (single) load_ranges(E, b, 0, ne, R, wsum);
    for (int t0 = tb; t0 < te; t0 += kNearThreads / 32) {
        int t = t0 + w;
        bool valid = t < te;
        double2 tz = valid ? E.sp_xy[t] : make_double2(0.0, 0.0);
        double acc = 0.0;
        float accf = 0.0f;
        for (int e0 = 0; e0 < ne; e0 += kNearRanges) {
            if (!single) {
                __syncthreads();
                load_ranges(E, b, e0, ne, R, wsum);
            }
            int T = R.pre[R.n];
            if (valid) {
                int r = 0;
                for (int v = lane; v < T; v += 32) {
                    while (R.pre[r + 1] <= v) ++r;
                    int s = R.beg[r] + (v - R.pre[r]);
                    double2 y = E.s_xy[s], st = str[s];
                    double wx = y.x - tz.x, wy = y.y - tz.y;
                    double n2 = wx * wx + wy * wy;
                    if (KERNEL == GQ_D) {
                        if (n2 == 0.0) continue;   // coincident source skipped
                        acc += (st.x * wx + st.y * wy) * gq_rcp(n2);
                    } else {                       // a coincident source gives log term 0
                        float tail;
                        acc = fma(st.x, gq_log_half_split(n2, lt, tail), acc);
                        accf = fmaf(gq_f32_rebased(st.x, qe), tail, accf);
                    }
                }
            }
        }
        if (KERNEL != GQ_D) acc = fma((double)accf, qscale, acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (valid && lane == 0) pot[t] = acc;
    }
}

template <int KERNEL>
__global__ void __launch_bounds__(kNearThreads) k_near_points(EvalView E, int nwork, const int *__restrict__ work,
                                                               double *__restrict__ pot) {
    __shared__ NearRanges R;
    __shared__ int wsum[kNearThreads / 32];
    __shared__ double lt[kGqLogN];
    for (int i = threadIdx.x; i < kGqLogN; i += kNearThreads) lt[i] = E.logt[i];
    near_points_box<KERNEL>(E, work[blockIdx.x], E.str, pot, R, wsum, lt);
}

// ------------------------------------------------------------------ Stage 5b: List 3 far
// M2QBXL, one thread per centre (centres of a box share their List 3 far
// boxes, so a warp reads the same multipoles).  Per far box d, with y = c - z_d,
// v = rho_d / y, s = r / y and At_k = A_k v^k:
//   Q_0 += A_0 log|y| + sum_k At_k
//   Q_m += (-1)^m s^m (sum_k C(m+k-1,k-1) At_k - A_0/m),   1 <= m <= q.
// The QBX order is a template parameter and the loops run k outer, m inner,
// so that At_k = A_k v^k is used as soon as it is formed (no array of p+1
// terms) and G_m = sum_k C(m+k-1, k-1) At_k accumulates in q+1 registers;
// (-r/y)^m carries the sign (-1)^m.
template <int PM, int QQ>
__global__ void __launch_bounds__(128) k_w_centres_q(EvalView E, int nc, const int *__restrict__ ctr_box_of,
                                                     const double2 *__restrict__ M, double2 *__restrict__ Qout) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int b = ctr_box_of[c];
    int beg = E.loff[3][b], end = E.loff[3][b + 1];
    if (beg == end) return;
    const int P = E.P, P1 = P + 1;
    double2 cz = E.sc_xy[c];
    double rc = E.sc_r[c];
    double2 acc[QQ + 1];
#pragma unroll
    for (int m = 0; m <= QQ; ++m) acc[m] = make_double2(0.0, 0.0);
    for (int i = beg; i < end; ++i) {
        int d = E.lidx[3][i];
        int l = E.blev[d];
        double rho = box_rho(E.R, l);
        double2 zd = box_centre(E.R, l, E.bix[d], E.biy[d]);
        double2 y = make_double2(cz.x - zd.x, cz.y - zd.y);
        double n2 = y.x * y.x + y.y * y.y, inv = gq_rcp(n2);
        double2 yinv = make_double2(y.x * inv, -y.y * inv);
        double2 v = cscale(yinv, rho), msv = cscale(yinv, -rc);
        const double2 *A = M + (size_t)d * P1;
        double A0 = A[0].x;
        double2 G[QQ + 1];
#pragma unroll
        for (int m = 0; m <= QQ; ++m) G[m] = make_double2(0.0, 0.0);
        double2 vk = v;
#pragma unroll
        for (int k = 1; k <= PM; ++k) {
            if (k <= P) {
                double2 at = cmul(A[k], vk);
                G[0] = cadd(G[0], at);
#pragma unroll
                for (int m = 1; m <= QQ; ++m) {
                    double cc = c_pascal[m][k];
                    G[m].x = fma(cc, at.x, G[m].x);
                    G[m].y = fma(cc, at.y, G[m].y);
                }
                vk = cmul(vk, v);
            }
        }
        acc[0].x += A0 * gq_log_half(n2, E.logt) + G[0].x;
        acc[0].y += G[0].y;
        double2 sm = make_double2(1.0, 0.0);
#pragma unroll
        for (int m = 1; m <= QQ; ++m) {
            sm = cmul(sm, msv);   // (-r/y)^m
            G[m].x -= A0 * (1.0 / m);
            acc[m] = cfma(sm, G[m], acc[m]);
        }
    }
    double2 *dst = Qout + (size_t)c * (QQ + 1);
#pragma unroll
    for (int m = 0; m <= QQ; ++m) dst[m] = cadd(dst[m], acc[m]);
}

template <int PM>
void launch_w_centres_q(gq_ctx *ctx, const EvalView &E, int nc, const int *owner, const double2 *M, double2 *Q) {
    switch (E.Q) {
#define GQ_CASE(v) case v: GQ_LAUNCH(ctx, (k_w_centres_q<PM, v>), gq_blocks(nc, 128), 128, 0, E, nc, owner, M, Q); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

void dispatch_w_centres_q(gq_ctx *ctx, const EvalView &E, int nc, const int *owner, const double2 *M, double2 *Q) {
    if (E.P <= 8) launch_w_centres_q<8>(ctx, E, nc, owner, M, Q);
    else if (E.P <= 16) launch_w_centres_q<16>(ctx, E, nc, owner, M, Q);
    else launch_w_centres_q<GQ_MAX_PFMM>(ctx, E, nc, owner, M, Q);
}

// M2P, one thread per point target: Phi += A_0 log|z| + sum_k A_k (rho/z)^k,
// z = t - z_d, by Horner's rule
__global__ void k_w_points(EvalView E, int npt, const int *__restrict__ pt_owner, const double2 *__restrict__ M,
                           double *__restrict__ pot) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npt) return;
    int b = pt_owner[t];
    int beg = E.loff[3][b], end = E.loff[3][b + 1];
    if (beg == end) return;
    int P = E.P, P1 = P + 1;
    double2 tz = E.sp_xy[t];
    double acc = 0.0;
    for (int i = beg; i < end; ++i) {
        int d = E.lidx[3][i];
        int l = E.blev[d];
        double rho = box_rho(E.R, l);
        double2 zd = box_centre(E.R, l, E.bix[d], E.biy[d]);
        double2 z = make_double2(tz.x - zd.x, tz.y - zd.y);
        double n2 = z.x * z.x + z.y * z.y, ri = rho * gq_rcp(n2);
        double2 v = make_double2(z.x * ri, -z.y * ri);
        const double2 *A = M + (size_t)d * P1;
        double2 h = A[P];
        for (int k = P - 1; k >= 1; --k) h = cfma(h, v, A[k]);
        h = cmul(h, v);
        acc += h.x + A[0].x * gq_log_half(n2, E.logt);
    }
    pot[t] += acc;
}

// ------------------------------------------------------------------ Stage 8
// L2QBXL by a Taylor shift, one thread per centre: with the box-scaled local
// expansion sum_k L_k z^k, z = (x - z_b)/rho, and eta = (c - z_b)/rho, the
// coefficients of the shifted polynomial in zeta = z - eta come from q+1
// passes of repeated synthetic division (pass i: b_k += eta b_{k+1} for
// k = p-1 .. i, after which b_i is final), i.e. sum_k C(k, m) L_k eta^(k-m)
// without binomials; Q_m += b_m (r/rho)^m.  rho is a power of two, so the
// scalings by 1/rho are exact.
template <int PM, int QQ>
__global__ void __launch_bounds__(128) k_l2qbxl_t(EvalView E, int nc, const int *__restrict__ ctr_box_of,
                                                  const double2 *__restrict__ L, double2 *__restrict__ Qout) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int P = E.P;
    int b = ctr_box_of[c];
    int l = E.blev[b];
    double irho = ldexp(1.0 / E.R.H, l);
    double2 zb = box_centre(E.R, l, E.bix[b], E.biy[b]);
    double2 cz = E.sc_xy[c];
    double2 eta = make_double2((cz.x - zb.x) * irho, (cz.y - zb.y) * irho);
    const double2 *B = L + (size_t)b * (P + 1);
    double2 bk[PM + 1];
#pragma unroll
    for (int k = 0; k <= PM; ++k) bk[k] = k <= P ? B[k] : make_double2(0.0, 0.0);
#pragma unroll
    for (int i = 0; i <= QQ; ++i)
#pragma unroll
        for (int k = PM - 1; k >= i; --k)
            if (k < P) bk[k] = cfma(eta, bk[k + 1], bk[k]);
    double s = E.sc_r[c] * irho, sm = 1.0;
    double2 *dst = Qout + (size_t)c * (QQ + 1);
#pragma unroll
    for (int m = 0; m <= QQ; ++m) {
        if (m <= P) dst[m] = cadd(dst[m], cscale(bk[m], sm));
        sm *= s;
    }
}

template <int PM>
void launch_l2qbxl_t(gq_ctx *ctx, const EvalView &E, int nc, const int *owner, const double2 *L, double2 *Q) {
    switch (E.Q) {
#define GQ_CASE(v) case v: GQ_LAUNCH(ctx, (k_l2qbxl_t<PM, v>), gq_blocks(nc, 128), 128, 0, E, nc, owner, L, Q); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

void dispatch_l2qbxl_t(gq_ctx *ctx, const EvalView &E, int nc, const int *owner, const double2 *L, double2 *Q) {
    if (E.P <= 8) launch_l2qbxl_t<8>(ctx, E, nc, owner, L, Q);
    else if (E.P <= 16) launch_l2qbxl_t<16>(ctx, E, nc, owner, L, Q);
    else launch_l2qbxl_t<GQ_MAX_PFMM>(ctx, E, nc, owner, L, Q);
}

// L2P: one thread per point target, Horner in the box-scaled variable
__global__ void k_l2p(EvalView E, int npt, const int *__restrict__ pt_owner, const double2 *__restrict__ L,
                      double *__restrict__ pot) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npt) return;
    int b = pt_owner[t];
    int l = E.blev[b];
    double rho = box_rho(E.R, l);
    double2 zb = box_centre(E.R, l, E.bix[b], E.biy[b]);
    double2 tz = E.sp_xy[t];
    double2 zeta = make_double2((tz.x - zb.x) / rho, (tz.y - zb.y) / rho);
    const double2 *B = L + (size_t)b * (E.P + 1);
    double2 h = B[E.P];
    for (int k = E.P - 1; k >= 0; --k) h = cfma(h, zeta, B[k]);
    pot[t] += h.x;
}

// final values at the targets (eq. qbx; two-sided targets average both centres)
__device__ __forceinline__ void final_target(int t, int kernel, int Q, const int *__restrict__ qcs,
                                             const int *__restrict__ kind, const int *__restrict__ ctr,
                                             const int *__restrict__ ctr_pos, const int *__restrict__ tgt_ptpos,
                                             const double *__restrict__ tgt_xy, const int *__restrict__ tgt_on,
                                             const double *__restrict__ base_n, const double2 *__restrict__ sc_xy,
                                             const double *__restrict__ sc_r, const double2 *__restrict__ Qc,
                                             const double2 *__restrict__ Qc2, const double *__restrict__ pot,
                                             const double *__restrict__ pot2, double *__restrict__ out) {
    int k = kind[t];
    if (k == 0) {
        int j = tgt_ptpos[t];
        out[t] = kernel == GQ_SP ? nan("") : -kInv2Pi * (pot[j] + (pot2 ? pot2[j] : 0.0));
        return;
    }
    double2 tz = make_double2(tgt_xy[2 * t], tgt_xy[2 * t + 1]);
    int nside = k == 2 ? 2 : 1;
    double sum = 0.0;
    for (int sd = 0; sd < nside; ++sd) {
        int cp = ctr_pos[ctr[t] + sd];
        double2 cz = sc_xy[cp];
        double r = sc_r[cp];
        double2 zeta = make_double2((tz.x - cz.x) / r, (tz.y - cz.y) / r);
        const double2 *B = Qc + (size_t)cp * (Q + 1);
        const double2 *B2 = Qc2 ? Qc2 + (size_t)cp * (Q + 1) : nullptr;
        const int q = qcs ? qcs[cp] : Q;
        auto coef = [&](int m) { return B2 ? cadd(B[m], B2[m]) : B[m]; };
        if (kernel == GQ_SP) {
            int node = tgt_on[t];
            if (node < 0) { sum = nan(""); break; }
            double2 h = cscale(coef(q), (double)q);
            for (int m = q - 1; m >= 1; --m) h = cfma(h, zeta, cscale(coef(m), (double)m));
            double2 n = make_double2(base_n[2 * node], base_n[2 * node + 1]);
            sum += -kInv2Pi * cmul(n, h).x / r;
        } else {
            double2 h = coef(q);
            for (int m = q - 1; m >= 0; --m) h = cfma(h, zeta, coef(m));
            sum += -kInv2Pi * h.x;
        }
    }
    out[t] = sum / nside;
}

__global__ void k_final(int nt, int kernel, int Q, const int *__restrict__ qcs, const int *__restrict__ kind,
                        const int *__restrict__ ctr,
                        const int *__restrict__ ctr_pos, const int *__restrict__ tgt_ptpos,
                        const double *__restrict__ tgt_xy, const int *__restrict__ tgt_on,
                        const double *__restrict__ base_n, const double2 *__restrict__ sc_xy,
                        const double *__restrict__ sc_r, const double2 *__restrict__ Qc,
                        const double2 *__restrict__ Qc2, const double *__restrict__ pot, const double *__restrict__ pot2,
                        double *__restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    final_target(t, kernel, Q, qcs, kind, ctr, ctr_pos, tgt_ptpos, tgt_xy, tgt_on, base_n, sc_xy, sc_r, Qc, Qc2, pot,
                 pot2, out);
}

// the operator at the base nodes (gq_apply): base node i is evaluated from its
// two centres 2i, 2i+1 and averaged, as an on-surface target of gq_eval would
// be (eq. qbx; principal value), and identity * mu_i is added
__global__ void k_final_base(int nbase, int kernel, int Q, const int *__restrict__ qcs, const int *__restrict__ ctr_pos,
                             const double *__restrict__ base_xy, const double *__restrict__ base_n,
                             const double2 *__restrict__ sc_xy, const double *__restrict__ sc_r,
                             const double2 *__restrict__ Qc, const double2 *__restrict__ Qc2, double identity,
                             const double *__restrict__ mu, double *__restrict__ out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nbase) return;
    double2 tz = make_double2(base_xy[2 * t], base_xy[2 * t + 1]);
    double sum = 0.0;
    for (int sd = 0; sd < 2; ++sd) {
        int cp = ctr_pos[2 * t + sd];
        double2 cz = sc_xy[cp];
        double r = sc_r[cp];
        double2 zeta = make_double2((tz.x - cz.x) / r, (tz.y - cz.y) / r);
        const double2 *B = Qc + (size_t)cp * (Q + 1);
        const double2 *B2 = Qc2 ? Qc2 + (size_t)cp * (Q + 1) : nullptr;
        const int q = qcs ? qcs[cp] : Q;
        auto coef = [&](int m) { return B2 ? cadd(B[m], B2[m]) : B[m]; };
        if (kernel == GQ_SP) {
            double2 h = cscale(coef(q), (double)q);
            for (int m = q - 1; m >= 1; --m) h = cfma(h, zeta, cscale(coef(m), (double)m));
            double2 n = make_double2(base_n[2 * t], base_n[2 * t + 1]);
            sum += -kInv2Pi * cmul(n, h).x / r;
        } else {
            double2 h = coef(q);
            for (int m = q - 1; m >= 0; --m) h = cfma(h, zeta, coef(m));
            sum += -kInv2Pi * h.x;
        }
    }
    out[t] = identity * mu[t] + sum / 2;
}

__global__ void k_export_qbx(int nc, int Q, const int *__restrict__ ctr_perm, const double *__restrict__ sc_r,
                             const double2 *__restrict__ Qc, const double2 *__restrict__ Qc2, double2 *__restrict__ out) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int c = (int)(t / (Q + 1)), m = (int)(t % (Q + 1));
    if (c >= nc) return;
    double r = sc_r[c], s = 1.0;
    for (int i = 0; i < m; ++i) s /= r;
    double2 v = Qc[(size_t)c * (Q + 1) + m];
    if (Qc2) v = cadd(v, Qc2[(size_t)c * (Q + 1) + m]);
    out[(size_t)ctr_perm[c] * (Q + 1) + m] = cscale(v, s);
}

// ------------------------------------------------------------------ mixed precision: FP32 direct sums
// Coordinates are stored relative to box centres so that the FP32 differences
// y - c do not cancel: a source is kept relative to its leaf centre, a centre
// or point target relative to its own box centre, and the offset between the
// two box centres is formed in FP64 once per source range.
struct MixedView {
    const float2 *s_rel, *str, *c_rel, *p_rel, *M;
    const float *c_r;
};

__device__ __forceinline__ float2 fcmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void k_rel_coords(int n, const double2 *__restrict__ xy, const int *__restrict__ owner, EvalView E,
                             float2 *__restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int b = owner[j];
    double2 z = box_centre(E.R, E.blev[b], E.bix[b], E.biy[b]);
    out[j] = make_float2((float)(xy[j].x - z.x), (float)(xy[j].y - z.y));
}

__global__ void k_to_float2(long long n, const double2 *__restrict__ in, float2 *__restrict__ out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = make_float2((float)in[j].x, (float)in[j].y);
}

__global__ void k_to_float(int n, const double *__restrict__ in, float *__restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[j] = (float)in[j];
}

struct NearRangesF {
    int beg[kNearRanges];
    int pre[kNearRanges + 1];
    float2 off[kNearRanges];   // centre of the source leaf minus centre of the target box
    int n;
};

__device__ void load_ranges_f(const EvalView &E, int b, double2 zb, int e0, int ne, NearRangesF &R, int *wsum) {
    int n0 = E.loff[0][b + 1] - E.loff[0][b], n2 = E.loff[2][b + 1] - E.loff[2][b];
    int cnt = min(kNearRanges, ne - e0);
    int lens[2] = {0, 0};
    for (int r = 0; r < 2; ++r) {
        int i = threadIdx.x * 2 + r;
        if (i < cnt) {
            int e = e0 + i, d;
            if (e < n0) d = E.lidx[0][E.loff[0][b] + e];
            else if (e < n0 + n2) d = E.lidx[2][E.loff[2][b] + e - n0];
            else d = E.lidx[4][E.loff[4][b] + e - n0 - n2];
            R.beg[i] = E.src_beg[d];
            lens[r] = E.src_end[d] - E.src_beg[d];
            double2 zd = box_centre(E.R, E.blev[d], E.bix[d], E.biy[d]);
            R.off[i] = make_float2((float)(zd.x - zb.x), (float)(zd.y - zb.y));
        }
    }
    int pre = block_excl_scan_128(lens[0] + lens[1], wsum);
    if (threadIdx.x * 2 < kNearRanges) R.pre[threadIdx.x * 2] = pre;
    if (threadIdx.x * 2 + 1 < kNearRanges) R.pre[threadIdx.x * 2 + 1] = pre + lens[0];
    if (threadIdx.x == kNearThreads - 1) R.pre[kNearRanges] = pre + lens[0] + lens[1];
    if (threadIdx.x == 0) R.n = cnt;
    __syncthreads();
}

template <int QQ, int KERNEL>
__global__ void __launch_bounds__(kNearThreads) k_near_centres_f32(EvalView E, MixedView X, int nwork,
                                                                    const int *__restrict__ work,
                                                                    double2 *__restrict__ Qout) {
    __shared__ NearRangesF R;
    __shared__ int wsum[kNearThreads / 32];
    int b = work[blockIdx.x];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ne = (E.loff[0][b + 1] - E.loff[0][b]) + (E.loff[2][b + 1] - E.loff[2][b]) + (E.loff[4][b + 1] - E.loff[4][b]);
    int cb = E.ctr_beg[b], ce = E.ctr_end[b];
    double2 zb = box_centre(E.R, E.blev[b], E.bix[b], E.biy[b]);
    bool single = ne <= kNearRanges;
    if (single) load_ranges_f(E, b, zb, 0, ne, R, wsum);
    for (int c0 = cb; c0 < ce; c0 += kNearThreads / 32) {
        int c = c0 + w;
        bool valid = c < ce;
        float2 cz = valid ? X.c_rel[c] : make_float2(0.f, 0.f);
        float rc = valid ? X.c_r[c] : 1.f;
        float rc2 = rc * rc;
        const int qc = (valid && E.qc) ? E.qc[c] : QQ;
        double2 czd = valid ? E.sc_xy[c] : make_double2(0.0, 0.0);
        double rcd = valid ? E.sc_r[c] : 1.0;
        float2 acc[QQ + 1];
        double2 acc64[QQ + 1];   // sources inside the expansion disk (|r/w| > 1): FP64
        bool used64 = false;
#pragma unroll
        for (int m = 0; m <= QQ; ++m) {
            acc[m] = make_float2(0.f, 0.f);
            acc64[m] = make_double2(0.0, 0.0);
        }
        for (int e0 = 0; e0 < ne; e0 += kNearRanges) {
            if (!single) {
                __syncthreads();
                load_ranges_f(E, b, zb, e0, ne, R, wsum);
            }
            int T = R.pre[R.n];
            if (valid) {
                int r = 0;
                for (int v = lane; v < T; v += 32) {
                    while (R.pre[r + 1] <= v) ++r;
                    int s = R.beg[r] + (v - R.pre[r]);
                    float2 y = X.s_rel[s], o = R.off[r], st = X.str[s];
                    float wx = (y.x + o.x) - cz.x, wy = (y.y + o.y) - cz.y;
                    float n2 = wx * wx + wy * wy;
                    if (n2 < rc2) {
                        used64 = true;
                        // rounding would be amplified by |r/w|^m: take this pair in FP64
                        double2 yd = E.s_xy[s], sd = E.str[s];
                        double dx = yd.x - czd.x, dy = yd.y - czd.y;
                        double d2 = dx * dx + dy * dy, dinv = 1.0 / d2;
                        double2 wi = make_double2(dx * dinv, -dy * dinv);
                        double2 uu = make_double2(rcd * wi.x, rcd * wi.y);
                        if (KERNEL == GQ_D) {
                            double2 t = cmul(sd, wi);
                            acc64[0] = cadd(acc64[0], t);
#pragma unroll
                            for (int m = 1; m <= QQ; ++m) {
                                t = cmul(t, uu);
                                acc64[m] = cadd(acc64[m], t);
                            }
                        } else {
                            acc64[0].x += sd.x * (0.5 * log(d2));
                            double2 t = make_double2(sd.x * uu.x, sd.x * uu.y);
                            acc64[1] = cadd(acc64[1], t);
#pragma unroll
                            for (int m = 2; m <= QQ; ++m) {
                                t = cmul(t, uu);
                                acc64[m] = cadd(acc64[m], t);
                            }
                        }
                        continue;
                    }
                    float inv = __fdividef(1.0f, n2);
                    float2 winv = make_float2(wx * inv, -wy * inv);
                    float2 u = make_float2(rc * winv.x, rc * winv.y);
                    if (KERNEL == GQ_D) {
                        float2 t = fcmul(st, winv);
                        acc[0].x += t.x;
                        acc[0].y += t.y;
#pragma unroll
                        for (int m = 1; m <= QQ; ++m) {
                            if (m > qc) break;
                            t = fcmul(t, u);
                            acc[m].x += t.x;
                            acc[m].y += t.y;
                        }
                    } else {
                        acc[0].x += st.x * 0.5f * logf(n2);
                        float2 t = make_float2(st.x * u.x, st.x * u.y);
                        acc[1].x += t.x;
                        acc[1].y += t.y;
#pragma unroll
                        for (int m = 2; m <= QQ; ++m) {
                            if (m > qc) break;
                            t = fcmul(t, u);
                            acc[m].x += t.x;
                            acc[m].y += t.y;
                        }
                    }
                }
            }
        }
        // warp sums by reduce-scatter in FP32 pairs (exact from the FP32 lane sums);
        // the FP64 part only where a lane of the warp used it
        const bool any64 = __any_sync(0xffffffffu, used64);
        dfl vals[2 * (QQ + 1)];
#pragma unroll
        for (int m = 0; m <= QQ; ++m) {
            vals[2 * m] = dfl{acc[m].x, 0.f};
            vals[2 * m + 1] = dfl{acc[m].y, 0.f};
        }
        int base, cnt;
        warp_reduce_scatter(vals, dfl{0.f, 0.f}, lane, [](dfl a, dfl x) { return dfl_add(a, x); },
                            [](dfl x, int o) {
                                return dfl{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
                            },
                            base, cnt);
        constexpr int NJ = (2 * (QQ + 1) + 31) / 32;
        double v64[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) v64[j] = 0.0;
        if (any64) {
            double d64[2 * (QQ + 1)];
#pragma unroll
            for (int m = 0; m <= QQ; ++m) {
                d64[2 * m] = acc64[m].x;
                d64[2 * m + 1] = acc64[m].y;
            }
            int b2, c2;
            warp_reduce_scatter(d64, 0.0, lane, [](double a, double x) { return a + x; },
                                [](double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }, b2, c2);
#pragma unroll
            for (int j = 0; j < NJ; ++j) v64[j] = d64[j];
        }
        if (valid) {
            double *dst = reinterpret_cast<double *>(Qout + (size_t)c * (QQ + 1));
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j < cnt) {
                    int i = base + j, m = i >> 1;
                    double x = dfl_to_double(vals[j]) + v64[j];
                    if (KERNEL != GQ_D && m >= 1) x *= -1.0 / m;
                    dst[i] = x;
                }
        }
    }
}

template <int KERNEL>
__global__ void __launch_bounds__(kNearThreads) k_near_points_f32(EvalView E, MixedView X, int nwork,
                                                                   const int *__restrict__ work,
                                                                   double *__restrict__ pot) {
    __shared__ NearRangesF R;
    __shared__ int wsum[kNearThreads / 32];
    int b = work[blockIdx.x];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ne = (E.loff[0][b + 1] - E.loff[0][b]) + (E.loff[2][b + 1] - E.loff[2][b]) + (E.loff[4][b + 1] - E.loff[4][b]);
    int tb = E.pt_beg[b], te = E.pt_end[b];
    double2 zb = box_centre(E.R, E.blev[b], E.bix[b], E.biy[b]);
    bool single = ne <= kNearRanges;
    if (single) load_ranges_f(E, b, zb, 0, ne, R, wsum);
    for (int t0 = tb; t0 < te; t0 += kNearThreads / 32) {
        int t = t0 + w;
        bool valid = t < te;
        float2 tz = valid ? X.p_rel[t] : make_float2(0.f, 0.f);
        float acc = 0.f;
        for (int e0 = 0; e0 < ne; e0 += kNearRanges) {
            if (!single) {
                __syncthreads();
                load_ranges_f(E, b, zb, e0, ne, R, wsum);
            }
            int T = R.pre[R.n];
            if (valid) {
                int r = 0;
                for (int v = lane; v < T; v += 32) {
                    while (R.pre[r + 1] <= v) ++r;
                    int s = R.beg[r] + (v - R.pre[r]);
                    float2 y = X.s_rel[s], o = R.off[r], st = X.str[s];
                    float wx = (y.x + o.x) - tz.x, wy = (y.y + o.y) - tz.y;
                    float n2 = wx * wx + wy * wy;
                    if (n2 == 0.f) continue;
                    if (KERNEL == GQ_D) acc += (st.x * wx + st.y * wy) * __fdividef(1.0f, n2);
                    else acc += st.x * 0.5f * logf(n2);
                }
            }
        }
        double dacc = (double)acc;
        for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
        if (valid && lane == 0) pot[t] = dacc;
    }
}

// M2P in FP32: thread per point target, Horner in v = rho / (t - z_d)
__global__ void k_w_points_f32(EvalView E, MixedView X, int npt, const int *__restrict__ pt_owner,
                               double *__restrict__ pot) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npt) return;
    int b = pt_owner[t];
    int beg = E.loff[3][b], end = E.loff[3][b + 1];
    if (beg == end) return;
    int P = E.P, P1 = P + 1;
    double2 tz = E.sp_xy[t];
    float acc = 0.f;
    for (int i = beg; i < end; ++i) {
        int d = E.lidx[3][i];
        int l = E.blev[d];
        double2 zd = box_centre(E.R, l, E.bix[d], E.biy[d]);
        float zx = (float)(tz.x - zd.x), zy = (float)(tz.y - zd.y);
        float rho = (float)box_rho(E.R, l);
        float n2 = zx * zx + zy * zy, inv = __fdividef(1.0f, n2);
        float2 v = make_float2(rho * zx * inv, -rho * zy * inv);
        const float2 *A = X.M + (size_t)d * P1;
        float2 h = A[P];
        for (int k = P - 1; k >= 1; --k) {
            h = fcmul(h, v);
            h.x += A[k].x;
            h.y += A[k].y;
        }
        h = fcmul(h, v);
        acc += h.x + A[0].x * 0.5f * logf(n2);
    }
    pot[t] += (double)acc;
}

// ------------------------------------------------------------------ split precision: double-FP32 pairs
// Coordinates, radii and strengths as FP32 pairs (gq_dfl.cuh), relative to box
// centres as in the FP32 tier: a source relative to its leaf centre, a centre
// relative to its own box centre; the offset between two box centres is a
// short dyadic number, exact in FP32.  Per centre, (r.hi, r.lo, 1/r^2 hi, lo).
struct SplitView {
    const float4 *s_rel, *str, *c_rel, *c_r, *p_rel;
    const float4 *M;     // multipoles, (re.hi, re.lo, im.hi, im.lo) per coefficient
    const float4 *lvl;   // per level l: [2l] = (rho, 1/rho), [2l+1] = (log rho, 1/rho^2)
    const float *logt;   // GqDflLogTable
    float H;             // root half-width (a power of two)
    float fb;            // sources with |w|^2 < fb r^2 are taken in FP64 (fb >= 1)
    bool near_pt;        // point-target pairs closer than 1/8 of the box half-width in FP64
};

__device__ __forceinline__ dflc dflc_add(dflc a, dflc b) { return dflc{dfl_add(a.re, b.re), dfl_add(a.im, b.im)}; }
__device__ __forceinline__ dflc dflc_sub(dflc a, dflc b) {
    return dflc{dfl_add(a.re, dfl_neg(b.re)), dfl_add(a.im, dfl_neg(b.im))};
}
__device__ __forceinline__ dflc dflc_scale(dflc a, dfl s) { return dflc{dfl_mul(a.re, s), dfl_mul(a.im, s)}; }
__device__ __forceinline__ dflc dflc_ld(float4 v) { return dflc{dfl{v.x, v.y}, dfl{v.z, v.w}}; }

// Centre of box b minus centre of box d, exact in FP32: both centres are odd
// multiples of their half-widths H 2^-l, which FP32 holds exactly for l <= 23,
// and the difference of two neighbouring boxes has few significant bits.
__device__ __forceinline__ float2 box_offset_f(float H, int lb, int ixb, int iyb, int ld, int ixd, int iyd) {
    float hb = ldexpf(H, -lb), hd = ldexpf(H, -ld);
    return make_float2(__fsub_rn(__fmul_rn((float)(2 * ixb + 1), hb), __fmul_rn((float)(2 * ixd + 1), hd)),
                       __fsub_rn(__fmul_rn((float)(2 * iyb + 1), hb), __fmul_rn((float)(2 * iyd + 1), hd)));
}

__global__ void k_level_split(int nlev, double H, float4 *__restrict__ out) {
    int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlev) return;
    double rho = ldexp(H, -l);
    dfl a = dfl_from_double(rho), b = dfl_from_double(1.0 / rho), c = dfl_from_double(log(rho)),
        d = dfl_from_double(1.0 / (rho * rho));
    out[2 * l] = make_float4(a.hi, a.lo, b.hi, b.lo);
    out[2 * l + 1] = make_float4(c.hi, c.lo, d.hi, d.lo);
}

__global__ void k_rel_coords_split(int n, const double2 *__restrict__ xy, const int *__restrict__ owner, EvalView E,
                                   float4 *__restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int b = owner[j];
    double2 z = box_centre(E.R, E.blev[b], E.bix[b], E.biy[b]);
    dfl x = dfl_from_double(xy[j].x - z.x), y = dfl_from_double(xy[j].y - z.y);
    out[j] = make_float4(x.hi, x.lo, y.hi, y.lo);
}

__global__ void k_radius_split(int n, const double *__restrict__ r, float4 *__restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    dfl a = dfl_from_double(r[j]), b = dfl_from_double(1.0 / (r[j] * r[j]));
    out[j] = make_float4(a.hi, a.lo, b.hi, b.lo);
}

__global__ void k_to_dfl4(long long n, const double2 *__restrict__ in, float4 *__restrict__ out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    dfl a = dfl_from_double(in[j].x), b = dfl_from_double(in[j].y);
    out[j] = make_float4(a.hi, a.lo, b.hi, b.lo);
}

// Direct interactions to centres with every per-pair step in FP32 pairs: the
// difference w = y - c, 1/|w|^2, 1/w, r/w, the power recurrence and the lane
// sums of the coefficients.  For S the logarithm is split as
// log|w| = log r + (1/2) log(|w|^2 / r^2), so that the pair logarithm sees
// arguments >= 1 of modest size and log r enters once per centre in FP64.
// Sources inside the expansion disk (|r/w| > 1) would amplify the rounding by
// |r/w|^m and are taken in FP64, as in the FP32 tier.
template <int QQ, int KERNEL>
__global__ void __launch_bounds__(kNearThreads) k_near_centres_split(EvalView E, SplitView X, int nwork,
                                                                      const int *__restrict__ work,
                                                                      double2 *__restrict__ Qout) {
    __shared__ NearRangesF R;
    __shared__ int wsum[kNearThreads / 32];
    __shared__ float lt[KERNEL == GQ_D ? 1 : 384];
    __shared__ double lt64[KERNEL == GQ_D ? 1 : kGqLogN];
    if (KERNEL != GQ_D) {
        for (int i = threadIdx.x; i < 384; i += kNearThreads) lt[i] = X.logt[i];
        for (int i = threadIdx.x; i < kGqLogN; i += kNearThreads) lt64[i] = E.logt[i];
    }
    int b = work[blockIdx.x];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ne = (E.loff[0][b + 1] - E.loff[0][b]) + (E.loff[2][b + 1] - E.loff[2][b]) + (E.loff[4][b + 1] - E.loff[4][b]);
    int cb = E.ctr_beg[b], ce = E.ctr_end[b];
    double2 zb = box_centre(E.R, E.blev[b], E.bix[b], E.biy[b]);
    bool single = ne <= kNearRanges;
    if (single) load_ranges_f(E, b, zb, 0, ne, R, wsum);
    for (int c0 = cb; c0 < ce; c0 += kNearThreads / 32) {
        int c = c0 + w;
        bool valid = c < ce;
        float4 c4 = valid ? X.c_rel[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 r4 = valid ? X.c_r[c] : make_float4(1.f, 0.f, 1.f, 0.f);
        dfl rc{r4.x, r4.y}, irc2{r4.z, r4.w};
        float rc2 = r4.x * r4.x;
        const int qc = (valid && E.qc) ? E.qc[c] : QQ;
        double2 czd = valid ? E.sc_xy[c] : make_double2(0.0, 0.0);
        double rcd = valid ? E.sc_r[c] : 1.0;
        dflc acc[QQ + 1];
        double2 acc64[QQ + 1];   // sources inside the expansion disk: FP64
#pragma unroll
        for (int m = 0; m <= QQ; ++m) {
            acc[m] = dflc{dfl{0.f, 0.f}, dfl{0.f, 0.f}};
            acc64[m] = make_double2(0.0, 0.0);
        }
        dfl acc_log{0.f, 0.f}, acc_str{0.f, 0.f};   // S: sum of st log(|w|^2/r^2), sum of st
        bool used64 = false;
        for (int e0 = 0; e0 < ne; e0 += kNearRanges) {
            if (!single) {
                __syncthreads();
                load_ranges_f(E, b, zb, e0, ne, R, wsum);
            }
            int T = R.pre[R.n];
            if (valid) {
                int r = 0, rcur = -1;
                dfl ex{0.f, 0.f}, ey{0.f, 0.f};   // source-box offset minus the centre
                for (int v = lane; v < T; v += 32) {
                    while (R.pre[r + 1] <= v) ++r;
                    if (r != rcur) {
                        float2 o = R.off[r];
                        ex = dfl_add_f(dfl{-c4.x, -c4.y}, o.x);
                        ey = dfl_add_f(dfl{-c4.z, -c4.w}, o.y);
                        rcur = r;
                    }
                    int s = R.beg[r] + (v - R.pre[r]);
                    float4 y4 = X.s_rel[s];
                    dfl wx = dfl_add(dfl{y4.x, y4.y}, ex), wy = dfl_add(dfl{y4.z, y4.w}, ey);
                    dfl n2 = dfl_add(dfl_sqr(wx), dfl_sqr(wy));
                    if (n2.hi < rc2 * X.fb) {
                        used64 = true;
                        double2 yd = E.s_xy[s], sd = E.str[s];
                        double dx = yd.x - czd.x, dy = yd.y - czd.y;
                        double d2 = dx * dx + dy * dy, dinv = 1.0 / d2;
                        double2 wi = make_double2(dx * dinv, -dy * dinv);
                        double2 uu = make_double2(rcd * wi.x, rcd * wi.y);
                        if (KERNEL == GQ_D) {
                            double2 t = cmul(sd, wi);
                            acc64[0] = cadd(acc64[0], t);
#pragma unroll
                            for (int m = 1; m <= QQ; ++m) {
                                t = cmul(t, uu);
                                acc64[m] = cadd(acc64[m], t);
                            }
                        } else {
                            acc64[0].x += sd.x * gq_log_half(d2, lt64);
                            double2 t = make_double2(sd.x * uu.x, sd.x * uu.y);
                            acc64[1] = cadd(acc64[1], t);
#pragma unroll
                            for (int m = 2; m <= QQ; ++m) {
                                t = cmul(t, uu);
                                acc64[m] = cadd(acc64[m], t);
                            }
                        }
                        continue;
                    }
                    float4 s4 = X.str[s];
                    dfl inv = dfl_rcp(n2);
                    dflc winv{dfl_mul(wx, inv), dfl_neg(dfl_mul(wy, inv))};
                    dflc u{dfl_mul(rc, winv.re), dfl_mul(rc, winv.im)};
                    dflc t;
                    if (KERNEL == GQ_D) {
                        t = dflc_mul(dflc{dfl{s4.x, s4.y}, dfl{s4.z, s4.w}}, winv);
                        dflc_acc(acc[0], t);
#pragma unroll
                        for (int m = 1; m <= QQ; ++m) {
                            if (m > qc) break;
                            t = dflc_mul(t, u);
                            dflc_acc(acc[m], t);
                        }
                    } else {
                        dfl st{s4.x, s4.y};
                        dfl lg = dfl_log(dfl_mul(n2, irc2), lt, lt + 128, lt + 256);
                        dfl_acc(acc_log, dfl_mul(st, lg));
                        dfl_acc(acc_str, st);
                        t = dflc{dfl_mul(st, u.re), dfl_mul(st, u.im)};
                        dflc_acc(acc[1], t);
#pragma unroll
                        for (int m = 2; m <= QQ; ++m) {
                            if (m > qc) break;
                            t = dflc_mul(t, u);
                            dflc_acc(acc[m], t);
                        }
                    }
                }
            }
        }
        // warp sums by reduce-scatter: pairs in the FP32 pipe, the FP64 part only
        // where a lane of the warp used it.  For S the constant term is folded
        // first: Q_0 = (1/2) sum st log(|w|^2/r^2) + log r sum st.
        const bool any64 = __any_sync(0xffffffffu, used64);
        if (KERNEL != GQ_D) {
            dfl lrc = dfl_log(dfl_sqr(rc), lt, lt + 128, lt + 256);   // log r^2
            acc[0].re = dfl_add(dfl_mul_f(dfl_two_sum(acc_log.hi, acc_log.lo), 0.5f),
                                dfl_mul(dfl_two_sum(acc_str.hi, acc_str.lo), dfl{0.5f * lrc.hi, 0.5f * lrc.lo}));
        }
        dfl vals[2 * (QQ + 1)];
#pragma unroll
        for (int m = 0; m <= QQ; ++m) {
            vals[2 * m] = dfl_two_sum(acc[m].re.hi, acc[m].re.lo);
            vals[2 * m + 1] = dfl_two_sum(acc[m].im.hi, acc[m].im.lo);
        }
        int base, cnt;
        warp_reduce_scatter(vals, dfl{0.f, 0.f}, lane, [](dfl a, dfl x) { return dfl_add(a, x); },
                            [](dfl x, int o) {
                                return dfl{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
                            },
                            base, cnt);
        constexpr int NJ = (2 * (QQ + 1) + 31) / 32;
        double v64[NJ];
#pragma unroll
        for (int j = 0; j < NJ; ++j) v64[j] = 0.0;
        if (any64) {
            double d64[2 * (QQ + 1)];
#pragma unroll
            for (int m = 0; m <= QQ; ++m) {
                d64[2 * m] = acc64[m].x;
                d64[2 * m + 1] = acc64[m].y;
            }
            int b2, c2;
            warp_reduce_scatter(d64, 0.0, lane, [](double a, double x) { return a + x; },
                                [](double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }, b2, c2);
#pragma unroll
            for (int j = 0; j < NJ; ++j) v64[j] = d64[j];
        }
        if (valid) {
            double *dst = reinterpret_cast<double *>(Qout + (size_t)c * (QQ + 1));
#pragma unroll
            for (int j = 0; j < NJ; ++j)
                if (j < cnt) {
                    int i = base + j, m = i >> 1;
                    double x = dfl_to_double(vals[j]) + v64[j];
                    if (KERNEL != GQ_D && m >= 1) x *= -1.0 / m;
                    dst[i] = x;
                }
        }
    }
}

// Potential at point targets from List 1 sources, every pair step in FP32
// pairs; pairs closer than 2^-50 fall back to FP64.
template <int KERNEL>
__global__ void __launch_bounds__(kNearThreads) k_near_points_split(EvalView E, SplitView X, int nwork,
                                                                     const int *__restrict__ work,
                                                                     double *__restrict__ pot) {
    __shared__ NearRangesF R;
    __shared__ int wsum[kNearThreads / 32];
    __shared__ float lt[KERNEL == GQ_D ? 1 : 384];
    if (KERNEL != GQ_D)
        for (int i = threadIdx.x; i < 384; i += kNearThreads) lt[i] = X.logt[i];
    int b = work[blockIdx.x];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ne = (E.loff[0][b + 1] - E.loff[0][b]) + (E.loff[2][b + 1] - E.loff[2][b]) + (E.loff[4][b + 1] - E.loff[4][b]);
    int tb = E.pt_beg[b], te = E.pt_end[b];
    double2 zb = box_centre(E.R, E.blev[b], E.bix[b], E.biy[b]);
    // below eps = 1e-10, pairs closer than 1/8 of the box half-width go to FP64: a
    // target that close to the curve sums large terms that cancel
    const float hb = ldexpf(X.H, -E.blev[b]) * 0.125f;
    const float near2 = X.near_pt ? hb * hb : 0x1p-100f;
    bool single = ne <= kNearRanges;
    if (single) load_ranges_f(E, b, zb, 0, ne, R, wsum);
    for (int t0 = tb; t0 < te; t0 += kNearThreads / 32) {
        int t = t0 + w;
        bool valid = t < te;
        float4 t4 = valid ? X.p_rel[t] : make_float4(0.f, 0.f, 0.f, 0.f);
        dfl acc{0.f, 0.f};
        double acc64 = 0.0;
        for (int e0 = 0; e0 < ne; e0 += kNearRanges) {
            if (!single) {
                __syncthreads();
                load_ranges_f(E, b, zb, e0, ne, R, wsum);
            }
            int T = R.pre[R.n];
            if (valid) {
                int r = 0, rcur = -1;
                dfl ex{0.f, 0.f}, ey{0.f, 0.f};
                for (int v = lane; v < T; v += 32) {
                    while (R.pre[r + 1] <= v) ++r;
                    if (r != rcur) {
                        float2 o = R.off[r];
                        ex = dfl_add_f(dfl{-t4.x, -t4.y}, o.x);
                        ey = dfl_add_f(dfl{-t4.z, -t4.w}, o.y);
                        rcur = r;
                    }
                    int s = R.beg[r] + (v - R.pre[r]);
                    float4 y4 = X.s_rel[s];
                    dfl wx = dfl_add(dfl{y4.x, y4.y}, ex), wy = dfl_add(dfl{y4.z, y4.w}, ey);
                    dfl n2 = dfl_add(dfl_sqr(wx), dfl_sqr(wy));
                    if (n2.hi < near2) {
                        double2 yd = E.s_xy[s], td = E.sp_xy[t], sd = E.str[s];
                        double dx = yd.x - td.x, dy = yd.y - td.y, d2 = dx * dx + dy * dy;
                        if (d2 == 0.0) continue;
                        if (KERNEL == GQ_D) acc64 += (sd.x * dx + sd.y * dy) / d2;
                        else acc64 += sd.x * (0.5 * log(d2));
                        continue;
                    }
                    float4 s4 = X.str[s];
                    if (KERNEL == GQ_D) {
                        dfl dot = dfl_dot2(s4.x, s4.y, wx.hi, wx.lo, s4.z, s4.w, wy.hi, wy.lo);
                        dfl_acc(acc, dfl_mul(dot, dfl_rcp(n2)));
                    } else {
                        dfl lg = dfl_log(n2, lt, lt + 128, lt + 256);
                        dfl_acc(acc, dfl_mul(dfl{s4.x, s4.y}, lg));
                    }
                }
            }
        }
        double dacc = (KERNEL == GQ_D ? 1.0 : 0.5) * dfl_to_double(acc) + acc64;
        for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
        if (valid && lane == 0) pot[t] = dacc;
    }
}

// M2P in FP32 pairs, one thread per point target, Horner in v = rho / (t - z_d);
// A_0 log|t - z_d| = A_0 (log rho + (1/2) log(|t - z_d|^2 / rho^2)).
__global__ void k_w_points_split(EvalView E, SplitView X, int npt, const int *__restrict__ pt_owner,
                                 double *__restrict__ pot) {
    __shared__ float lt[384];
    for (int i = threadIdx.x; i < 384; i += blockDim.x) lt[i] = X.logt[i];
    __syncthreads();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npt) return;
    int b = pt_owner[t];
    int beg = E.loff[3][b], end = E.loff[3][b + 1];
    if (beg == end) return;
    int P = E.P, P1 = P + 1;
    int lb = E.blev[b], ixb = E.bix[b], iyb = E.biy[b];
    float4 t4 = X.p_rel[t];
    dfl acc{0.f, 0.f};
    for (int i = beg; i < end; ++i) {
        int d = E.lidx[3][i];
        int l = E.blev[d];
        float2 off = box_offset_f(X.H, lb, ixb, iyb, l, E.bix[d], E.biy[d]);
        dfl zx = dfl_add_f(dfl{t4.x, t4.y}, off.x), zy = dfl_add_f(dfl{t4.z, t4.w}, off.y);
        dfl n2 = dfl_add(dfl_sqr(zx), dfl_sqr(zy));
        dfl inv = dfl_rcp(n2);
        float4 la = X.lvl[2 * l], lb4 = X.lvl[2 * l + 1];
        dfl rho{la.x, la.y};
        dflc v{dfl_mul(rho, dfl_mul(zx, inv)), dfl_neg(dfl_mul(rho, dfl_mul(zy, inv)))};
        const float4 *A = X.M + (size_t)d * P1;
        dflc h = dflc_ld(A[P]);
        for (int k = P - 1; k >= 1; --k) h = dflc_add(dflc_mul(h, v), dflc_ld(A[k]));
        h = dflc_mul(h, v);
        dfl lg = dfl_log(dfl_mul(n2, dfl{lb4.z, lb4.w}), lt, lt + 128, lt + 256);
        dfl lz = dfl_add(dfl{0.5f * lg.hi, 0.5f * lg.lo}, dfl{lb4.x, lb4.y});
        float4 a0 = A[0];
        dfl_acc(acc, h.re);
        dfl_acc(acc, dfl_mul(dfl{a0.x, a0.y}, lz));
    }
    pot[t] += dfl_to_double(acc);
}

// M2QBXL in FP32 pairs, one thread per centre.  With y = c - z_d, v = rho/y,
// omega = (z - c)/y and At_k = A_k v^k, the local expansion of
// sum_k At_k (1 + omega)^-k is built by Horner's rule in (1 + omega)^-1 on
// a series truncated after omega^q: from k = K down to 1, add At_k to the
// constant term, then divide the series by (1 + omega), which is the
// recurrence S_m <- S_m - S_{m-1}.  The coefficient of omega^m equals
// (-1)^m sum_k C(m+k-1, k-1) At_k, the same sum as the FP64 kernel forms with
// the binomial table, and Q_m += (r/y)^m (S_m - (-1)^m A_0/m).  The powers
// v^k run downwards from v^K, K = P unless |v|^P < 2^-80, where K is cut so
// that v^K keeps its low part above FP32's normal range (the terms beyond are
// below 2^-80 A_k).
template <int QQ>
__global__ void __launch_bounds__(128) k_w_centres_split(EvalView E, SplitView X, int nc,
                                                         const int *__restrict__ ctr_box_of, double2 *__restrict__ Qout) {
    __shared__ float lt[384];
    for (int i = threadIdx.x; i < 384; i += blockDim.x) lt[i] = X.logt[i];
    __syncthreads();
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int b = ctr_box_of[c];
    int beg = E.loff[3][b], end = E.loff[3][b + 1];
    if (beg == end) return;
    const int P = E.P, P1 = P + 1;
    int lb = E.blev[b], ixb = E.bix[b], iyb = E.biy[b];
    float4 c4 = X.c_rel[c], r4 = X.c_r[c];
    dfl rc{r4.x, r4.y};
    dflc acc[QQ + 1];
#pragma unroll
    for (int m = 0; m <= QQ; ++m) acc[m] = dflc{dfl{0.f, 0.f}, dfl{0.f, 0.f}};
    for (int i = beg; i < end; ++i) {
        int d = E.lidx[3][i];
        int l = E.blev[d];
        float2 off = box_offset_f(X.H, lb, ixb, iyb, l, E.bix[d], E.biy[d]);
        dfl yx = dfl_add_f(dfl{c4.x, c4.y}, off.x), yy = dfl_add_f(dfl{c4.z, c4.w}, off.y);
        dfl n2 = dfl_add(dfl_sqr(yx), dfl_sqr(yy));
        dfl inv = dfl_rcp(n2);
        dflc yinv{dfl_mul(yx, inv), dfl_neg(dfl_mul(yy, inv))};
        float4 la = X.lvl[2 * l], lb4 = X.lvl[2 * l + 1];
        dfl rho{la.x, la.y}, irho{la.z, la.w};
        dflc v = dflc_scale(yinv, rho), sv = dflc_scale(yinv, rc);
        dflc vinv{dfl_mul(yx, irho), dfl_mul(yy, irho)};
        int K = P;
        float av2 = v.re.hi * v.re.hi + v.im.hi * v.im.hi;
        if ((float)P * __log2f(av2) < -160.f) K = max(1, min(P, (int)(-160.f / __log2f(av2))));
        dflc vk{dfl{1.f, 0.f}, dfl{0.f, 0.f}}, base = v;
        for (int e = K; e; e >>= 1) {
            if (e & 1) vk = dflc_mul(vk, base);
            if (e > 1) base = dflc_mul(base, base);
        }
        const float4 *A = X.M + (size_t)d * P1;
        dflc S[QQ + 1];
#pragma unroll
        for (int m = 0; m <= QQ; ++m) S[m] = dflc{dfl{0.f, 0.f}, dfl{0.f, 0.f}};
        for (int k = K; k >= 1; --k) {
            S[0] = dflc_add(S[0], dflc_mul(dflc_ld(A[k]), vk));
#pragma unroll
            for (int m = 1; m <= QQ; ++m) S[m] = dflc_sub(S[m], S[m - 1]);
            vk = dflc_mul(vk, vinv);
        }
        dfl A0{A[0].x, A[0].y};
        dfl lg = dfl_log(dfl_mul(n2, dfl{lb4.z, lb4.w}), lt, lt + 128, lt + 256);
        dfl ly = dfl_add(dfl{0.5f * lg.hi, 0.5f * lg.lo}, dfl{lb4.x, lb4.y});
        dflc_acc(acc[0], dflc{dfl_add(S[0].re, dfl_mul(A0, ly)), S[0].im});
        dflc sm = sv;
#pragma unroll
        for (int m = 1; m <= QQ; ++m) {
            float ih = __frcp_rn((float)m);
            dfl a = dfl_mul(A0, dfl{ih, fmaf(-(float)m, ih, 1.0f) * ih});   // A_0 / m
            dflc g{(m & 1) ? dfl_add(S[m].re, a) : dfl_add(S[m].re, dfl_neg(a)), S[m].im};
            dflc_acc(acc[m], dflc_mul(sm, g));
            sm = dflc_mul(sm, sv);
        }
    }
    double2 *dst = Qout + (size_t)c * (QQ + 1);
#pragma unroll
    for (int m = 0; m <= QQ; ++m)
        dst[m] = make_double2(dst[m].x + dfl_to_double(acc[m].re), dst[m].y + dfl_to_double(acc[m].im));
}

void dispatch_w_centres_split(gq_ctx *ctx, const EvalView &E, const SplitView &X, int nc, const int *owner,
                              double2 *Q) {
    switch (E.Q) {
#define GQ_CASE(v) case v: GQ_LAUNCH(ctx, k_w_centres_split<v>, gq_blocks(nc, 128), 128, 0, E, X, nc, owner, Q); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

// P2M (Stage 2) in FP32 pairs for the mixed tiers: the sums of k_p2m with the
// box-relative source coordinates, the strengths, the powers of u and the lane
// sums in pairs (lazy accumulators, normalised before the group butterfly).
// Writes the pair multipoles M2 of the source leaves.
template <int PM>
__global__ void k_p2m_split(EvalView E, SplitView X, int nwork, const int *__restrict__ work,
                            float4 *__restrict__ M2) {
    int wid = (blockIdx.x * blockDim.x + threadIdx.x) / kP2MG, lane = threadIdx.x % kP2MG;
    // whole groups leave together; the shuffles below stay inside a group
    if (wid >= nwork) return;
    int b = work[wid];
    int l = E.blev[b], P = E.P;
    const float irh = X.lvl[2 * l].z;   // 1/rho, a power of two: exact in FP32
    const dfl zero{0.f, 0.f};
    dflc acc[PM + 1];
#pragma unroll
    for (int k = 0; k <= PM; ++k) acc[k] = dflc{zero, zero};
    for (int s = E.src_beg[b] + lane; s < E.src_end[b]; s += kP2MG) {
        float4 y = X.s_rel[s];
        dflc u{dfl{y.x * irh, y.y * irh}, dfl{y.z * irh, y.w * irh}};
        dflc q = dflc_ld(X.str[s]);
        dflc t;
        if (E.kernel == GQ_D) {
            t = dflc{dfl{q.re.hi * irh, q.re.lo * irh}, dfl{q.im.hi * irh, q.im.lo * irh}};
        } else {
            dfl_acc(acc[0].re, q.re);
            t = dflc{dfl_mul(q.re, u.re), dfl_mul(q.re, u.im)};
        }
        dflc_acc(acc[1], t);
#pragma unroll
        for (int k = 2; k <= PM; ++k)
            if (k <= P) {
                t = dflc_mul(t, u);
                dflc_acc(acc[k], t);
            }
    }
    const unsigned gmask = ((1u << kP2MG) - 1u) << (threadIdx.x & 31 & ~(kP2MG - 1));
#pragma unroll
    for (int k = 0; k <= PM; ++k)
        if (k <= P) {
            dflc v{dfl_two_sum(acc[k].re.hi, acc[k].re.lo), dfl_two_sum(acc[k].im.hi, acc[k].im.lo)};
            for (int o = kP2MG / 2; o > 0; o >>= 1) {
                dflc w{dfl{__shfl_xor_sync(gmask, v.re.hi, o), __shfl_xor_sync(gmask, v.re.lo, o)},
                       dfl{__shfl_xor_sync(gmask, v.im.hi, o), __shfl_xor_sync(gmask, v.im.lo, o)}};
                v = dflc_add(v, w);
            }
            acc[k] = v;
        }
#pragma unroll
    for (int k = 0; k <= PM; ++k)
        if (k <= P && k % kP2MG == lane) {
            dflc v = acc[k];
            if (k >= 1) {
                if (E.kernel == GQ_D) {
                    v = dflc{dfl_neg(v.re), dfl_neg(v.im)};
                } else {
                    float ih = __frcp_rn((float)k);
                    dfl mik{-ih, -(fmaf(-(float)k, ih, 1.0f) * ih)};   // -1/k
                    v = dflc{dfl_mul(v.re, mik), dfl_mul(v.im, mik)};
                }
            }
            M2[(size_t)b * (P + 1) + k] = make_float4(v.re.hi, v.re.lo, v.im.hi, v.im.lo);
        }
}

// M2M (Stage 2) in FP32 pairs: k_m2m_t with the quadrant matrices and the
// multipoles in pairs, one thread per (parent, m), one lazy sum over children.
__global__ void k_m2m_split(EvalView E, int lstart, int lend, const float4 *__restrict__ T2,
                            float4 *__restrict__ M2) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int P1 = E.P + 1;
    int b = lstart + (int)(t / P1), m = (int)(t % P1);
    if (b >= lend) return;
    int4 c4 = E.bchild[b];
    int ch[4] = {c4.x, c4.y, c4.z, c4.w};
    if (ch[0] < 0 && ch[1] < 0 && ch[2] < 0 && ch[3] < 0) return;  // leaf
    if (E.sub_src[b] == 0) return;
    const dfl zero{0.f, 0.f};
    dflc acc{zero, zero};
    for (int q = 0; q < 4; ++q) {
        int c = ch[q];
        if (c < 0 || E.sub_src[c] == 0) continue;
        const float4 *A = M2 + (size_t)c * P1;
        if (m == 0) {
            dflc_acc(acc, dflc_ld(A[0]));
            continue;
        }
        const float4 *Tq = T2 + ((size_t)q * kTN + m) * kTN;
        dflc t0 = dflc_ld(__ldg(&Tq[0]));
        dfl a0 = dflc_ld(A[0]).re;
        dflc_acc(acc, dflc{dfl_mul(t0.re, a0), dfl_mul(t0.im, a0)});
        for (int k = 1; k <= m; ++k) dflc_acc(acc, dflc_mul(dflc_ld(__ldg(&Tq[k])), dflc_ld(A[k])));
    }
    dfl re = dfl_two_sum(acc.re.hi, acc.re.lo), im = dfl_two_sum(acc.im.hi, acc.im.lo);
    M2[(size_t)b * P1 + m] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// L2L (Stage 7) in FP32 pairs: k_l2l_t with the quadrant matrices and the
// local expansions in pairs, one thread per (child, m).
__global__ void k_l2l_split(EvalView E, int lstart, int lend, const float4 *__restrict__ U2,
                            float4 *__restrict__ L2) {
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    int P1 = E.P + 1;
    int c = lstart + (int)(t / P1), m = (int)(t % P1);
    if (c >= lend || E.sub_tgt[c] == 0) return;
    int p = E.bparent[c];
    int q = (E.bix[c] & 1) | ((E.biy[c] & 1) << 1);
    const float4 *B = L2 + (size_t)p * P1;
    const float4 *Uq = U2 + ((size_t)q * kTN + m) * kTN;
    float4 *dst = L2 + (size_t)c * P1 + m;
    dflc acc = dflc_ld(*dst);
    for (int k = m; k <= E.P; ++k) dflc_acc(acc, dflc_mul(dflc_ld(__ldg(&Uq[k])), dflc_ld(B[k])));
    dfl re = dfl_two_sum(acc.re.hi, acc.re.lo), im = dfl_two_sum(acc.im.hi, acc.im.lo);
    *dst = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// out += in as pairs (in FP64): folds the FP64 P2L terms into the pair locals
__global__ void k_add_to_dfl4(long long n, const double2 *__restrict__ in, float4 *__restrict__ out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float4 v = out[j];
    dfl a = dfl_from_double(in[j].x), b = dfl_from_double(in[j].y);
    dfl re = dfl_add(dfl{v.x, v.y}, a), im = dfl_add(dfl{v.z, v.w}, b);
    out[j] = make_float4(re.hi, re.lo, im.hi, im.lo);
}

// L2QBXL (Stage 8) in FP32 pairs: the Taylor shift of k_l2qbxl_t on the
// pair local expansions, with eta = (c - z_b)/rho and r/rho from the pair
// box-relative centre coordinates and radius (scalings by the power of two
// 1/rho exact), adding into the FP64 QBX coefficients.
template <int PM, int QQ>
__global__ void __launch_bounds__(128) k_l2qbxl_split(EvalView E, SplitView X, int nc,
                                                      const int *__restrict__ ctr_box_of,
                                                      const float4 *__restrict__ L2, double2 *__restrict__ Qout) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    const int P = E.P;
    int b = ctr_box_of[c];
    const float irh = X.lvl[2 * E.blev[b]].z;   // 1/rho, a power of two
    float4 c4 = X.c_rel[c], r4 = X.c_r[c];
    dflc eta{dfl{c4.x * irh, c4.y * irh}, dfl{c4.z * irh, c4.w * irh}};
    const float4 *B = L2 + (size_t)b * (P + 1);
    const dfl zero{0.f, 0.f};
    dflc bk[PM + 1];
#pragma unroll
    for (int k = 0; k <= PM; ++k) bk[k] = k <= P ? dflc_ld(B[k]) : dflc{zero, zero};
#pragma unroll
    for (int i = 0; i <= QQ; ++i)
#pragma unroll
        for (int k = PM - 1; k >= i; --k)
            if (k < P) bk[k] = dflc_add(bk[k], dflc_mul(eta, bk[k + 1]));
    const dfl sr{r4.x * irh, r4.y * irh};
    dfl sm{1.f, 0.f};
    double2 *dst = Qout + (size_t)c * (QQ + 1);
#pragma unroll
    for (int m = 0; m <= QQ; ++m) {
        if (m <= P)
            dst[m] = make_double2(dst[m].x + dfl_to_double(dfl_mul(bk[m].re, sm)),
                                  dst[m].y + dfl_to_double(dfl_mul(bk[m].im, sm)));
        sm = dfl_mul(sm, sr);
    }
}

template <int PM>
void launch_l2qbxl_split(gq_ctx *ctx, const EvalView &E, const SplitView &X, int nc, const int *owner,
                         const float4 *L2, double2 *Q) {
    switch (E.Q) {
#define GQ_CASE(v) case v: GQ_LAUNCH(ctx, (k_l2qbxl_split<PM, v>), gq_blocks(nc, 128), 128, 0, E, X, nc, owner, L2, Q); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

void dispatch_l2qbxl_split(gq_ctx *ctx, const EvalView &E, const SplitView &X, int nc, const int *owner,
                           const float4 *L2, double2 *Q) {
    if (E.P <= 8) launch_l2qbxl_split<8>(ctx, E, X, nc, owner, L2, Q);
    else if (E.P <= 16) launch_l2qbxl_split<16>(ctx, E, X, nc, owner, L2, Q);
    else launch_l2qbxl_split<GQ_MAX_PFMM>(ctx, E, X, nc, owner, L2, Q);
}

__global__ void k_from_dfl4(long long n, const float4 *__restrict__ in, double2 *__restrict__ out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float4 v = in[j];
    out[j] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

// M2L (Stage 4) in FP32 pairs for the mixed tiers: the factored translation of
// k_m2l -- At_k = A_k delta^-k, G_m = sum_k C(m+k-1, k-1) At_k, then
// L_m += (-1)^m delta^-m (G_m - A_0/m) and L_0 += A_0 log(rho |delta|) + G_0 --
// with the multipoles, delta^-k, the binomials and every product and sum in
// pairs (about 2^-46 relative per operation; the G_m sums in lazy
// accumulators), adding into the pair local expansions L2.  Groups of G
// lanes, lane g the order index, as in k_m2l.
// The binomial rows sit in shared memory with an odd row stride (in 8-byte
// words), so that the G lanes of a group, each reading its own row, hit
// distinct banks.
template <int G>
__global__ void k_m2l_split(EvalView E, SplitView X, int nwork, const int *__restrict__ work,
                            const float4 *__restrict__ dtab2, const float2 *__restrict__ logtab2,
                            const float2 *__restrict__ binom2, float4 *__restrict__ L2) {
    extern __shared__ float2 pasc2[];   // [P+1][RS]: C(m+k-1, k-1) as (hi, lo)
    const int P = E.P, P1 = P + 1, RS = P1 | 1;
    for (int i = threadIdx.x; i < P1 * P1; i += blockDim.x) {
        int m = i / P1, k = i % P1;
        pasc2[m * RS + k] = k >= 1 ? binom2[(m + k - 1) * kBinN + (k - 1)] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    int lane = threadIdx.x & 31, g = lane % G;
    long long grp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / G;
    bool act = grp < nwork;
    int b = act ? work[grp] : 0;
    int beg = act ? E.loff[1][b] : 0, end = act ? E.loff[1][b + 1] : 0;
    int n = end - beg, nmax = n;
    for (int o = G; o < 32; o <<= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    int l = E.blev[b], bx = E.bix[b], by = E.biy[b];
    const float4 lv = X.lvl[2 * l + 1];
    const dfl logrho{lv.x, lv.y};
    float ih = g >= 1 ? __frcp_rn((float)g) : 0.f;
    const dfl ig{ih, g >= 1 ? fmaf(-(float)g, ih, 1.0f) * ih : 0.f};   // 1/g
    const dfl zero{0.f, 0.f};
    dflc acc{zero, zero};
    const float2 *prow = pasc2 + (g <= P ? g : 0) * RS;
    for (int i = 0; i < nmax; ++i) {
        bool valid = i < n;
        int d = valid ? E.lidx[1][beg + i] : b;
        int off = valid ? (by - E.biy[d] + 5) * 11 + (bx - E.bix[d] + 5) : 0;
        dflc A = (valid && g <= P) ? dflc_ld(X.M[(size_t)d * P1 + g]) : dflc{zero, zero};
        dflc tk = dflc_ld(dtab2[off * 32 + g]);                 // delta^-g
        dflc At = g >= 1 ? dflc_mul(A, tk) : dflc{zero, zero};
        dfl A0{__shfl_sync(0xffffffffu, A.re.hi, 0, G), __shfl_sync(0xffffffffu, A.re.lo, 0, G)};
        dflc Gm{zero, zero};
        for (int k = 1; k <= P; ++k) {
            float xh = __shfl_sync(0xffffffffu, At.re.hi, k, G), xl = __shfl_sync(0xffffffffu, At.re.lo, k, G);
            float yh = __shfl_sync(0xffffffffu, At.im.hi, k, G), yl = __shfl_sync(0xffffffffu, At.im.lo, k, G);
            float2 c = prow[k];
            dfl_mac_lazy(Gm.re, c.x, c.y, xh, xl);
            dfl_mac_lazy(Gm.im, c.x, c.y, yh, yl);
        }
        if (!valid) continue;
        Gm.re = dfl_two_sum(Gm.re.hi, Gm.re.lo);
        Gm.im = dfl_two_sum(Gm.im.hi, Gm.im.lo);
        if (g == 0) {
            float2 lt = logtab2[off];
            dflc_acc(acc, dflc{dfl_add(dfl_mul(A0, dfl_add(logrho, dfl{lt.x, lt.y})), Gm.re), Gm.im});
        } else if (g <= P) {
            dflc t{dfl_add(Gm.re, dfl_neg(dfl_mul(A0, ig))), Gm.im};
            dflc sg = (g & 1) ? dflc{dfl_neg(tk.re), dfl_neg(tk.im)} : tk;
            dflc_acc(acc, dflc_mul(sg, t));
        }
    }
    if (act && g <= P) {
        float4 *dst = L2 + (size_t)b * P1 + g;
        float4 o = *dst;
        dfl re = dfl_add(dfl{o.x, o.y}, dfl_two_sum(acc.re.hi, acc.re.lo));
        dfl im = dfl_add(dfl{o.z, o.w}, dfl_two_sum(acc.im.hi, acc.im.lo));
        *dst = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
}

template <int QQ>
void launch_near_centres_split(gq_ctx *ctx, const EvalView &E, const SplitView &X, int nwork, const int *work,
                               double2 *Q) {
    auto kd = k_near_centres_split<QQ, GQ_D>;
    auto ks = k_near_centres_split<QQ, GQ_S>;
    GQ_LAUNCH(ctx, (E.kernel == GQ_D ? kd : ks), nwork, kNearThreads, 0, E, X, nwork, work, Q);
}

void dispatch_near_centres_split(gq_ctx *ctx, const EvalView &E, const SplitView &X, int nwork, const int *work,
                                 double2 *Q) {
    switch (E.Q) {
#define GQ_CASE(v) case v: launch_near_centres_split<v>(ctx, E, X, nwork, work, Q); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

template <int QQ>
void launch_near_centres_f32(gq_ctx *ctx, const EvalView &E, const MixedView &X, int nwork, const int *work,
                             double2 *Q) {
    auto kd = k_near_centres_f32<QQ, GQ_D>;
    auto ks = k_near_centres_f32<QQ, GQ_S>;
    GQ_LAUNCH(ctx, (E.kernel == GQ_D ? kd : ks), nwork, kNearThreads, 0, E, X, nwork, work, Q);
}

void dispatch_near_centres_f32(gq_ctx *ctx, const EvalView &E, const MixedView &X, int nwork, const int *work,
                               double2 *Q) {
    switch (E.Q) {
#define GQ_CASE(v) case v: launch_near_centres_f32<v>(ctx, E, X, nwork, work, Q); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

// Several densities on one geometry at once: the per-pair geometry (w, |w|^2,
// its reciprocal, log|w|, r/w) and the powers (r/w)^m are formed once and
// serve ND densities, each of which adds only its strength times the power.
// strm: ND strength arrays of the sorted sources, sstride apart; Qm: ND
// coefficient arrays [nc][q+1], qstride apart.  Same layout and sums as
// k_near_centres otherwise.
template <int QQ, int KERNEL, int ND>
__device__ void near_centres_multi_box(const EvalView &E, int b, const double2 *__restrict__ strm, long long sstride,
                                       double2 *__restrict__ Qm, long long qstride, NearRanges &R, int *wsum,
                                       const double *lt) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int ne = (E.loff[0][b + 1] - E.loff[0][b]) + (E.loff[2][b + 1] - E.loff[2][b]) + (E.loff[4][b + 1] - E.loff[4][b]);
    int cb = E.ctr_beg[b], ce = E.ctr_end[b];
    bool single = ne <= kNearRanges;
    if (single) load_ranges(E, b, 0, ne, R, wsum);
    else __syncthreads();
    for (int c0 = cb; c0 < ce; c0 += kNearThreads / 32) {
        int c = c0 + w;
        bool valid = c < ce;
        double2 cz = valid ? E.sc_xy[c] : make_double2(0.0, 0.0);
        double rc = valid ? E.sc_r[c] : 1.0;
        const int qc = (valid && E.qc) ? E.qc[c] : QQ;
        double2 acc[ND][QQ + 1];
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int m = 0; m <= QQ; ++m) acc[d][m] = make_double2(0.0, 0.0);
        for (int e0 = 0; e0 < ne; e0 += kNearRanges) {
            if (!single) {
                __syncthreads();
                load_ranges(E, b, e0, ne, R, wsum);
            }
            int T = R.pre[R.n];
            if (valid) {
                int r = 0;
                for (int v = lane; v < T; v += 32) {
                    while (R.pre[r + 1] <= v) ++r;
                    int s = R.beg[r] + (v - R.pre[r]);
                    double2 y = E.s_xy[s];
                    double2 st[ND];
#pragma unroll
                    for (int d = 0; d < ND; ++d) st[d] = strm[d * sstride + s];
                    double wx = y.x - cz.x, wy = y.y - cz.y;
                    double n2 = wx * wx + wy * wy;
                    double inv = gq_rcp(n2);
                    if (KERNEL == GQ_D) {
                        double2 bm = make_double2(wx * inv, -wy * inv);   // (1/w) (r/w)^m
                        double2 u = make_double2(rc * bm.x, rc * bm.y);
#pragma unroll
                        for (int d = 0; d < ND; ++d) acc[d][0] = cfma(st[d], bm, acc[d][0]);
#pragma unroll
                        for (int m = 1; m <= QQ; ++m) {
                            if (m > qc) break;
                            bm = cmul(bm, u);
#pragma unroll
                            for (int d = 0; d < ND; ++d) acc[d][m] = cfma(st[d], bm, acc[d][m]);
                        }
                    } else {
                        double ir = rc * inv;
                        double2 u = make_double2(wx * ir, -wy * ir), pw = u;
                        double lg = gq_log_half(n2, lt);
#pragma unroll
                        for (int d = 0; d < ND; ++d) {
                            acc[d][0].x = fma(st[d].x, lg, acc[d][0].x);
                            acc[d][1].x = fma(st[d].x, pw.x, acc[d][1].x);
                            acc[d][1].y = fma(st[d].x, pw.y, acc[d][1].y);
                        }
#pragma unroll
                        for (int m = 2; m <= QQ; ++m) {
                            if (m > qc) break;
                            pw = cmul(pw, u);
#pragma unroll
                            for (int d = 0; d < ND; ++d) {
                                acc[d][m].x = fma(st[d].x, pw.x, acc[d][m].x);
                                acc[d][m].y = fma(st[d].x, pw.y, acc[d][m].y);
                            }
                        }
                    }
                }
            }
        }
        constexpr int NV = 2 * (QQ + 1);
        double vals[ND * NV];
#pragma unroll
        for (int d = 0; d < ND; ++d)
#pragma unroll
            for (int m = 0; m <= QQ; ++m) {
                vals[d * NV + 2 * m] = acc[d][m].x;
                vals[d * NV + 2 * m + 1] = acc[d][m].y;
            }
        int base, cnt;
        warp_reduce_scatter(vals, 0.0, lane, [](double a, double x) { return a + x; },
                            [](double x, int o) { return __shfl_xor_sync(0xffffffffu, x, o); }, base, cnt);
        if (valid) {
#pragma unroll
            for (int j = 0; j < (ND * NV + 31) / 32; ++j)
                if (j < cnt) {
                    int i = base + j, d = i / NV, k = i - d * NV, m = k >> 1;
                    double x = vals[j];
                    if (KERNEL != GQ_D && m >= 1) x *= -1.0 / m;
                    reinterpret_cast<double *>(Qm + d * qstride + (size_t)c * (QQ + 1))[k] = x;
                }
        }
    }
}


template <int QQ, int KERNEL, int ND>
__global__ void __launch_bounds__(kNearThreads) k_near_centres_multi(EvalView E, int nwork, const int *__restrict__ work,
                                                                      const double2 *__restrict__ strm, long long sstride,
                                                                      double2 *__restrict__ Qm, long long qstride) {
    __shared__ NearRanges R;
    __shared__ int wsum[kNearThreads / 32];
    __shared__ double lt[KERNEL == GQ_D ? 1 : kGqLogN];
    if (KERNEL != GQ_D)
        for (int i = threadIdx.x; i < kGqLogN; i += kNearThreads) lt[i] = E.logt[i];
    near_centres_multi_box<QQ, KERNEL, ND>(E, work[blockIdx.x], strm, sstride, Qm, qstride, R, wsum, lt);
}

template <int QQ, int ND>
void launch_near_centres_multi(gq_ctx *ctx, const EvalView &E, int nwork, const int *work, const double2 *strm,
                               long long sstride, double2 *Qm, long long qstride) {
    auto kd = k_near_centres_multi<QQ, GQ_D, ND>;
    auto ks = k_near_centres_multi<QQ, GQ_S, ND>;
    GQ_LAUNCH(ctx, (E.kernel == GQ_D ? kd : ks), nwork, kNearThreads, 0, E, nwork, work, strm, sstride, Qm, qstride);
}

template <int ND>
void dispatch_near_centres_multi(gq_ctx *ctx, const EvalView &E, int nwork, const int *work, const double2 *strm,
                                 long long sstride, double2 *Qm, long long qstride) {
    switch (E.Q) {
#define GQ_CASE(v) case v: launch_near_centres_multi<v, ND>(ctx, E, nwork, work, strm, sstride, Qm, qstride); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

template <int QQ>
void launch_near_centres(gq_ctx *ctx, const EvalView &E, int nwork, const int *work, double2 *Q) {
    auto kd = k_near_centres<QQ, GQ_D>;
    auto ks = k_near_centres<QQ, GQ_S>;
    if (E.kernel == GQ_D)
        GQ_LAUNCH(ctx, kd, nwork, kNearThreads, 0, E, nwork, work, Q);
    else
        GQ_LAUNCH(ctx, ks, nwork, kNearThreads, 0, E, nwork, work, Q);
}

void dispatch_near_centres(gq_ctx *ctx, const EvalView &E, int nwork, const int *work, double2 *Q) {
    switch (E.Q) {
#define GQ_CASE(v) case v: launch_near_centres<v>(ctx, E, nwork, work, Q); break;
        GQ_CASE(1) GQ_CASE(2) GQ_CASE(3) GQ_CASE(4) GQ_CASE(5) GQ_CASE(6) GQ_CASE(7) GQ_CASE(8)
        GQ_CASE(9) GQ_CASE(10) GQ_CASE(11) GQ_CASE(12) GQ_CASE(13) GQ_CASE(14) GQ_CASE(15) GQ_CASE(16)
#undef GQ_CASE
        default: throw gq_error{GQ_ERR_INVALID, "p_qbx out of range"};
    }
}

__global__ void k_tgt_ptpos(int npt, const int *__restrict__ pt_perm, int *__restrict__ out) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < npt) out[pt_perm[j]] = j;
}


// ------------------------------------------------------------------ persistent batched evaluation
// One launch covers the direct interactions and the final sums of every
// geometry and density of a batch (the FMM passes run before it, per
// geometry).  Work items, taken in order from a counter by CTAs of
// kNearThreads threads:
//   NEAR4/NEAR2/NEAR1 (geometry, first box, first density): the direct part of
//     the QBX coefficients (Stages 3, 5a, 6a) of `tile` target boxes for 4, 2
//     or 1 densities at once (per-pair geometry and powers shared);
//   NEARPT (geometry, box, density): the direct potential at point targets;
//   FINAL (geometry, first target, density): eq. qbx at 256 targets.
// All NEAR/NEARPT items precede every FINAL item.  A FINAL item first waits
// until its geometry's direct items are done (a per-geometry counter; the
// items it waits for were taken earlier by running CTAs and wait for nothing,
// so the wait ends); the wait is bounded by limit_ns, after which the kernel
// sets *err and skips the item (later waits return at once).
enum { BI_NEAR4 = 0, BI_NEAR2 = 1, BI_NEAR1 = 2, BI_NEARPT = 3, BI_FINAL = 4 };

struct BatchItem {
    int type, geom, a, b;
};

struct BatchGeomDev {
    EvalView E;
    const int *ctr_boxes, *pt_boxes;
    int tile;                          // target boxes per NEAR item
    const double2 *strm;               // [nd][nsrc] strengths
    long long sstride;
    double2 *Qn;                       // [nd][nc][q+1] direct parts
    const double2 *Qf;                 // [nd][nc][q+1] far parts (FMM passes)
    long long qstride;
    double *potn;                      // [nd][npt] direct point potentials
    const double *potf;                // [nd][npt] far point potentials
    long long pstride;
    const unsigned int *qexp;          // [nd] largest strength exponent per density
    double *out;                       // [nd][nt]
    int nt, kernel, items;             // items: NEAR + NEARPT items of this geometry
    const int *kind, *ctr, *ctr_pos, *tgt_ptpos, *tgt_on;
    const double *tgt_xy, *base_n;
};

template <int QQ, int KERNEL>
__global__ void __launch_bounds__(kNearThreads) k_batch_persistent(const BatchGeomDev *__restrict__ G,
                                                                    const BatchItem *__restrict__ items, int nitems,
                                                                    const double *__restrict__ logt, int *next,
                                                                    int *done, unsigned long long limit_ns,
                                                                    int *err) {
    __shared__ NearRanges R;
    __shared__ int wsum[kNearThreads / 32];
    __shared__ double lt[KERNEL == GQ_D ? 1 : kGqLogN];
    __shared__ int sitem, sok;
    if (KERNEL != GQ_D)
        for (int i = threadIdx.x; i < kGqLogN; i += kNearThreads) lt[i] = logt[i];
    for (;;) {
        if (threadIdx.x == 0) sitem = atomicAdd(next, 1);
        __syncthreads();
        const int it = sitem;
        __syncthreads();   // every thread has the item before thread 0 takes the next
        if (it >= nitems) break;
        const BatchItem I = items[it];
        const BatchGeomDev &g = G[I.geom];
        if (I.type <= BI_NEAR1) {
            const int n0 = I.a, n1 = min(I.a + g.tile, g.E.nwork_ctr);
            for (int j = n0; j < n1; ++j) {
                const int b = g.ctr_boxes[j];
                const double2 *st = g.strm + I.b * g.sstride;
                double2 *q = g.Qn + I.b * g.qstride;
                if (I.type == BI_NEAR4) near_centres_multi_box<QQ, KERNEL, 4>(g.E, b, st, g.sstride, q, g.qstride, R, wsum, lt);
                else if (I.type == BI_NEAR2) near_centres_multi_box<QQ, KERNEL, 2>(g.E, b, st, g.sstride, q, g.qstride, R, wsum, lt);
                else near_centres_multi_box<QQ, KERNEL, 1>(g.E, b, st, g.sstride, q, g.qstride, R, wsum, lt);
                __syncthreads();
            }
        } else if (I.type == BI_NEARPT) {
            EvalView E = g.E;
            E.qexp = g.qexp + I.b;
            near_points_box<KERNEL>(E, g.pt_boxes[I.a], g.strm + I.b * g.sstride, g.potn + I.b * g.pstride, R, wsum,
                                    lt);
            __syncthreads();
        } else {
            if (threadIdx.x == 0) {
                const volatile int *dv = done + I.geom;
                const unsigned long long t0 = gqtc_globaltimer();
                int ok = 1;
                while (*dv < g.items) {
                    if (*(volatile int *)err || gqtc_globaltimer() - t0 > limit_ns) {
                        atomicExch(err, 1);
                        ok = 0;
                        break;
                    }
                }
                __threadfence();
                sok = ok;
            }
            __syncthreads();
            const int t = I.a + threadIdx.x;
            if (sok && t < g.nt)
                final_target(t, g.kernel, g.E.Q, g.E.qc, g.kind, g.ctr, g.ctr_pos, g.tgt_ptpos, g.tgt_xy, g.tgt_on,
                             g.base_n, g.E.sc_xy, g.E.sc_r, g.Qf + I.b * g.qstride, g.Qn + I.b * g.qstride,
                             g.potf + I.b * g.pstride, g.potn + I.b * g.pstride, g.out + (size_t)I.b * g.nt);
            continue;
        }
        // a direct item is done: every thread's writes are visible device-wide
        // before the count moves
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(done + I.geom, 1);
    }
}

}  // namespace

// ------------------------------------------------------------------ tables (per geometry)
// Constant tables (log tables, binomials, same-level M2L offsets, M2M/L2L
// quadrant matrices): built on the host once per device and kept for the
// life of the process (about 200 KB); each geometry adds the target -> point
// map of its current build.
struct ConstTables {
    const double *logt = nullptr;     // GqLogTable
    const float *dlogt = nullptr;     // GqDflLogTable
    const double *binom = nullptr;    // [64][64]
    const double2 *dtab = nullptr;    // [121][32] delta^-k
    const double *logtab = nullptr;   // [121] log|delta|
    const double2 *tm2m = nullptr;    // [4][kTN][kTN] M2M matrices
    const double2 *tl2l = nullptr;    // [4][kTN][kTN] L2L matrices
    const float4 *dtab2 = nullptr;    // dtab as FP32 pairs (re.hi, re.lo, im.hi, im.lo)
    const float2 *logtab2 = nullptr;  // logtab as FP32 pairs
    const float2 *binom2 = nullptr;   // binom as FP32 pairs
    const float4 *tm2m2 = nullptr;    // tm2m as FP32 pairs
    const float4 *tl2l2 = nullptr;    // tl2l as FP32 pairs
};

struct EvalTables : ConstTables {
    dbuf<int> tgt_ptpos;     // [nt] target -> sorted point index
};

static void host_const_tables(std::vector<double> &bn, std::vector<double2> &dt, std::vector<double> &lt,
                              std::vector<double2> &tm, std::vector<double2> &tl) {
    bn.assign(kBinN * kBinN, 0.0);
    for (int n = 0; n < kBinN; ++n) {
        bn[n * kBinN] = 1.0;
        for (int k = 1; k <= n; ++k) bn[n * kBinN + k] = bn[(n - 1) * kBinN + k - 1] + (k <= n - 1 ? bn[(n - 1) * kBinN + k] : 0.0);
    }
    dt.assign(121 * 32, make_double2(0.0, 0.0));
    lt.assign(121, 0.0);
    for (int dy = -5; dy <= 5; ++dy)
        for (int dx = -5; dx <= 5; ++dx) {
            int off = (dy + 5) * 11 + (dx + 5);
            double re = 2.0 * dx, im = 2.0 * dy, n2 = re * re + im * im;
            double ir = n2 > 0 ? re / n2 : 0.0, ii = n2 > 0 ? -im / n2 : 0.0;
            double pr = 1.0, pi = 0.0;
            for (int k = 0; k < 32; ++k) {
                dt[off * 32 + k] = make_double2(pr, pi);
                double nr = pr * ir - pi * ii, ni = pr * ii + pi * ir;
                pr = nr; pi = ni;
            }
            lt[off] = n2 > 0 ? 0.5 * log(n2) : 0.0;
        }
    // translation matrices for the four child quadrants, in long double
    tm.assign((size_t)4 * kTN * kTN, make_double2(0.0, 0.0));
    tl.assign(tm.size(), make_double2(0.0, 0.0));
    std::vector<long double> C((size_t)(2 * kTN) * (2 * kTN), 0.0L);
    auto Cb = [&](int n, int k) -> long double & { return C[(size_t)n * (2 * kTN) + k]; };
    for (int n = 0; n < 2 * kTN; ++n) {
        Cb(n, 0) = 1.0L;
        for (int k = 1; k <= n; ++k) Cb(n, k) = Cb(n - 1, k - 1) + (k <= n - 1 ? Cb(n - 1, k) : 0.0L);
    }
    for (int q = 0; q < 4; ++q) {
        long double ex = (q & 1) ? 0.5L : -0.5L, ey = (q & 2) ? 0.5L : -0.5L;
        std::vector<long double> pr(kTN + 1), pi(kTN + 1);   // eta^j
        pr[0] = 1.0L;
        pi[0] = 0.0L;
        for (int j = 1; j <= kTN; ++j) {
            pr[j] = pr[j - 1] * ex - pi[j - 1] * ey;
            pi[j] = pr[j - 1] * ey + pi[j - 1] * ex;
        }
        for (int m = 0; m < kTN; ++m)
            for (int k = 0; k < kTN; ++k) {
                size_t i = ((size_t)q * kTN + m) * kTN + k;
                if (m >= 1 && k == 0) tm[i] = make_double2((double)(-pr[m] / m), (double)(-pi[m] / m));
                if (m >= 1 && k >= 1 && k <= m) {
                    long double f = Cb(m - 1, k - 1) * ldexpl(1.0L, -k);
                    tm[i] = make_double2((double)(f * pr[m - k]), (double)(f * pi[m - k]));
                }
                if (k >= m) {
                    long double f = Cb(k, m) * ldexpl(1.0L, -m);
                    tl[i] = make_double2((double)(f * pr[k - m]), (double)(f * pi[k - m]));
                }
            }
    }
}

template <class T>
static const T *upload_const(const T *h, size_t n) {
    void *d = nullptr;
    GQ_CUDA(cudaMalloc(&d, sizeof(T) * n));
    GQ_CUDA(cudaMemcpy(d, h, sizeof(T) * n, cudaMemcpyHostToDevice));
    return (const T *)d;
}

static const ConstTables &const_tables(int dev) {
    static std::mutex mu;
    static std::map<int, ConstTables> per_dev;
    std::lock_guard<std::mutex> lk(mu);
    auto it = per_dev.find(dev);
    if (it != per_dev.end()) return it->second;
    int cur = 0;
    GQ_CUDA(cudaGetDevice(&cur));
    GQ_CUDA(cudaSetDevice(dev));
    std::vector<double> bn, lt;
    std::vector<double2> dt, tm, tl;
    host_const_tables(bn, dt, lt, tm, tl);
    std::vector<double> pc((GQ_MAX_PQBX + 1) * 33, 0.0);
    for (int m = 0; m <= GQ_MAX_PQBX; ++m)
        for (int k = 1; k <= 32; ++k) pc[m * 33 + k] = bn[(m + k - 1) * kBinN + (k - 1)];
    GQ_CUDA(cudaMemcpyToSymbol(c_pascal, pc.data(), sizeof(double) * pc.size()));
    GqLogTable LT;
    gq_log_table_host(&LT);
    GqDflLogTable DT;
    gq_dfl_log_table_host(&DT);
    ConstTables C;
    C.logt = upload_const((const double *)&LT, kGqLogN);
    C.dlogt = upload_const((const float *)&DT, 384);
    C.binom = upload_const(bn.data(), bn.size());
    C.dtab = upload_const(dt.data(), dt.size());
    C.logtab = upload_const(lt.data(), lt.size());
    C.tm2m = upload_const(tm.data(), tm.size());
    C.tl2l = upload_const(tl.data(), tl.size());
    auto split = [](double x) {
        float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    };
    std::vector<float4> dt2(dt.size());
    for (size_t i = 0; i < dt.size(); ++i) {
        float2 a = split(dt[i].x), b = split(dt[i].y);
        dt2[i] = make_float4(a.x, a.y, b.x, b.y);
    }
    std::vector<float2> lt2(lt.size()), bn2(bn.size());
    for (size_t i = 0; i < lt.size(); ++i) lt2[i] = split(lt[i]);
    for (size_t i = 0; i < bn.size(); ++i) bn2[i] = split(bn[i]);
    C.dtab2 = upload_const(dt2.data(), dt2.size());
    C.logtab2 = upload_const(lt2.data(), lt2.size());
    C.binom2 = upload_const(bn2.data(), bn2.size());
    std::vector<float4> tm2(tm.size());
    for (size_t i = 0; i < tm.size(); ++i) {
        float2 a = split(tm[i].x), b = split(tm[i].y);
        tm2[i] = make_float4(a.x, a.y, b.x, b.y);
    }
    C.tm2m2 = upload_const(tm2.data(), tm2.size());
    for (size_t i = 0; i < tl.size(); ++i) {
        float2 a = split(tl[i].x), b = split(tl[i].y);
        tm2[i] = make_float4(a.x, a.y, b.x, b.y);
    }
    C.tl2l2 = upload_const(tm2.data(), tm2.size());
    GQ_CUDA(cudaSetDevice(cur));
    return per_dev.emplace(dev, C).first->second;
}

static void make_tables(gq_geom *g, EvalTables &T) {
    static_cast<ConstTables &>(T) = const_tables(g->ctx->device);
    T.tgt_ptpos.alloc(g->nt);
    if (g->npt) GQ_LAUNCH(g->ctx, k_tgt_ptpos, gq_blocks(g->npt, 256), 256, 0, g->npt, (const int *)g->pt_perm.p, T.tgt_ptpos.p);
}

// tables are owned by the geometry through this registry
static std::mutex g_tab_mu;
static std::map<gq_geom *, EvalTables *> g_tabs;

void gq_tables_release(gq_geom *g) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto it = g_tabs.find(g);
    if (it != g_tabs.end()) {
        delete it->second;
        g_tabs.erase(it);
    }
}

static EvalTables &get_tables(gq_geom *g) {
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto it = g_tabs.find(g);
    if (it != g_tabs.end()) return *it->second;
    EvalTables *T = new EvalTables;
    make_tables(g, *T);
    g_tabs[g] = T;
    return *T;
}

void gq_eval_all(gq_geom *g, int kernel, const double *dens_dev, double *out_dev, gq_stats *stt,
                 const double2 *qn_pre, const double *apply_identity, const EvalFar *far) {
    // apply_identity != null: the operator at the base nodes (gq_apply); the
    // point-target stages are skipped and out_dev has one value per base node.
    // far != null: strengths and the FMM passes only, their parts of the QBX
    // coefficients and point potentials written to far->Q, far->pot (the
    // batched evaluation does the direct parts and the final sums itself).
    const bool at_base = apply_identity != nullptr;
    const bool fmm_only = far != nullptr;
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    EvalTables &T = get_tables(g);
    int P = g->prm.p_fmm, Qn = g->prm.p_qbx, P1 = P + 1, Q1 = Qn + 1;
    int kin = kernel == GQ_SP ? GQ_S : kernel;
    EvalView E;
    E.R = g->root;
    E.P = P;
    E.Q = Qn;
    E.kernel = kin;
    E.blev = g->blev; E.bix = g->bix; E.biy = g->biy; E.bparent = g->bparent; E.bchild = g->bchild;
    E.src_beg = g->src_beg; E.src_end = g->src_end;
    E.ctr_beg = g->ctr_beg; E.ctr_end = g->ctr_end; E.pt_beg = g->pt_beg; E.pt_end = g->pt_end;
    E.sub_src = g->sub_src; E.sub_tgt = g->sub_tgt;
    E.s_xy = g->s_xy; E.str = g->strength; E.sc_xy = g->sc_xy; E.sc_r = g->sc_r; E.sp_xy = g->sp_xy;
    for (int i = 0; i < 6; ++i) { E.loff[i] = g->list_off[i]; E.lidx[i] = g->list_idx[i]; }
    E.binom = T.binom;
    E.qc = g->has_qc ? (const int *)g->q_ctr.p : nullptr;
    E.logt = T.logt;

    g->strength.alloc(g->nsrc);
    E.str = g->strength;
    g->qexp.alloc(1);
    E.qexp = g->qexp;
    g->M.alloc((size_t)g->nbox * P1);
    g->L.alloc((size_t)g->nbox * P1);
    g->Q.alloc((size_t)g->nc * Q1);    // List 3 far + box-local part of the QBX coefficients
    g->Qn.alloc((size_t)g->nc * Q1);   // direct part
    g->pot.alloc(g->npt);
    g->potn.alloc(g->npt);
    double2 *Qb = fmm_only ? far->Q : g->Q.p;      // after the allocations: the
    double *potb = fmm_only ? far->pot : g->pot.p; // first call sets the pointers
    if (!g->s2) {
        GQ_CUDA(cudaStreamCreateWithFlags(&g->s2, cudaStreamNonBlocking));
        GQ_CUDA(cudaEventCreateWithFlags(&g->ev_str, cudaEventDisableTiming));
        GQ_CUDA(cudaEventCreateWithFlags(&g->ev_near, cudaEventDisableTiming));
    }
    // The direct part may run on a second stream, concurrently with the FMM passes
    // (GQ_OVERLAP=1); by default both run in order on the context's stream: the
    // direct kernels alone keep the FP64 pipe busy, so concurrency gains nothing.
    static const bool overlap = getenv("GQ_OVERLAP") && getenv("GQ_OVERLAP")[0] == '1';
    cudaStream_t s2 = overlap ? g->s2 : st;
    gq_ctx ctx2 = *ctx;   // launches of the direct part
    ctx2.stream = s2;
    ctx2.launches = 0;

    // stage events (only when statistics are requested); the direct stages run on
    // the second stream, concurrently with the FMM passes
    enum { S0, S_STR, S_FMM, S_M2M, S_M2L, S_P2L, S_L2L, S_WC, S_WP, S_L2Q, S_END, N_BEG, N_CTR, N_PT, NEV };
    cudaEvent_t ev[NEV];
    bool timed = stt != nullptr;
    if (timed)
        for (int i = 0; i < NEV; ++i) GQ_CUDA(cudaEventCreate(&ev[i]));
    auto mark = [&](int i, cudaStream_t on) {
        if (timed) GQ_CUDA(cudaEventRecord(ev[i], on));
    };
    mark(S0, st);
    int64_t l0 = ctx->launches;

    // A1
    GQ_CUDA(cudaMemsetAsync(g->qexp.p, 0, sizeof(unsigned int), st));
    GQ_LAUNCH(ctx, k_strengths, gq_blocks(g->nsrc, 256), 256, 0, g->nsrc, g->nu, g->nb, (const int *)g->src_perm,
              (const double *)g->interp, dens_dev, (const double *)g->s_w, (const double2 *)g->s_n, kin, g->strength.p,
              g->qexp.p);
    const bool mixed = g->prm.precision == GQ_PREC_MIXED || g->prm.precision == GQ_PREC_MIXED_FMM;
    const bool f32 = mixed && g->prm.eps >= kF32TierEps;
    const bool split = mixed && g->prm.eps >= 1e-12 && g->prm.eps < kF32TierEps;
    MixedView X{};
    if (f32) {
        if (!g->mixed_ready) {
            g->s_rel.alloc(g->nsrc);
            g->c_rel.alloc(g->nc);
            g->c_rf.alloc(g->nc);
            g->p_rel.alloc(g->npt);
            if (g->nsrc) GQ_LAUNCH(ctx, k_rel_coords, gq_blocks(g->nsrc, 256), 256, 0, g->nsrc, (const double2 *)g->s_xy,
                                   (const int *)g->src_owner, E, g->s_rel.p);
            if (g->nc) {
                GQ_LAUNCH(ctx, k_rel_coords, gq_blocks(g->nc, 256), 256, 0, g->nc, (const double2 *)g->sc_xy,
                          (const int *)g->ctr_owner, E, g->c_rel.p);
                GQ_LAUNCH(ctx, k_to_float, gq_blocks(g->nc, 256), 256, 0, g->nc, (const double *)g->sc_r, g->c_rf.p);
            }
            if (g->npt) GQ_LAUNCH(ctx, k_rel_coords, gq_blocks(g->npt, 256), 256, 0, g->npt, (const double2 *)g->sp_xy,
                                  (const int *)g->pt_owner, E, g->p_rel.p);
            g->mixed_ready = true;
        }
        g->str_f.alloc(g->nsrc);
        g->M_f.alloc((size_t)g->nbox * P1);
        if (g->nsrc) GQ_LAUNCH(ctx, k_to_float2, gq_blocks(g->nsrc, 256), 256, 0, (long long)g->nsrc,
                               (const double2 *)g->strength, g->str_f.p);
        X.s_rel = g->s_rel; X.str = g->str_f; X.c_rel = g->c_rel; X.p_rel = g->p_rel; X.M = g->M_f; X.c_r = g->c_rf;
    }
    SplitView SX{};
    // List 3 far at centres runs in pairs in both mixed tiers (exact FP32 box offsets need l <= 23)
    const bool split_w = (split || f32) && g->nlev <= 24;
    // GQ_PREC_MIXED_FMM: the FMM passes (P2M, M2M, M2L, L2L, L2QBXL) in pairs down
    // to eps = 1e-10: the M2L rounding, amplified by the binomial sums' cancellation
    // (at most about 25x for the same-level offsets |delta| >= 4), stays near 1e-13
    // relative, below eps/5 there; at smaller eps, and in GQ_PREC_MIXED, they stay FP64
    const bool m2l_split =
        g->prm.precision == GQ_PREC_MIXED_FMM && (split || f32) && g->prm.eps >= 1e-10;
    if (split || f32) {
        if (!g->split_ready) {
            g->s_rel2.alloc(g->nsrc);
            g->c_rel2.alloc(g->nc);
            g->c_r2.alloc(g->nc);
            if (g->nsrc) GQ_LAUNCH(ctx, k_rel_coords_split, gq_blocks(g->nsrc, 256), 256, 0, g->nsrc,
                                   (const double2 *)g->s_xy, (const int *)g->src_owner, E, g->s_rel2.p);
            if (g->nc) {
                GQ_LAUNCH(ctx, k_rel_coords_split, gq_blocks(g->nc, 256), 256, 0, g->nc, (const double2 *)g->sc_xy,
                          (const int *)g->ctr_owner, E, g->c_rel2.p);
                GQ_LAUNCH(ctx, k_radius_split, gq_blocks(g->nc, 256), 256, 0, g->nc, (const double *)g->sc_r, g->c_r2.p);
            }
            g->p_rel2.alloc(g->npt);
            if (g->npt) GQ_LAUNCH(ctx, k_rel_coords_split, gq_blocks(g->npt, 256), 256, 0, g->npt,
                                  (const double2 *)g->sp_xy, (const int *)g->pt_owner, E, g->p_rel2.p);
            g->lvl2.alloc(2 * (size_t)g->nlev);
            GQ_LAUNCH(ctx, k_level_split, 1, 64, 0, g->nlev, g->root.H, g->lvl2.p);
            g->split_ready = true;
        }
        g->M2.alloc((size_t)g->nbox * P1);
        if (m2l_split) g->L2.alloc((size_t)g->nbox * P1);
        if (split || m2l_split) {
            g->str2.alloc(g->nsrc);
            if (g->nsrc) GQ_LAUNCH(ctx, k_to_dfl4, gq_blocks(g->nsrc, 256), 256, 0, (long long)g->nsrc,
                                   (const double2 *)g->strength, g->str2.p);
        }
        SX.s_rel = g->s_rel2; SX.str = g->str2; SX.c_rel = g->c_rel2; SX.c_r = g->c_r2; SX.p_rel = g->p_rel2;
        SX.M = g->M2; SX.lvl = g->lvl2; SX.logt = T.dlogt; SX.H = (float)g->root.H;
        // only the sources inside the disk go to FP64: widening that region to |r/w| > 1/2
        // lowered the added D rounding on a small grid from 1.6e-13 to 1.45e-13 only, and
        // its divergent FP64 lanes tripled the kernel time
        SX.fb = 1.0f;
        SX.near_pt = g->prm.eps < 1e-10;
    }
    mark(S_STR, st);
    GQ_CUDA(cudaEventRecord(g->ev_str, st));

    // ---- Stages 3, 5a, 6a (direct interactions) on the second stream
    GQ_CUDA(cudaStreamWaitEvent(s2, g->ev_str, 0));
    mark(N_BEG, s2);
    if (g->n_ctr_boxes && !fmm_only) {
        if (f32) dispatch_near_centres_f32(&ctx2, E, X, g->n_ctr_boxes, g->ctr_boxes, g->Qn.p);
        else if (split) dispatch_near_centres_split(&ctx2, E, SX, g->n_ctr_boxes, g->ctr_boxes, g->Qn.p);
        else if (!qn_pre) dispatch_near_centres(&ctx2, E, g->n_ctr_boxes, g->ctr_boxes, g->Qn.p);
    }
    mark(N_CTR, s2);
    if (g->n_pt_boxes && !at_base && !fmm_only) {
        if (f32) {
            auto kd = k_near_points_f32<GQ_D>;
            auto ks = k_near_points_f32<GQ_S>;
            GQ_LAUNCH((&ctx2), (kin == GQ_D ? kd : ks), g->n_pt_boxes, kNearThreads, 0, E, X, g->n_pt_boxes,
                      (const int *)g->pt_boxes, g->potn.p);
        } else if (split) {
            auto kd = k_near_points_split<GQ_D>;
            auto ks = k_near_points_split<GQ_S>;
            GQ_LAUNCH((&ctx2), (kin == GQ_D ? kd : ks), g->n_pt_boxes, kNearThreads, 0, E, SX, g->n_pt_boxes,
                      (const int *)g->pt_boxes, g->potn.p);
        } else {
            auto kd = k_near_points<GQ_D>;
            auto ks = k_near_points<GQ_S>;
            GQ_LAUNCH((&ctx2), (kin == GQ_D ? kd : ks), g->n_pt_boxes, kNearThreads, 0, E, g->n_pt_boxes,
                      (const int *)g->pt_boxes, g->potn.p);
        }
    }
    mark(N_PT, s2);
    GQ_CUDA(cudaEventRecord(g->ev_near, s2));

    // ---- FMM passes on the context's stream
    mark(S_FMM, st);
    GQ_CUDA(cudaMemsetAsync(g->M.p, 0, sizeof(double2) * g->nbox * P1, st));
    if (m2l_split) {
        GQ_CUDA(cudaMemsetAsync(g->M2.p, 0, sizeof(float4) * g->nbox * P1, st));
        GQ_CUDA(cudaMemsetAsync(g->L2.p, 0, sizeof(float4) * g->nbox * P1, st));
    }
    GQ_CUDA(cudaMemsetAsync(g->L.p, 0, sizeof(double2) * g->nbox * P1, st));
    GQ_CUDA(cudaMemsetAsync(Qb, 0, sizeof(double2) * g->nc * Q1, st));
    if (g->npt && !at_base) GQ_CUDA(cudaMemsetAsync(potb, 0, sizeof(double) * g->npt, st));
    // Stage 2 (in pairs wherever M2L runs in pairs: the multipoles then live in
    // M2 and the FP64 copy is made from them for the FP64 consumers)
    if (g->n_leaf_src) {
        if (m2l_split) {
            auto k8 = k_p2m_split<8>;
            auto k16 = k_p2m_split<16>;
            auto k32 = k_p2m_split<GQ_MAX_PFMM>;
            GQ_LAUNCH(ctx, (P <= 8 ? k8 : P <= 16 ? k16 : k32), gq_blocks((long long)g->n_leaf_src * kP2MG, 128),
                      128, 0, E, SX, g->n_leaf_src, (const int *)g->leaf_src_boxes, g->M2.p);
        } else {
            auto k8 = k_p2m<8>;
            auto k16 = k_p2m<16>;
            auto k32 = k_p2m<GQ_MAX_PFMM>;
            GQ_LAUNCH(ctx, (P <= 8 ? k8 : P <= 16 ? k16 : k32), gq_blocks((long long)g->n_leaf_src * kP2MG, 128),
                      128, 0, E, g->n_leaf_src, (const int *)g->leaf_src_boxes, g->M.p);
        }
    }
    for (int l = g->nlev - 2; l >= 0; --l) {
        int s = g->level_start_h[l], e = g->level_start_h[l + 1];
        if (m2l_split)
            GQ_LAUNCH(ctx, k_m2m_split, gq_blocks((long long)(e - s) * P1, 128), 128, 0, E, s, e, T.tm2m2, g->M2.p);
        else if (g->m2m_level_start_h[l + 1] > g->m2m_level_start_h[l])
            GQ_LAUNCH(ctx, k_m2m_t, gq_blocks(g->m2m_level_start_h[l + 1] - g->m2m_level_start_h[l], 128 / P1),
                      (128 / P1) * P1, 0, E, (const int *)g->m2m_boxes, g->m2m_level_start_h[l],
                      g->m2m_level_start_h[l + 1], (const double2 *)T.tm2m, g->M.p);
    }
    mark(S_M2M, st);
    if (m2l_split)
        GQ_LAUNCH(ctx, k_from_dfl4, gq_blocks((long long)g->nbox * P1, 256), 256, 0, (long long)g->nbox * P1,
                  (const float4 *)g->M2, g->M.p);
    else if (split_w)   // multipoles as FP32 pairs for the pair List 3 far kernels
        GQ_LAUNCH(ctx, k_to_dfl4, gq_blocks((long long)g->nbox * P1, 256), 256, 0, (long long)g->nbox * P1,
                  (const double2 *)g->M, g->M2.p);
    // Stage 4
    if (g->n_far_boxes) {
        int G = P1 <= 16 ? 16 : 32;
        if (m2l_split) {
            size_t sm = sizeof(float2) * P1 * (P1 | 1);
            auto k16 = k_m2l_split<16>;
            auto k32 = k_m2l_split<32>;
            GQ_LAUNCH(ctx, (G == 16 ? k16 : k32), gq_blocks((long long)g->n_far_boxes * G, 128), 128, sm, E, SX,
                      g->n_far_boxes, (const int *)g->far_boxes, T.dtab2, T.logtab2, T.binom2, g->L2.p);
        } else if (gq_m2l_tc_supported(g)) {
            gq_m2l_tc(g, (const double2 *)g->M, g->L.p);   // FP64-accurate, on the tensor cores
        } else {
            size_t sm = sizeof(double) * P1 * P1;
            auto k16 = k_m2l<16>;
            auto k32 = k_m2l<32>;
            GQ_LAUNCH(ctx, (G == 16 ? k16 : k32), gq_blocks((long long)g->n_far_boxes * G, 128), 128, sm, E,
                      g->n_far_boxes, (const int *)g->far_boxes, (const double2 *)g->M, (const double2 *)T.dtab,
                      (const double *)T.logtab, g->L.p);
        }
    }
    mark(S_M2L, st);
    if (g->n_far_boxes) {
        // Stage 6b
        GQ_LAUNCH(ctx, k_p2l, gq_blocks((long long)g->n_far_boxes * 32, 128), 128, 0, E, g->n_far_boxes,
                  (const int *)g->far_boxes, g->L.p);
    }
    mark(S_P2L, st);
    // Stage 7 (in pairs wherever M2L runs in pairs: the FP64 P2L terms are
    // folded into the pair locals first, and the FP64 copy is made at the end)
    if (m2l_split)
        GQ_LAUNCH(ctx, k_add_to_dfl4, gq_blocks((long long)g->nbox * P1, 256), 256, 0, (long long)g->nbox * P1,
                  (const double2 *)g->L, g->L2.p);
    for (int l = 1; l < g->nlev; ++l) {
        int s = g->level_start_h[l], e = g->level_start_h[l + 1];
        if (m2l_split)
            GQ_LAUNCH(ctx, k_l2l_split, gq_blocks((long long)(e - s) * P1, 128), 128, 0, E, s, e, T.tl2l2, g->L2.p);
        else
            GQ_LAUNCH(ctx, k_l2l_t, gq_blocks(e - s, 128 / P1), (128 / P1) * P1, 0, E, s, e,
                      (const double2 *)T.tl2l, g->L.p);
    }
    if (m2l_split)
        GQ_LAUNCH(ctx, k_from_dfl4, gq_blocks((long long)g->nbox * P1, 256), 256, 0, (long long)g->nbox * P1,
                  (const float4 *)g->L2, g->L.p);
    if (f32)
        GQ_LAUNCH(ctx, k_to_float2, gq_blocks((long long)g->nbox * P1, 256), 256, 0, (long long)g->nbox * P1,
                  (const double2 *)g->M, g->M_f.p);
    mark(S_L2L, st);
    // Stage 5b
    if (g->nc && split_w) {
        dispatch_w_centres_split(ctx, E, SX, g->nc, (const int *)g->ctr_owner, Qb);
    } else if (g->nc) {
        if (gq_w_tc_supported(g)) gq_w_centres_tc(g, E.R, (const double2 *)g->M, T.logt, Qb);
        else dispatch_w_centres_q(ctx, E, g->nc, (const int *)g->ctr_owner, (const double2 *)g->M, Qb);
    }
    mark(S_WC, st);
    if (g->npt && !at_base) {
        if (f32)
            GQ_LAUNCH(ctx, k_w_points_f32, gq_blocks(g->npt, 128), 128, 0, E, X, g->npt, (const int *)g->pt_owner,
                      potb);
        else if (split_w)
            GQ_LAUNCH(ctx, k_w_points_split, gq_blocks(g->npt, 128), 128, 0, E, SX, g->npt, (const int *)g->pt_owner,
                      potb);
        else
            GQ_LAUNCH(ctx, k_w_points, gq_blocks(g->npt, 128), 128, 0, E, g->npt, (const int *)g->pt_owner,
                      (const double2 *)g->M, potb);
    }
    mark(S_WP, st);
    // Stage 8
    if (g->nc)
        if (m2l_split)
            dispatch_l2qbxl_split(ctx, E, SX, g->nc, (const int *)g->ctr_owner, (const float4 *)g->L2, Qb);
        else
            dispatch_l2qbxl_t(ctx, E, g->nc, (const int *)g->ctr_owner, (const double2 *)g->L, Qb);
    if (g->npt && !at_base)
        GQ_LAUNCH(ctx, k_l2p, gq_blocks(g->npt, 128), 128, 0, E, g->npt, (const int *)g->pt_owner, (const double2 *)g->L,
                  potb);
    mark(S_L2Q, st);
    // join the direct part, then evaluate at the targets
    GQ_CUDA(cudaStreamWaitEvent(st, g->ev_near, 0));
    // the direct part of the QBX coefficients: this call's, or formed beforehand
    // for several densities at once (gq_eval_multi)
    const bool use_pre = qn_pre && !f32 && !split;
    const double2 *qn_use = use_pre ? qn_pre : (const double2 *)g->Qn;
    g->qn_last = qn_use;
    if (fmm_only) {
        // the direct parts and the final sums are the caller's
    } else if (at_base) {
        if (g->nbase)
            GQ_LAUNCH(ctx, k_final_base, gq_blocks(g->nbase, 256), 256, 0, g->nbase, kernel, Qn, E.qc,
                      (const int *)g->ctr_pos, (const double *)g->base_xy, (const double *)g->base_n,
                      (const double2 *)g->sc_xy, (const double *)g->sc_r, (const double2 *)g->Q, qn_use,
                      *apply_identity, dens_dev, out_dev);
    } else if (g->nt)
        GQ_LAUNCH(ctx, k_final, gq_blocks(g->nt, 256), 256, 0, g->nt, kernel, Qn, E.qc, (const int *)g->t_kind,
                  (const int *)g->t_ctr, (const int *)g->ctr_pos, (const int *)T.tgt_ptpos, (const double *)g->tgt_xy,
                  (const int *)g->tgt_on, (const double *)g->base_n, (const double2 *)g->sc_xy,
                  (const double *)g->sc_r, (const double2 *)g->Q, qn_use, (const double *)g->pot,
                  (const double *)g->potn, out_dev);
    mark(S_END, st);
    ctx->launches += ctx2.launches;
    if (timed) {
        GQ_CUDA(cudaEventSynchronize(ev[S_END]));
        {
            int tce = gq_m2l_tc_error(g);
            GQ_REQUIRE(tce != 2, GQ_ERR_UNSUPPORTED, "tensor-core M2L: a List 2 entry outside the offset window");
            GQ_REQUIRE(tce == 0, GQ_ERR_TIMEOUT, "tensor-core M2L: a bounded wait gave up");
        }
        auto el = [&](int a, int b2) {
            float ms = 0;
            GQ_CUDA(cudaEventElapsedTime(&ms, ev[a], ev[b2]));
            return (double)ms;
        };
        stt->ms_total = el(S0, S_END);
        stt->ms_stage[0] = el(S0, S_STR);
        stt->ms_stage[1] = el(S_FMM, S_M2M);
        stt->ms_stage[2] = el(S_M2M, S_M2L);
        stt->ms_stage[3] = el(S_M2L, S_P2L);
        stt->ms_stage[4] = el(S_P2L, S_L2L);
        stt->ms_stage[5] = el(N_BEG, N_CTR);
        stt->ms_stage[6] = el(N_CTR, N_PT);
        stt->ms_stage[7] = el(S_L2L, S_WC);
        stt->ms_stage[8] = el(S_WC, S_WP);
        stt->ms_stage[9] = el(S_WP, S_L2Q);
        stt->ms_stage[10] = el(S_L2Q, S_END);
        stt->kernel_launches = ctx->launches - l0;
        for (int i = 0; i < NEV; ++i) cudaEventDestroy(ev[i]);
    }
    g->have_eval = true;
    g->last_kernel = kernel;
}

// Which FP64 translations the next gq_eval of g runs on the tensor cores (the
// conditions of the dispatch in gq_eval_all).
void gq_tensor_paths_impl(gq_geom *g, int *m2l_tc, int *m2qbxl_tc) {
    const bool mixed = g->prm.precision == GQ_PREC_MIXED || g->prm.precision == GQ_PREC_MIXED_FMM;
    const bool f32 = mixed && g->prm.eps >= kF32TierEps;
    const bool split = mixed && g->prm.eps >= 1e-12 && g->prm.eps < kF32TierEps;
    const bool split_w = (split || f32) && g->nlev <= 24;
    const bool m2l_split = g->prm.precision == GQ_PREC_MIXED_FMM && (split || f32) && g->prm.eps >= 1e-10;
    *m2l_tc = !m2l_split && gq_m2l_tc_supported(g) ? 1 : 0;
    *m2qbxl_tc = !split_w && g->nc > 0 && gq_w_tc_supported(g) ? 1 : 0;
}

// the evaluation views a batch item needs
static void gq_batch_geom_view(gq_geom *g, int kernel, BatchGeomDev &out) {
    EvalTables &T = get_tables(g);
    EvalView E{};
    E.R = g->root;
    E.P = g->prm.p_fmm;
    E.Q = g->prm.p_qbx;
    E.kernel = kernel == GQ_SP ? GQ_S : kernel;
    E.blev = g->blev; E.bix = g->bix; E.biy = g->biy; E.bparent = g->bparent; E.bchild = g->bchild;
    E.src_beg = g->src_beg; E.src_end = g->src_end;
    E.ctr_beg = g->ctr_beg; E.ctr_end = g->ctr_end; E.pt_beg = g->pt_beg; E.pt_end = g->pt_end;
    E.sub_src = g->sub_src; E.sub_tgt = g->sub_tgt;
    E.s_xy = g->s_xy; E.sc_xy = g->sc_xy; E.sc_r = g->sc_r; E.sp_xy = g->sp_xy;
    for (int i = 0; i < 6; ++i) { E.loff[i] = g->list_off[i]; E.lidx[i] = g->list_idx[i]; }
    E.binom = T.binom;
    E.qc = g->has_qc ? (const int *)g->q_ctr.p : nullptr;
    E.logt = T.logt;
    E.nwork_ctr = g->n_ctr_boxes;
    out.E = E;
    out.ctr_boxes = g->ctr_boxes;
    out.pt_boxes = g->pt_boxes;
    out.kernel = kernel;
    out.nt = g->nt;
    out.kind = g->t_kind;
    out.ctr = g->t_ctr;
    out.ctr_pos = g->ctr_pos;
    out.tgt_ptpos = T.tgt_ptpos;
    out.tgt_on = g->tgt_on;
    out.tgt_xy = g->tgt_xy;
    out.base_n = g->base_n;
}

// ------------------------------------------------------------------ persistent batch plan
struct gq_bplan {
    gq_ctx *ctx = nullptr;
    int kernel = 0, ndens = 0, q = 0, tile = 1, stall_geom = -1;
    std::vector<gq_geom *> geoms;
    std::vector<BatchGeomDev> hG;
    std::vector<const double *> dens;
    std::vector<double *> out;
    std::vector<std::unique_ptr<dbuf<double2>>> strm, Qn, Qf;
    std::vector<std::unique_ptr<dbuf<double>>> potn, potf;
    std::vector<std::unique_ptr<dbuf<unsigned int>>> qexp;
    dbuf<BatchGeomDev> G;
    dbuf<BatchItem> items;
    int nitems = 0;
    dbuf<int> next, done, err;
    const double *logt = nullptr;
};

bool gq_bplan_supported(const std::vector<gq_geom *> &geoms, int kernel) {
    if (geoms.empty() || (kernel != GQ_S && kernel != GQ_D && kernel != GQ_SP)) return false;
    const int q = geoms[0]->prm.p_qbx;
    if (q != 5 && q != 8) return false;
    for (auto *g : geoms)
        if (g->prm.precision != GQ_PREC_FP64 || g->prm.p_qbx != q || !g->built) return false;
    return true;
}

// The item list for `tile` target boxes per direct item (uploaded; the
// stream is synchronised, so no launch reads the old list afterwards).
// Every direct item precedes every final item.
void gq_bplan_retile(gq_bplan *P, int tile) {
    std::vector<BatchItem> near, fin;
    for (size_t i = 0; i < P->geoms.size(); ++i) {
        gq_geom *g = P->geoms[i];
        int items = 0;
        for (int j = 0; j < g->n_ctr_boxes; j += tile) {
            int d0 = 0;
            for (; d0 + 4 <= P->ndens; d0 += 4, ++items) near.push_back({BI_NEAR4, (int)i, j, d0});
            for (; d0 + 2 <= P->ndens; d0 += 2, ++items) near.push_back({BI_NEAR2, (int)i, j, d0});
            for (; d0 < P->ndens; ++d0, ++items) near.push_back({BI_NEAR1, (int)i, j, d0});
        }
        for (int j = 0; j < g->n_pt_boxes; ++j)
            for (int d = 0; d < P->ndens; ++d, ++items) near.push_back({BI_NEARPT, (int)i, j, d});
        for (int d = 0; d < P->ndens; ++d)
            for (int t = 0; t < g->nt; t += kNearThreads) fin.push_back({BI_FINAL, (int)i, t, d});
        P->hG[i].tile = tile;
        P->hG[i].items = items + ((int)i == P->stall_geom ? 1 : 0);
    }
    std::vector<BatchItem> all(near);
    all.insert(all.end(), fin.begin(), fin.end());
    P->tile = tile;
    P->nitems = (int)all.size();
    P->items.alloc(all.size());
    cudaStream_t st = P->ctx->stream;
    GQ_CUDA(cudaStreamSynchronize(st));
    GQ_CUDA(cudaMemcpyAsync(P->G.p, P->hG.data(), sizeof(BatchGeomDev) * P->hG.size(), cudaMemcpyHostToDevice, st));
    if (!all.empty())
        GQ_CUDA(cudaMemcpyAsync(P->items.p, all.data(), sizeof(BatchItem) * all.size(), cudaMemcpyHostToDevice, st));
    GQ_CUDA(cudaStreamSynchronize(st));
}

// Buffers and device descriptors for `kernel` and `ndens` densities of every
// geometry, and the item list for `tile`.  The geometries' evaluation tables
// must exist (an eager evaluation has run).  stall_geom >= 0 makes that
// geometry's final items wait for one item more than exist (a test of the
// bounded wait).
gq_bplan *gq_bplan_new(gq_ctx *ctx, int kernel, int ndens, const std::vector<gq_geom *> &geoms,
                       const double *const *dens, double *const *out, int tile, int stall_geom) {
    std::unique_ptr<gq_bplan> P(new gq_bplan);
    P->ctx = ctx;
    P->kernel = kernel;
    P->ndens = ndens;
    P->q = geoms[0]->prm.p_qbx;
    P->stall_geom = stall_geom;
    P->geoms = geoms;
    P->dens.assign(dens, dens + geoms.size());
    P->out.assign(out, out + geoms.size());
    const int Q1 = P->q + 1;
    P->hG.resize(geoms.size());
    for (size_t i = 0; i < geoms.size(); ++i) {
        gq_geom *g = geoms[i];
        P->strm.emplace_back(new dbuf<double2>);
        P->Qn.emplace_back(new dbuf<double2>);
        P->Qf.emplace_back(new dbuf<double2>);
        P->potn.emplace_back(new dbuf<double>);
        P->potf.emplace_back(new dbuf<double>);
        P->qexp.emplace_back(new dbuf<unsigned int>);
        const long long ss = g->nsrc, qs = (long long)g->nc * Q1, ps = g->npt > 0 ? g->npt : 1;
        P->strm[i]->alloc((size_t)ndens * ss);
        P->Qn[i]->alloc((size_t)ndens * qs);
        P->Qf[i]->alloc((size_t)ndens * qs);
        P->potn[i]->alloc((size_t)ndens * ps);
        P->potf[i]->alloc((size_t)ndens * ps);
        P->qexp[i]->alloc(ndens);
        BatchGeomDev &G = P->hG[i];
        gq_batch_geom_view(g, kernel, G);
        if (i == 0) P->logt = G.E.logt;
        G.strm = P->strm[i]->p;
        G.sstride = ss;
        G.Qn = P->Qn[i]->p;
        G.Qf = P->Qf[i]->p;
        G.qstride = qs;
        G.potn = P->potn[i]->p;
        G.potf = P->potf[i]->p;
        G.pstride = ps;
        G.qexp = P->qexp[i]->p;
        G.out = out[i];
    }
    P->G.alloc(P->hG.size());
    P->next.alloc(1);
    P->done.alloc(geoms.size());
    P->err.alloc(1);
    GQ_CUDA(cudaMemsetAsync(P->err.p, 0, sizeof(int), ctx->stream));
    gq_bplan_retile(P.get(), tile);
    return P.release();
}

int gq_bplan_tile(const gq_bplan *P) { return P->tile; }

void gq_bplan_free(gq_bplan *P) { delete P; }

// Record geometry i's evaluations without their direct parts: strengths and
// the FMM passes of every density into the plan's far buffers (on g->ctx).
void gq_bplan_fmm(gq_bplan *P, int i) {
    gq_geom *g = P->geoms[i];
    const int Q1 = P->q + 1;
    cudaStream_t st = g->ctx->stream;
    for (int d = 0; d < P->ndens; ++d) {
        EvalFar far{P->Qf[i]->p + (size_t)d * g->nc * Q1, P->potf[i]->p + (size_t)d * (g->npt > 0 ? g->npt : 1)};
        gq_eval_all(g, P->kernel, P->dens[i] + (size_t)d * g->nbase, nullptr, nullptr, nullptr, nullptr, &far);
        if (g->nsrc)
            GQ_CUDA(cudaMemcpyAsync(P->strm[i]->p + (size_t)d * g->nsrc, g->strength.p, sizeof(double2) * g->nsrc,
                                    cudaMemcpyDeviceToDevice, st));
        GQ_CUDA(cudaMemcpyAsync(P->qexp[i]->p + d, g->qexp.p, sizeof(unsigned int), cudaMemcpyDeviceToDevice, st));
    }
}

// Record the persistent launch (counters cleared first) on ctx's stream.
void gq_bplan_persistent(gq_bplan *P, gq_ctx *ctx, int grid, unsigned long long limit_ns) {
    cudaStream_t st = ctx->stream;
    GQ_CUDA(cudaMemsetAsync(P->next.p, 0, sizeof(int), st));
    GQ_CUDA(cudaMemsetAsync(P->done.p, 0, sizeof(int) * P->geoms.size(), st));
    const int kin = P->kernel == GQ_SP ? GQ_S : P->kernel;
#define GQ_BP(QV)                                                                                                 \
    if (P->q == QV) {                                                                                             \
        auto ks = k_batch_persistent<QV, GQ_S>;                                                                   \
        auto kd = k_batch_persistent<QV, GQ_D>;                                                                   \
        GQ_LAUNCH(ctx, (kin == GQ_D ? kd : ks), grid, kNearThreads, 0, (const BatchGeomDev *)P->G.p,             \
                  (const BatchItem *)P->items.p, P->nitems, P->logt, P->next.p, P->done.p, limit_ns, P->err.p);   \
        return;                                                                                                   \
    }
    GQ_BP(5)
    GQ_BP(8)
#undef GQ_BP
    throw gq_error{GQ_ERR_UNSUPPORTED, "persistent batch: p_qbx not compiled"};
}

// the device error word (synchronises): nonzero when a bounded wait gave up;
// cleared by the read
int gq_bplan_error(gq_bplan *P) {
    int h = 0;
    cudaStream_t st = P->ctx->stream;
    GQ_CUDA(cudaMemcpyAsync(&h, P->err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaMemsetAsync(P->err.p, 0, sizeof(int), st));
    GQ_CUDA(cudaStreamSynchronize(st));
    return h;
}

// Several densities on one geometry: the direct part of the QBX coefficients
// for all of them by the multi-density kernel (FP64 mode), then the rest of
// the evaluation per density.  The mixed-precision tiers evaluate one density
// after another.
void gq_eval_multi(gq_geom *g, int kernel, int nd, const double *const *dens, double *const *out) {
    const bool mixed = g->prm.precision == GQ_PREC_MIXED || g->prm.precision == GQ_PREC_MIXED_FMM;
    const bool f32 = mixed && g->prm.eps >= kF32TierEps;
    const bool split = mixed && g->prm.eps >= 1e-12 && g->prm.eps < kF32TierEps;
    if (nd <= 1 || f32 || split || g->n_ctr_boxes == 0) {
        for (int d = 0; d < nd; ++d) gq_eval_all(g, kernel, dens[d], out[d], nullptr);
        return;
    }
    gq_ctx *ctx = g->ctx;
    EvalTables &T = get_tables(g);
    int kin = kernel == GQ_SP ? GQ_S : kernel;
    const int Q1 = g->prm.p_qbx + 1;
    const long long sstride = g->nsrc, qstride = (long long)g->nc * Q1;
    g->strm.alloc((size_t)nd * g->nsrc);
    g->Qm.alloc((size_t)nd * qstride);
    for (int d = 0; d < nd; ++d)
        if (g->nsrc)
            GQ_LAUNCH(ctx, k_strengths, gq_blocks(g->nsrc, 256), 256, 0, g->nsrc, g->nu, g->nb, (const int *)g->src_perm,
                      (const double *)g->interp, dens[d], (const double *)g->s_w, (const double2 *)g->s_n, kin,
                      g->strm.p + d * sstride, (unsigned int *)nullptr);
    EvalView E{};
    E.R = g->root;
    E.P = g->prm.p_fmm;
    E.Q = g->prm.p_qbx;
    E.kernel = kin;
    E.blev = g->blev; E.bix = g->bix; E.biy = g->biy; E.bparent = g->bparent; E.bchild = g->bchild;
    E.src_beg = g->src_beg; E.src_end = g->src_end;
    E.ctr_beg = g->ctr_beg; E.ctr_end = g->ctr_end; E.pt_beg = g->pt_beg; E.pt_end = g->pt_end;
    E.sub_src = g->sub_src; E.sub_tgt = g->sub_tgt;
    E.s_xy = g->s_xy; E.sc_xy = g->sc_xy; E.sc_r = g->sc_r; E.sp_xy = g->sp_xy;
    for (int i = 0; i < 6; ++i) { E.loff[i] = g->list_off[i]; E.lidx[i] = g->list_idx[i]; }
    E.binom = T.binom;
    E.qc = g->has_qc ? (const int *)g->q_ctr.p : nullptr;
    E.logt = T.logt;
    int d0 = 0;
    for (; d0 + 4 <= nd; d0 += 4)
        dispatch_near_centres_multi<4>(ctx, E, g->n_ctr_boxes, g->ctr_boxes, g->strm.p + d0 * sstride, sstride,
                                       g->Qm.p + d0 * qstride, qstride);
    for (; d0 + 2 <= nd; d0 += 2)
        dispatch_near_centres_multi<2>(ctx, E, g->n_ctr_boxes, g->ctr_boxes, g->strm.p + d0 * sstride, sstride,
                                       g->Qm.p + d0 * qstride, qstride);
    for (; d0 < nd; ++d0)
        dispatch_near_centres_multi<1>(ctx, E, g->n_ctr_boxes, g->ctr_boxes, g->strm.p + d0 * sstride, sstride,
                                       g->Qm.p + d0 * qstride, qstride);
    for (int d = 0; d < nd; ++d) gq_eval_all(g, kernel, dens[d], out[d], nullptr, g->Qm.p + d * qstride);
}

void gq_export_qbx_impl(gq_geom *g, double *host) {
    int Q1 = g->prm.p_qbx + 1;
    dbuf<double2> tmp;
    tmp.alloc((size_t)g->nc * Q1);
    GQ_LAUNCH(g->ctx, k_export_qbx, gq_blocks((long long)g->nc * Q1, 256), 256, 0, g->nc, g->prm.p_qbx,
              (const int *)g->ctr_perm, (const double *)g->sc_r, (const double2 *)g->Q,
              g->qn_last ? g->qn_last : (const double2 *)g->Qn, tmp.p);
    GQ_CUDA(cudaMemcpyAsync(host, tmp.p, sizeof(double2) * g->nc * Q1, cudaMemcpyDeviceToHost, g->ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(g->ctx->stream));
}

// ====================================================================== no-allocation evaluation
// gq_eval_noalloc: the evaluation of gq_eval for callers that cannot allocate
// device memory at call time.  Its working memory (source strengths, box
// multipole and local expansions, QBX coefficients, point-target potentials,
// translation tables) lives in one file-scope device array of fixed size.
// It launches the kernels gq_eval launches in FP64 mode, with the direct and
// List 3 far/local parts of the QBX coefficients summed in one array.
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;   // 16 MiB per device, held until exit
constexpr size_t kNoAllocTableBytes = size_t(256) << 10;
// table offsets inside the array (bytes)
constexpr size_t kNaBinom = 0;                  // [64][64] doubles, 32 KiB
constexpr size_t kNaDtab = 32768;               // [121][32] double2, 61,952 B
constexpr size_t kNaLogtab = 98304;             // [121] doubles
constexpr size_t kNaLogt = 99328;               // GqLogTable
constexpr size_t kNaM2M = 131072;               // [4][kTN][kTN] double2, 61,504 B
constexpr size_t kNaL2L = 196608;               // [4][kTN][kTN] double2
constexpr size_t kNaQexp = 261888;              // one unsigned int, written by every call
static_assert(kNaLogt + sizeof(double) * kGqLogN <= kNaM2M, "log table overlaps the M2M matrices");
static_assert(kNaL2L + sizeof(double2) * 4 * kTN * kTN <= kNaQexp, "tables exceed their region");
static_assert(kNaQexp + 256 <= kNoAllocTableBytes, "exponent slot outside the table region");

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
    bool ready = false;
    unsigned char *base = nullptr;   // device address of g_noalloc_scratch
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

// Once per device, with that device current (checked): resolve the device
// address of the scratch array (host code cannot use the symbol itself) and
// store the read-only translation tables at its start.  The copies finish
// before the slot is marked ready, so no later launch on any stream can read
// a partly written table.
NoAllocDevice &noalloc_setup(int dev) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    GQ_REQUIRE(dev >= 0 && dev < 64, GQ_ERR_UNSUPPORTED, "gq_eval_noalloc: device index >= 64");
    int cur = -1;
    GQ_CUDA(cudaGetDevice(&cur));
    GQ_REQUIRE(cur == dev, GQ_ERR_STATE, "gq_eval_noalloc: the context's device must be the current device");
    NoAllocDevice &D = g_noalloc_dev[dev];
    if (D.ready) return D;
    void *ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) throw gq_error{GQ_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
    std::vector<double> bn, lt;
    std::vector<double2> dt, tm, tl;
    host_const_tables(bn, dt, lt, tm, tl);
    unsigned char *base = (unsigned char *)ptr;
    GQ_CUDA(cudaMemcpy(base + kNaBinom, bn.data(), sizeof(double) * bn.size(), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaMemcpy(base + kNaDtab, dt.data(), sizeof(double2) * dt.size(), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaMemcpy(base + kNaLogtab, lt.data(), sizeof(double) * lt.size(), cudaMemcpyHostToDevice));
    GqLogTable LT;
    gq_log_table_host(&LT);
    GQ_CUDA(cudaMemcpy(base + kNaLogt, &LT, sizeof(LT), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaMemcpy(base + kNaM2M, tm.data(), sizeof(double2) * tm.size(), cudaMemcpyHostToDevice));
    GQ_CUDA(cudaMemcpy(base + kNaL2L, tl.data(), sizeof(double2) * tl.size(), cudaMemcpyHostToDevice));
    std::vector<double> pc((GQ_MAX_PQBX + 1) * 33, 0.0);
    for (int m = 0; m <= GQ_MAX_PQBX; ++m)
        for (int k = 1; k <= 32; ++k) pc[m * 33 + k] = bn[(m + k - 1) * kBinN + (k - 1)];
    GQ_CUDA(cudaMemcpyToSymbol(c_pascal, pc.data(), sizeof(double) * pc.size()));
    GQ_CUDA(cudaDeviceSynchronize());
    D.base = base;
    D.ready = true;
    return D;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

size_t gq_noalloc_capacity() { return kNoAllocBytes - kNoAllocTableBytes; }

size_t gq_noalloc_need(const gq_geom *g) {
    size_t P1 = g->prm.p_fmm + 1, Q1 = g->prm.p_qbx + 1;
    return align256(sizeof(double2) * g->nsrc) + 2 * align256(sizeof(double2) * g->nbox * P1) +
           align256(sizeof(double2) * g->nc * Q1) + align256(sizeof(double) * (g->npt ? g->npt : 1)) +
           align256(sizeof(int) * (g->nt ? g->nt : 1));
}

void gq_eval_noalloc_impl(gq_geom *g, int kernel, const double *dens_dev, double *out_dev) {
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    size_t need = gq_noalloc_need(g);
    if (need > gq_noalloc_capacity())
        throw gq_error{GQ_ERR_UNSUPPORTED, "gq_eval_noalloc: problem needs " + std::to_string(need) +
                                               " bytes of scratch, the fixed array holds " +
                                               std::to_string(gq_noalloc_capacity())};
    NoAllocDevice &D = noalloc_setup(ctx->device);
    const double *binom = (const double *)(D.base + kNaBinom);
    const double2 *dtab = (const double2 *)(D.base + kNaDtab);
    const double *logtab = (const double *)(D.base + kNaLogtab);
    const double2 *tm2m = (const double2 *)(D.base + kNaM2M);
    const double2 *tl2l = (const double2 *)(D.base + kNaL2L);
    unsigned int *qexp = (unsigned int *)(D.base + kNaQexp);
    unsigned char *w = D.base + kNoAllocTableBytes;
    int P = g->prm.p_fmm, Qn = g->prm.p_qbx, P1 = P + 1, Q1 = Qn + 1;
    double2 *str = (double2 *)w;  w += align256(sizeof(double2) * g->nsrc);
    double2 *M = (double2 *)w;    w += align256(sizeof(double2) * g->nbox * P1);
    double2 *L = (double2 *)w;    w += align256(sizeof(double2) * g->nbox * P1);
    double2 *Qc = (double2 *)w;   w += align256(sizeof(double2) * g->nc * Q1);
    double *pot = (double *)w;    w += align256(sizeof(double) * (g->npt ? g->npt : 1));
    int *ptpos = (int *)w;
    int kin = kernel == GQ_SP ? GQ_S : kernel;
    EvalView E;
    E.R = g->root;
    E.P = P;
    E.Q = Qn;
    E.kernel = kin;
    E.blev = g->blev; E.bix = g->bix; E.biy = g->biy; E.bparent = g->bparent; E.bchild = g->bchild;
    E.src_beg = g->src_beg; E.src_end = g->src_end;
    E.ctr_beg = g->ctr_beg; E.ctr_end = g->ctr_end; E.pt_beg = g->pt_beg; E.pt_end = g->pt_end;
    E.sub_src = g->sub_src; E.sub_tgt = g->sub_tgt;
    E.s_xy = g->s_xy; E.str = str; E.sc_xy = g->sc_xy; E.sc_r = g->sc_r; E.sp_xy = g->sp_xy;
    for (int i = 0; i < 6; ++i) { E.loff[i] = g->list_off[i]; E.lidx[i] = g->list_idx[i]; }
    E.binom = binom;
    E.qc = g->has_qc ? (const int *)g->q_ctr.p : nullptr;
    E.logt = (const double *)(D.base + kNaLogt);
    E.qexp = qexp;

    // the array keeps the previous call's contents: clear the accumulators
    GQ_CUDA(cudaMemsetAsync(M, 0, sizeof(double2) * g->nbox * P1, st));
    GQ_CUDA(cudaMemsetAsync(L, 0, sizeof(double2) * g->nbox * P1, st));
    GQ_CUDA(cudaMemsetAsync(Qc, 0, sizeof(double2) * g->nc * Q1, st));
    if (g->npt) GQ_LAUNCH(ctx, k_tgt_ptpos, gq_blocks(g->npt, 256), 256, 0, g->npt, (const int *)g->pt_perm.p, ptpos);
    GQ_CUDA(cudaMemsetAsync(qexp, 0, sizeof(unsigned int), st));
    GQ_LAUNCH(ctx, k_strengths, gq_blocks(g->nsrc, 256), 256, 0, g->nsrc, g->nu, g->nb, (const int *)g->src_perm,
              (const double *)g->interp, dens_dev, (const double *)g->s_w, (const double2 *)g->s_n, kin, str, qexp);
    if (g->n_leaf_src) {
        auto k8 = k_p2m<8>;
        auto k16 = k_p2m<16>;
        auto k32 = k_p2m<GQ_MAX_PFMM>;
        GQ_LAUNCH(ctx, (P <= 8 ? k8 : P <= 16 ? k16 : k32), gq_blocks((long long)g->n_leaf_src * kP2MG, 128), 128, 0,
                  E, g->n_leaf_src, (const int *)g->leaf_src_boxes, M);
    }
    for (int l = g->nlev - 2; l >= 0; --l) {
        int s = g->level_start_h[l], e = g->level_start_h[l + 1];
        GQ_LAUNCH(ctx, k_m2m_t, gq_blocks(e - s, 128 / P1), (128 / P1) * P1, 0, E, (const int *)nullptr, s, e, tm2m,
                  M);
    }
    if (g->n_far_boxes) {
        size_t sm = sizeof(double) * P1 * P1;
        auto k16 = k_m2l<16>;
        auto k32 = k_m2l<32>;
        int G = P1 <= 16 ? 16 : 32;
        GQ_LAUNCH(ctx, (G == 16 ? k16 : k32), gq_blocks((long long)g->n_far_boxes * G, 128), 128, sm, E,
                  g->n_far_boxes, (const int *)g->far_boxes, (const double2 *)M, dtab, logtab, L);
        GQ_LAUNCH(ctx, k_p2l, gq_blocks((long long)g->n_far_boxes * 32, 128), 128, 0, E, g->n_far_boxes,
                  (const int *)g->far_boxes, L);
    }
    for (int l = 1; l < g->nlev; ++l) {
        int s = g->level_start_h[l], e = g->level_start_h[l + 1];
        GQ_LAUNCH(ctx, k_l2l_t, gq_blocks(e - s, 128 / P1), (128 / P1) * P1, 0, E, s, e, tl2l, L);
    }
    // the direct part writes the coefficients, the List 3 far and local parts add to them
    if (g->n_ctr_boxes) dispatch_near_centres(ctx, E, g->n_ctr_boxes, g->ctr_boxes, Qc);
    if (g->n_pt_boxes) {
        auto kd = k_near_points<GQ_D>;
        auto ks = k_near_points<GQ_S>;
        GQ_LAUNCH(ctx, (kin == GQ_D ? kd : ks), g->n_pt_boxes, kNearThreads, 0, E, g->n_pt_boxes,
                  (const int *)g->pt_boxes, pot);
    }
    if (g->nc) {
        dispatch_w_centres_q(ctx, E, g->nc, (const int *)g->ctr_owner, (const double2 *)M, Qc);
        dispatch_l2qbxl_t(ctx, E, g->nc, (const int *)g->ctr_owner, (const double2 *)L, Qc);
    }
    if (g->npt) {
        GQ_LAUNCH(ctx, k_w_points, gq_blocks(g->npt, 128), 128, 0, E, g->npt, (const int *)g->pt_owner,
                  (const double2 *)M, pot);
        GQ_LAUNCH(ctx, k_l2p, gq_blocks(g->npt, 128), 128, 0, E, g->npt, (const int *)g->pt_owner, (const double2 *)L,
                  pot);
    }
    if (g->nt)
        GQ_LAUNCH(ctx, k_final, gq_blocks(g->nt, 256), 256, 0, g->nt, kernel, Qn, E.qc, (const int *)g->t_kind,
                  (const int *)g->t_ctr, (const int *)g->ctr_pos, (const int *)ptpos, (const double *)g->tgt_xy,
                  (const int *)g->tgt_on, (const double *)g->base_n, (const double2 *)g->sc_xy,
                  (const double *)g->sc_r, (const double2 *)Qc, (const double2 *)nullptr, (const double *)pot,
                  (const double *)nullptr, out_dev);
}
