// gq_lists.cu -- interaction lists of Sec. 4.3.2 (Definitions 1-8) for the
// target-confinement quadtree, as CSR arrays over boxes: one enumeration pass
// writes each box's entries to fixed-capacity scratch rows and counts them, a
// prefix scan gives the CSR offsets, and a compaction copies the rows; if a
// row overflows, a second enumeration fills the CSR rows directly.
//
// Same-level neighbours come from a 5x5 window of box indices per box, built
// level by level from the parent's window (no searches).
//
// All relations are integer tests on box coordinates measured in units of
// half a level-30 box: a level-l box has half-width h = 2^(30-l) and centre
// (2 ix + 1) h.  With d the l-inf distance of two box centres:
//   adjacent(a, b)    d <= h_a + h_b        (closed squares intersect; a box
//                                            is adjacent to itself)
//   2-colleagues      same level, d <= 4 h
//   a < TCR(b)        d >= 3 h_a + (1 + t_f) h_b
//   TCR(a) < b        d >= 3 (1 + t_f) h_a + h_b
// with t_f = tf_num / tf_den handled exactly by clearing the denominator.
// With the disk-shaped TCR (tcr_shape 1, the appendix corrigendum's variant)
// the two separations are l-inf distances between a square and a disk,
// tested exactly as an l2 distance from the disk's centre to a grown square
// (disk_clear below).
//
// Which boxes carry which list: List 1, 3 close/far and 4 close for boxes
// owning targets (centres or point targets); List 2 and 4 far for boxes
// with targets anywhere in their subtree.  Only boxes with sources in their
// subtree are entered.
#include "gq_internal.cuh"

void gq_build_far_boxes(gq_geom *g);

namespace {

constexpr int kT = 128;
constexpr int kStack = 128;

struct TreeView {
    int nlev;
    const int *level_start;
    const uint64_t *bkey;
    const int *blev, *bix, *biy, *bparent;
    const int4 *bchild;
    const int *sub_src, *sub_tgt, *own_tgt;
    const int *win;   // [nbox][25]: box at (ix + dx, iy + dy) of the same level, dx, dy in [-2, 2], or -1
    int64_t tn, td;
    int shape;    // TCR: 0 square, 1 disk
    int demote;
};

__device__ __forceinline__ int child_q(int4 c, int q) { return q == 0 ? c.x : q == 1 ? c.y : q == 2 ? c.z : c.w; }

struct IBox {
    int l;
    int64_t x, y;  // box coordinates at level l
};

__device__ __forceinline__ int64_t ih(int l) { return (int64_t)1 << (GQ_KEYBITS - l); }
__device__ __forceinline__ int64_t i64abs(int64_t a) { return a < 0 ? -a : a; }
__device__ __forceinline__ int64_t dcen(IBox a, IBox b) {
    int64_t dx = i64abs((2 * a.x + 1) * ih(a.l) - (2 * b.x + 1) * ih(b.l));
    int64_t dy = i64abs((2 * a.y + 1) * ih(a.l) - (2 * b.y + 1) * ih(b.l));
    return dx > dy ? dx : dy;
}
__device__ __forceinline__ bool adjacent(IBox a, IBox b) { return dcen(a, b) <= ih(a.l) + ih(b.l); }
// Disk-shaped TCR: the l-inf distance between a square S(c_s, h) and a disk
// D(c_d, rho) is at least s exactly when the l2 distance from c_d to the
// closed square S(c_s, h + s) is at least rho, i.e.
//   max(X - T, 0)^2 + max(Y - T, 0)^2 >= rho^2,   T = h + s,
// X, Y the absolute centre differences; exact with 128-bit squares.
__device__ __forceinline__ bool disk_clear(int64_t X, int64_t Y, int64_t T, int64_t rho) {
    const __int128 ex = X > T ? (__int128)(X - T) : (__int128)0;
    const __int128 ey = Y > T ? (__int128)(Y - T) : (__int128)0;
    return ex * ex + ey * ey >= (__int128)rho * rho;
}
__device__ __forceinline__ int64_t dax(IBox a, IBox b) { return i64abs((2 * a.x + 1) * ih(a.l) - (2 * b.x + 1) * ih(b.l)); }
__device__ __forceinline__ int64_t day(IBox a, IBox b) { return i64abs((2 * a.y + 1) * ih(a.l) - (2 * b.y + 1) * ih(b.l)); }
// a < TCR(b): l-inf distance between a and TCR(b) >= 2|a|
__device__ __forceinline__ bool sep_a_tcrb(const TreeView &T, IBox a, IBox b) {
    if (T.shape == 1)
        return disk_clear(T.td * dax(a, b), T.td * day(a, b), 3 * T.td * ih(a.l), (T.td + T.tn) * ih(b.l));
    return T.td * dcen(a, b) >= 3 * T.td * ih(a.l) + (T.td + T.tn) * ih(b.l);
}
// TCR(a) < b: l-inf distance between TCR(a) and b >= 2|a|(1 + t_f)
__device__ __forceinline__ bool sep_tcra_b(const TreeView &T, IBox a, IBox b) {
    if (T.shape == 1)
        return disk_clear(T.td * dax(a, b), T.td * day(a, b), T.td * ih(b.l) + 2 * (T.td + T.tn) * ih(a.l),
                          (T.td + T.tn) * ih(a.l));
    return T.td * dcen(a, b) >= 3 * (T.td + T.tn) * ih(a.l) + T.td * ih(b.l);
}
__device__ __forceinline__ IBox ibox(const TreeView &T, int b) { return IBox{T.blev[b], T.bix[b], T.biy[b]}; }
__device__ __forceinline__ bool is_leaf(const TreeView &T, int b) {
    int4 c = T.bchild[b];
    return c.x < 0 && c.y < 0 && c.z < 0 && c.w < 0;
}

// 5x5 windows of same-level boxes, one level at a time from the parent's
// window: the box at (X, Y) is child (X & 1) + 2 (Y & 1) of the parent-level
// box at (X >> 1, Y >> 1), which lies in the parent's window.
__global__ void k_windows(int lstart, int lend, const int *__restrict__ bparent, const int *__restrict__ bix,
                          const int *__restrict__ biy, const int4 *__restrict__ bchild, int *__restrict__ win) {
    int b = lstart + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= lend) return;
    int p = bparent[b];
    int x = bix[b], y = biy[b];
    int *w = win + (size_t)b * 25;
    if (p < 0) {
        for (int i = 0; i < 25; ++i) w[i] = -1;
        w[12] = b;
        return;
    }
    const int *pw = win + (size_t)p * 25;
    int px = x >> 1, py = y >> 1;
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            int X = x + dx, Y = y + dy, d = -1;
            if (X >= 0 && Y >= 0) {
                int q = pw[((Y >> 1) - py + 2) * 5 + ((X >> 1) - px + 2)];
                if (q >= 0) d = child_q(bchild[q], (X & 1) | ((Y & 1) << 1));
            }
            w[(dy + 2) * 5 + dx + 2] = d;
        }
}

__device__ __forceinline__ int wlook(const TreeView &T, int b, int dx, int dy) {
    return T.win[(size_t)b * 25 + (dy + 2) * 5 + dx + 2];
}

// Level restriction (Sec. 4.6 remark): leaf b is in violation when a box two
// levels deeper touches it; such a box is a grandchild of one of b's eight
// same-level neighbours (its level-l ancestor touches b and is not b).
__global__ void k_balance_check(int nbox, int max_level, const int *__restrict__ blev, const int *__restrict__ bix,
                                const int *__restrict__ biy, const int4 *__restrict__ bchild,
                                const uint64_t *__restrict__ bkey, const int *__restrict__ win,
                                const int *__restrict__ belig, uint64_t *__restrict__ out, int *__restrict__ nout) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int4 c = bchild[b];
    if (c.x >= 0 || c.y >= 0 || c.z >= 0 || c.w >= 0) return;   // not a leaf
    const int l = blev[b];
    if (belig[b] <= 0 || l >= max_level) return;
    IBox me{l, bix[b], biy[b]};
    bool viol = false;
    for (int dy = -1; dy <= 1 && !viol; ++dy)
        for (int dx = -1; dx <= 1 && !viol; ++dx) {
            if (dx == 0 && dy == 0) continue;
            int n = win[(size_t)b * 25 + (dy + 2) * 5 + dx + 2];
            if (n < 0) continue;
            int4 nc = bchild[n];
            int ch[4] = {nc.x, nc.y, nc.z, nc.w};
            for (int q = 0; q < 4 && !viol; ++q) {
                if (ch[q] < 0) continue;
                int4 gc = bchild[ch[q]];
                int gg[4] = {gc.x, gc.y, gc.z, gc.w};
                for (int r = 0; r < 4; ++r)
                    if (gg[r] >= 0 && adjacent(IBox{l + 2, bix[gg[r]], biy[gg[r]]}, me)) {
                        viol = true;
                        break;
                    }
            }
        }
    if (viol) out[atomicAdd(nout, 1)] = ((uint64_t)l << 60) | bkey[b];
}

enum { LU = 0, LV = 1, LWC = 2, LWF = 3, LXC = 4, LXF = 5 };
// stack modes
enum { M_OWN = 0, M_COLL = 1, M_FARCLOSE = 2, M_LEAVES_WC = 3 };

// Row capacities of the one-pass fill (entries per box and list): List 2 holds
// at most 75 boxes, List 4 close 42 and List 4 far 63; Lists 1 and 3 have no
// fixed bound, and a box that exceeds a capacity sends the build to the
// second enumeration pass, which fills the exact CSR rows.
constexpr int kRowCap[6] = {64, 80, 128, 96, 48, 64};

enum { E_COUNT = 0, E_FILL = 1, E_ROWS = 2 };

// scratch rows: list i's rows (cap[i] slots each) start at base[i]
struct RowTable {
    int cap[6];
    long long base[6];
};

struct Emitter {
    int mode;   // E_COUNT: count only; E_FILL: write the CSR rows; E_ROWS: write capped scratch rows
    int cnt[6];
    int cap[6];
    int *dst[6];
    __device__ void emit(int which, int d) {
        int c = cnt[which]++;
        if (mode == E_FILL || (mode == E_ROWS && c < cap[which])) dst[which][c] = d;
    }
};

__device__ void push_children(const TreeView &T, int b, int mode, int *stk, int &sp, int *err) {
    int4 c = T.bchild[b];
    int cc[4] = {c.x, c.y, c.z, c.w};
    for (int q = 3; q >= 0; --q) {
        if (cc[q] < 0) continue;
        if (sp >= kStack) { *err = 1; return; }
        stk[sp++] = (cc[q] << 3) | mode;
    }
}

// Depth-first walk of the boxes on the stack.  Modes: M_OWN collects the
// source leaves of b's subtree (List 1); M_COLL descends a 2-colleague's
// subtree through boxes adjacent to b (adjacent leaves -> List 1, the first
// non-adjacent boxes -> List 3, Def. 3); M_FARCLOSE splits a List 3 box into
// List 3 far (d < TCR(b), Def. 5) or, through its descendants, List 3 close
// leaves (Def. 4), demoting far boxes with fewer than `demote` sources to
// their leaves (Remark 1); M_LEAVES_WC emits the leaves of a demoted box.
__device__ void drain(const TreeView &T, IBox B, int *stk, int &sp, Emitter &E, int *err) {
    while (sp > 0) {
        int e = stk[--sp];
        int d = e >> 3, mode = e & 7;
        if (T.sub_src[d] == 0) continue;
        bool leaf = is_leaf(T, d);
        IBox D = ibox(T, d);
        if (mode == M_OWN) {
            if (leaf) E.emit(LU, d);
            else push_children(T, d, M_OWN, stk, sp, err);
        } else if (mode == M_COLL) {
            if (!adjacent(D, B)) {
                if (sp >= kStack) { *err = 1; return; }
                stk[sp++] = (d << 3) | M_FARCLOSE;
            } else if (leaf) {
                E.emit(LU, d);
            } else {
                push_children(T, d, M_COLL, stk, sp, err);
            }
        } else if (mode == M_FARCLOSE) {
            if (sep_a_tcrb(T, D, B)) {
                if (T.sub_src[d] < T.demote) {
                    if (sp >= kStack) { *err = 1; return; }
                    stk[sp++] = (d << 3) | M_LEAVES_WC;
                } else {
                    E.emit(LWF, d);
                }
            } else if (leaf) {
                E.emit(LWC, d);
            } else {
                push_children(T, d, M_FARCLOSE, stk, sp, err);
            }
        } else {
            if (leaf) E.emit(LWC, d);
            else push_children(T, d, M_LEAVES_WC, stk, sp, err);
        }
        if (*err) return;
    }
}

__device__ void enumerate(const TreeView &T, int b, Emitter &E, int *err) {
    if (T.sub_tgt[b] == 0) return;
    const bool tb = T.own_tgt[b] > 0;
    const IBox B = ibox(T, b);
    const int l = B.l;
    int stk[kStack];
    int sp = 0;

    // ancestors of b by level: anc[m] is the level-m box containing b
    int anc[GQ_KEYBITS + 1];
    anc[l] = b;
    for (int m = l; m > 0; --m) anc[m - 1] = T.bparent[anc[m]];

    // ---- List 2: children of the 2-colleagues of parent(b), 2-well-separated from b
    if (l >= 1) {
        int64_t px = B.x >> 1, py = B.y >> 1;
        for (int64_t jy = 2 * (py - 2); jy <= 2 * (py + 2) + 1; ++jy)
            for (int64_t jx = 2 * (px - 2); jx <= 2 * (px + 2) + 1; ++jx) {
                if (i64abs(jx - B.x) <= 2 && i64abs(jy - B.y) <= 2) continue;
                if (jx < 0 || jy < 0) continue;
                int q = wlook(T, anc[l - 1], (int)((jx >> 1) - px), (int)((jy >> 1) - py));
                int d = q >= 0 ? child_q(T.bchild[q], (int)((jx & 1) | ((jy & 1) << 1))) : -1;
                if (d >= 0 && T.sub_src[d] > 0) E.emit(LV, d);
            }
    }

    if (tb) {
        // ---- List 1 (a): leaves of b's own subtree, b included
        stk[sp++] = (b << 3) | M_OWN;
        drain(T, B, stk, sp, E, err);
        if (*err) return;
        // ---- List 1 (b): coarser or same-level leaves adjacent to b
        for (int m = 0; m <= l; ++m) {
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy) continue;
                    int d = wlook(T, anc[m], dx, dy);
                    if (d < 0 || !is_leaf(T, d) || T.sub_src[d] == 0) continue;
                    if (adjacent(ibox(T, d), B)) E.emit(LU, d);
                }
        }
    }
    // ---- descendants of the 2-colleagues: finer adjacent leaves (List 1) and List 3
    for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
            if (!dx && !dy) continue;
            int t = wlook(T, b, dx, dy);
            if (!tb || t < 0 || is_leaf(T, t) || T.sub_src[t] == 0) continue;
            push_children(T, t, M_COLL, stk, sp, err);
            drain(T, B, stk, sp, E, err);
            if (*err) return;
        }

    // ---- List 4 close / far: source leaves that are 2-colleagues of b or of an ancestor
    for (int m = 0; m <= l; ++m) {
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                if (!dx && !dy) continue;
                int d = wlook(T, anc[m], dx, dy);
                if (d < 0 || !is_leaf(T, d) || T.sub_src[d] == 0) continue;
                IBox D = ibox(T, d);
                bool in_upto_l = false, in_upto_lm1 = false, in_b = false;
                for (int j = m; j <= l; ++j) {
                    IBox W{j, B.x >> (l - j), B.y >> (l - j)};
                    bool mem;
                    if (j == m) {
                        mem = !adjacent(D, W);                        // Def. 6, first part
                    } else {
                        IBox Wp{j - 1, B.x >> (l - j + 1), B.y >> (l - j + 1)};
                        mem = adjacent(D, Wp) && !adjacent(D, W);   // Def. 6, second part
                    }
                    if (mem) {
                        in_upto_l = true;
                        if (j <= l - 1) in_upto_lm1 = true;
                        if (j == l) in_b = true;
                    }
                }
                bool far_b = sep_tcra_b(T, B, D);
                if (tb && in_upto_l && !far_b) E.emit(LXC, d);      // Def. 7
                bool close_par = false;
                if (l >= 1) {
                    IBox Pb{l - 1, B.x >> 1, B.y >> 1};
                    close_par = in_upto_lm1 && !sep_tcra_b(T, Pb, D);
                }
                if ((in_b || close_par) && far_b) E.emit(LXF, d);   // Def. 8
            }
    }
}

struct ListPtrs {
    const int *off[6];
    int *idx[6];
    int *cnt[6];
};

// One enumeration per box.  E_ROWS (the default pass): entries go to row b of
// the scratch table and the counts to cnt; a count above its row's capacity
// raises *ovf.  E_COUNT counts only; E_FILL writes the CSR rows at off[i][b].
__global__ void k_lists(TreeView T, int nbox, int mode, ListPtrs LP, RowTable R, int *__restrict__ rows, int *err,
                        int *ovf) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    Emitter E;
    E.mode = mode;
    for (int i = 0; i < 6; ++i) {
        E.cnt[i] = 0;
        E.cap[i] = R.cap[i];
        if (mode == E_FILL) E.dst[i] = LP.idx[i] + LP.off[i][b];
        else if (mode == E_ROWS) E.dst[i] = rows + R.base[i] + (long long)b * R.cap[i];
    }
    int e = 0;
    enumerate(T, b, E, &e);
    if (e) atomicExch(err, 1);
    if (mode != E_FILL) {
        bool over = false;
        for (int i = 0; i < 6; ++i) {
            LP.cnt[i][b] = E.cnt[i];
            over |= E.cnt[i] > R.cap[i];
        }
        if (over && mode == E_ROWS) atomicExch(ovf, 1);
    }
}

// the scratch rows into the CSR arrays: one warp per box
__global__ void k_lists_compact(int nbox, ListPtrs LP, RowTable R, const int *__restrict__ rows) {
    int b = (int)(((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (b >= nbox) return;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const int o = LP.off[i][b], n = LP.off[i][b + 1] - o;
        const int *src = rows + R.base[i] + (long long)b * R.cap[i];
        for (int j = lane; j < n; j += 32) LP.idx[i][o + j] = src[j];
    }
}

}  // namespace

void gq_balance_violations(gq_geom *g, const int *belig, std::vector<uint64_t> &out) {
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    int nbox = g->nbox;
    dbuf<int> win, n;
    dbuf<uint64_t> keys;
    win.alloc((size_t)nbox * 25);
    keys.alloc(nbox);
    n.alloc(1);
    for (int l = 0; l < g->nlev; ++l) {
        int s0 = g->level_start_h[l], s1 = g->level_start_h[l + 1];
        GQ_LAUNCH(ctx, k_windows, gq_blocks(s1 - s0, kT), kT, 0, s0, s1, (const int *)g->bparent.p,
                  (const int *)g->bix.p, (const int *)g->biy.p, (const int4 *)g->bchild.p, win.p);
    }
    GQ_CUDA(cudaMemsetAsync(n.p, 0, sizeof(int), st));
    GQ_LAUNCH(ctx, k_balance_check, gq_blocks(nbox, kT), kT, 0, nbox, g->prm.max_level, (const int *)g->blev.p,
              (const int *)g->bix.p, (const int *)g->biy.p, (const int4 *)g->bchild.p, (const uint64_t *)g->bkey.p,
              (const int *)win.p, belig, keys.p, n.p);
    int h = 0;
    GQ_CUDA(cudaMemcpyAsync(&h, n.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaStreamSynchronize(st));
    out.resize(h);
    if (h) {
        GQ_CUDA(cudaMemcpyAsync(out.data(), keys.p, sizeof(uint64_t) * h, cudaMemcpyDeviceToHost, st));
        GQ_CUDA(cudaStreamSynchronize(st));
    }
}

void gq_build_lists(gq_geom *g) {
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    TreeView T;
    T.nlev = g->nlev;
    T.level_start = g->level_start.p;
    T.bkey = g->bkey.p;
    T.blev = g->blev.p;
    T.bix = g->bix.p;
    T.biy = g->biy.p;
    T.bchild = g->bchild.p;
    T.bparent = g->bparent.p;
    T.sub_src = g->sub_src.p;
    T.sub_tgt = g->sub_tgt.p;
    T.own_tgt = g->own_tgt.p;
    T.tn = g->prm.tf_num;
    T.td = g->prm.tf_den;
    T.shape = g->prm.tcr_shape;
    T.demote = g->prm.w3_demote;
    int nbox = g->nbox;
    dbuf<int> win;
    win.alloc((size_t)nbox * 25);
    for (int l = 0; l < g->nlev; ++l) {
        int s0 = g->level_start_h[l], s1 = g->level_start_h[l + 1];
        GQ_LAUNCH(ctx, k_windows, gq_blocks(s1 - s0, kT), kT, 0, s0, s1, (const int *)g->bparent.p,
                  (const int *)g->bix.p, (const int *)g->biy.p, (const int4 *)g->bchild.p, win.p);
    }
    T.win = win.p;
    dbuf<int> cnt[6], err, tmp, rows;
    ListPtrs LP;
    for (int i = 0; i < 6; ++i) {
        cnt[i].alloc(nbox);
        g->list_off[i].alloc(nbox + 1);
        LP.off[i] = g->list_off[i].p;
        LP.cnt[i] = cnt[i].p;
        LP.idx[i] = nullptr;
    }
    // err[0]: a traversal stack overflowed; err[1]: a scratch row overflowed
    err.alloc(2);
    GQ_CUDA(cudaMemsetAsync(err.p, 0, 2 * sizeof(int), st));
    tmp.alloc(gq_scan_tmp_size(nbox));
    RowTable R;
    long long rows_n = 0;
    for (int i = 0; i < 6; ++i) {
        R.cap[i] = g->list_row_cap > 0 ? g->list_row_cap : kRowCap[i];
        R.base[i] = rows_n;
        rows_n += (long long)nbox * R.cap[i];
    }
    rows.alloc((size_t)rows_n);
    GQ_LAUNCH(ctx, k_lists, gq_blocks(nbox, kT), kT, 0, T, nbox, (int)E_ROWS, LP, R, rows.p, err.p, err.p + 1);
    int tot[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 6; ++i) {
        gq_exclusive_scan(ctx, cnt[i].p, g->list_off[i].p, nbox, tmp.p);
        GQ_CUDA(cudaMemcpyAsync(&tot[i], g->list_off[i].p + nbox, sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    int herr[2] = {0, 0};
    GQ_CUDA(cudaMemcpyAsync(herr, err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < 6; ++i) {
        g->list_size[i] = tot[i];
        g->list_idx[i].alloc(tot[i]);
        LP.idx[i] = g->list_idx[i].p;
    }
    if (herr[1] == 0) {
        GQ_LAUNCH(ctx, k_lists_compact, gq_blocks((long long)nbox * 32, 256), 256, 0, nbox, LP, R, (const int *)rows.p);
    } else {   // a row overflowed: enumerate again into the exact CSR rows
        GQ_LAUNCH(ctx, k_lists, gq_blocks(nbox, kT), kT, 0, T, nbox, (int)E_FILL, LP, R, (int *)nullptr, err.p,
                  err.p + 1);
        GQ_CUDA(cudaMemcpyAsync(herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        GQ_CUDA(cudaStreamSynchronize(st));
    }
    g->lists_fill_passes = herr[1] == 0 ? 1 : 2;
    int herr0 = herr[0];
    GQ_REQUIRE(herr0 == 0, GQ_ERR_UNSUPPORTED, "list construction: traversal stack overflow");
    gq_build_far_boxes(g);
}
