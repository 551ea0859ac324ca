// gq_tree.cu -- Stage 1 of the GIGAQBX Algorithm (Sec. 4.4) and its inputs:
// QBX centres (Sec. 2.2.2), target association, the root box, Morton keys,
// each centre's deepest admissible level (target confinement region, Sec.
// 4.3) and the level-by-level subdivision (Sec. 4.3: a box subdivides when it
// owns more than n_max particles eligible for its children; empty children
// are pruned; a centre whose disk does not fit the child's TCR stays).
//
// Compiled with -fmad=false: every floating-point operation that decides an
// integer result (keys, levels, association) rounds separately, so the
// results are reproducible bit for bit by any IEEE-754 implementation that
// performs the same operations.
#include <math.h>

#include <algorithm>
#include <memory>

#include <stdio.h>
#include <stdlib.h>

#include <utility>
#include <vector>

#include "gq_internal.cuh"

namespace {

constexpr int kT = 256;

// ------------------------------------------------------------------ A2: centres
__global__ void k_centres(int nbase, int nb, const double *__restrict__ base_xy, const double *__restrict__ base_n,
                          const double *__restrict__ panel_len, double radius_factor, double *__restrict__ c_xy,
                          double *__restrict__ c_r) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nbase) return;
    double r = radius_factor * panel_len[i / nb];
    for (int side = 0; side < 2; ++side) {
        double sg = side ? 1.0 : -1.0;
        int c = 2 * i + side;
        c_xy[2 * c] = base_xy[2 * i] + (sg * r) * base_n[2 * i];
        c_xy[2 * c + 1] = base_xy[2 * i + 1] + (sg * r) * base_n[2 * i + 1];
        c_r[c] = r;
    }
}

// ------------------------------------------------------------------ reductions
// mode 0: centres (x, y, r) -> min/max of x, y and max r
// mode 1: root box extent over sources, point targets and centre disks
struct Ext {
    double x0, x1, y0, y1, rmax;
};
__device__ void ext_merge(Ext &a, const Ext &b) {
    a.x0 = fmin(a.x0, b.x0); a.x1 = fmax(a.x1, b.x1);
    a.y0 = fmin(a.y0, b.y0); a.y1 = fmax(a.y1, b.y1);
    a.rmax = fmax(a.rmax, b.rmax);
}

__global__ void k_extent(int mode, int nsrc, const double *__restrict__ up_xy, int npt, const int *__restrict__ pt_tgt,
                         const double *__restrict__ tgt_xy, int nc, const double *__restrict__ c_xy,
                         const double *__restrict__ c_r, Ext *__restrict__ part) {
    Ext e{INFINITY, -INFINITY, INFINITY, -INFINITY, 0.0};
    long long total = mode == 0 ? nc : (long long)nsrc + npt + nc;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        Ext v;
        if (mode == 0) {
            double x = c_xy[2 * i], y = c_xy[2 * i + 1];
            v = Ext{x, x, y, y, c_r[i]};
        } else if (i < nsrc) {
            double x = up_xy[2 * i], y = up_xy[2 * i + 1];
            v = Ext{x, x, y, y, 0.0};
        } else if (i < nsrc + npt) {
            int t = pt_tgt[i - nsrc];
            double x = tgt_xy[2 * t], y = tgt_xy[2 * t + 1];
            v = Ext{x, x, y, y, 0.0};
        } else {
            long long c = i - nsrc - npt;
            double x = c_xy[2 * c], y = c_xy[2 * c + 1], r = c_r[c];
            v = Ext{x - r, x + r, y - r, y + r, r};
        }
        ext_merge(e, v);
    }
    __shared__ Ext sh[kT];
    sh[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) ext_merge(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

Ext device_extent(gq_geom *g, int mode) {
    const int nblk = 304;
    dbuf<Ext> part;
    part.alloc(nblk);
    GQ_LAUNCH(g->ctx, k_extent, nblk, kT, 0, mode, g->nsrc, (const double *)g->up_xy, g->npt,
              (const int *)g->pt_tgt, (const double *)g->tgt_xy, g->nc, (const double *)g->c_xy,
              (const double *)g->c_r, part.p);
    std::vector<Ext> h(nblk);
    GQ_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(Ext) * nblk, cudaMemcpyDeviceToHost, g->ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(g->ctx->stream));
    Ext e{INFINITY, -INFINITY, INFINITY, -INFINITY, 0.0};
    for (auto &v : h) {
        e.x0 = fmin(e.x0, v.x0); e.x1 = fmax(e.x1, v.x1);
        e.y0 = fmin(e.y0, v.y0); e.y1 = fmax(e.y1, v.y1);
        e.rmax = fmax(e.rmax, v.rmax);
    }
    return e;
}

// ------------------------------------------------------------------ A3: association
// Grid cells of the association search: cell index floor((x - x0) * inv_cell)
// for centres and targets alike.  The map is monotone in x and within a few
// ulps of (x - x0) / cell, so a centre within 0.8 cell widths of a target
// (the search radius is below that) is in a cell adjacent to the target's.
__global__ void k_cell_of_centre(int nc, const double *__restrict__ c_xy, double x0, double y0, double inv_cell,
                                 int ncx, int ncy, uint32_t *__restrict__ key, int *__restrict__ val) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nc) return;
    int gx = (int)floor((c_xy[2 * c] - x0) * inv_cell), gy = (int)floor((c_xy[2 * c + 1] - y0) * inv_cell);
    gx = min(max(gx, 0), ncx - 1);
    gy = min(max(gy, 0), ncy - 1);
    key[c] = (uint32_t)(gy * ncx + gx);
    val[c] = c;
}

// targets in grid-cell order, so that a warp of k_associate walks the same
// cells and candidate lists: off-surface targets by cell (targets outside the
// searched grid after them), on-surface targets last
__global__ void k_cell_of_target(int nt, const double *__restrict__ tgt_xy, const int *__restrict__ tgt_on, double x0,
                                 double y0, double inv_cell, int ncx, int ncy, uint32_t *__restrict__ key,
                                 int *__restrict__ val) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    uint32_t ncell = (uint32_t)ncx * (uint32_t)ncy, k;
    if (tgt_on[t] >= 0) {
        k = ncell + 1;
    } else {
        double fgx = floor((tgt_xy[2 * t] - x0) * inv_cell), fgy = floor((tgt_xy[2 * t + 1] - y0) * inv_cell);
        if (fgx >= -1 && fgx <= ncx && fgy >= -1 && fgy <= ncy) {
            int gx = min(max((int)fgx, 0), ncx - 1), gy = min(max((int)fgy, 0), ncy - 1);
            k = (uint32_t)gy * (uint32_t)ncx + (uint32_t)gx;
        } else {
            k = ncell;
        }
    }
    key[t] = k;
    val[t] = t;
}

// centres in cell order as float (x, y, threshold, 1/r): the threshold bounds
// the squared distance of any centre the exact test could accept
__global__ void k_cell_floats(int n, const int *__restrict__ items, const double *__restrict__ c_xy,
                              const double *__restrict__ c_r, double slack, double delta, float4 *__restrict__ cf) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int c = items[k];
    double lim = slack * c_r[c] * 1.001 + delta;
    cf[k] = make_float4((float)c_xy[2 * c], (float)c_xy[2 * c + 1], __double2float_ru(lim * lim * 1.001),
                        (float)(1.0 / c_r[c]));
}

__global__ void k_cell_bounds(int n, const uint32_t *__restrict__ key, int *__restrict__ start, int *__restrict__ end) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t k = key[i];
    if (i == 0 || key[i - 1] != k) start[k] = i;
    if (i == n - 1 || key[i + 1] != k) end[k] = i + 1;
}

// On-surface targets use the centre pair of their base node; an off-surface
// target takes the centre minimising |t-c|^2/r^2 (lowest id on ties) if that
// ratio is <= slack^2, else it is a point target.
//
// The candidates of the 3 x 3 cells around the target are scanned twice in
// FP32.  With df the FP32 distance (|df - |t - c|| <= delta), every candidate
// has rho = |t - c| / r in [lo, hi] = [(df - delta) / r, (df + delta) / r]
// (each widened by 1e-5 for the FP32 roundings).  The first scan finds the
// smallest hi; the exact minimiser, and every candidate tied with it, has
// lo <= rho <= rho_min <= that bound, so the second scan evaluates the exact
// FP64 key only for candidates with lo at or below it.
__global__ void k_associate(int nt, const int *__restrict__ order, const double *__restrict__ tgt_xy,
                            const int *__restrict__ tgt_on,
                            const double *__restrict__ c_xy, const double *__restrict__ c_r,
                            const int *__restrict__ cell_items, const float4 *__restrict__ cell_f,
                            const int *__restrict__ cstart, const int *__restrict__ cend, double x0, double y0,
                            double inv_cell, int ncx, int ncy, double slack2, float delta, int have_grid,
                            int *__restrict__ kind, int *__restrict__ ctr, int *__restrict__ is_pt) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int t = order ? order[i] : i;
    if (tgt_on[t] >= 0) {
        kind[t] = 2; ctr[t] = 2 * tgt_on[t]; is_pt[t] = 0;
        return;
    }
    double tx = tgt_xy[2 * t], ty = tgt_xy[2 * t + 1];
    float txf = (float)tx, tyf = (float)ty;
    int best = -1;
    double bestk = INFINITY;
    double fgx = floor((tx - x0) * inv_cell), fgy = floor((ty - y0) * inv_cell);
    if (have_grid && fgx >= -1 && fgx <= ncx && fgy >= -1 && fgy <= ncy) {
        const int gx = (int)fgx, gy = (int)fgy;
        const int y_lo = max(gy - 1, 0), y_hi = min(gy + 1, ncy - 1);
        const int x_lo = max(gx - 1, 0), x_hi = min(gx + 1, ncx - 1);
        float hmin = INFINITY;   // smallest upper bound of rho over the candidates
        for (int yy = y_lo; yy <= y_hi; ++yy)
            for (int xx = x_lo; xx <= x_hi; ++xx) {
                const int cid = yy * ncx + xx;
                for (int k = cstart[cid]; k < cend[cid]; ++k) {
                    const float4 f = cell_f[k];
                    const float fx = txf - f.x, fy = tyf - f.y;
                    const float d2f = fx * fx + fy * fy;
                    if (d2f > f.z) continue;     // cannot pass the slack test
                    hmin = fminf(hmin, (sqrtf(d2f) + delta) * f.w * 1.00001f);
                }
            }
        for (int yy = y_lo; yy <= y_hi; ++yy)
            for (int xx = x_lo; xx <= x_hi; ++xx) {
                const int cid = yy * ncx + xx;
                for (int k = cstart[cid]; k < cend[cid]; ++k) {
                    const float4 f = cell_f[k];
                    const float fx = txf - f.x, fy = tyf - f.y;
                    const float d2f = fx * fx + fy * fy;
                    if (d2f > f.z) continue;
                    if ((sqrtf(d2f) - delta) * f.w * 0.99999f > hmin) continue;   // lo above the bound
                    const int c = cell_items[k];
                    const double dx = tx - c_xy[2 * c], dy = ty - c_xy[2 * c + 1];
                    const double d2 = dx * dx + dy * dy;
                    const double key = d2 / (c_r[c] * c_r[c]);
                    if (key < bestk || (key == bestk && c < best)) {
                        bestk = key;
                        best = c;
                    }
                }
            }
    }
    if (best >= 0 && bestk <= slack2) { kind[t] = 1; ctr[t] = best; is_pt[t] = 0; }
    else { kind[t] = 0; ctr[t] = -1; is_pt[t] = 1; }
}

__global__ void k_compact_index(int n, const int *__restrict__ flag, const int *__restrict__ pos, int *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && flag[i]) out[pos[i]] = i;
}

// ------------------------------------------------------------------ A4: keys and centre levels
// u is a power of two, so (v - lo) * (1/u) equals (v - lo) / u exactly
__device__ __forceinline__ uint64_t key1(double v, double lo, double inv_u) {
    double f = floor((v - lo) * inv_u);
    const double kmax = (double)((1ll << GQ_KEYBITS) - 1);
    if (f < 0) return 0;
    if (f > kmax) return (uint64_t)kmax;
    return (uint64_t)f;
}

// combined particle array: [0, nsrc) sources, [nsrc, nsrc+nc) centres, then point targets
__global__ void k_keys(int nsrc, int nc, int npt, const double *__restrict__ up_xy, const double *__restrict__ c_xy,
                       const double *__restrict__ c_r, const int *__restrict__ pt_tgt, const double *__restrict__ tgt_xy,
                       RootInfo R, double inv_u, double tcr_scale, double kappa_H, int tcr_shape, int max_level,
                       uint64_t *__restrict__ key, int *__restrict__ val, int *__restrict__ elig,
                       int *__restrict__ c_lc) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)nsrc + nc + npt;
    if (i >= n) return;
    double x, y;
    int e = 31;  // sources and point targets may descend to any level
    if (i < nsrc) {
        x = up_xy[2 * i]; y = up_xy[2 * i + 1];
    } else if (i < nsrc + nc) {
        int c = (int)(i - nsrc);
        x = c_xy[2 * c]; y = c_xy[2 * c + 1];
    } else {
        int t = pt_tgt[i - nsrc - nc];
        x = tgt_xy[2 * t]; y = tgt_xy[2 * t + 1];
    }
    uint64_t kx = key1(x, R.lo_x, inv_u), ky = key1(y, R.lo_y, inv_u);
    if (i >= nsrc && i < nsrc + nc) {
        // deepest level whose TCR (half-width, or with the disk-shaped TCR
        // radius, |b|(1 + t_f)) holds the whole disk, for every box on the key path
        int c = (int)(i - nsrc);
        double r = c_r[c];
        int lc = -1, l0 = 0;
        // Levels l with r <= kappa H 2^-l (and at most 23, so that the key's
        // rounding, one level-30 unit, is below 1/64 of the box) hold the disk
        // with a margin of a tenth of the box whatever the rounding, so the
        // scan below would pass them: it starts after them.
        if (kappa_H > 0 && r > 0) {
            l0 = min(ilogb(kappa_H / r), min(max_level, GQ_KEYBITS - 7));
            l0 = max(l0, 0);
            lc = l0 - 1;
        }
        for (int l = l0; l <= max_level; ++l) {
            int64_t ix = (int64_t)(kx >> (GQ_KEYBITS - l)), iy = (int64_t)(ky >> (GQ_KEYBITS - l));
            double hb = ldexp(R.H, -l);
            double bx = R.lo_x + (double)(2 * ix + 1) * hb;
            double by = R.lo_y + (double)(2 * iy + 1) * hb;
            double dx = x - bx, dy = y - by;
            double d = tcr_shape == 1 ? sqrt(dx * dx + dy * dy) : fmax(fabs(dx), fabs(dy));
            d += r;
            if (d <= hb * tcr_scale) lc = l; else break;
        }
        e = lc < 0 ? 0 : lc;
        c_lc[c] = e;
    }
    key[i] = gq_morton(kx, ky);
    val[i] = (int)i;
    elig[i] = e;
}

__global__ void k_gather_int(long long n, const int *__restrict__ idx, const int *__restrict__ src, int *__restrict__ dst) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

// ------------------------------------------------------------------ A4: level-by-level subdivision
__device__ int lower_bound_prefix(const uint64_t *K, int lo, int hi, int shift, uint64_t target) {
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if ((K[mid] >> shift) < target) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// For each box at level l: subdivide if it holds more than n_max particles
// eligible for level l+1; a child exists if its quadrant holds one.
// forced: sorted keys (level << 60) | Morton key of boxes subdivided whatever
// their count (level restriction); belig[j]: the count, kept for the balance check
__device__ bool key_forced(const uint64_t *forced, int n, uint64_t k) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (forced[mid] < k) lo = mid + 1; else hi = mid;
    }
    return lo < n && forced[lo] == k;
}

__global__ void k_subdivide(int nl, int l, int max_level, int n_max, const uint64_t *__restrict__ K,
                            const int *__restrict__ P, const uint64_t *__restrict__ bkey, const int *__restrict__ bbeg,
                            const int *__restrict__ bend, int *__restrict__ nchild, int4 *__restrict__ cbeg,
                            int4 *__restrict__ cend, const uint64_t *__restrict__ forced, int nforced,
                            int *__restrict__ belig) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nl) return;
    int beg = bbeg[j], end = bend[j];
    int S = P[end] - P[beg];
    belig[j] = S;
    int cnt = 0;
    int cb[4] = {-1, -1, -1, -1}, ce[4] = {-1, -1, -1, -1};
    bool sub = S > n_max || (S > 0 && nforced > 0 && key_forced(forced, nforced, ((uint64_t)l << 60) | bkey[j]));
    if (sub && l < max_level) {
        int shift = 2 * (GQ_KEYBITS - (l + 1));
        uint64_t base = bkey[j] << 2;
        int bnd[5];
        bnd[0] = beg;
        bnd[4] = end;
        for (int q = 1; q < 4; ++q) bnd[q] = lower_bound_prefix(K, beg, end, shift, base + q);
        for (int q = 0; q < 4; ++q) {
            if (P[bnd[q + 1]] - P[bnd[q]] >= 1) {
                cb[q] = bnd[q]; ce[q] = bnd[q + 1];
                ++cnt;
            }
        }
    }
    nchild[j] = cnt;
    cbeg[j] = make_int4(cb[0], cb[1], cb[2], cb[3]);
    cend[j] = make_int4(ce[0], ce[1], ce[2], ce[3]);
}

__global__ void k_emit_children(int nl, int next_start, const uint64_t *__restrict__ bkey, const int *__restrict__ coff,
                                const int4 *__restrict__ cbeg, const int4 *__restrict__ cend, int this_start,
                                int4 *__restrict__ child, uint64_t *__restrict__ nkey, int *__restrict__ nbeg,
                                int *__restrict__ nend, int *__restrict__ npar) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nl) return;
    int cb[4] = {cbeg[j].x, cbeg[j].y, cbeg[j].z, cbeg[j].w};
    int ce[4] = {cend[j].x, cend[j].y, cend[j].z, cend[j].w};
    int ch[4] = {-1, -1, -1, -1};
    int o = coff[j];
    for (int q = 0; q < 4; ++q) {
        if (cb[q] < 0) continue;
        nkey[o] = (bkey[j] << 2) | (uint64_t)q;
        nbeg[o] = cb[q];
        nend[o] = ce[q];
        npar[o] = this_start + j;
        ch[q] = next_start + o;
        ++o;
    }
    child[j] = make_int4(ch[0], ch[1], ch[2], ch[3]);
}

// Ownership (Sec. 4.3): a particle descends from the root into the child
// holding it while it is eligible for that child's level and the child
// exists; the box where it stops owns it.  One walk per particle once the
// box tree is final (the levels' child tables in bchild).
__global__ void k_owner_walk(long long n, int nlev, const uint64_t *__restrict__ K, const int *__restrict__ elig,
                             const int4 *__restrict__ bchild, int *__restrict__ owner) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t k = K[i];
    const int e = elig[i];
    int o = 0;
    for (int l = 0; l + 1 < nlev && e >= l + 1; ++l) {
        int4 c = bchild[o];
        int q = (int)((k >> (2 * (GQ_KEYBITS - (l + 1)))) & 3);
        int nc = q == 0 ? c.x : q == 1 ? c.y : q == 2 ? c.z : c.w;
        if (nc < 0) break;
        o = nc;
    }
    owner[i] = o;
}

// de-interleave a Morton key into box coordinates
__device__ __forceinline__ uint32_t compact_bits(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
    x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
    x = (x | (x >> 16)) & 0x00000000ffffffffull;
    return (uint32_t)x;
}

__global__ void k_box_final(int nl, int start, int l, const uint64_t *__restrict__ lkey, const int *__restrict__ lpar,
                            const int4 *__restrict__ lchild, uint64_t *__restrict__ bkey, int *__restrict__ blev,
                            int *__restrict__ bix, int *__restrict__ biy, int *__restrict__ bparent,
                            int4 *__restrict__ bchild) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nl) return;
    int b = start + j;
    uint64_t k = lkey[j];
    bkey[b] = k;
    blev[b] = l;
    bix[b] = (int)compact_bits(k);
    biy[b] = (int)compact_bits(k >> 1);
    bparent[b] = lpar[j];
    bchild[b] = lchild ? lchild[j] : make_int4(-1, -1, -1, -1);
}

// ------------------------------------------------------------------ per-type arrays
__global__ void k_type_flags(long long n, const int *__restrict__ V, int lo, int hi, int *__restrict__ flag) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = V[i] >= lo && V[i] < hi;
}

__global__ void k_type_compact(long long n, const int *__restrict__ flag, const int *__restrict__ pos,
                               const int *__restrict__ V, const int *__restrict__ owner, const uint64_t *__restrict__ K,
                               int lo, int *__restrict__ out_id, int *__restrict__ out_owner,
                               uint64_t *__restrict__ out_key) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !flag[i]) return;
    int p = pos[i];
    out_id[p] = V[i] - lo;
    out_owner[p] = owner[i];
    if (out_key) out_key[p] = K[i];
}

__global__ void k_ranges(int n, const int *__restrict__ owner, int *__restrict__ beg, int *__restrict__ end) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int o = owner[j];
    if (j == 0 || owner[j - 1] != o) beg[o] = j;
    if (j == n - 1 || owner[j + 1] != o) end[o] = j + 1;
}

__global__ void k_subtree_src(int nbox, const uint64_t *__restrict__ bkey, const int *__restrict__ blev,
                              const uint64_t *__restrict__ skey, int nsrc, int *__restrict__ sb, int *__restrict__ se) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int shift = 2 * (GQ_KEYBITS - blev[b]);
    uint64_t k = bkey[b];
    int lo = 0, hi = nsrc;
    while (lo < hi) { int m = (lo + hi) >> 1; if ((skey[m] >> shift) < k) lo = m + 1; else hi = m; }
    int a = lo;
    hi = nsrc;
    while (lo < hi) { int m = (lo + hi) >> 1; if ((skey[m] >> shift) <= k) lo = m + 1; else hi = m; }
    sb[b] = a;
    se[b] = lo;
}

__global__ void k_box_counts(int nbox, const int *__restrict__ ssb, const int *__restrict__ sse,
                             const int *__restrict__ cb, const int *__restrict__ ce, const int *__restrict__ pb,
                             const int *__restrict__ pe, int *__restrict__ sub_src, int *__restrict__ own_tgt,
                             int *__restrict__ sub_tgt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    sub_src[b] = sse[b] - ssb[b];
    int t = (ce[b] - cb[b]) + (pe[b] - pb[b]);
    own_tgt[b] = t;
    sub_tgt[b] = t;
}

__global__ void k_sub_tgt_level(int start, int end, const int4 *__restrict__ bchild, int *__restrict__ sub_tgt) {
    int b = start + blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= end) return;
    int4 c = bchild[b];
    int s = sub_tgt[b];
    if (c.x >= 0) s += sub_tgt[c.x];
    if (c.y >= 0) s += sub_tgt[c.y];
    if (c.z >= 0) s += sub_tgt[c.z];
    if (c.w >= 0) s += sub_tgt[c.w];
    sub_tgt[b] = s;
}

__global__ void k_gather_sources(int n, const int *__restrict__ perm, const double *__restrict__ xy,
                                 const double *__restrict__ w, const double *__restrict__ nrm, double2 *__restrict__ oxy,
                                 double *__restrict__ ow, double2 *__restrict__ on) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int i = perm[j];
    oxy[j] = make_double2(xy[2 * i], xy[2 * i + 1]);
    ow[j] = w[i];
    on[j] = make_double2(nrm[2 * i], nrm[2 * i + 1]);
}

__global__ void k_gather_centres(int n, const int *__restrict__ perm, const double *__restrict__ xy,
                                 const double *__restrict__ r, double2 *__restrict__ oxy, double *__restrict__ orr,
                                 int *__restrict__ pos) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int c = perm[j];
    oxy[j] = make_double2(xy[2 * c], xy[2 * c + 1]);
    orr[j] = r[c];
    pos[c] = j;
}

__global__ void k_gather_points(int n, const int *__restrict__ perm_pt, const int *__restrict__ pt_tgt,
                                const double *__restrict__ txy, int *__restrict__ perm_out, double2 *__restrict__ oxy) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int t = pt_tgt[perm_pt[j]];
    perm_out[j] = t;
    oxy[j] = make_double2(txy[2 * t], txy[2 * t + 1]);
}

__global__ void k_flag_nonempty(int n, const int *__restrict__ beg, const int *__restrict__ end, int *__restrict__ flag) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < n) flag[b] = end[b] > beg[b];
}

// boxes whose multipole the upward pass forms from their children's (M2M):
// not a leaf, sources in the subtree
__global__ void k_flag_parents(int n, const int4 *__restrict__ bchild, const int *__restrict__ sub_src,
                               int *__restrict__ flag) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    int4 c = bchild[b];
    flag[b] = (c.x >= 0 || c.y >= 0 || c.z >= 0 || c.w >= 0) && sub_src[b] > 0;
}

}  // namespace

// compact indices i in [0, n) with flag[i] != 0 into out (ascending); returns the
// count.  The scan's buffers belong to the geometry (grown, never freed during a
// build), so nothing goes back to the shared pool while the kernels may still
// read it and no second synchronisation is needed.
static int compact_flags(gq_geom *g, const int *flag, long long n, dbuf<int> &out) {
    g->cf_pos.alloc(n + 1);
    g->cf_tmp.alloc(gq_scan_tmp_size(n));
    gq_exclusive_scan(g->ctx, flag, g->cf_pos.p, n, g->cf_tmp.p);
    int cnt = 0;
    GQ_CUDA(cudaMemcpyAsync(&cnt, g->cf_pos.p + n, sizeof(int), cudaMemcpyDeviceToHost, g->ctx->stream));
    GQ_CUDA(cudaStreamSynchronize(g->ctx->stream));
    out.alloc(cnt);
    if (n > 0)
        GQ_LAUNCH(g->ctx, k_compact_index, gq_blocks(n, kT), kT, 0, (int)n, flag, (const int *)g->cf_pos.p, out.p);
    return cnt;
}

// ------------------------------------------------------------------ public stages
void gq_form_centres(gq_geom *g) {
    g->nc = 2 * g->nbase;
    g->c_xy.alloc(2 * (size_t)g->nc);
    g->c_r.alloc(g->nc);
    g->c_lc.alloc(g->nc);
    GQ_LAUNCH(g->ctx, k_centres, gq_blocks(g->nbase, kT), kT, 0, g->nbase, g->nb, (const double *)g->base_xy,
              (const double *)g->base_n, (const double *)g->panel_len, g->prm.radius_factor, g->c_xy.p, g->c_r.p);
}

static void associate(gq_geom *g) {
    gq_ctx *ctx = g->ctx;
    int nt = g->nt, nc = g->nc;
    g->t_kind.alloc(nt);
    g->t_ctr.alloc(nt);
    dbuf<int> &is_pt = g->cf_flag;   // read by the compaction after this function returns
    is_pt.alloc(nt);
    Ext ce = device_extent(g, 0);
    double slack = g->prm.assoc_slack;
    double cell = 1.25 * slack * ce.rmax;
    int have_grid = (nc > 0 && cell > 0);
    const double inv_cell = have_grid ? 1.0 / cell : 0.0;
    int ncx = 1, ncy = 1;
    if (have_grid) {
        double fx = floor((ce.x1 - ce.x0) / cell) + 1, fy = floor((ce.y1 - ce.y0) / cell) + 1;
        GQ_REQUIRE(fx * fy < 4.0e8, GQ_ERR_UNSUPPORTED, "association grid too fine (centre radii vary too much)");
        ncx = (int)fx;
        ncy = (int)fy;
    }
    long long ncell = (long long)ncx * ncy;
    double delta_assoc = 0.0;
    dbuf<uint32_t> ckey;
    dbuf<int> cval, cstart, cend;
    dbuf<float4> cf;
    ckey.alloc(nc);
    cval.alloc(nc);
    cf.alloc(nc);
    cstart.alloc(ncell);
    cend.alloc(ncell);
    GQ_CUDA(cudaMemsetAsync(cstart.p, 0, sizeof(int) * ncell, ctx->stream));
    GQ_CUDA(cudaMemsetAsync(cend.p, 0, sizeof(int) * ncell, ctx->stream));
    if (have_grid) {
        GQ_LAUNCH(ctx, k_cell_of_centre, gq_blocks(nc, kT), kT, 0, nc, (const double *)g->c_xy, ce.x0, ce.y0, inv_cell,
                  ncx, ncy, ckey.p, cval.p);
        int bits = 1;
        while ((1ll << bits) < ncell) ++bits;
        gq_radix_sort_pairs32(ctx, ckey.p, cval.p, nc, bits);
        GQ_LAUNCH(ctx, k_cell_bounds, gq_blocks(nc, kT), kT, 0, nc, (const uint32_t *)ckey.p, cstart.p, cend.p);
        // float prefilter margin: rounding of coordinates of magnitude <= X to float moves a
        // distance by at most 3 X 2^-24; searched targets lie within two cells of the centres
        double X = fmax(fmax(fabs(ce.x0), fabs(ce.x1)), fmax(fabs(ce.y0), fabs(ce.y1))) + 2.0 * cell;
        double delta = 16.0 * X * 0x1p-24;
        delta_assoc = delta;
        GQ_LAUNCH(ctx, k_cell_floats, gq_blocks(nc, kT), kT, 0, nc, (const int *)cval.p, (const double *)g->c_xy,
                  (const double *)g->c_r, slack, delta, cf.p);
    }
    dbuf<uint32_t> tkey;
    dbuf<int> torder;
    if (have_grid && nt > 0) {
        tkey.alloc(nt);
        torder.alloc(nt);
        GQ_LAUNCH(ctx, k_cell_of_target, gq_blocks(nt, kT), kT, 0, nt, (const double *)g->tgt_xy,
                  (const int *)g->tgt_on, ce.x0, ce.y0, inv_cell, ncx, ncy, tkey.p, torder.p);
        int bits = 1;
        while ((1ll << bits) < ncell + 2) ++bits;
        gq_radix_sort_pairs32(ctx, tkey.p, torder.p, nt, bits);
    }
    if (nt > 0)
        GQ_LAUNCH(ctx, k_associate, gq_blocks(nt, kT), kT, 0, nt, (const int *)torder.p, (const double *)g->tgt_xy,
                  (const int *)g->tgt_on,
                  (const double *)g->c_xy, (const double *)g->c_r, (const int *)cval.p, (const float4 *)cf.p,
                  (const int *)cstart.p, (const int *)cend.p, ce.x0, ce.y0, inv_cell, ncx, ncy, slack * slack,
                  (float)(delta_assoc * 1.001), have_grid, g->t_kind.p,
                  g->t_ctr.p, is_pt.p);
    g->npt = compact_flags(g, is_pt.p, nt, g->pt_tgt);
}

// Root square (Sec. 4.3): half-width H a power of two with 2H >= extent (1 + 2^-20),
// lower corner on a multiple of u = 2H / 2^30.
static RootInfo make_root(const Ext &e) {
    double ext = fmax(e.x1 - e.x0, e.y1 - e.y0);
    if (!(ext > 0)) ext = 1.0;
    double target = 0.5 * ext * (1.0 + 0x1p-20);
    int ex;
    double m = frexp(target, &ex);
    RootInfo R;
    R.H = (m == 0.5) ? ldexp(1.0, ex - 1) : ldexp(1.0, ex);
    R.u = ldexp(R.H, 1 - GQ_KEYBITS);
    R.lo_x = floor(e.x0 / R.u) * R.u;
    R.lo_y = floor(e.y0 / R.u) * R.u;
    return R;
}

struct LevelBufs {
    dbuf<uint64_t> key;
    dbuf<int> beg, end, par, elig;
    dbuf<int4> child;
    int n = 0;
};

// Optional phase timing of the build (environment variable GQ_BUILD_TIMING set):
// CUDA events between phases, printed to stderr when the build ends.
struct PhaseTimer {
    cudaStream_t st;
    bool on;
    std::vector<std::pair<const char *, cudaEvent_t>> ev;
    explicit PhaseTimer(cudaStream_t s) : st(s), on(getenv("GQ_BUILD_TIMING") != nullptr) { mark("start"); }
    void mark(const char *name) {
        if (!on) return;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        cudaEventRecord(e, st);
        ev.emplace_back(name, e);
    }
    ~PhaseTimer() {
        if (!on || ev.empty()) return;
        cudaEventSynchronize(ev.back().second);
        fprintf(stderr, "gq_build phases (ms):");
        for (size_t i = 1; i < ev.size(); ++i) {
            float ms = 0;
            cudaEventElapsedTime(&ms, ev[i - 1].second, ev[i].second);
            fprintf(stderr, " %s %.3f", ev[i].first, ms);
        }
        fprintf(stderr, "\n");
        for (auto &e : ev) cudaEventDestroy(e.second);
    }
};

void gq_build_all(gq_geom *g) {
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    GQ_REQUIRE(g->targets_set, GQ_ERR_STATE, "gq_build: targets not set");
    PhaseTimer pt(st);
    associate(g);
    pt.mark("associate");

    // ---- root and keys
    Ext re = device_extent(g, 1);
    GQ_REQUIRE(std::isfinite(re.x0) && std::isfinite(re.x1) && std::isfinite(re.y0) && std::isfinite(re.y1),
               GQ_ERR_UNSUPPORTED, "non-finite coordinates");
    g->root = make_root(re);
    const long long N = (long long)g->nsrc + g->nc + g->npt;
    dbuf<uint64_t> K;
    dbuf<int> V, elig0, elig;
    K.alloc(N);
    V.alloc(N);
    elig0.alloc(N);
    elig.alloc(N);
    double tcr_scale = (double)(g->prm.tf_den + g->prm.tf_num) / (double)g->prm.tf_den;
    // A disk of radius r centred in a level-l box lies at distance at most
    // c0 (h + u) from the box centre (c0 = 1 for the square TCR, sqrt 2 for
    // the disk; h the half-width, u one level-30 unit <= h/64): with
    // r <= kappa h, kappa = 0.8 (scale - c0 - 1/32), the fit holds with room.
    const double c0 = g->prm.tcr_shape == 1 ? 1.4143 : 1.0;
    const double kappa = 0.8 * (tcr_scale - c0 - 1.0 / 32.0);
    const double kappa_H = kappa > 0 ? kappa * g->root.H : 0.0;
    GQ_LAUNCH(ctx, k_keys, gq_blocks(N, kT), kT, 0, g->nsrc, g->nc, g->npt, (const double *)g->up_xy,
              (const double *)g->c_xy, (const double *)g->c_r, (const int *)g->pt_tgt, (const double *)g->tgt_xy,
              g->root, 1.0 / g->root.u, tcr_scale, kappa_H, g->prm.tcr_shape, g->prm.max_level, K.p, V.p, elig0.p,
              g->c_lc.p);
    gq_radix_sort_pairs(ctx, K.p, V.p, N, 2 * GQ_KEYBITS);
    GQ_LAUNCH(ctx, k_gather_int, gq_blocks(N, kT), kT, 0, N, (const int *)V.p, (const int *)elig0.p, elig.p);

    pt.mark("keys_sort");
    // ---- level-by-level subdivision (a lambda: the level restriction runs it
    // again with the subdivisions it forces)
    std::vector<int> lstart;
    dbuf<int> belig;   // per box: particles eligible for its children
    dbuf<int> flag, P, scan_tmp, owner, nchild, coff, ctmp;
    dbuf<int4> cbeg, cend;
    auto build_levels = [&](const uint64_t *forced, int nforced) {
        // ---- level-by-level subdivision
        std::vector<std::unique_ptr<LevelBufs>> lv;
        lv.emplace_back(new LevelBufs);
        lv[0]->n = 1;
        lv[0]->key.alloc(1);
        lv[0]->beg.alloc(1);
        lv[0]->end.alloc(1);
        lv[0]->par.alloc(1);
        {
            uint64_t k0 = 0;
            int b0 = 0, e0 = (int)N, p0 = -1;
            GQ_CUDA(cudaMemcpyAsync(lv[0]->key.p, &k0, sizeof(k0), cudaMemcpyHostToDevice, st));
            GQ_CUDA(cudaMemcpyAsync(lv[0]->beg.p, &b0, sizeof(int), cudaMemcpyHostToDevice, st));
            GQ_CUDA(cudaMemcpyAsync(lv[0]->end.p, &e0, sizeof(int), cudaMemcpyHostToDevice, st));
            GQ_CUDA(cudaMemcpyAsync(lv[0]->par.p, &p0, sizeof(int), cudaMemcpyHostToDevice, st));
            GQ_CUDA(cudaStreamSynchronize(st));
        }
        flag.alloc(N);
        P.alloc(N + 1);
        scan_tmp.alloc(gq_scan_tmp_size(N));
        lstart = {0, 1};
        for (int l = 0;; ++l) {
            LevelBufs &cur = *lv[l];
            int nl = cur.n;
            // prefix counts of the particles eligible at level l + 1 (elig > l)
            gq_exclusive_scan_above(ctx, (const int *)elig.p, l, P.p, N, scan_tmp.p);
            nchild.alloc(nl);
            coff.alloc(nl + 1);
            cbeg.alloc(nl);
            cend.alloc(nl);
            ctmp.alloc(gq_scan_tmp_size(nl));
            cur.elig.alloc(nl);
            GQ_LAUNCH(ctx, k_subdivide, gq_blocks(nl, kT), kT, 0, nl, l, g->prm.max_level, g->prm.n_max,
                      (const uint64_t *)K.p, (const int *)P.p, (const uint64_t *)cur.key.p, (const int *)cur.beg.p,
                      (const int *)cur.end.p, nchild.p, cbeg.p, cend.p, forced, nforced, cur.elig.p);
            gq_exclusive_scan(ctx, nchild.p, coff.p, nl, ctmp.p);
            int total = 0;
            GQ_CUDA(cudaMemcpyAsync(&total, coff.p + nl, sizeof(int), cudaMemcpyDeviceToHost, st));
            GQ_CUDA(cudaStreamSynchronize(st));
            cur.child.alloc(nl);
            lv.emplace_back(new LevelBufs);
            LevelBufs &nxt = *lv[l + 1];
            nxt.n = total;
            nxt.key.alloc(total);
            nxt.beg.alloc(total);
            nxt.end.alloc(total);
            nxt.par.alloc(total);
            int next_start = lstart[l + 1];
            GQ_LAUNCH(ctx, k_emit_children, gq_blocks(nl, kT), kT, 0, nl, next_start, (const uint64_t *)cur.key.p,
                      (const int *)coff.p, (const int4 *)cbeg.p, (const int4 *)cend.p, lstart[l], cur.child.p, nxt.key.p,
                      nxt.beg.p, nxt.end.p, nxt.par.p);
            if (total == 0) {
                lv.pop_back();
                break;
            }
            lstart.push_back(lstart[l + 1] + total);
        }
        g->nlev = (int)lv.size();
        g->nbox = lstart[g->nlev];
        g->level_start_h.assign(lstart.begin(), lstart.begin() + g->nlev + 1);
        g->level_start.alloc(g->nlev + 1);
        GQ_CUDA(cudaMemcpyAsync(g->level_start.p, g->level_start_h.data(), sizeof(int) * (g->nlev + 1),
                                cudaMemcpyHostToDevice, st));

        pt.mark("levels");
        // ---- final box arrays
        int nbox = g->nbox;
        belig.alloc(nbox);
        g->bkey.alloc(nbox);
        g->blev.alloc(nbox);
        g->bix.alloc(nbox);
        g->biy.alloc(nbox);
        g->bparent.alloc(nbox);
        g->bchild.alloc(nbox);
        for (int l = 0; l < g->nlev; ++l) {
            LevelBufs &B = *lv[l];
            GQ_LAUNCH(ctx, k_box_final, gq_blocks(B.n, kT), kT, 0, B.n, lstart[l], l, (const uint64_t *)B.key.p,
                      (const int *)B.par.p, (const int4 *)B.child.p, g->bkey.p, g->blev.p, g->bix.p, g->biy.p,
                      g->bparent.p, g->bchild.p);
            GQ_CUDA(cudaMemcpyAsync(belig.p + lstart[l], B.elig.p, sizeof(int) * B.n, cudaMemcpyDeviceToDevice, st));
        }
        owner.alloc(N);
        GQ_LAUNCH(ctx, k_owner_walk, gq_blocks(N, kT), kT, 0, N, g->nlev, (const uint64_t *)K.p, (const int *)elig.p,
                  (const int4 *)g->bchild.p, owner.p);
    };
    build_levels(nullptr, 0);
    if (g->prm.level_restrict) {
        // Sec. 4.6 level restriction: subdivide, and rebuild, while a leaf owning a
        // particle eligible for children touches a box two levels deeper
        std::vector<uint64_t> forced;
        dbuf<uint64_t> dforced;
        for (int it = 0;; ++it) {
            std::vector<uint64_t> add;
            gq_balance_violations(g, belig.p, add);
            if (add.empty()) break;
            GQ_REQUIRE(it < 64, GQ_ERR_UNSUPPORTED, "level restriction did not converge");
            forced.insert(forced.end(), add.begin(), add.end());
            std::sort(forced.begin(), forced.end());
            forced.erase(std::unique(forced.begin(), forced.end()), forced.end());
            dforced.alloc(forced.size());
            GQ_CUDA(cudaMemcpyAsync(dforced.p, forced.data(), sizeof(uint64_t) * forced.size(),
                                    cudaMemcpyHostToDevice, st));
            build_levels(dforced.p, (int)forced.size());
        }
    }

    pt.mark("box_arrays");
    const int nbox = g->nbox;
    // ---- per-type arrays
    dbuf<int> pos;
    pos.alloc(N + 1);
    // sources (Morton order)
    dbuf<uint64_t> skey;
    skey.alloc(g->nsrc);
    g->src_perm.alloc(g->nsrc);
    g->src_owner.alloc(g->nsrc);
    GQ_LAUNCH(ctx, k_type_flags, gq_blocks(N, kT), kT, 0, N, (const int *)V.p, 0, g->nsrc, flag.p);
    gq_exclusive_scan(ctx, flag.p, pos.p, N, scan_tmp.p);
    GQ_LAUNCH(ctx, k_type_compact, gq_blocks(N, kT), kT, 0, N, (const int *)flag.p, (const int *)pos.p,
              (const int *)V.p, (const int *)owner.p, (const uint64_t *)K.p, 0, g->src_perm.p, g->src_owner.p,
              skey.p);
    // centres (Morton order, then stable by owner box)
    dbuf<int> cid_m, cown_m;
    cid_m.alloc(g->nc);
    cown_m.alloc(g->nc);
    GQ_LAUNCH(ctx, k_type_flags, gq_blocks(N, kT), kT, 0, N, (const int *)V.p, g->nsrc, g->nsrc + g->nc, flag.p);
    gq_exclusive_scan(ctx, flag.p, pos.p, N, scan_tmp.p);
    GQ_LAUNCH(ctx, k_type_compact, gq_blocks(N, kT), kT, 0, N, (const int *)flag.p, (const int *)pos.p,
              (const int *)V.p, (const int *)owner.p, (const uint64_t *)K.p, g->nsrc, cid_m.p, cown_m.p,
              (uint64_t *)nullptr);
    {
        dbuf<uint32_t> ok;
        ok.alloc(g->nc);
        static_assert(sizeof(uint32_t) == sizeof(int), "");
        GQ_CUDA(cudaMemcpyAsync(ok.p, cown_m.p, sizeof(int) * g->nc, cudaMemcpyDeviceToDevice, st));
        int bits = 1;
        while ((1ll << bits) < nbox) ++bits;
        gq_radix_sort_pairs32(ctx, ok.p, cid_m.p, g->nc, bits);
        g->ctr_perm.alloc(g->nc);
        g->ctr_owner.alloc(g->nc);
        GQ_CUDA(cudaMemcpyAsync(g->ctr_perm.p, cid_m.p, sizeof(int) * g->nc, cudaMemcpyDeviceToDevice, st));
        GQ_CUDA(cudaMemcpyAsync(g->ctr_owner.p, ok.p, sizeof(int) * g->nc, cudaMemcpyDeviceToDevice, st));
        GQ_CUDA(cudaStreamSynchronize(st));
    }
    // point targets (Morton order)
    dbuf<int> pid_m;
    pid_m.alloc(g->npt);
    g->pt_owner.alloc(g->npt);
    GQ_LAUNCH(ctx, k_type_flags, gq_blocks(N, kT), kT, 0, N, (const int *)V.p, g->nsrc + g->nc,
              g->nsrc + g->nc + g->npt, flag.p);
    gq_exclusive_scan(ctx, flag.p, pos.p, N, scan_tmp.p);
    GQ_LAUNCH(ctx, k_type_compact, gq_blocks(N, kT), kT, 0, N, (const int *)flag.p, (const int *)pos.p,
              (const int *)V.p, (const int *)owner.p, (const uint64_t *)K.p, g->nsrc + g->nc, pid_m.p,
              g->pt_owner.p, (uint64_t *)nullptr);

    pt.mark("type_arrays");
    // ---- box ranges and counts
    for (dbuf<int> *a : {&g->src_beg, &g->src_end, &g->ctr_beg, &g->ctr_end, &g->pt_beg, &g->pt_end, &g->ssub_beg,
                         &g->ssub_end, &g->sub_src, &g->sub_tgt, &g->own_tgt}) {
        a->alloc(nbox);
        GQ_CUDA(cudaMemsetAsync(a->p, 0, sizeof(int) * nbox, st));
    }
    if (g->nsrc) GQ_LAUNCH(ctx, k_ranges, gq_blocks(g->nsrc, kT), kT, 0, g->nsrc, (const int *)g->src_owner.p, g->src_beg.p, g->src_end.p);
    if (g->nc) GQ_LAUNCH(ctx, k_ranges, gq_blocks(g->nc, kT), kT, 0, g->nc, (const int *)g->ctr_owner.p, g->ctr_beg.p, g->ctr_end.p);
    if (g->npt) GQ_LAUNCH(ctx, k_ranges, gq_blocks(g->npt, kT), kT, 0, g->npt, (const int *)g->pt_owner.p, g->pt_beg.p, g->pt_end.p);
    GQ_LAUNCH(ctx, k_subtree_src, gq_blocks(nbox, kT), kT, 0, nbox, (const uint64_t *)g->bkey.p, (const int *)g->blev.p,
              (const uint64_t *)skey.p, g->nsrc, g->ssub_beg.p, g->ssub_end.p);
    GQ_LAUNCH(ctx, k_box_counts, gq_blocks(nbox, kT), kT, 0, nbox, (const int *)g->ssub_beg.p, (const int *)g->ssub_end.p,
              (const int *)g->ctr_beg.p, (const int *)g->ctr_end.p, (const int *)g->pt_beg.p, (const int *)g->pt_end.p,
              g->sub_src.p, g->own_tgt.p, g->sub_tgt.p);
    for (int l = g->nlev - 1; l >= 0; --l) {
        int s = lstart[l], e = lstart[l + 1];
        GQ_LAUNCH(ctx, k_sub_tgt_level, gq_blocks(e - s, kT), kT, 0, s, e, (const int4 *)g->bchild.p, g->sub_tgt.p);
    }

    pt.mark("ranges");
    // ---- gathered particle data
    g->s_xy.alloc(g->nsrc);
    g->s_w.alloc(g->nsrc);
    g->s_n.alloc(g->nsrc);
    if (g->nsrc) GQ_LAUNCH(ctx, k_gather_sources, gq_blocks(g->nsrc, kT), kT, 0, g->nsrc, (const int *)g->src_perm.p,
              (const double *)g->up_xy, (const double *)g->up_w, (const double *)g->up_n, g->s_xy.p, g->s_w.p, g->s_n.p);
    g->sc_xy.alloc(g->nc);
    g->sc_r.alloc(g->nc);
    g->ctr_pos.alloc(g->nc);
    if (g->nc) GQ_LAUNCH(ctx, k_gather_centres, gq_blocks(g->nc, kT), kT, 0, g->nc, (const int *)g->ctr_perm.p,
              (const double *)g->c_xy, (const double *)g->c_r, g->sc_xy.p, g->sc_r.p, g->ctr_pos.p);
    g->pt_perm.alloc(g->npt);
    g->sp_xy.alloc(g->npt);
    if (g->npt) GQ_LAUNCH(ctx, k_gather_points, gq_blocks(g->npt, kT), kT, 0, g->npt, (const int *)pid_m.p,
              (const int *)g->pt_tgt, (const double *)g->tgt_xy, g->pt_perm.p, g->sp_xy.p);

    pt.mark("gather");
    // ---- work lists
    dbuf<int> bflag;
    bflag.alloc(nbox);
    GQ_LAUNCH(ctx, k_flag_nonempty, gq_blocks(nbox, kT), kT, 0, nbox, (const int *)g->src_beg.p, (const int *)g->src_end.p, bflag.p);
    g->n_leaf_src = compact_flags(g, bflag.p, nbox, g->leaf_src_boxes);
    GQ_LAUNCH(ctx, k_flag_nonempty, gq_blocks(nbox, kT), kT, 0, nbox, (const int *)g->ctr_beg.p, (const int *)g->ctr_end.p, bflag.p);
    g->n_ctr_boxes = compact_flags(g, bflag.p, nbox, g->ctr_boxes);
    GQ_LAUNCH(ctx, k_flag_nonempty, gq_blocks(nbox, kT), kT, 0, nbox, (const int *)g->pt_beg.p, (const int *)g->pt_end.p, bflag.p);
    g->n_pt_boxes = compact_flags(g, bflag.p, nbox, g->pt_boxes);
    // the M2M parents, kept in box order, so that level l's are the entries
    // from the compaction offset of its first box to that of the next level's
    GQ_LAUNCH(ctx, k_flag_parents, gq_blocks(nbox, kT), kT, 0, nbox, (const int4 *)g->bchild.p,
              (const int *)g->sub_src.p, bflag.p);
    g->n_m2m_boxes = compact_flags(g, bflag.p, nbox, g->m2m_boxes);
    dbuf<int> m2m_ls;
    m2m_ls.alloc(g->nlev + 1);
    GQ_LAUNCH(ctx, k_gather_int, gq_blocks(g->nlev + 1, kT), kT, 0, (long long)(g->nlev + 1),
              (const int *)g->level_start.p, (const int *)g->cf_pos.p, m2m_ls.p);
    g->m2m_level_start_h.assign(g->nlev + 1, 0);
    GQ_CUDA(cudaMemcpyAsync(g->m2m_level_start_h.data(), m2m_ls.p, sizeof(int) * (g->nlev + 1),
                            cudaMemcpyDeviceToHost, st));
    GQ_CUDA(cudaStreamSynchronize(st));
    pt.mark("work_lists");

    gq_build_lists(g);
    pt.mark("lists");
}

// flags boxes with a nonempty V or X-far list (computed after the lists)
__global__ void k_flag_far(int nbox, const int *__restrict__ voff, const int *__restrict__ xoff, int *__restrict__ flag) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nbox) flag[b] = (voff[b + 1] > voff[b]) || (xoff[b + 1] > xoff[b]);
}

void gq_build_far_boxes(gq_geom *g) {
    dbuf<int> &bflag = g->cf_flag;   // read by the compaction after this function returns
    bflag.alloc(g->nbox);
    GQ_LAUNCH(g->ctx, k_flag_far, gq_blocks(g->nbox, kT), kT, 0, g->nbox, (const int *)g->list_off[1].p,
              (const int *)g->list_off[5].p, bflag.p);
    g->n_far_boxes = compact_flags(g, bflag.p, g->nbox, g->far_boxes);
}
