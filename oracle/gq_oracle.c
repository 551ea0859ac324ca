/*
 * gq_oracle.c -- plain serial FP64 oracle for GIGAQBX.
 *
 * TEST INFRASTRUCTURE ONLY: called by tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  Written from the
 * paper (Wala & Kloeckner 2018); shares nothing with the CUDA path.
 * Compile with -ffp-contract=off: the decisions that feed integer results
 * (keys, centre levels, association) must round every operation separately.
 *
 * Threads: built with -fopenmp, the evaluation loops (O1 and Stages 2-8 of
 * O2) run over boxes, centres and targets in parallel (orc_set_threads);
 * every output is still summed by one thread in the serial order, so the
 * results are bit for bit those of one thread.  The tree and lists stay
 * serial.
 *
 * GQ_ORC_MUT (default 0) plants one deliberate mistake when compiled with
 * -DGQ_ORC_MUT=k; tests/test_oracle_mutations.py builds such variants to show
 * that the pins catch each of them.  Normal builds never set it.
 *
 * Conventions (Sec. 2.1, eqs. slp/dlp/qbx, and Sec. 3.1):
 *   complex potential Phi with   S mu(x) = -(1/2pi) Re Phi_S(x),
 *                                D mu(x) = -(1/2pi) Re Phi_D(x),
 *   Phi_S(z) = sum_j q_j log(z - y_j),   q_j = w_j mu_j,
 *   Phi_D(z) = sum_j d_j / (y_j - z),    d_j = w_j mu_j (n1 + i n2)_j
 *   (n . grad_y log|y - x| = Re(n / (y - x))).
 *   Multipole about c, w = y - c:  S: a_0 = q, a_k = -q w^k / k     (eq. multipole)
 *                                  D: a_0 = 0, a_k = -d w^(k-1)
 *   Local about c:                 S: b_0 = q log(c - y), b_m = -q / (m w^m)   (eq. local)
 *                                  D: b_m = d / w^(m+1)
 *   M2M (eq. m2m), M2L (eq. m2l, with the a_0 term's sign as obtained by
 *   expanding log z about y: (-1)^(m+1) a_0 / (m y^m); the printed (-1)^m is
 *   a typo), L2L (eq. l2l).
 *
 * Target confinement region: the closed l-inf ball (square) of radius
 * |b|(1 + t_f) (Sec. 4.3), or, with tcr_shape = 1, the closed l2 disk of that
 * radius (the variant named in the appendix corrigendum; reading: every
 * definition of Sec. 4.3 kept with the disk as the set).
 */
#ifndef GQ_ORC_MUT
#define GQ_ORC_MUT 0
#endif
#include "gq_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* number of threads for the evaluation loops (1 = serial) */
static int g_threads = 1;
int orc_set_threads(int n) {
#ifdef _OPENMP
    g_threads = n < 1 ? 1 : n;
#else
    (void)n;
    g_threads = 1;
#endif
    return g_threads;
}
int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

typedef double complex cplx;

#define KEYBITS 30
#define TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------ utils */
typedef struct { int *v; int n, cap; } ivec;
static void iv_push(ivec *a, int x) {
    if (a->n == a->cap) { a->cap = a->cap ? 2 * a->cap : 8; a->v = realloc(a->v, sizeof(int) * a->cap); }
    a->v[a->n++] = x;
}
static void iv_free(ivec *a) { free(a->v); a->v = NULL; a->n = a->cap = 0; }

typedef struct {
    int level; int64_t ix, iy; int parent; int child[4];
    ivec src, ctr, tgt;     /* owned particles */
    int sub_src, sub_tgt;   /* subtree counts (sources; centres + point targets) */
    double cx, cy, h;       /* geometric centre and half-width */
} obox;

typedef struct { int n; int *off; int *idx; } csr;

struct orc_state {
    orc_geom g; orc_params p;
    /* copies of inputs */
    double *ref_b, *ref_u, *base_xy, *base_n, *up_xy, *up_n, *up_w, *panel_len, *tgt_xy;
    int *tgt_on;
    int nbase, nsrc;
    /* centres (A2) */
    int nc; double *c_xy, *c_r; int *c_lc;
    /* association (A3): kind 0 = point target, 1 = one-sided QBX, 2 = two-sided QBX */
    int *t_kind, *t_ctr;
    int npt; int *pt_tgt; int *tgt_pt;  /* point-target list and inverse map (-1) */
    /* root (A4) */
    double lo_x, lo_y, H, u;
    int64_t *s_kx, *s_ky, *c_kx, *c_ky, *p_kx, *p_ky;
    /* tree */
    int nbox, capbox; obox *box;
    /* level restriction: boxes subdivided regardless of their particle count,
     * keys (level << 60) | morton(ix, iy), sorted */
    uint64_t *forced; int nforced;
    int *src_owner, *ctr_owner, *pt_owner;
    /* lists */
    csr L[ORC_NLISTS], LB[ORC_NLISTS];
    int have_brute;
    double binom[128][128];
};

static void *xdup(const void *p, size_t n) { void *q = malloc(n ? n : 1); if (n) memcpy(q, p, n); return q; }

/* ------------------------------------------------------------------ create */
orc_state *orc_create(const orc_geom *g, const orc_params *p) {
    orc_state *s = calloc(1, sizeof(orc_state));
    s->g = *g; s->p = *p;
    s->nbase = g->npanels * g->nb;
    s->nsrc = g->npanels * g->nu;
    s->ref_b = xdup(g->ref_b, sizeof(double) * g->nb);
    s->ref_u = xdup(g->ref_u, sizeof(double) * g->nu);
    s->base_xy = xdup(g->base_xy, sizeof(double) * 2 * s->nbase);
    s->base_n = xdup(g->base_n, sizeof(double) * 2 * s->nbase);
    s->up_xy = xdup(g->up_xy, sizeof(double) * 2 * s->nsrc);
    s->up_n = xdup(g->up_n, sizeof(double) * 2 * s->nsrc);
    s->up_w = xdup(g->up_w, sizeof(double) * s->nsrc);
    s->panel_len = xdup(g->panel_len, sizeof(double) * g->npanels);
    s->tgt_xy = xdup(g->tgt_xy, sizeof(double) * 2 * g->ntargets);
    s->tgt_on = xdup(g->tgt_onsurf, sizeof(int) * g->ntargets);
    for (int n = 0; n < 128; ++n) {
        s->binom[n][0] = 1.0;
        for (int k = 1; k <= n; ++k) s->binom[n][k] = s->binom[n - 1][k - 1] + (k <= n - 1 ? s->binom[n - 1][k] : 0.0);
    }
    return s;
}

static void free_lists(csr *L) {
    for (int i = 0; i < ORC_NLISTS; ++i) { free(L[i].off); free(L[i].idx); L[i].off = L[i].idx = NULL; L[i].n = 0; }
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free(s->ref_b); free(s->ref_u); free(s->base_xy); free(s->base_n); free(s->up_xy); free(s->up_n);
    free(s->up_w); free(s->panel_len); free(s->tgt_xy); free(s->tgt_on);
    free(s->c_xy); free(s->c_r); free(s->c_lc); free(s->t_kind); free(s->t_ctr); free(s->pt_tgt); free(s->tgt_pt);
    free(s->s_kx); free(s->s_ky); free(s->c_kx); free(s->c_ky); free(s->p_kx); free(s->p_ky);
    for (int b = 0; b < s->nbox; ++b) { iv_free(&s->box[b].src); iv_free(&s->box[b].ctr); iv_free(&s->box[b].tgt); }
    free(s->box); free(s->src_owner); free(s->ctr_owner); free(s->pt_owner); free(s->forced);
    free_lists(s->L); free_lists(s->LB);
    free(s);
}

/* ------------------------------------------------------------------ A2: centres
 * Sec. 2.2.2: centres at t -/+ r n(t) with r proportional to the length of
 * the panel containing t.  Centre 2i is on the interior side (-n) of base
 * node i, centre 2i+1 on the exterior side (+n). */
static void form_centres(orc_state *s) {
    s->nc = 2 * s->nbase;
    s->c_xy = malloc(sizeof(double) * 2 * s->nc);
    s->c_r = malloc(sizeof(double) * s->nc);
    s->c_lc = malloc(sizeof(int) * s->nc);
    for (int i = 0; i < s->nbase; ++i) {
        int panel = i / s->g.nb;
        double r = (GQ_ORC_MUT == 17 ? 0.5 : 1.0) * s->p.radius_factor * s->panel_len[panel];
        for (int side = 0; side < 2; ++side) {
            double sg = (side ? 1.0 : -1.0) * (GQ_ORC_MUT == 18 ? -1.0 : 1.0);
            int c = 2 * i + side;
            s->c_xy[2 * c] = s->base_xy[2 * i] + sg * r * s->base_n[2 * i];
            s->c_xy[2 * c + 1] = s->base_xy[2 * i + 1] + sg * r * s->base_n[2 * i + 1];
            s->c_r[c] = r;
        }
    }
}

/* ------------------------------------------------------------------ A3: association
 * On-surface targets (given with their base node) use both centres of that
 * node and average the two one-sided values.  An off-surface target joins
 * the centre minimising |t-c|^2 / r^2 (lowest id on ties) if that ratio is
 * at most slack^2 (Sec. 2.2.2 allows a slack of up to 20%); otherwise it is
 * an ordinary point target of the FMM.  The nearest centre is found through
 * a uniform bucket grid whose cells are wider than any admissible distance,
 * so the result equals the exhaustive minimum. */
static void associate(orc_state *s) {
    int nt = s->g.ntargets;
    s->t_kind = malloc(sizeof(int) * (nt ? nt : 1));
    s->t_ctr = malloc(sizeof(int) * (nt ? nt : 1));
    s->tgt_pt = malloc(sizeof(int) * (nt ? nt : 1));
    double slack2 = s->p.assoc_slack * s->p.assoc_slack;
    double rmax = 0, x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
    for (int c = 0; c < s->nc; ++c) {
        if (s->c_r[c] > rmax) rmax = s->c_r[c];
        x0 = fmin(x0, s->c_xy[2 * c]); x1 = fmax(x1, s->c_xy[2 * c]);
        y0 = fmin(y0, s->c_xy[2 * c + 1]); y1 = fmax(y1, s->c_xy[2 * c + 1]);
    }
    double cell = 1.25 * s->p.assoc_slack * rmax;
    int ncx = 1, ncy = 1;
    if (s->nc > 0 && cell > 0) {
        ncx = (int)floor((x1 - x0) / cell) + 1;
        ncy = (int)floor((y1 - y0) / cell) + 1;
    }
    int *cstart = calloc((size_t)ncx * ncy + 1, sizeof(int));
    int *citems = malloc(sizeof(int) * (s->nc ? s->nc : 1));
    int *ccell = malloc(sizeof(int) * (s->nc ? s->nc : 1));
    for (int c = 0; c < s->nc; ++c) {
        int gx = (int)floor((s->c_xy[2 * c] - x0) / cell), gy = (int)floor((s->c_xy[2 * c + 1] - y0) / cell);
        if (gx < 0) gx = 0; if (gx >= ncx) gx = ncx - 1;
        if (gy < 0) gy = 0; if (gy >= ncy) gy = ncy - 1;
        ccell[c] = gy * ncx + gx; cstart[ccell[c] + 1]++;
    }
    for (int i = 0; i < ncx * ncy; ++i) cstart[i + 1] += cstart[i];
    int *fillp = malloc(sizeof(int) * ((size_t)ncx * ncy + 1));
    memcpy(fillp, cstart, sizeof(int) * ((size_t)ncx * ncy + 1));
    for (int c = 0; c < s->nc; ++c) citems[fillp[ccell[c]]++] = c;   /* ascending ids per cell */
    free(fillp); free(ccell);

    s->npt = 0;
    s->pt_tgt = malloc(sizeof(int) * (nt ? nt : 1));
    for (int t = 0; t < nt; ++t) {
        s->tgt_pt[t] = -1;
        if (s->tgt_on[t] >= 0) { s->t_kind[t] = 2; s->t_ctr[t] = 2 * s->tgt_on[t]; continue; }
        double tx = s->tgt_xy[2 * t], ty = s->tgt_xy[2 * t + 1];
        int best = -1; double bestk = INFINITY;
        double fgx = floor((tx - x0) / cell), fgy = floor((ty - y0) / cell);
        if (s->nc > 0 && cell > 0 && fgx >= -1 && fgx <= ncx && fgy >= -1 && fgy <= ncy) {
            int gx = (int)fgx, gy = (int)fgy;
            for (int yy = gy - 1; yy <= gy + 1; ++yy) {
                if (yy < 0 || yy >= ncy) continue;
                for (int xx = gx - 1; xx <= gx + 1; ++xx) {
                    if (xx < 0 || xx >= ncx) continue;
                    int cellid = yy * ncx + xx;
                    for (int k = cstart[cellid]; k < cstart[cellid + 1]; ++k) {
                        int c = citems[k];
                        double dx = tx - s->c_xy[2 * c], dy = ty - s->c_xy[2 * c + 1];
                        double d2 = dx * dx + dy * dy;
                        double key = d2 / (s->c_r[c] * s->c_r[c]);
                        if (key < bestk || (key == bestk && c < best)) { bestk = key; best = c; }
                    }
                }
            }
        }
        if (best >= 0 && bestk <= (GQ_ORC_MUT == 8 ? s->p.assoc_slack : slack2)) { s->t_kind[t] = 1; s->t_ctr[t] = best; }
        else { s->t_kind[t] = 0; s->t_ctr[t] = -1; s->tgt_pt[t] = s->npt; s->pt_tgt[s->npt++] = t; }
    }
    free(cstart); free(citems);
}

/* ------------------------------------------------------------------ A4: root, keys, centre levels
 * The root is a square holding all sources, point targets and every centre's
 * whole disk (Sec. 4.3).  Its half-width H is a power of two and its corner
 * a multiple of u = 2H / 2^30, so that every box centre is an exact binary
 * fraction.  Keys: k = floor((x - lo) / u), clamped to [0, 2^30). */
static void root_and_keys(orc_state *s) {
    double x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY;
    for (int i = 0; i < s->nsrc; ++i) {
        x0 = fmin(x0, s->up_xy[2 * i]); x1 = fmax(x1, s->up_xy[2 * i]);
        y0 = fmin(y0, s->up_xy[2 * i + 1]); y1 = fmax(y1, s->up_xy[2 * i + 1]);
    }
    for (int k = 0; k < s->npt; ++k) {
        int t = s->pt_tgt[k];
        x0 = fmin(x0, s->tgt_xy[2 * t]); x1 = fmax(x1, s->tgt_xy[2 * t]);
        y0 = fmin(y0, s->tgt_xy[2 * t + 1]); y1 = fmax(y1, s->tgt_xy[2 * t + 1]);
    }
    for (int c = 0; c < s->nc; ++c) {
        x0 = fmin(x0, s->c_xy[2 * c] - s->c_r[c]); x1 = fmax(x1, s->c_xy[2 * c] + s->c_r[c]);
        y0 = fmin(y0, s->c_xy[2 * c + 1] - s->c_r[c]); y1 = fmax(y1, s->c_xy[2 * c + 1] + s->c_r[c]);
    }
    double ext = fmax(x1 - x0, y1 - y0);
    if (!(ext > 0)) ext = 1.0;
    double target = 0.5 * ext * (1.0 + 0x1p-20);
    int e; double m = frexp(target, &e);          /* target = m 2^e, m in [0.5, 1) */
    s->H = (m == 0.5) ? ldexp(1.0, e - 1) : ldexp(1.0, e);
    s->u = ldexp(s->H, 1 - KEYBITS);
    s->lo_x = floor(x0 / s->u) * s->u;
    s->lo_y = floor(y0 / s->u) * s->u;

    int64_t kmax = ((int64_t)1 << KEYBITS) - 1;
#define KEY(v, lo) ({ double _f = floor(((v) - (lo)) / s->u); int64_t _k = (_f < 0) ? 0 : (_f > (double)kmax ? kmax : (int64_t)_f); _k; })
    s->s_kx = malloc(sizeof(int64_t) * (s->nsrc ? s->nsrc : 1)); s->s_ky = malloc(sizeof(int64_t) * (s->nsrc ? s->nsrc : 1));
    for (int i = 0; i < s->nsrc; ++i) { s->s_kx[i] = KEY(s->up_xy[2 * i], s->lo_x); s->s_ky[i] = KEY(s->up_xy[2 * i + 1], s->lo_y); }
    s->c_kx = malloc(sizeof(int64_t) * (s->nc ? s->nc : 1)); s->c_ky = malloc(sizeof(int64_t) * (s->nc ? s->nc : 1));
    for (int c = 0; c < s->nc; ++c) { s->c_kx[c] = KEY(s->c_xy[2 * c], s->lo_x); s->c_ky[c] = KEY(s->c_xy[2 * c + 1], s->lo_y); }
    s->p_kx = malloc(sizeof(int64_t) * (s->npt ? s->npt : 1)); s->p_ky = malloc(sizeof(int64_t) * (s->npt ? s->npt : 1));
    for (int k = 0; k < s->npt; ++k) { int t = s->pt_tgt[k]; s->p_kx[k] = KEY(s->tgt_xy[2 * t], s->lo_x); s->p_ky[k] = KEY(s->tgt_xy[2 * t + 1], s->lo_y); }
#undef KEY

    /* Centre level L_c (Sec. 4.3, TCR): the deepest level l such that the
     * centre's disk lies in TCR(b_l) = B_inf(|b_l|(1 + t_f), centre(b_l)) (or,
     * with the disk-shaped TCR, the l2 disk of that radius) for every box
     * b_0..b_l on its key path (fitting is monotone in l). */
    double tcr_scale = (double)(s->p.tf_den + s->p.tf_num) / (double)s->p.tf_den;
    for (int c = 0; c < s->nc; ++c) {
        int lc = -1;
        for (int l = 0; l <= s->p.max_level; ++l) {
            int64_t ix = s->c_kx[c] >> (KEYBITS - l), iy = s->c_ky[c] >> (KEYBITS - l);
            double hb = ldexp(s->H, -l);
            double bx = s->lo_x + (double)(2 * ix + 1) * hb;
            double by = s->lo_y + (double)(2 * iy + 1) * hb;
            double dx = s->c_xy[2 * c] - bx, dy = s->c_xy[2 * c + 1] - by;
            /* the disk lies in the square TCR when its l-inf distance plus r fits the
             * half-width, in the disk TCR when its l2 distance plus r fits the radius */
            double d = s->p.tcr_shape == 1
                           ? (GQ_ORC_MUT == 21 ? fmax(fabs(dx), fabs(dy)) : sqrt(dx * dx + dy * dy))
                           : fmax(fabs(dx), fabs(dy));
            d += (GQ_ORC_MUT == 16 ? 0.0 : s->c_r[c]);
            if (d <= hb * (GQ_ORC_MUT == 15 ? 1.0 : tcr_scale)) lc = l; else break;
        }
        s->c_lc[c] = lc < 0 ? 0 : lc;
    }
}

/* ------------------------------------------------------------------ A4: tree (Stage 1)
 * Repeatedly subdivide every box that owns more than n_max particles
 * eligible for its children (sources, point targets, centres whose disk
 * fits the child's TCR); empty children are pruned; centres that do not fit
 * stay in the parent (Sec. 4.3, Algorithm Stage 1). */
static int new_box(orc_state *s, int level, int64_t ix, int64_t iy, int parent) {
    if (s->nbox == s->capbox) {
        s->capbox = s->capbox ? 2 * s->capbox : 64;
        s->box = realloc(s->box, sizeof(obox) * s->capbox);
    }
    obox *b = &s->box[s->nbox];
    memset(b, 0, sizeof(obox));
    b->level = level; b->ix = ix; b->iy = iy; b->parent = parent;
    for (int q = 0; q < 4; ++q) b->child[q] = -1;
    b->h = ldexp(s->H, -level);
    b->cx = s->lo_x + (double)(2 * ix + 1) * b->h;
    b->cy = s->lo_y + (double)(2 * iy + 1) * b->h;
    return s->nbox++;
}

static int quadrant(int64_t kx, int64_t ky, int child_level) {
    int sh = KEYBITS - child_level;
    return (int)((kx >> sh) & 1) | (int)(((ky >> sh) & 1) << 1);
}

static uint64_t morton2(int64_t ix, int64_t iy) {
    uint64_t k = 0;
    for (int i = 0; i < KEYBITS; ++i) k |= (((uint64_t)ix >> i) & 1) << (2 * i) | (((uint64_t)iy >> i) & 1) << (2 * i + 1);
    return k;
}
static uint64_t box_key(int level, int64_t ix, int64_t iy) { return ((uint64_t)level << 60) | morton2(ix, iy); }
static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}
static int key_in(const uint64_t *keys, int n, uint64_t k) {
    return n > 0 && bsearch(&k, keys, n, sizeof(uint64_t), cmp_u64) != NULL;
}

static void build_tree(orc_state *s) {
    new_box(s, 0, 0, 0, -1);
    for (int i = 0; i < s->nsrc; ++i) iv_push(&s->box[0].src, i);
    for (int c = 0; c < s->nc; ++c) iv_push(&s->box[0].ctr, c);
    for (int k = 0; k < s->npt; ++k) iv_push(&s->box[0].tgt, k);
    int fbeg = 0, fend = 1;
    while (fbeg < fend) {
        for (int b = fbeg; b < fend; ++b) {
            int lev = s->box[b].level;
            if (lev >= s->p.max_level) continue;
            int elig = s->box[b].src.n + s->box[b].tgt.n;
            for (int k = 0; k < s->box[b].ctr.n; ++k) if (s->c_lc[s->box[b].ctr.v[k]] > lev) elig++;
            if (elig <= s->p.n_max &&
                !(elig > 0 && key_in(s->forced, s->nforced, box_key(lev, s->box[b].ix, s->box[b].iy))))
                continue;
            int cl = lev + 1;
            int cnt[4] = {0, 0, 0, 0};
            for (int k = 0; k < s->box[b].src.n; ++k) { int i = s->box[b].src.v[k]; cnt[quadrant(s->s_kx[i], s->s_ky[i], cl)]++; }
            for (int k = 0; k < s->box[b].tgt.n; ++k) { int i = s->box[b].tgt.v[k]; cnt[quadrant(s->p_kx[i], s->p_ky[i], cl)]++; }
            for (int k = 0; k < s->box[b].ctr.n; ++k) { int i = s->box[b].ctr.v[k]; if (s->c_lc[i] > lev) cnt[quadrant(s->c_kx[i], s->c_ky[i], cl)]++; }
            for (int q = 0; q < 4; ++q) {
                if (!cnt[q]) continue;
                int64_t ix = 2 * s->box[b].ix + (q & 1), iy = 2 * s->box[b].iy + (q >> 1);
                int nb = new_box(s, cl, ix, iy, b);     /* may move s->box */
                s->box[b].child[q] = nb;
            }
            obox *B = &s->box[b];
            for (int k = 0; k < B->src.n; ++k) { int i = B->src.v[k]; iv_push(&s->box[B->child[quadrant(s->s_kx[i], s->s_ky[i], cl)]].src, i); }
            for (int k = 0; k < B->tgt.n; ++k) { int i = B->tgt.v[k]; iv_push(&s->box[B->child[quadrant(s->p_kx[i], s->p_ky[i], cl)]].tgt, i); }
            ivec keep = {0};
            for (int k = 0; k < B->ctr.n; ++k) {
                int i = B->ctr.v[k];
                if (s->c_lc[i] > lev) iv_push(&s->box[B->child[quadrant(s->c_kx[i], s->c_ky[i], cl)]].ctr, i);
                else iv_push(&keep, i);
            }
            iv_free(&B->src); iv_free(&B->tgt); iv_free(&B->ctr);
            B->ctr = keep;
        }
        fbeg = fend; fend = s->nbox;
    }
    /* owners and subtree counts (children always have larger indices) */
    s->src_owner = malloc(sizeof(int) * (s->nsrc ? s->nsrc : 1));
    s->ctr_owner = malloc(sizeof(int) * (s->nc ? s->nc : 1));
    s->pt_owner = malloc(sizeof(int) * (s->npt ? s->npt : 1));
    for (int b = 0; b < s->nbox; ++b) {
        obox *B = &s->box[b];
        for (int k = 0; k < B->src.n; ++k) s->src_owner[B->src.v[k]] = b;
        for (int k = 0; k < B->ctr.n; ++k) s->ctr_owner[B->ctr.v[k]] = b;
        for (int k = 0; k < B->tgt.n; ++k) s->pt_owner[B->tgt.v[k]] = b;
        B->sub_src = B->src.n; B->sub_tgt = B->ctr.n + B->tgt.n;
    }
    for (int b = s->nbox - 1; b > 0; --b) {
        int par = s->box[b].parent;
        s->box[par].sub_src += s->box[b].sub_src;
        s->box[par].sub_tgt += s->box[b].sub_tgt;
    }
}

/* ------------------------------------------------------------------ integer box geometry
 * Coordinates in units of half the finest (level-30) box width: a level-l
 * box has half-width h = 2^(30-l) and centre (2 ix + 1) h.  All relations of
 * Sec. 4.3.1 reduce to integer comparisons of the l-inf centre distance. */
static inline int64_t i64abs(int64_t a) { return a < 0 ? -a : a; }
static inline int64_t bh(const obox *b) { return (int64_t)1 << (KEYBITS - b->level); }
static inline int64_t dcen(const obox *a, const obox *b) {
    int64_t dx = i64abs((2 * a->ix + 1) * bh(a) - (2 * b->ix + 1) * bh(b));
    int64_t dy = i64abs((2 * a->iy + 1) * bh(a) - (2 * b->iy + 1) * bh(b));
    return dx > dy ? dx : dy;
}
/* 'adjacent': the closed squares intersect.  A box is adjacent to itself
 * (List 1 counts the self-interaction among the adjacent ones), to its
 * ancestors and to its descendants. */
static inline int adjacent(const obox *a, const obox *b) {
    return GQ_ORC_MUT == 6 ? dcen(a, b) < bh(a) + bh(b) : dcen(a, b) <= bh(a) + bh(b);
}
/* k-colleagues with k = 2: same level, inside B_inf(5|b|, c_b). */
static inline int colleague2(const obox *a, const obox *b) { return a->level == b->level && dcen(a, b) <= 4 * bh(b); }
/* Disk-shaped TCR (appendix corrigendum), the definitions of Sec. 4.3 kept:
 * the l-inf distance between a square S(c_s, h) and a disk D(c_d, rho) is at
 * least s exactly when D misses the open square of half-width h + s around
 * c_s, i.e. when the l2 distance from c_d to the closed square S(c_s, h + s)
 * is at least rho:  max(X - T, 0)^2 + max(Y - T, 0)^2 >= rho^2  with X, Y the
 * absolute centre differences and T = h + s.  Integer arithmetic (units of
 * the level-30 half-width, scaled by td), squares in 128 bits. */
static inline int disk_clear(int64_t X, int64_t Y, int64_t T, int64_t rho) {
    __int128 ex = X > T ? (__int128)(X - T) : (GQ_ORC_MUT == 20 ? (__int128)(X - T) : 0);
    __int128 ey = Y > T ? (__int128)(Y - T) : (GQ_ORC_MUT == 20 ? (__int128)(Y - T) : 0);
    return ex * ex + ey * ey >= (__int128)rho * rho;
}
static inline void dxy(const obox *a, const obox *b, int64_t *X, int64_t *Y) {
    *X = i64abs((2 * a->ix + 1) * bh(a) - (2 * b->ix + 1) * bh(b));
    *Y = i64abs((2 * a->iy + 1) * bh(a) - (2 * b->iy + 1) * bh(b));
}
/* a < TCR(b): the l-inf distance between a and TCR(b) is at least 2|a|; for
 * the square TCR, dist >= 3|a| + |b|(1 + t_f) */
static inline int sep_a_tcrb_p(int shape, int64_t tn, int64_t td, const obox *a, const obox *b) {
    if (shape == 1) {
        int64_t X, Y;
        dxy(a, b, &X, &Y);
        return disk_clear(td * X, td * Y, 3 * td * bh(a), (td + tn) * bh(b));
    }
    return td * dcen(a, b) >= 3 * td * bh(a) + (GQ_ORC_MUT == 14 ? td : td + tn) * bh(b);
}
/* TCR(a) < b: the l-inf distance between TCR(a) and b is at least
 * 2|a|(1 + t_f); for the square TCR, dist >= 3|a|(1 + t_f) + |b| */
static inline int sep_tcra_b_p(int shape, int64_t tn, int64_t td, const obox *a, const obox *b) {
    if (shape == 1) {
        int64_t X, Y;
        dxy(a, b, &X, &Y);
        return disk_clear(td * X, td * Y, td * bh(b) + 2 * (td + tn) * bh(a), (td + tn) * bh(a));
    }
    return td * dcen(a, b) >= 3 * (GQ_ORC_MUT == 13 ? td : td + tn) * bh(a) + td * bh(b);
}
static inline int sep_a_tcrb(const orc_state *s, const obox *a, const obox *b) {
    return sep_a_tcrb_p(s->p.tcr_shape, s->p.tf_num, s->p.tf_den, a, b);
}
static inline int sep_tcra_b(const orc_state *s, const obox *a, const obox *b) {
    return sep_tcra_b_p(s->p.tcr_shape, s->p.tf_num, s->p.tf_den, a, b);
}
static inline int is_leaf(const obox *b) { return b->child[0] < 0 && b->child[1] < 0 && b->child[2] < 0 && b->child[3] < 0; }
static int is_strict_desc(const orc_state *s, int d, int a) {
    for (int w = s->box[d].parent; w >= 0; w = s->box[w].parent) if (w == a) return 1;
    return 0;
}
static int anc_at(const orc_state *s, int b, int level) {
    while (b >= 0 && s->box[b].level > level) b = s->box[b].parent;
    return b;
}

/* which boxes carry lists: U, W, X^close for boxes owning targets;
 * V and X^far for boxes with targets in their subtree. */
static int owns_targets(const orc_state *s, int b) { return s->box[b].ctr.n + s->box[b].tgt.n > 0; }

/* ------------------------------------------------------------------ A5: lists, O2
 * Built with recursively formed 2-colleague sets: colleagues of b are the
 * children of the colleagues of parent(b) within two boxes of b. */
typedef struct { ivec l[ORC_NLISTS]; } boxlists;

static void collect_leaves(const orc_state *s, int d, ivec *out) {
    if (s->box[d].sub_src == 0) return;
    if (is_leaf(&s->box[d])) { iv_push(out, d); return; }
    for (int q = 0; q < 4; ++q) if (s->box[d].child[q] >= 0) collect_leaves(s, s->box[d].child[q], out);
}

static void w_farclose(const orc_state *s, int b, int d, boxlists *bl) {
    const obox *B = &s->box[b], *D = &s->box[d];
    if (D->sub_src == 0) return;
    if (sep_a_tcrb(s, D, B)) {
        if (GQ_ORC_MUT != 10 && D->sub_src < s->p.w3_demote) collect_leaves(s, d, &bl->l[ORC_WC]);  /* Remark 1 */
        else iv_push(&bl->l[ORC_WF], d);
        return;
    }
    if (is_leaf(D)) { iv_push(&bl->l[ORC_WC], d); return; }
    for (int q = 0; q < 4; ++q) if (D->child[q] >= 0) w_farclose(s, b, D->child[q], bl);
}

/* descend a colleague's subtree: adjacent leaves -> List 1, first
 * non-adjacent boxes -> List 3 (then split close/far) */
static void u_w_descend(const orc_state *s, int b, int d, boxlists *bl, int want_targets) {
    const obox *B = &s->box[b], *D = &s->box[d];
    if (D->sub_src == 0) return;
    if (!adjacent(D, B)) { if (want_targets) w_farclose(s, b, d, bl); return; }
    if (is_leaf(D)) { if (want_targets) iv_push(&bl->l[ORC_U], d); return; }
    for (int q = 0; q < 4; ++q) if (D->child[q] >= 0) u_w_descend(s, b, D->child[q], bl, want_targets);
}

static void build_lists_o2(orc_state *s) {
    ivec *coll = calloc(s->nbox, sizeof(ivec));
    iv_push(&coll[0], 0);
    for (int b = 1; b < s->nbox; ++b) {
        int P = s->box[b].parent;
        for (int k = 0; k < coll[P].n; ++k) {
            const obox *C = &s->box[coll[P].v[k]];
            for (int q = 0; q < 4; ++q) {
                int d = C->child[q];
                if (d >= 0 && colleague2(&s->box[d], &s->box[b])) iv_push(&coll[b], d);
            }
        }
    }
    boxlists *bl = calloc(s->nbox, sizeof(boxlists));
    for (int b = 0; b < s->nbox; ++b) {
        const obox *B = &s->box[b];
        if (B->sub_tgt == 0) continue;
        int tb = owns_targets(s, b);
        /* List 2 */
        if (B->parent >= 0) {
            int P = B->parent;
            for (int k = 0; k < coll[P].n; ++k) {
                const obox *C = &s->box[coll[P].v[k]];
                for (int q = 0; q < 4; ++q) {
                    int d = C->child[q];
                    if (d >= 0 && !colleague2(&s->box[d], B) && s->box[d].sub_src > 0) iv_push(&bl[b].l[ORC_V], d);
                }
            }
        }
        if (tb) {
            /* List 1: leaves of b's own subtree (b included) */
            collect_leaves(s, b, &bl[b].l[ORC_U]);
            /* List 1: coarser or same-level adjacent leaves */
            for (int a = b; a >= 0; a = s->box[a].parent)
                for (int k = 0; k < coll[a].n; ++k) {
                    int d = coll[a].v[k];
                    const obox *D = &s->box[d];
                    if (d != a && is_leaf(D) && D->sub_src > 0 && adjacent(D, B)) iv_push(&bl[b].l[ORC_U], d);
                }
        }
        /* finer adjacent leaves (List 1) and List 3 from colleagues' subtrees */
        for (int k = 0; k < coll[b].n; ++k) {
            int t = coll[b].v[k];
            if (t == b || is_leaf(&s->box[t])) continue;
            for (int q = 0; q < 4; ++q) if (s->box[t].child[q] >= 0) u_w_descend(s, b, s->box[t].child[q], &bl[b], tb);
        }
        /* List 4 close / far: candidates are source leaves that are
         * 2-colleagues of b or of one of its ancestors. */
        int chain[KEYBITS + 2]; int lb = B->level;
        for (int a = b; a >= 0; a = s->box[a].parent) chain[s->box[a].level] = a;
        for (int m = 0; m <= lb; ++m) {
            int a = chain[m];
            for (int k = 0; k < coll[a].n; ++k) {
                int d = coll[a].v[k];
                const obox *D = &s->box[d];
                if (d == a || !is_leaf(D) || D->sub_src == 0) continue;
                /* membership in List 4 of chain[j] (Def. 6) */
                int inX_upto_l = 0, inX_upto_lm1 = 0, inX_b = 0;
                for (int j = m; j <= lb; ++j) {
                    int w = chain[j], mem;
                    if (j == m) mem = !adjacent(D, &s->box[w]);
                    else mem = adjacent(D, &s->box[chain[j - 1]]) && !adjacent(D, &s->box[w]);
                    if (mem) { inX_upto_l = 1; if (j <= lb - 1) inX_upto_lm1 = 1; if (j == lb) inX_b = 1; }
                }
                int close_b = inX_upto_l && !sep_tcra_b(s, B, D);
                if (close_b && tb) iv_push(&bl[b].l[ORC_XC], d);
                int close_par = 0;
                if (lb >= 1) close_par = inX_upto_lm1 && !sep_tcra_b(s, &s->box[chain[lb - 1]], D);
                if ((inX_b || close_par) && sep_tcra_b(s, B, D)) iv_push(&bl[b].l[ORC_XF], d);
            }
        }
    }
    for (int i = 0; i < ORC_NLISTS; ++i) {
        csr *L = &s->L[i];
        L->n = s->nbox;
        L->off = calloc(s->nbox + 1, sizeof(int));
        for (int b = 0; b < s->nbox; ++b) L->off[b + 1] = L->off[b] + bl[b].l[i].n;
        L->idx = malloc(sizeof(int) * (L->off[s->nbox] ? L->off[s->nbox] : 1));
        for (int b = 0; b < s->nbox; ++b) if (bl[b].l[i].n) memcpy(L->idx + L->off[b], bl[b].l[i].v, sizeof(int) * bl[b].l[i].n);
    }
    for (int b = 0; b < s->nbox; ++b) { iv_free(&coll[b]); for (int i = 0; i < ORC_NLISTS; ++i) iv_free(&bl[b].l[i]); }
    free(coll); free(bl);
}

/* ------------------------------------------------------------------ A5: lists, O3 brute force
 * Every pair (b, d) is tested against Definitions 1-8 as printed, including
 * the Remark 1 demotion of small List 3 far boxes. */
static int inW3(const orc_state *s, int b, int d) {            /* Def. 3 */
    const obox *B = &s->box[b], *D = &s->box[d];
    if (D->level <= B->level) return 0;
    int t = anc_at(s, d, B->level);
    if (!colleague2(&s->box[t], B)) return 0;
    if (adjacent(D, B)) return 0;
    for (int w = D->parent; w != t; w = s->box[w].parent) if (!adjacent(&s->box[w], B)) return 0;
    return 1;
}
static int inW3orDesc(const orc_state *s, int b, int d) {
    for (int a = d; a >= 0; a = s->box[a].parent) if (inW3(s, b, a)) return 1;
    return 0;
}
static int w3far_raw(const orc_state *s, int b, int d) {       /* Def. 5 */
    if (!inW3orDesc(s, b, d) || !sep_a_tcrb(s, &s->box[d], &s->box[b])) return 0;
    for (int w = s->box[d].parent; w >= 0; w = s->box[w].parent)
        if (inW3orDesc(s, b, w) && sep_a_tcrb(s, &s->box[w], &s->box[b])) return 0;
    return 1;
}
static int inX4(const orc_state *s, int w, int d) {            /* Def. 6 */
    const obox *W = &s->box[w], *D = &s->box[d];
    if (!is_leaf(D) || D->sub_src == 0) return 0;
    if (D->level == W->level) return colleague2(D, W) && !adjacent(D, W);
    if (D->level < W->level && W->parent >= 0) {
        int a = anc_at(s, w, D->level);
        return colleague2(D, &s->box[a]) && adjacent(D, &s->box[W->parent]) && !adjacent(D, W);
    }
    return 0;
}
static int x4close(const orc_state *s, int b, int d) {          /* Def. 7 */
    int any = 0;
    for (int w = b; w >= 0; w = s->box[w].parent) if (inX4(s, w, d)) { any = 1; break; }
    return any && !sep_tcra_b(s, &s->box[b], &s->box[d]);
}

int orc_lists_bruteforce(orc_state *s) {
    boxlists *bl = calloc(s->nbox, sizeof(boxlists));
    for (int b = 0; b < s->nbox; ++b) {
        const obox *B = &s->box[b];
        if (B->sub_tgt == 0) continue;
        int tb = owns_targets(s, b);
        for (int d = 0; d < s->nbox; ++d) {
            const obox *D = &s->box[d];
            if (D->sub_src == 0) continue;
            int leaf = is_leaf(D);
            if (tb && leaf && (d == b || is_strict_desc(s, d, b) || adjacent(D, B))) iv_push(&bl[b].l[ORC_U], d);   /* Def. 1 */
            if (D->level == B->level && B->level >= 1 && colleague2(&s->box[D->parent], &s->box[B->parent]) && !colleague2(D, B))
                iv_push(&bl[b].l[ORC_V], d);                                                                   /* Def. 2 */
            if (tb) {
                int far = w3far_raw(s, b, d);
                if (far && D->sub_src >= s->p.w3_demote) iv_push(&bl[b].l[ORC_WF], d);                       /* Def. 5 */
                if (leaf) {
                    int close = inW3orDesc(s, b, d) && !sep_a_tcrb(s, D, B);                                   /* Def. 4 */
                    if (!close) /* Remark 1: leaf below (or equal to) a demoted far box */
                        for (int a = d; a >= 0; a = s->box[a].parent)
                            if (w3far_raw(s, b, a) && s->box[a].sub_src < s->p.w3_demote) { close = 1; break; }
                    if (close) iv_push(&bl[b].l[ORC_WC], d);
                }
                if (x4close(s, b, d)) iv_push(&bl[b].l[ORC_XC], d);
            }
            /* Def. 8 */
            int xf = 0;
            if (sep_tcra_b(s, B, D)) {
                if (inX4(s, b, d)) xf = 1;
                if (!xf && B->parent >= 0 && x4close(s, B->parent, d)) xf = 1;
            }
            if (xf) iv_push(&bl[b].l[ORC_XF], d);
        }
    }
    free_lists(s->LB);
    for (int i = 0; i < ORC_NLISTS; ++i) {
        csr *L = &s->LB[i];
        L->n = s->nbox;
        L->off = calloc(s->nbox + 1, sizeof(int));
        for (int b = 0; b < s->nbox; ++b) L->off[b + 1] = L->off[b] + bl[b].l[i].n;
        L->idx = malloc(sizeof(int) * (L->off[s->nbox] ? L->off[s->nbox] : 1));
        for (int b = 0; b < s->nbox; ++b) if (bl[b].l[i].n) memcpy(L->idx + L->off[b], bl[b].l[i].v, sizeof(int) * bl[b].l[i].n);
    }
    for (int b = 0; b < s->nbox; ++b) for (int i = 0; i < ORC_NLISTS; ++i) iv_free(&bl[b].l[i]);
    free(bl);
    s->have_brute = 1;
    return 0;
}

static void free_tree(orc_state *s) {
    for (int b = 0; b < s->nbox; ++b) { iv_free(&s->box[b].src); iv_free(&s->box[b].ctr); iv_free(&s->box[b].tgt); }
    free(s->box); s->box = NULL; s->nbox = s->capbox = 0;
    free(s->src_owner); free(s->ctr_owner); free(s->pt_owner);
    s->src_owner = s->ctr_owner = s->pt_owner = NULL;
}

/* Level restriction (Sec. 4.6, remark on level-restricted quadtrees: adjacent
 * leaves' levels differ by at most one).  Reading: a leaf a at level l is in
 * violation when some box at level l + 2 touches it (closed squares
 * intersect; a deeper box touching a has such an ancestor).  A leaf in
 * violation that owns a particle eligible for children (and l < max_level) is
 * subdivided as in Stage 1 -- empty children pruned, centres moving only when
 * their disk fits the child's TCR -- by rebuilding the tree from the root
 * with the subdivision forced; repeat until no such leaf is left.  A leaf with
 * no particle eligible for children cannot be refined and keeps its
 * violation.  Candidates: the 20 level-(l+2) positions around a, looked up
 * among the existing boxes. */
static int balance_pass(orc_state *s) {
    int maxl = 0;
    for (int b = 0; b < s->nbox; ++b) if (s->box[b].level > maxl) maxl = s->box[b].level;
    uint64_t *keys = malloc(sizeof(uint64_t) * (size_t)(s->nbox > 0 ? s->nbox : 1));
    for (int b = 0; b < s->nbox; ++b) keys[b] = box_key(s->box[b].level, s->box[b].ix, s->box[b].iy);
    qsort(keys, s->nbox, sizeof(uint64_t), cmp_u64);
    int nnew = 0;
    uint64_t *add = malloc(sizeof(uint64_t) * (size_t)(s->nbox > 0 ? s->nbox : 1));
    for (int b = 0; b < s->nbox; ++b) {
        const obox *B = &s->box[b];
        int leaf = B->child[0] < 0 && B->child[1] < 0 && B->child[2] < 0 && B->child[3] < 0;
        int l = B->level;
        if (!leaf || l + 2 > maxl || l >= s->p.max_level) continue;
        int elig = B->src.n + B->tgt.n;
        for (int k = 0; k < B->ctr.n; ++k) if (s->c_lc[B->ctr.v[k]] > l) elig++;
        if (elig == 0) continue;
        int viol = 0;
        int64_t n2 = (int64_t)1 << (l + 2);
        for (int64_t Y = 4 * B->iy - 1; Y <= 4 * B->iy + 4 && !viol; ++Y)
            for (int64_t X = 4 * B->ix - 1; X <= 4 * B->ix + 4 && !viol; ++X) {
                if (X < 0 || Y < 0 || X >= n2 || Y >= n2) continue;
                if (X >= 4 * B->ix && X < 4 * B->ix + 4 && Y >= 4 * B->iy && Y < 4 * B->iy + 4) continue;
                if (GQ_ORC_MUT == 19 && (X < 4 * B->ix || X > 4 * B->ix + 3) && (Y < 4 * B->iy || Y > 4 * B->iy + 3))
                    continue;   /* planted mistake: corner neighbours ignored */
                if (key_in(keys, s->nbox, box_key(l + 2, X, Y))) viol = 1;
            }
        if (viol) add[nnew++] = box_key(l, B->ix, B->iy);
    }
    free(keys);
    if (nnew) {
        s->forced = realloc(s->forced, sizeof(uint64_t) * (s->nforced + nnew));
        memcpy(s->forced + s->nforced, add, sizeof(uint64_t) * nnew);
        s->nforced += nnew;
        qsort(s->forced, s->nforced, sizeof(uint64_t), cmp_u64);
    }
    free(add);
    return nnew;
}

int orc_build(orc_state *s) {
    form_centres(s);
    associate(s);
    root_and_keys(s);
    build_tree(s);
    while (s->p.level_restrict && balance_pass(s) > 0) {
        free_tree(s);
        build_tree(s);
    }
    build_lists_o2(s);
    return 0;
}

/* ------------------------------------------------------------------ accessors */
int orc_sep_test(int shape, int tn, int td, int which, int la, int64_t ixa, int64_t iya, int lb, int64_t ixb,
                 int64_t iyb) {
    obox a, b;
    memset(&a, 0, sizeof a);
    memset(&b, 0, sizeof b);
    a.level = la; a.ix = ixa; a.iy = iya;
    b.level = lb; b.ix = ixb; b.iy = iyb;
    return which == 0 ? sep_a_tcrb_p(shape, tn, td, &a, &b) : sep_tcra_b_p(shape, tn, td, &a, &b);
}

int orc_nbox(const orc_state *s) { return s->nbox; }
int orc_ncentres(const orc_state *s) { return s->nc; }
int orc_npoint_targets(const orc_state *s) { return s->npt; }
void orc_root(const orc_state *s, double out[4]) { out[0] = s->lo_x; out[1] = s->lo_y; out[2] = s->H; out[3] = s->u; }
void orc_boxes(const orc_state *s, int *level, int64_t *ix, int64_t *iy, int *parent,
               int *nsrc, int *nctr, int *ntgt, int *sub_src, int *sub_tgt) {
    for (int b = 0; b < s->nbox; ++b) {
        const obox *B = &s->box[b];
        level[b] = B->level; ix[b] = B->ix; iy[b] = B->iy; parent[b] = B->parent;
        nsrc[b] = B->src.n; nctr[b] = B->ctr.n; ntgt[b] = B->tgt.n; sub_src[b] = B->sub_src; sub_tgt[b] = B->sub_tgt;
    }
}
void orc_centres(const orc_state *s, double *xy, double *r, int *lc) {
    memcpy(xy, s->c_xy, sizeof(double) * 2 * s->nc); memcpy(r, s->c_r, sizeof(double) * s->nc);
    memcpy(lc, s->c_lc, sizeof(int) * s->nc);
}
void orc_assoc(const orc_state *s, int *kind, int *ctr) {
    memcpy(kind, s->t_kind, sizeof(int) * s->g.ntargets); memcpy(ctr, s->t_ctr, sizeof(int) * s->g.ntargets);
}
void orc_owners(const orc_state *s, int *src_owner, int *ctr_owner, int *tgt_owner) {
    memcpy(src_owner, s->src_owner, sizeof(int) * s->nsrc);
    memcpy(ctr_owner, s->ctr_owner, sizeof(int) * s->nc);
    for (int t = 0; t < s->g.ntargets; ++t) tgt_owner[t] = s->tgt_pt[t] >= 0 ? s->pt_owner[s->tgt_pt[t]] : -1;
}
int64_t orc_list_size(const orc_state *s, int which, int brute) {
    const csr *L = brute ? &s->LB[which] : &s->L[which];
    return L->off ? L->off[L->n] : 0;
}
void orc_list(const orc_state *s, int which, int brute, int *off, int *idx) {
    const csr *L = brute ? &s->LB[which] : &s->L[which];
    memcpy(off, L->off, sizeof(int) * (L->n + 1));
    memcpy(idx, L->idx, sizeof(int) * L->off[L->n]);
}

/* ------------------------------------------------------------------ A1: upsampling
 * Lagrange interpolation on the panel's reference nodes (Sec. 2.2.1:
 * density upsampled to the quadrature node count). */
void orc_upsample(const orc_state *s, const double *mu_base, double *mu_up) {
    int nb = s->g.nb, nu = s->g.nu;
    for (int P = 0; P < s->g.npanels; ++P)
        for (int j = 0; j < nu; ++j) {
            double t = s->ref_u[j], acc = 0;
            for (int i = 0; i < nb; ++i) {
                double li = 1.0;
                for (int k = 0; k < nb; ++k) if (k != i) li *= (t - s->ref_b[k]) / (s->ref_b[i] - s->ref_b[k]);
                acc += li * mu_base[P * nb + i];
            }
            mu_up[P * nu + j] = acc;
        }
}

/* ------------------------------------------------------------------ expansions (Sec. 3.1) */
static cplx cpow_int(cplx z, int n) { cplx r = 1; for (int i = 0; i < n; ++i) r *= z; return r; }

/* source strength: S -> q = w mu (real, stored as complex), D -> d = w mu n */
static void strengths(const orc_state *s, int kernel, const double *mu_base, cplx *str) {
    double *mu = malloc(sizeof(double) * s->nsrc);
    orc_upsample(s, mu_base, mu);
    for (int i = 0; i < s->nsrc; ++i) {
        double wm = s->up_w[i] * mu[i];
        if (kernel == ORC_D) str[i] = wm * (s->up_n[2 * i] + I * s->up_n[2 * i + 1]);
        else str[i] = wm;
    }
    free(mu);
}

static inline cplx pt(const double *xy, int i) { return xy[2 * i] + I * xy[2 * i + 1]; }

/* local coefficients about c (order q) of one source: eq. (local) / eq. (qbx) */
static void p2local(int kernel, int q, cplx c, cplx y, cplx str, cplx *beta) {
    cplx w = y - c;
    if (kernel == ORC_D) {
        for (int m = 0; m <= q; ++m) beta[m] += str / cpow_int(w, GQ_ORC_MUT == 5 ? m : m + 1);
    } else {
        beta[0] += str * clog(c - y);
        for (int m = 1; m <= q; ++m) beta[m] += -str / (m * cpow_int(w, m));
    }
}
/* potential Phi at t of one source */
static cplx p2pot(int kernel, cplx t, cplx y, cplx str) {
    if (kernel == ORC_D) return str / (y - t);
    return str * clog(t - y);
}
/* multipole coefficients (order p) about c of one source: eq. (multipole) */
static void p2mpole(int kernel, int p, cplx c, cplx y, cplx str, cplx *a) {
    cplx w = y - c;
    if (kernel == ORC_D) {
        for (int k = 1; k <= p; ++k) a[k] += -str * cpow_int(w, GQ_ORC_MUT == 12 ? k : k - 1);
    } else {
        a[0] += str;
        for (int k = 1; k <= p; ++k) a[k] += -str * cpow_int(w, k) / (GQ_ORC_MUT == 3 ? 1 : k);
    }
}
/* eq. (m2m): shift multipole from c_old to c_new, y = c_new - c_old */
static void m2m(const double binom[128][128], int p, cplx y, const cplx *a, cplx *out) {
    out[0] += a[0];
    for (int m = 1; m <= p; ++m) {
        cplx acc = -a[0] * cpow_int(-y, m) / m;
        for (int k = 1; k <= m; ++k)
            acc += (GQ_ORC_MUT == 2 ? binom[m][k - 1] : binom[m - 1][k - 1]) * a[k] * cpow_int(-y, m - k);
        out[m] += acc;
    }
}
/* eq. (m2l) with the a_0 sign fixed: multipole at 0 -> local at y (orders p_in, p_out) */
static void m2l(const double binom[128][128], int p_in, int p_out, cplx y, const cplx *a, cplx *out) {
    cplx acc = a[0] * clog(y);
    for (int k = 1; k <= p_in; ++k) acc += a[k] / cpow_int(y, k);
    out[0] += acc;
    for (int m = 1; m <= p_out; ++m) {
        double sg = (m % 2) ? -1.0 : 1.0;                    /* (-1)^m */
        acc = (GQ_ORC_MUT == 1 ? sg : -sg) * a[0] / (m * cpow_int(y, m));
        for (int k = 1; k <= p_in; ++k) acc += sg * binom[m + k - 1][GQ_ORC_MUT == 9 ? k : k - 1] * a[k] / cpow_int(y, m + k);
        out[m] += acc;
    }
}
/* eq. (l2l): local at 0 (order p_in) -> local at y (order p_out) */
static void l2l(const double binom[128][128], int p_in, int p_out, cplx y, const cplx *b, cplx *out) {
    for (int m = 0; m <= p_out; ++m) {
        cplx acc = 0;
        for (int k = m; k <= p_in; ++k) acc += binom[k][m] * b[k] * cpow_int(GQ_ORC_MUT == 4 ? -y : y, k - m);
        out[m] += acc;
    }
}
static cplx eval_local(int p, cplx c, const cplx *b, cplx t) {
    cplx acc = 0;
    for (int k = 0; k <= p; ++k) acc += b[k] * cpow_int(t - c, k);
    return acc;
}
static cplx eval_local_deriv(int p, cplx c, const cplx *b, cplx t) {
    cplx acc = 0;
    for (int k = 1; k <= p; ++k) acc += (GQ_ORC_MUT == 11 ? 1.0 : (double)k) * b[k] * cpow_int(t - c, k - 1);
    return acc;
}
static cplx eval_mpole(int p, cplx c, const cplx *a, cplx t) {
    cplx acc = a[0] * clog(t - c);
    for (int k = 1; k <= p; ++k) acc += a[k] / cpow_int(t - c, k);
    return acc;
}

/* ------------------------------------------------------------------ O2: Stages 2-8 */
static void final_values(orc_state *s, int kernel, const int *target_mask, const cplx *Q,
                         const cplx *pot_pt, double *value) {
    int q = s->p.p_qbx;
#pragma omp parallel for schedule(static) num_threads(g_threads)
    for (int t = 0; t < s->g.ntargets; ++t) {
        if (target_mask && !target_mask[t]) continue;
        cplx tt = pt(s->tgt_xy, t);
        if (s->t_kind[t] == 0) {
            value[t] = (kernel == ORC_SP) ? NAN : -creal(pot_pt[s->tgt_pt[t]]) / TWO_PI;
            continue;
        }
        int nside = s->t_kind[t] == 2 ? 2 : 1;
        double acc = 0;
        for (int k = 0; k < nside; ++k) {
            int c = s->t_ctr[t] + k;
            cplx cc = pt(s->c_xy, c);
            if (kernel == ORC_SP) {
                int node = s->tgt_on[t];
                cplx n = (node >= 0) ? pt(s->base_n, node) : NAN;
                acc += -creal(n * eval_local_deriv(q, cc, Q + (size_t)c * (q + 1), tt)) / TWO_PI;
            } else {
                acc += -creal(eval_local(q, cc, Q + (size_t)c * (q + 1), tt)) / TWO_PI;
            }
        }
        value[t] = GQ_ORC_MUT == 7 ? acc : acc / nside;
    }
}

static void mark_needed(orc_state *s, const int *target_mask, char *need_c, char *need_p) {
    for (int t = 0; t < s->g.ntargets; ++t) {
        if (target_mask && !target_mask[t]) continue;
        if (s->t_kind[t] == 0) need_p[s->tgt_pt[t]] = 1;
        else { need_c[s->t_ctr[t]] = 1; if (s->t_kind[t] == 2) need_c[s->t_ctr[t] + 1] = 1; }
    }
}

int orc_eval(orc_state *s, int kernel, const double *density_base, const int *target_mask,
             double *value, double *qbx_out) {
    int p = s->p.p_fmm, q = s->p.p_qbx, kin = (kernel == ORC_SP) ? ORC_S : kernel;
    size_t P1 = p + 1, Q1 = q + 1;
    cplx *str = malloc(sizeof(cplx) * s->nsrc);
    strengths(s, kin, density_base, str);
    char *need_c = calloc(s->nc + 1, 1), *need_p = calloc(s->npt + 1, 1);
    mark_needed(s, target_mask, need_c, need_p);
    char *need_box = calloc(s->nbox, 1), *need_far = calloc(s->nbox, 1);
    for (int c = 0; c < s->nc; ++c) if (need_c[c]) need_box[s->ctr_owner[c]] = 1;
    for (int k = 0; k < s->npt; ++k) if (need_p[k]) need_box[s->pt_owner[k]] = 1;
    for (int b = 0; b < s->nbox; ++b) if (need_box[b]) for (int a = b; a >= 0; a = s->box[a].parent) need_far[a] = 1;

    /* Stage 2: multipoles, leaves then postorder M2M (children have larger indices) */
    cplx *M = calloc((size_t)s->nbox * P1, sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 64) num_threads(g_threads)
    for (int b = 0; b < s->nbox; ++b) {
        obox *B = &s->box[b];
        cplx cb = B->cx + I * B->cy;
        for (int k = 0; k < B->src.n; ++k) { int i = B->src.v[k]; p2mpole(kin, p, cb, pt(s->up_xy, i), str[i], M + b * P1); }
    }
    for (int b = s->nbox - 1; b > 0; --b) {
        obox *B = &s->box[b];
        if (B->sub_src == 0) continue;
        obox *Pb = &s->box[B->parent];
        cplx y = (Pb->cx + I * Pb->cy) - (B->cx + I * B->cy);
        m2m(s->binom, p, y, M + b * P1, M + B->parent * P1);
    }
    /* Stages 4, 6b, 7: box local expansions, top down (parents first) */
    cplx *L = calloc((size_t)s->nbox * P1, sizeof(cplx));
    /* boxes are numbered level by level: one level at a time, a box's parent
     * (previous level) is complete before the box reads it */
    for (int lb = 0; lb < s->nbox;) {
        int le = lb;
        while (le < s->nbox && s->box[le].level == s->box[lb].level) ++le;
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int b = lb; b < le; ++b) {
        if (!need_far[b]) continue;
        obox *B = &s->box[b];
        cplx cb = B->cx + I * B->cy;
        if (B->parent >= 0) {
            obox *Pb = &s->box[B->parent];
            l2l(s->binom, p, p, cb - (Pb->cx + I * Pb->cy), L + B->parent * P1, L + b * P1);
        }
        for (int k = s->L[ORC_V].off[b]; k < s->L[ORC_V].off[b + 1]; ++k) {
            int d = s->L[ORC_V].idx[k];
            m2l(s->binom, p, p, cb - (s->box[d].cx + I * s->box[d].cy), M + d * P1, L + b * P1);
        }
        for (int k = s->L[ORC_XF].off[b]; k < s->L[ORC_XF].off[b + 1]; ++k) {
            obox *D = &s->box[s->L[ORC_XF].idx[k]];
            for (int j = 0; j < D->src.n; ++j) { int i = D->src.v[j]; p2local(kin, p, cb, pt(s->up_xy, i), str[i], L + b * P1); }
        }
    }
        lb = le;
    }
    /* Stages 3, 5, 6a, 8 for centres and point targets */
    cplx *Q = calloc((size_t)s->nc * Q1 + 1, sizeof(cplx));
    cplx *pot = calloc((size_t)s->npt + 1, sizeof(cplx));
    const int near_lists[3] = {ORC_U, ORC_WC, ORC_XC};
#pragma omp parallel for schedule(dynamic, 4) num_threads(g_threads)
    for (int b = 0; b < s->nbox; ++b) {
        if (!need_box[b]) continue;
        obox *B = &s->box[b];
        cplx cb = B->cx + I * B->cy;
        for (int kk = 0; kk < B->ctr.n; ++kk) {
            int c = B->ctr.v[kk];
            if (!need_c[c]) continue;
            cplx cc = pt(s->c_xy, c);
            cplx *beta = Q + (size_t)c * Q1;
            for (int li = 0; li < 3; ++li) {
                const csr *Ls = &s->L[near_lists[li]];
                for (int k = Ls->off[b]; k < Ls->off[b + 1]; ++k) {
                    obox *D = &s->box[Ls->idx[k]];
                    for (int j = 0; j < D->src.n; ++j) { int i = D->src.v[j]; p2local(kin, q, cc, pt(s->up_xy, i), str[i], beta); }
                }
            }
            for (int k = s->L[ORC_WF].off[b]; k < s->L[ORC_WF].off[b + 1]; ++k) {
                int d = s->L[ORC_WF].idx[k];
                m2l(s->binom, p, q, cc - (s->box[d].cx + I * s->box[d].cy), M + d * P1, beta);
            }
            l2l(s->binom, p, q, cc - cb, L + b * P1, beta);
        }
        for (int kk = 0; kk < B->tgt.n; ++kk) {
            int k_ = B->tgt.v[kk];
            if (!need_p[k_]) continue;
            cplx tt = pt(s->tgt_xy, s->pt_tgt[k_]);
            cplx acc = 0;
            for (int li = 0; li < 3; ++li) {
                const csr *Ls = &s->L[near_lists[li]];
                for (int k = Ls->off[b]; k < Ls->off[b + 1]; ++k) {
                    obox *D = &s->box[Ls->idx[k]];
                    for (int j = 0; j < D->src.n; ++j) {
                        int i = D->src.v[j];
                        cplx y = pt(s->up_xy, i);
                        if (y == tt) continue;   /* coincident source: skipped */
                        acc += p2pot(kin, tt, y, str[i]);
                    }
                }
            }
            for (int k = s->L[ORC_WF].off[b]; k < s->L[ORC_WF].off[b + 1]; ++k) {
                int d = s->L[ORC_WF].idx[k];
                acc += eval_mpole(p, s->box[d].cx + I * s->box[d].cy, M + d * P1, tt);
            }
            acc += eval_local(p, cb, L + b * P1, tt);
            pot[k_] = acc;
        }
    }
    final_values(s, kernel, target_mask, Q, pot, value);
    if (qbx_out)
        for (int c = 0; c < s->nc; ++c) if (need_c[c])
            for (int m = 0; m <= q; ++m) { qbx_out[2 * (c * Q1 + m)] = creal(Q[c * Q1 + m]); qbx_out[2 * (c * Q1 + m) + 1] = cimag(Q[c * Q1 + m]); }
    free(str); free(need_c); free(need_p); free(need_box); free(need_far); free(M); free(L); free(Q); free(pot);
    return 0;
}

/* ------------------------------------------------------------------ O1: direct QBX, eq. (qbx) */
int orc_direct(orc_state *s, int kernel, const double *density_base, const int *target_mask,
               double *value, double *qbx_out) {
    int q = s->p.p_qbx, kin = (kernel == ORC_SP) ? ORC_S : kernel;
    size_t Q1 = q + 1;
    cplx *str = malloc(sizeof(cplx) * s->nsrc);
    strengths(s, kin, density_base, str);
    char *need_c = calloc(s->nc + 1, 1), *need_p = calloc(s->npt + 1, 1);
    mark_needed(s, target_mask, need_c, need_p);
    cplx *Q = calloc((size_t)s->nc * Q1 + 1, sizeof(cplx));
    cplx *pot = calloc((size_t)s->npt + 1, sizeof(cplx));
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int c = 0; c < s->nc; ++c) {
        if (!need_c[c]) continue;
        cplx cc = pt(s->c_xy, c);
        for (int i = 0; i < s->nsrc; ++i) p2local(kin, q, cc, pt(s->up_xy, i), str[i], Q + c * Q1);
    }
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
    for (int k = 0; k < s->npt; ++k) {
        if (!need_p[k]) continue;
        cplx tt = pt(s->tgt_xy, s->pt_tgt[k]), acc = 0;
        for (int i = 0; i < s->nsrc; ++i) { cplx y = pt(s->up_xy, i); if (y != tt) acc += p2pot(kin, tt, y, str[i]); }
        pot[k] = acc;
    }
    final_values(s, kernel, target_mask, Q, pot, value);
    if (qbx_out)
        for (int c = 0; c < s->nc; ++c) if (need_c[c])
            for (int m = 0; m <= q; ++m) { qbx_out[2 * (c * Q1 + m)] = creal(Q[c * Q1 + m]); qbx_out[2 * (c * Q1 + m) + 1] = cimag(Q[c * Q1 + m]); }
    free(str); free(need_c); free(need_p); free(Q); free(pot);
    return 0;
}

/* ------------------------------------------------------------------ single operators */
static double g_binom[128][128];
static int g_binom_ready = 0;
static void ensure_binom(void) {
    if (g_binom_ready) return;
    for (int n = 0; n < 128; ++n) {
        g_binom[n][0] = 1.0;
        for (int k = 1; k <= n; ++k) g_binom[n][k] = g_binom[n - 1][k - 1] + (k <= n - 1 ? g_binom[n - 1][k] : 0.0);
    }
    g_binom_ready = 1;
}
static cplx rd(const double *v, int i) { return v[2 * i] + I * v[2 * i + 1]; }
static void wr(double *v, int i, cplx z) { v[2 * i] = creal(z); v[2 * i + 1] = cimag(z); }

void orc_op_p2m(int kernel, int p, const double *c, int n, const double *y, const double *str, double *a) {
    cplx *A = calloc(p + 1, sizeof(cplx));
    for (int i = 0; i < n; ++i) p2mpole(kernel, p, rd(c, 0), rd(y, i), rd(str, i), A);
    for (int k = 0; k <= p; ++k) wr(a, k, A[k]);
    free(A);
}
void orc_op_m2m(int p, const double *c_old, const double *c_new, const double *a, double *out) {
    ensure_binom();
    cplx *A = malloc(sizeof(cplx) * (p + 1)), *O = calloc(p + 1, sizeof(cplx));
    for (int k = 0; k <= p; ++k) A[k] = rd(a, k);
    m2m(g_binom, p, rd(c_new, 0) - rd(c_old, 0), A, O);
    for (int k = 0; k <= p; ++k) wr(out, k, O[k]);
    free(A); free(O);
}
void orc_op_m2l(int p_in, int p_out, const double *c_m, const double *c_l, const double *a, double *out) {
    ensure_binom();
    cplx *A = malloc(sizeof(cplx) * (p_in + 1)), *O = calloc(p_out + 1, sizeof(cplx));
    for (int k = 0; k <= p_in; ++k) A[k] = rd(a, k);
    m2l(g_binom, p_in, p_out, rd(c_l, 0) - rd(c_m, 0), A, O);
    for (int k = 0; k <= p_out; ++k) wr(out, k, O[k]);
    free(A); free(O);
}
void orc_op_p2l(int kernel, int p, const double *c, int n, const double *y, const double *str, double *b) {
    cplx *B = calloc(p + 1, sizeof(cplx));
    for (int i = 0; i < n; ++i) p2local(kernel, p, rd(c, 0), rd(y, i), rd(str, i), B);
    for (int k = 0; k <= p; ++k) wr(b, k, B[k]);
    free(B);
}
void orc_op_l2l(int p_in, int p_out, const double *c_old, const double *c_new, const double *b, double *out) {
    ensure_binom();
    cplx *B = malloc(sizeof(cplx) * (p_in + 1)), *O = calloc(p_out + 1, sizeof(cplx));
    for (int k = 0; k <= p_in; ++k) B[k] = rd(b, k);
    l2l(g_binom, p_in, p_out, rd(c_new, 0) - rd(c_old, 0), B, O);
    for (int k = 0; k <= p_out; ++k) wr(out, k, O[k]);
    free(B); free(O);
}
void orc_op_eval_local(int p, const double *c, const double *b, int n, const double *t, double *phi) {
    cplx *B = malloc(sizeof(cplx) * (p + 1));
    for (int k = 0; k <= p; ++k) B[k] = rd(b, k);
    for (int i = 0; i < n; ++i) wr(phi, i, eval_local(p, rd(c, 0), B, rd(t, i)));
    free(B);
}
void orc_op_eval_mpole(int p, const double *c, const double *a, int n, const double *t, double *phi) {
    cplx *A = malloc(sizeof(cplx) * (p + 1));
    for (int k = 0; k <= p; ++k) A[k] = rd(a, k);
    for (int i = 0; i < n; ++i) wr(phi, i, eval_mpole(p, rd(c, 0), A, rd(t, i)));
    free(A);
}
