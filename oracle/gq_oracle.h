/*
 * gq_oracle.h -- plain, slow, serial FP64 CPU oracle for GIGAQBX
 * (Wala & Kloeckner, "A Fast Algorithm with Error Bounds for Quadrature by
 * Expansion", 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may call this library.  It shares no code with
 * the CUDA path (no headers, helpers, tables or constant generators).
 *
 * Contents
 *   O1  direct (unaccelerated) QBX, eq. (qbx) of Sec. 2.1
 *   O2  the GIGAQBX FMM, Stages 1-8 of the Algorithm in Sec. 4.4, written
 *       with unscaled textbook expansions (Sec. 3.1, eqs. multipole, m2m,
 *       m2l, local, l2l) and straightforward loops
 *   O3  brute-force interaction lists straight from Definitions 1-8 of
 *       Sec. 4.3.2 by enumerating all box pairs (small trees only)
 *
 * Parity status: every function is pinned by the CPU tests (closed forms on
 * the unit circle, Green's identity, operator exactness and the error bounds
 * of Lemmas 1-3, brute-force lists and the interaction partition invariant,
 * O2 against O1 within the Theorem's bound).
 */
#ifndef GQ_ORACLE_H
#define GQ_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int npanels, nb, nu;          /* panels, base nodes / panel, quadrature nodes / panel */
    const double *ref_b, *ref_u;  /* reference Gauss-Legendre nodes in [-1,1] (nb, nu) */
    const double *base_xy;        /* [npanels*nb][2] base nodes */
    const double *base_n;         /* [npanels*nb][2] unit outward normals */
    const double *up_xy, *up_n;   /* [npanels*nu][2] quadrature nodes / normals */
    const double *up_w;           /* [npanels*nu] quadrature weights (arc length) */
    const double *panel_len;      /* [npanels] panel arc lengths */
    int ntargets;
    const double *tgt_xy;         /* [ntargets][2] */
    const int *tgt_onsurf;        /* base node index (two-sided on-surface) or -1 */
} orc_geom;

typedef struct {
    int p_qbx, p_fmm, n_max;
    int tf_num, tf_den;           /* target confinement factor t_f = tf_num/tf_den */
    int w3_demote;                /* List 3 far boxes with fewer sources go direct */
    int max_level;                /* <= 30 */
    double radius_factor;         /* expansion radius = radius_factor * panel length */
    double assoc_slack;           /* off-surface target joins a centre if |t-c|/r <= slack */
    int level_restrict;           /* 1: balance the tree (Sec. 4.6, level-restriction remark) */
    int tcr_shape;                /* TCR(b): 0 the closed l-inf ball (square) of radius |b|(1 + t_f)
                                     (Sec. 4.3), 1 the closed l2 disk of that radius (the variant of
                                     the appendix corrigendum) */
} orc_params;

enum { ORC_U = 0, ORC_V = 1, ORC_WC = 2, ORC_WF = 3, ORC_XC = 4, ORC_XF = 5, ORC_NLISTS = 6 };
enum { ORC_S = 0, ORC_D = 1, ORC_SP = 2 };

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_geom *g, const orc_params *p);
void orc_destroy(orc_state *s);
/* Stages A2-A5: centres, target association, root, keys, tree, lists (O2). */
int orc_build(orc_state *s);
/* The adequate-separation relations of Sec. 4.3 (Def. "adequate separation")
 * for two boxes given by level and index, with TCR shape `shape` (as
 * orc_params.tcr_shape) and t_f = tn / td: which 0 tests a |> TCR(b), which 1
 * tests TCR(a) |> b.  Exposed for tests of the relations themselves. */
int orc_sep_test(int shape, int tn, int td, int which, int la, int64_t ixa, int64_t iya, int lb, int64_t ixb,
                 int64_t iyb);
/* O3: brute-force lists into a second list set. */
int orc_lists_bruteforce(orc_state *s);

/* Accessors (arrays sized by the matching count). */
int orc_nbox(const orc_state *s);
int orc_ncentres(const orc_state *s);
int orc_npoint_targets(const orc_state *s);
void orc_root(const orc_state *s, double out[4]);  /* lo_x, lo_y, H, u */
void orc_boxes(const orc_state *s, int *level, int64_t *ix, int64_t *iy, int *parent,
               int *nsrc, int *nctr, int *ntgt, int *sub_src, int *sub_tgt);
void orc_centres(const orc_state *s, double *xy, double *r, int *lc);
void orc_assoc(const orc_state *s, int *kind, int *ctr);
void orc_owners(const orc_state *s, int *src_owner, int *ctr_owner, int *tgt_owner);
int64_t orc_list_size(const orc_state *s, int which, int brute);
void orc_list(const orc_state *s, int which, int brute, int *off, int *idx);

/* A1: Lagrange upsampling of a base-node density to the quadrature nodes. */
void orc_upsample(const orc_state *s, const double *mu_base, double *mu_up);

/* O2.  kernel: ORC_S, ORC_D or ORC_SP (normal derivative of S, QBX targets
 * only).  target_mask (may be NULL = all) selects the targets computed;
 * value[nt] receives the result (unselected entries untouched).  qbx_out
 * (may be NULL) receives [nc][p_qbx+1] complex coefficients (interleaved
 * re,im) for the centres that were needed. */
/* Threads of the evaluation loops (OpenMP builds; 1 = serial, the default).
 * Results do not depend on it.  Returns the count in effect. */
int orc_set_threads(int n);
/* Processors OpenMP sees (1 without OpenMP). */
int orc_max_threads(void);

int orc_eval(orc_state *s, int kernel, const double *density_base, const int *target_mask,
             double *value, double *qbx_out);
/* O1: direct QBX / direct point sums, same conventions. */
int orc_direct(orc_state *s, int kernel, const double *density_base, const int *target_mask,
               double *value, double *qbx_out);

/* Single translation operators (unscaled, complex interleaved), used to pin
 * the oracle against brute force and the bounds of Lemmas 1-3. */
void orc_op_p2m(int kernel, int p, const double *c, int n, const double *y,
                const double *str, double *a);
void orc_op_m2m(int p, const double *c_old, const double *c_new, const double *a, double *out);
void orc_op_m2l(int p_in, int p_out, const double *c_m, const double *c_l, const double *a,
                double *out);
void orc_op_p2l(int kernel, int p, const double *c, int n, const double *y,
                const double *str, double *b);
void orc_op_l2l(int p_in, int p_out, const double *c_old, const double *c_new, const double *b,
                double *out);
void orc_op_eval_local(int p, const double *c, const double *b, int n, const double *t,
                       double *phi);
void orc_op_eval_mpole(int p, const double *c, const double *a, int n, const double *t,
                       double *phi);

#ifdef __cplusplus
}
#endif
#endif
