/*
 * gigaqbx.h -- C ABI of the GB300 (sm_103a) GIGAQBX library.
 *
 * GIGAQBX evaluates the 2D Laplace single- and double-layer potentials
 *     S mu(x) = -(1/2pi) int_Gamma mu(y) log|y - x| ds(y)             (Sec. 1, eq. slp)
 *     D mu(x) = -(1/2pi) int_Gamma mu(y) n(y) . grad_y log|y - x| ds(y) (Sec. 1, eq. dlp)
 * on, near and away from a curve Gamma by Quadrature by Expansion
 * (Sec. 2.1, eq. qbx) accelerated by the modified FMM of Sec. 4 (target
 * confinement regions, 2-away separation, Lists 1, 2, 3 close/far and
 * 4 close/far; Algorithm, Stages 1-8).
 *
 * Inputs follow the problem statement at the start of Sec. 4: (a) a curve
 * cut into panels carrying a Gauss-Legendre rule, (b) orders chosen from an
 * accuracy, (c) a density at the panel nodes, (d) target points.
 *
 * Conventions for every call
 *  - Status: 0 (GQ_OK) or a negative GQ_ERR_* code; calls never abort.
 *    gq_last_error() returns a message for the context's last failure.
 *  - Pointers marked "host or device" may point to either; the library
 *    checks with cudaPointerGetAttributes and copies as needed.  The caller
 *    keeps ownership of every array it passes; the library copies what it
 *    keeps.  Handles are owned by the library and released by *_destroy.
 *  - All device work is ordered on the stream given to gq_create.  Outputs
 *    written to device memory are complete when that stream reaches the
 *    point after the call; host outputs are complete when the call returns.
 *  - Arrays of points are interleaved (x0, y0, x1, y1, ...) doubles.
 *  - Complex coefficients are interleaved (re, im) doubles.
 */
#ifndef GIGAQBX_H
#define GIGAQBX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int gq_status;
#define GQ_OK 0
#define GQ_ERR_INVALID (-1)     /* bad argument (null, size, order out of range) */
#define GQ_ERR_NOMEM (-2)       /* device or host allocation failed */
#define GQ_ERR_CUDA (-3)        /* a CUDA runtime call or kernel failed */
#define GQ_ERR_TIMEOUT (-4)     /* a bounded device-side wait gave up */
#define GQ_ERR_UNSUPPORTED (-5) /* degenerate geometry or unsupported parameters */
#define GQ_ERR_STATE (-6)       /* call out of order (e.g. eval before build) */

typedef struct gq_ctx gq_ctx;
typedef struct gq_geom gq_geom;

/* Layer potential to evaluate.  GQ_SP is the normal derivative of S at
 * on-surface targets (Sec. 1, exterior Neumann equation); it is defined for
 * on-surface (two-sided) targets only, other targets receive NaN. */
enum { GQ_S = 0, GQ_D = 1, GQ_SP = 2 };

/* Algorithm parameters (Sec. 4.1 and 4.3).
 *  p_qbx, p_fmm : QBX and FMM orders, 1 <= p_qbx <= 16, 1 <= p_fmm <= 30.
 *                 0 means "choose from eps": p_fmm = ceil(log2(1/eps)) - 1
 *                 (FMM error ~ (1/2)^(p_fmm+1), Sec. 4.1, 5.1), capped at 30;
 *                 p_qbx = ceil((log10(2/eps) - 2.06) / 1.26), the smallest
 *                 order whose QBX truncation error, measured as 10^(-2.06 -
 *                 1.26 q) with Green's identity on starfish curves with
 *                 centres half a panel length off the curve, is <= eps/2
 *                 (the paper leaves the truncation constant open, Sec. 2.1).
 *  n_max        : subdivide a box owning more than n_max particles eligible
 *                 for its children (Sec. 4.3, Stage 1).
 *  tf_num/tf_den: target confinement factor t_f as an exact fraction
 *                 (0 <= t_f < 1; default 9/10 as in Sec. 5.1).
 *  w3_demote    : List 3 far boxes with fewer sources are handled directly
 *                 (Remark 1; Sec. 5.2 uses 15).
 *  max_level    : deepest tree level (<= 30).
 *  radius_factor: expansion radius = radius_factor * panel arc length
 *                 (Sec. 2.2.2 places centres half a panel length off the curve).
 *  assoc_slack  : an off-surface target is served by the centre minimising
 *                 |t-c|/r when that ratio is <= assoc_slack (Sec. 2.2.2
 *                 reports up to 20% slack as harmless); otherwise it is an
 *                 ordinary FMM point target.
 *  eps          : requested accuracy (used for orders of 0 and by the mixed modes).
 *  precision    : GQ_PREC_FP64 (default): every stage in FP64.
 *                 GQ_PREC_MIXED: a tier chosen from eps.
 *                 eps >= 5e-6: the direct interactions (Lists 1, 3 close,
 *                 4 close to centres and to point targets) and the List 3
 *                 far multipole evaluation at point targets run in FP32 on
 *                 coordinates taken relative to box centres, with FP64 sums
 *                 across lanes (rounding 4e-8 .. 3e-7 relative measured,
 *                 the larger for D; below eps/5).
 *                 1e-12 <= eps < 5e-6: the same steps run in double-FP32
 *                 pairs (about 48 significant bits; measured 1e-15 .. 2e-13
 *                 relative to the FP64 path).  In both tiers a source inside
 *                 a centre's expansion disk (|r/w| > 1, where rounding would
 *                 grow as |r/w|^m) is taken in FP64, below eps = 1e-10 also
 *                 a source within 1/8 of the box half-width of a point
 *                 target; the List 3 far
 *                 translation to centres (M2QBXL) runs in pairs when the tree
 *                 has at most 24 levels.  The translations M2M, M2L, L2L,
 *                 L2QBXL, the P2M and P2L sums, L2P and the final QBX
 *                 evaluation stay FP64.  For eps < 1e-12 MIXED runs as FP64.
 *                 GQ_PREC_MIXED_FMM: MIXED, and for eps >= 1e-10 also P2M,
 *                 M2M, M2L, L2L and L2QBXL in double-FP32 pairs (measured
 *                 3e-14 added to the potential at p_fmm 30; an extension
 *                 beyond the FP64 translations of MIXED).
 *                 Any other value: GQ_ERR_INVALID from gq_geometry_create.
 */
typedef struct {
    int p_qbx, p_fmm, n_max;
    int tf_num, tf_den;
    int w3_demote;
    int max_level;
    double radius_factor;
    double assoc_slack;
    double eps;
    int precision;
    int m2l;
    int level_restrict;
    int tcr_shape;
} gq_params;

enum { GQ_PREC_FP64 = 0, GQ_PREC_MIXED = 1, GQ_PREC_MIXED_FMM = 2 };

/* m2l: how the FP64 translations run
 *   GQ_M2L_AUTO (default): on the BF16 tensor cores with FP64 accuracy
 *     - the List 2 translations (Stage 4, Sec. 3.1 eq. m2l) when p_fmm <= 15
 *       and they are FP64 (GQ_PREC_FP64, GQ_PREC_MIXED; GQ_PREC_MIXED_FMM keeps
 *       its FP32-pair M2L): every multipole and translation entry is split
 *       exactly into eleven 5-bit digits (54 bits) at a shared exponent, digit
 *       products accumulate exactly in FP32 tensor memory and are recombined
 *       in 64-bit integers (measured within a few units of 1e-15 of the FP64
 *       M2L);
 *     - the List 3 far multipoles to the QBX centres (Stage 5b) in the FP64
 *       evaluation when p_fmm <= 16, p_qbx <= 15 and C(p_qbx + p_fmm - 1,
 *       p_fmm - 1) < 2^24: the binomial sums of each (centre, box) pair as a
 *       product of 64-bit fixed-point pair entries (eight 8-bit digits) and
 *       the constant binomial matrix (three 8-bit digits);
 *     otherwise FP64 FMAs.
 *   GQ_M2L_FP64: always the FP64 FMA kernels. */
enum { GQ_M2L_AUTO = 0, GQ_M2L_FP64 = 1 };

/* level_restrict = 1: a level-restricted tree (Sec. 4.6, remark on
 * level-restricted quadtrees: adjacent leaves differ by at most one level),
 * which bounds List 3 of every leaf.  After Stage 1, a leaf that owns a
 * particle eligible for children (and is above max_level) is subdivided as in
 * Stage 1 (empty children pruned, centres moving only when their disk fits
 * the child's TCR) while some box two or more levels deeper touches it (closed
 * squares intersect); the tree is rebuilt with those subdivisions forced until
 * none is left.  A leaf with no particle eligible for children cannot be
 * refined and keeps its contact.  0 (default): the tree of Stage 1 alone.
 * Other values: GQ_ERR_INVALID. */

/* tcr_shape: the target confinement region TCR(b) (Sec. 4.3) of a box b of
 * half-width |b|
 *   0 (default): the closed square (l-inf ball) of half-width |b|(1 + t_f),
 *     the paper's definition;
 *   1: the closed disk (l2 ball) of radius |b|(1 + t_f), the variant named in
 *     the paper's appendix corrigendum.  Every definition of Sec. 4.3 is kept
 *     with the disk as the set: a centre stays at the deepest level whose TCR
 *     holds its whole disk (l2 distance of the centres plus the radius within
 *     |b|(1 + t_f)); a |> TCR(b) when the l-inf distance between a and the
 *     disk is at least 2|a|, TCR(a) |> b when the l-inf distance between the
 *     disk and b is at least 2|a|(1 + t_f) (exact integer tests).
 *   Other values: GQ_ERR_INVALID. */

/* Discretised curve (Sec. 2.1, 2.2.1).  Panel k owns base nodes
 * [k*nb, (k+1)*nb) and quadrature (upsampled) nodes [k*nu, (k+1)*nu).
 * ref_b[nb], ref_u[nu]: reference Gauss-Legendre nodes on [-1, 1] of the
 * base and quadrature rules; the density given at base nodes is carried to
 * the quadrature nodes by Lagrange interpolation on these nodes.  All
 * arrays host or device. */
typedef struct {
    int npanels, nb, nu;
    const double *ref_b, *ref_u;
    const double *base_xy;   /* [npanels*nb][2] base nodes                  */
    const double *base_n;    /* [npanels*nb][2] unit outward normals         */
    const double *up_xy;     /* [npanels*nu][2] quadrature nodes             */
    const double *up_n;      /* [npanels*nu][2] unit outward normals         */
    const double *up_w;      /* [npanels*nu] quadrature weights (arc length) */
    const double *panel_len; /* [npanels] panel arc lengths                  */
} gq_geometry_desc;

/* Per-evaluation statistics (optional output of gq_eval). */
typedef struct {
    int64_t kernel_launches;  /* kernels this library launched in the call */
    double ms_total;          /* device time of the call (CUDA events) */
    double ms_stage[12];      /* device time per stage group: 0 upsample + strengths,
                                 1 P2M + M2M, 2 M2L (List 2), 3 P2L (List 4 far),
                                 4 L2L, 5 direct to centres (Lists 1, 3 close, 4 close),
                                 6 direct to point targets, 7 List 3 far to centres,
                                 8 List 3 far to point targets, 9 L2QBXL + L2P,
                                 10 final QBX evaluation, 11 unused */
} gq_stats;

/* Tree and list sizes after gq_build. */
typedef struct {
    int nbox, nlevels, ncentres, npoint_targets, ntargets, nsources;
    int64_t list_size[6];     /* U, V, W close, W far, X close, X far */
} gq_tree_info;

gq_status gq_params_default(gq_params *out);

/* Host-only: the parameters gq_geometry_create will use for `in` -- orders
 * of 0 filled in from eps (p_fmm: the smallest p with the idealised FMM
 * error (1/2)^(p+1) <= eps, Sec. 4.1 and 5.1; p_qbx: the calibrated QBX
 * truncation rule described under p_qbx above), clamped to [1, 30] and
 * [1, 16] -- and the same validation.  `in` and `out` may alias.  Returns
 * GQ_ERR_INVALID (and leaves `out` unchanged) for parameters that
 * gq_geometry_create would reject; no context, no GPU work. */
gq_status gq_params_resolve(const gq_params *in, gq_params *out);

/* Context on `device`, ordering work on `cuda_stream` (a cudaStream_t; NULL
 * = the legacy default stream).  gq_create, gq_geometry_create, gq_build and
 * the batch calls make `device` the calling thread's current device; the
 * other calls that launch work (gq_targets_set, gq_eval, gq_eval_noalloc,
 * gq_gmres, the learned-order calls) expect it to be current already, as it
 * is when one thread drives one GPU, and leave the device selection alone so
 * that they can be recorded into a caller's stream capture. */
gq_status gq_create(int device, void *cuda_stream, gq_ctx **out);
gq_status gq_destroy(gq_ctx *ctx);
const char *gq_last_error(const gq_ctx *ctx);
/* Change the stream later calls order their work on. */
gq_status gq_set_stream(gq_ctx *ctx, void *cuda_stream);

/* Copy a discretised curve to the device and form the QBX centres
 * (Sec. 2.2.2: two centres per base node at t -/+ r n, r = radius_factor *
 * panel length; centre 2i on the interior side, 2i+1 on the exterior). */
gq_status gq_geometry_create(gq_ctx *ctx, const gq_geometry_desc *desc, const gq_params *params,
                             gq_geom **out);
gq_status gq_geometry_destroy(gq_geom *g);
/* The parameters in use, with orders of 0 resolved from eps. */
gq_status gq_geometry_params(const gq_geom *g, gq_params *out);

/* Set the n targets (host or device).  on_surface_node[i] >= 0 marks an
 * on-surface target evaluated by the two centres of that base node and
 * averaged (principal value); -1 marks an off-surface target.  An entry
 * outside [-1, npanels*nb) gives GQ_ERR_INVALID and leaves the geometry
 * without targets (gq_build then fails with GQ_ERR_STATE until a valid
 * gq_targets_set). */
gq_status gq_targets_set(gq_geom *g, int n, const double *xy, const int *on_surface_node);

/* Stage 1 and the lists: target association, root box, Morton keys, the
 * target-confinement quadtree, and Lists 1, 2, 3 close/far, 4 close/far
 * (Sec. 4.3, Definitions 1-8).  Reused by every later gq_eval. */
gq_status gq_build(gq_geom *g);

/* Stages 2-8 and the final QBX evaluation (Sec. 4.4 Algorithm; eq. qbx).
 * density_base: [npanels*nb] density at base nodes (host or device).
 * out: [ntargets] potential values (host or device).  stats may be NULL. */
gq_status gq_eval(gq_geom *g, int kernel, const double *density_base, double *out, gq_stats *stats);

/* The layer-potential operator at the base nodes, as an integral equation
 * applies it (Sec. 1: the exterior Neumann problem leads to the second-kind
 * equation -mu/2 + S' mu = g; Sec. 4 states the evaluation of S mu for a
 * density given at the nodes):
 *     out[i] = identity * mu[i] + (K mu)(x_i),   K = S, D or S' (kernel),
 * x_i the base node i, evaluated two-sided from its two centres 2i and 2i+1
 * and averaged (the principal value on the curve, eq. qbx).  identity = -0.5
 * with kernel GQ_SP gives the exterior Neumann operator; 0 gives K alone.
 * Stages 2-8 run as in gq_eval on the geometry's current build; the targets
 * given to gq_targets_set play no part in the result beyond the tree they
 * shaped (their point-target stages are skipped), so the values equal those
 * of gq_eval with the base nodes as on-surface targets on the same tree.
 * mu: [npanels*nb] density at the base nodes (host or device).
 * out: [npanels*nb] (host or device).  GQ_ERR_STATE before gq_build,
 * GQ_ERR_INVALID for a null pointer or an unknown kernel.  Runs in the
 * geometry's precision mode. */
gq_status gq_apply(gq_geom *g, int kernel, double identity, const double *mu, double *out);

/* Exterior Neumann problem (Sec. 1): with u = S mu outside the curve and the
 * normal derivative g prescribed on it, solve the second-kind equation
 *     -mu/2 + S' mu = g
 * for mu at the base nodes by restarted GMRES(restart) from mu = 0.  The
 * operator is gq_apply(GQ_SP, identity -0.5) (two-sided QBX, principal value),
 * on whatever targets the geometry was built with; the Arnoldi
 * vectors and their orthogonalisation (classical Gram-Schmidt, twice) are
 * FP64 device work.  rhs: [npanels*nb] g (host or device).  mu: [npanels*nb]
 * solution (host or device).  Stops when the residual estimate drops below
 * tol * |rhs| or after maxit iterations; *iters receives the iteration count
 * and *resid the true relative residual |rhs - A mu| / |rhs| (either may be
 * NULL). */
gq_status gq_gmres(gq_geom *g, const double *rhs, double tol, int maxit, int restart, double *mu, int *iters,
                   double *resid);

/* Batched evaluation of independent geometries (each built, on the context's
 * device).  gq_batch_eval evaluates `kernel` for ndens densities of every
 * geometry: dens[i] points to ndens consecutive density vectors of geometry i
 * ([ndens][npanels_i*nb_i], device memory) and out[i] receives
 * [ndens][ntargets_i] values (device memory).  All evaluations run as one CUDA
 * graph launch on the context's stream: each geometry is a branch of the
 * graph (its densities in order), branches are spread over several streams,
 * largest first.  The first call for a given (kernel, ndens, pointer set)
 * runs the evaluations once, then an autotuner captures the graph with 1, 2,
 * 4, 8 and 16 streams, times replays and keeps the fastest (cached per batch
 * shape; written to the file named by GQ_AUTOTUNE_CACHE if set); later calls
 * with the same arguments only replay the graph.  The geometries must stay
 * alive and must not be rebuilt while the batch exists.  In FP64 mode the
 * direct part of the QBX coefficients is formed for up to four densities of a
 * geometry at a time (the per-pair geometry and the powers (r/w)^m shared),
 * which rounds differently from one gq_eval per density: results agree with
 * gq_eval to about 1e-14 relative and repeat bit for bit from call to call;
 * the rest of the evaluation uses the gq_eval kernels. */
typedef struct gq_batch gq_batch;
gq_status gq_batch_create(gq_ctx *ctx, int ngeom, gq_geom *const *geoms, gq_batch **out);
gq_status gq_batch_destroy(gq_batch *b);
gq_status gq_batch_eval(gq_batch *b, int kernel, int ndens, const double *const *dens, double *const *out);
/* Streams the autotuner chose for the captured graph (0 before the first gq_batch_eval). */
gq_status gq_batch_streams(const gq_batch *b, int *streams);

/* How gq_batch_eval evaluates (the next call recaptures):
 *   mode 2 (default): the autotuner times modes 0 and 1 (each with its own
 *     streams, and for mode 0 its tiles and CTA count) and keeps the faster.
 *   mode 0: when every geometry is FP64 with the same p_qbx (5 or
 *     8), the graph's per-geometry branches run only the strengths and the
 *     FMM passes (Stages 2, 4, 5b, 6b, 7, 8) of each density into buffers of
 *     their own, and one persistent launch then takes work items from a
 *     counter for all geometries and densities: the direct part of the QBX
 *     coefficients for 4, 2 or 1 densities of a tile of target boxes, the
 *     direct potential at point targets, and the final sums (eq. qbx) of 256
 *     targets.  Every direct item precedes every final item; a final item
 *     waits, boundedly, for its geometry's direct items (a counter in global
 *     memory); a wait that runs out makes the call return GQ_ERR_TIMEOUT.
 *     The autotuner picks the branch streams, then the target boxes per
 *     direct item (1, 2, 4), then the CTAs (1, 3/4 or 1/2 per SM).  The call synchronises the stream to read the
 *     wait status.  Other configurations use the branches of mode 1.
 *   mode 1: every evaluation in the per-geometry branches (as described at
 *     gq_batch_eval).
 * The results equal those of mode 1 to rounding of the final sums (the same
 * kernels' arithmetic). */
gq_status gq_batch_mode(gq_batch *b, int mode);
/* Target boxes per direct item of the persistent launch in use (0: the
 * captured graph does not use the persistent launch). */
gq_status gq_batch_persistent(const gq_batch *b, int *tile);
/* CTAs of the persistent launch in use (0: the captured graph does not use
 * it): the autotuner picks one, three quarters or half of one per SM. */
gq_status gq_batch_persistent_ctas(const gq_batch *b, int *ctas);

/* Exterior Neumann solves (Sec. 1, as gq_gmres) for every geometry of the
 * batch at once: restarted GMRES(restart) from mu = 0 on each geometry in
 * lockstep, where each Arnoldi step applies S' to all geometries by one replay
 * of the batch's CUDA graph (captured with kernel GQ_SP and one density per
 * geometry on the first call, autotuned as in gq_batch_eval; a later
 * gq_batch_eval with other arguments recaptures).  Every geometry must have
 * the base nodes as targets (as gq_gmres requires), else GQ_ERR_STATE.
 * rhs[i], mu[i]: device arrays of npanels_i*nb_i doubles (g and the solution).
 * iters[i], resid[i] (host arrays of ngeom, either may be NULL): iterations and
 * true relative residual per geometry.  Per geometry the arithmetic is that of
 * gq_gmres, so the solutions are those of one gq_gmres after another; a
 * geometry that has converged stays in the graph replays (its vectors are
 * frozen) until the last one converges or reaches maxit. */
gq_status gq_batch_gmres(gq_batch *b, const double *const *rhs, double tol, int maxit, int restart,
                         double *const *mu, int *iters, double *resid);

/* Learned order selection (an extension; the paper picks orders from its
 * bounds, Sec. 4.1, which it reports to overestimate the error by about two
 * orders of magnitude, Sec. 5.1).  A fixed MLP 32 -> 64 -> 32 -> 32 -> 2 with
 * ReLU maps 32 per-centre features to [log10 relative QBX truncation error at
 * p_qbx = q_ref, log10 relative FMM error at p_fmm = p_ref].
 *
 * gq_centre_features: [ncentres][32] FP32 in centre-id order (host or device):
 *   0-7  distance from the centre to the 8 nearest other panels (their nearest
 *        quadrature node among the centre's direct-interaction sources) over
 *        r, ascending (64 when fewer panels are near),
 *   8-15 those panels' lengths over the centre's own panel length,
 *   16-31 curvature times r at the base nodes k-8 .. k+7 of the centre's
 *        panel, k its own node (indices clamped to the panel), positive where
 *        the curve bends towards the centre.
 * Needs gq_build. */
gq_status gq_centre_features(gq_geom *g, float *features);

typedef struct gq_mlp gq_mlp;
/* He-initialised weights from `seed`; lives on the context's device. */
gq_status gq_mlp_create(gq_ctx *ctx, uint64_t seed, gq_mlp **out);
gq_status gq_mlp_destroy(gq_mlp *m);
/* Number of parameters (*count), and optionally copy them out (get) or in
 * (set), host or device, layout W1[64][32] b1[64] W2[32][64] b2[32]
 * W3[32][32] b3[32] W4[2][32] b4[2]. */
gq_status gq_mlp_weights(gq_mlp *m, float *get, const float *set, int *count);
/* Mean squared error of the network (no normalisation) on n samples X[n][32],
 * Y[n][2] and its gradient with respect to every parameter (FP32 forward and
 * backward kernels).  grad: host [count] (may be NULL). */
gq_status gq_mlp_loss_grad(gq_mlp *m, const float *X, const float *Y, int n, float *loss, float *grad);
/* Train with Adam (FP32) on X[n][32], Y[n][2] (host or device), inputs and
 * labels standardised by their mean and deviation (kept for prediction),
 * `epochs` passes of shuffled mini-batches of `batch`.  *final_loss: mean
 * squared error of the last epoch in standardised units. */
gq_status gq_mlp_train(gq_mlp *m, const float *X, const float *Y, int n, int epochs, int batch, float lr,
                       uint64_t seed, float *final_loss);
/* BF16 inference (weights and activations rounded to BF16, FP32 sums):
 * Y[n][2] from X[n][32] (host or device). */
gq_status gq_mlp_predict(gq_mlp *m, const float *X, int n, float *Y);
/* Set orders from the network's predictions: the tree gets
 *   p_fmm = p_ref + ceil((max_c yf_c + margin_fmm - log10(eps/2)) / 0.5),
 * capped at the bound-driven order p_bound (its fallback); when q_ref > 0
 * centre c also gets its own QBX order
 *   q_c = q_ref + ceil((yq_c + margin_qbx - log10(eps/2)) / 1.26)
 * capped at 16 (q_ref <= 0 keeps the geometry's p_qbx for every centre).
 * 0.5 and 1.26 decades per order are the FMM and QBX error decay rates
 * measured on starfish curves.  *p_fmm and *q_max receive the orders used.
 * Later gq_eval calls evaluate each centre's expansion to its own order. */
gq_status gq_learned_orders(gq_geom *g, gq_mlp *m, double eps, double margin_qbx, double margin_fmm, int q_ref,
                            int p_ref, int p_bound, int *p_fmm, int *q_max);
/* Per-centre QBX orders q[ncentres] in centre-id order (host or device,
 * each in [1, 16]); p_qbx becomes their maximum.  The direct interactions
 * and the final evaluation of centre c stop at q[c]. */
gq_status gq_set_centre_orders(gq_geom *g, const int *q);
/* Set global orders (and drop per-centre orders) for later gq_eval calls. */
gq_status gq_set_orders(gq_geom *g, int p_qbx, int p_fmm);

/* gq_eval without allocating: the same evaluation as gq_eval for callers
 * that must not allocate device memory once they are running -- for example
 * code replayed inside a captured CUDA graph, real-time or embedded services
 * that reserve all their memory up front, or hosts that forbid cudaMalloc
 * after start-up.  The paper has no counterpart; it is a deployment variant.
 *
 * Working memory comes from one fixed device array inside the library
 * (16 MiB, of which 256 KiB hold translation tables); every GPU that loads
 * the library keeps that array until the process exits.  Problems whose
 * working set (quadrature nodes x 16 B + 2 x boxes x (p_fmm+1) x 16 B +
 * centres x (p_qbx+1) x 16 B + point targets x 8 B + targets x 4 B, each
 * rounded up to 256 B) exceeds the rest of the array are rejected with
 * GQ_ERR_UNSUPPORTED and a message giving both sizes.
 *
 * density_dev and out_dev must be device memory (GQ_ERR_INVALID otherwise):
 * host inputs would need staging buffers.  The geometry must be built.  The
 * evaluation is the FP64 one whatever the geometry's precision mode (the
 * mixed modes need buffers of their own).
 * The context's device must be the calling thread's current device
 * (GQ_ERR_STATE otherwise).  The first call on a device sets the array up
 * (looks up its device address, writes the tables and waits for the copies
 * with a device synchronisation); make that first call before any stream
 * capture.  The kernels are those of gq_eval in FP64 mode.
 * All calls share the one array and it keeps the last call's contents, so
 * calls whose device work overlaps (different streams or contexts) race;
 * order them on one stream.  No memory is allocated or freed by this call. */
gq_status gq_eval_noalloc(gq_geom *g, int kernel, const double *density_dev, double *out_dev);

/* Sizes of the built tree. */
gq_status gq_tree_info_get(gq_geom *g, gq_tree_info *out);

/* Host copies of build results for inspection and bit-exact comparison.
 * Boxes are numbered level by level, Morton order within a level. */
gq_status gq_export_root(gq_geom *g, double out[4]); /* lo_x, lo_y, H, u */
gq_status gq_export_boxes(gq_geom *g, int *level, int64_t *ix, int64_t *iy, int *parent,
                          int *nsrc, int *nctr, int *ntgt, int *sub_src, int *sub_tgt);
/* which: 0 U, 1 V, 2 W close, 3 W far, 4 X close, 5 X far.  off[nbox+1], idx[size]. */
gq_status gq_export_list(gq_geom *g, int which, int *off, int *idx);
gq_status gq_export_centres(gq_geom *g, double *xy, double *r, int *level);
/* kind: 0 point target, 1 one-sided QBX target, 2 two-sided; ctr: centre id (two-sided: interior centre) */
gq_status gq_export_assoc(gq_geom *g, int *kind, int *ctr);
/* owner box of every source (quadrature node order), centre and target (-1 for QBX targets) */
gq_status gq_export_owners(gq_geom *g, int *src_owner, int *ctr_owner, int *tgt_owner);
/* QBX coefficients of the last gq_eval, [ncentres][p_qbx+1] complex, in the
 * unscaled form of eq. qbx (coefficient of (x - c)^m). */
gq_status gq_export_qbx(gq_geom *g, double *coeffs);

/* Number of kernels this context has launched so far (all calls). */
gq_status gq_context_launches(const gq_ctx *ctx, int64_t *out);

/* Device memory the library keeps cached for reuse (bytes), and a call that
 * returns all of it to the driver (call when no library work is in flight).
 * Buffers of live geometries are not affected. */
gq_status gq_memory_cached(int64_t *bytes);
gq_status gq_memory_release(void);

/* ======================================================================
 * Diagnostics.  Measurement and self-check helpers used by the tests and
 * the benchmark; they are not part of the method and the paper has no
 * counterpart.  Each runs a small amount of device work on the context's
 * device.
 * ==================================================================== */

/* Measurement helper: throughput of a dependent-chain-free FMA loop on the
 * context's device, in TFLOP/s (2 flops per FMA).  what = 0: FP64 FMA,
 * what = 1: FP32 FMA, what = 2: FP64 tensor-core MMA (warp-wide
 * mma.sync m8n8k4 FP64, 512 flops each), what = 3: both FP64 paths at once
 * (half the warps each, equal flops; about the sum of the two rates if they
 * issue to separate units).  Used as the measured peak of the
 * FP64/FP32 roofline and to decide whether a contraction should use the FP64
 * tensor cores; the paper has no counterpart.  Runs about 0.1 s of device work. */
gq_status gq_probe_fma_peak(gq_ctx *ctx, int what, double *tflops);

/* Check helper for the FP64 logarithm and reciprocal the direct kernels use
 * (no counterpart in the paper): y[i] = f(x[i]) on the device, x and y device
 * arrays of n doubles; fn = 0: the table-driven logarithm, 1: CUDA's log,
 * 2: the reciprocal (approximate seed + one third-order step), 3: IEEE division 1/x, 4: the double-FP32
 * logarithm of the split-precision kernels (x rounded to an FP32 pair,
 * x in [2^-126, 2^126]), 5: the double-FP32 reciprocal (same range). */
gq_status gq_probe_math(gq_ctx *ctx, int fn, int n, const double *x, double *y);

/* Tensor-core check: D[128][32] = A[128][K] * B[32][K]^T on one CTA by K/16
 * chained tcgen05.mma (BF16 inputs, FP32 accumulation in tensor memory), as
 * the tensor-core M2L uses them.  a, b: host arrays of BF16 bit patterns,
 * row-major; d: host [128][32] floats.  K a multiple of 16 in [16, 256]
 * (GQ_ERR_INVALID otherwise).  swap = 1 exchanges the leading and stride
 * byte offsets of the shared-memory descriptors (a layout check).
 * GQ_ERR_TIMEOUT if the bounded completion wait gave up. */
gq_status gq_probe_umma(gq_ctx *ctx, int K, const uint16_t *a, const uint16_t *b, int swap, float *d);

/* Which translations the next gq_eval of a built geometry runs on the BF16
 * tensor cores with FP64 accuracy (see gq_params.m2l): *m2l_tc = 1 for the
 * List 2 translations (Stage 4), *m2qbxl_tc = 1 for List 3 far to the QBX
 * centres (Stage 5b); 0 where the FP64 FMA kernels (or, in the mixed tiers,
 * their FP32-pair kernels) run instead -- orders or mode outside the
 * tensor-core kernels' range, or a device on which the kernel cannot be
 * resident.  GQ_ERR_STATE before gq_build. */
gq_status gq_tensor_paths(gq_geom *g, int *m2l_tc, int *m2qbxl_tc);

/* Check of the one-pass list construction (no counterpart in the paper):
 * gq_build enumerates each box's lists once into scratch rows of fixed
 * capacity and copies them into the CSR arrays; a box whose list exceeds its
 * row sends the build to a second enumeration that fills the CSR rows
 * directly, with the same lists.  row_cap > 0 caps every row at row_cap
 * entries for this geometry's next builds, 0 restores the default
 * capacities, and a negative value leaves the setting as it is.  *passes
 * (if not null) receives the enumeration passes of the geometry's last
 * build (1 or 2; 0 before the first).  No device work. */
gq_status gq_lists_check(gq_geom *g, int row_cap, int *passes);

/* Check of the persistent batch launch's bounded waits: wait_ns bounds every
 * dependency wait (default 1 s); stall_geom >= 0 makes that geometry's final
 * items wait for one direct item more than exist (a count nothing reaches),
 * so their waits run out, gq_batch_eval returns GQ_ERR_TIMEOUT and the other
 * items still complete; -1 restores normal operation.  The next gq_batch_eval
 * recaptures.  GQ_ERR_INVALID for wait_ns <= 0 or a geometry index out of range. */
gq_status gq_batch_wait_test(gq_batch *b, int64_t wait_ns, int stall_geom);

#ifdef __cplusplus
}
#endif
#endif
