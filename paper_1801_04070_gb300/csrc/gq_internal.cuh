// gq_internal.cuh -- shared declarations of the GIGAQBX CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gigaqbx.h"

#define GQ_KEYBITS 30
#define GQ_MAX_PQBX 16
#define GQ_MAX_PFMM 30

// ------------------------------------------------------------------ errors
struct gq_error {
    gq_status code;
    std::string msg;
};

#define GQ_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            throw gq_error{GQ_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
    } while (0)
#define GQ_CHECK_LAUNCH() GQ_CUDA(cudaGetLastError())
#define GQ_REQUIRE(cond, code, text) \
    do {                             \
        if (!(cond)) throw gq_error{code, text}; \
    } while (0)

// ------------------------------------------------------------------ device memory
// Caching allocator (gq_alloc.cu): blocks come in power-of-two size classes per
// device; a released block goes back to its class's free list instead of to
// cudaFree, so steady-state builds and evaluations allocate nothing from the
// driver and never hit cudaFree's implicit device synchronisation.  On an
// allocation failure the device's cached blocks are freed and the call retried.
// A block released while kernels still read it may be handed out again: every
// user in this library releases only after the last use on the same stream or
// after synchronising with it.
void *gq_dev_alloc(size_t bytes, size_t *cap, int *device);
void gq_dev_free(void *p, size_t cap, int device);
size_t gq_dev_cached_bytes();
void gq_dev_release_cache();

template <class T>
struct dbuf {
    T *p = nullptr;
    size_t n = 0;
    size_t cap = 0;
    int dev = 0;
    dbuf() = default;
    dbuf(const dbuf &) = delete;
    dbuf &operator=(const dbuf &) = delete;
    ~dbuf() { release(); }
    void release() {
        if (p) gq_dev_free(p, cap, dev);
        p = nullptr;
        n = 0;
        cap = 0;
    }
    void alloc(size_t count) {
        if (count <= n && p) return;
        release();
        size_t bytes = (count ? count : 1) * sizeof(T);
        p = (T *)gq_dev_alloc(bytes, &cap, &dev);
        n = count;
    }
    void swap(dbuf &o) {
        T *tp = p; p = o.p; o.p = tp;
        size_t tn = n; n = o.n; o.n = tn;
        size_t tc = cap; cap = o.cap; o.cap = tc;
        int td = dev; dev = o.dev; o.dev = td;
    }
    operator T *() const { return p; }
};

struct gq_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string last_error;
    int64_t launches = 0;   // kernels launched by this context
};

// box-centre geometry broadcast to kernels
struct RootInfo {
    double lo_x, lo_y, H, u;
};

struct gq_geom {
    gq_ctx *ctx = nullptr;
    gq_params prm{};
    int npanels = 0, nb = 0, nu = 0, nbase = 0, nsrc = 0, nc = 0, nt = 0;
    // geometry (device, original order)
    dbuf<double> base_xy, base_n, up_xy, up_n, up_w, panel_len, interp;  // interp [nu][nb]
    dbuf<double> c_xy, c_r;
    dbuf<int> c_lc;
    // targets
    dbuf<double> tgt_xy;
    dbuf<int> tgt_on;
    bool targets_set = false;
    bool targets_are_base_nodes = false;   // target i is on-surface at base node i, nt == nbase
    // association
    dbuf<int> t_kind, t_ctr;
    int npt = 0;
    dbuf<int> pt_tgt;   // point target k -> target index (ascending)
    // root
    RootInfo root{};
    // tree
    bool built = false;
    int nbox = 0, nlev = 0;
    std::vector<int> level_start_h;  // [nlev+1]
    dbuf<int> level_start;
    dbuf<uint64_t> bkey;             // Morton key at the box's level
    dbuf<int> blev, bix, biy, bparent;
    dbuf<int4> bchild;
    dbuf<int> sub_src, sub_tgt, own_tgt;
    dbuf<int> src_beg, src_end;      // owned sources (leaves) in sorted-source order
    dbuf<int> ssub_beg, ssub_end;    // subtree sources in sorted-source order
    dbuf<int> ctr_beg, ctr_end;      // owned centres in sorted-centre order
    dbuf<int> pt_beg, pt_end;        // owned point targets in sorted-point order
    // sorted particle data
    dbuf<int> src_perm;              // sorted source j -> quadrature node id
    dbuf<double2> s_xy;              // sorted source positions
    dbuf<double> s_w;                // sorted weights
    dbuf<double2> s_n;               // sorted normals
    dbuf<int> src_owner;             // sorted source j -> owner box
    dbuf<int> ctr_perm;              // sorted centre position -> centre id
    dbuf<int> ctr_pos;               // centre id -> sorted position
    dbuf<double2> sc_xy;             // sorted centres
    dbuf<double> sc_r;
    dbuf<int> ctr_owner;             // sorted centre -> owner box
    dbuf<int> pt_perm;               // sorted point target -> target index
    dbuf<double2> sp_xy;
    dbuf<int> pt_owner;              // sorted point target -> owner box
    // lists (CSR over boxes): 0 U, 1 V, 2 WC, 3 WF, 4 XC, 5 XF
    dbuf<int> list_off[6], list_idx[6];
    int64_t list_size[6] = {0, 0, 0, 0, 0, 0};
    int list_row_cap = 0;            // scratch row capacity override of the list fill (0: per-list defaults)
    int lists_fill_passes = 0;       // enumeration passes of the last list construction (1 or 2)
    // work lists for the evaluation
    dbuf<int> leaf_src_boxes;  int n_leaf_src = 0;   // leaves owning sources
    dbuf<int> ctr_boxes;       int n_ctr_boxes = 0;  // boxes owning centres
    dbuf<int> pt_boxes;        int n_pt_boxes = 0;   // boxes owning point targets
    dbuf<int> far_boxes;       int n_far_boxes = 0;  // boxes with V or X far entries
    dbuf<int> m2m_boxes;       int n_m2m_boxes = 0;  // non-leaf boxes with sources below, by level
    std::vector<int> m2m_level_start_h;              // [nlev+1] level l's part of m2m_boxes
    // evaluation buffers
    dbuf<double2> strength;          // sorted sources: S -> (q, 0), D -> d
    dbuf<unsigned int> qexp;         // largest biased exponent of the strengths (one value)
    dbuf<double2> M, L;              // [nbox][p_fmm+1] box-scaled expansions
    dbuf<double2> Q;                 // [nc][p_qbx+1] r-scaled QBX coefficients (sorted centres): far part
    dbuf<double2> Qn;                // the same, direct part
    dbuf<double> pot;                // sorted point targets: Re Phi, far part
    dbuf<double> potn;               // the same, direct part
    cudaStream_t s2 = nullptr;       // second stream for the direct part of an evaluation
    cudaEvent_t ev_str = nullptr, ev_near = nullptr;
    dbuf<double> out_dev;            // [nt] staging for host outputs
    dbuf<double> dens_dev;           // [nbase] staging for host inputs
    int last_kernel = -1;
    bool have_eval = false;
    // learned orders: per-centre QBX order (sorted centre order), used when has_qc
    bool has_qc = false;
    dbuf<int> q_ctr;
    // mixed precision (FP32 direct sums): coordinates relative to box centres
    bool mixed_ready = false;
    dbuf<float2> s_rel;   // sorted sources minus their leaf centre
    dbuf<float2> c_rel;   // sorted centres minus their owner-box centre
    dbuf<float> c_rf;     // centre radii
    dbuf<float2> p_rel;   // sorted point targets minus their leaf centre
    dbuf<float2> str_f;   // strengths
    dbuf<float2> M_f;     // multipoles (List 3 far evaluation at point targets)
    // split precision (double-FP32 direct sums): the same relative coordinates as pairs
    bool split_ready = false;
    dbuf<float4> s_rel2;  // (x.hi, x.lo, y.hi, y.lo)
    dbuf<float4> c_rel2;
    dbuf<float4> c_r2;    // (r.hi, r.lo, (1/r^2).hi, (1/r^2).lo)
    dbuf<float4> str2;    // (re.hi, re.lo, im.hi, im.lo)
    // several densities at once (gq_eval_multi): strengths and direct coefficients per density
    dbuf<double2> strm, Qm;
    const double2 *qn_last = nullptr;   // direct coefficients of the last evaluation
    dbuf<float4> p_rel2;  // sorted point targets minus their leaf centre
    dbuf<float4> M2;      // multipoles
    dbuf<float4> L2;      // local expansions
    dbuf<float4> lvl2;    // per level: (rho, 1/rho), (log rho, 1/rho^2)
    // tensor-core M2L (gq_m2l_tc.cu): tiles of the current build, multipole digits
    // scratch of compact_flags and of its callers' flags (kept between calls)
    dbuf<int> cf_pos, cf_tmp, cf_flag;
    // M2QBXL on the tensor cores: (centre, List 3 far box) pairs of the build
    bool wtc_ready = false;
    int wtc_npairs = 0;
    dbuf<int> wtc_pstart, wtc_pc, wtc_pd;
    dbuf<double2> wtc_contrib;
    bool tc_ready = false;
    dbuf<int> tc_tile_box, tc_slot_src, tc_tile_q, tc_err, tc_lexp, tc_counter, tc_ntiles_dev, tc_cnt;
    dbuf<unsigned> tc_tile_mask;
    dbuf<uint16_t> tc_mdig;
};

// ------------------------------------------------------------------ launch helpers
inline int gq_blocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    return (int)(b < 1 ? 1 : b);
}

// ------------------------------------------------------------------ primitives (gq_prims.cu)
// Exclusive prefix sum of n ints: out[0..n] (out[n] = total).  tmp sized by scan_tmp_size.
size_t gq_scan_tmp_size(long long n);
void gq_exclusive_scan(gq_ctx *ctx, const int *in, int *out, long long n, int *tmp);
// the same for the flags vals[i] > thresh (computed on the fly)
void gq_exclusive_scan_above(gq_ctx *ctx, const int *vals, int thresh, int *out, long long n, int *tmp);
// nonzero when a scan's bounded look-back wait gave up since the last call (cleared; synchronous)
int gq_scan_error_take();
// Stable LSD radix sort of (key, value) pairs on key bits [0, bits).  In/out may alias
// the temporaries: results are returned in keys/vals.
void gq_radix_sort_pairs(gq_ctx *ctx, uint64_t *keys, int *vals, long long n, int bits);
void gq_radix_sort_pairs32(gq_ctx *ctx, uint32_t *keys, int *vals, long long n, int bits);

// ------------------------------------------------------------------ stages
void gq_build_all(gq_geom *g);                 // gq_tree.cu
void gq_build_lists(gq_geom *g);               // gq_lists.cu
// Keys (level << 60) | Morton key of the leaves that violate the level
// restriction (a box two levels deeper touches them) and own a particle
// eligible for children (belig[b] > 0); synchronises the stream.
void gq_balance_violations(gq_geom *g, const int *belig, std::vector<uint64_t> &out);
// far parts of one evaluation for the batched path (see gq_eval_all)
struct EvalFar {
    double2 *Q;     // [nc][p_qbx+1] QBX coefficients from List 3 far and the box locals
    double *pot;    // [npt] point potentials from List 3 far and the box locals
};
void gq_eval_all(gq_geom *g, int kernel, const double *dens_dev, double *out_dev, gq_stats *st,
                 const double2 *qn_pre = nullptr, const double *apply_identity = nullptr,
                 const EvalFar *far = nullptr);                                            // gq_fmm.cu
void gq_eval_multi(gq_geom *g, int kernel, int nd, const double *const *dens, double *const *out);
void gq_export_qbx_impl(gq_geom *g, double *host);  // gq_fmm.cu
double gq_probe_fma(gq_ctx *ctx, int what);         // gq_probe.cu
void gq_probe_math_impl(gq_ctx *ctx, int fn, int n, const double *x_dev, double *y_dev);
void gq_probe_umma_impl(gq_ctx *ctx, int K, const uint16_t *A_host, const uint16_t *B_host, int swap, float *D_host);
void gq_eval_noalloc_impl(gq_geom *g, int kernel, const double *dens_dev, double *out_dev);  // gq_fmm.cu
// persistent batched evaluation (gq_fmm.cu): direct parts and final sums of
// all geometries and densities in one launch after per-geometry FMM passes
struct gq_bplan;
bool gq_bplan_supported(const std::vector<gq_geom *> &geoms, int kernel);
gq_bplan *gq_bplan_new(gq_ctx *ctx, int kernel, int ndens, const std::vector<gq_geom *> &geoms,
                       const double *const *dens, double *const *out, int tile, int stall_geom);
void gq_bplan_free(gq_bplan *P);
void gq_bplan_retile(gq_bplan *P, int tile);
int gq_bplan_tile(const gq_bplan *P);
void gq_bplan_fmm(gq_bplan *P, int i);
void gq_bplan_persistent(gq_bplan *P, gq_ctx *ctx, int grid, unsigned long long limit_ns);
int gq_bplan_error(gq_bplan *P);
bool gq_m2l_tc_supported(const gq_geom *g);                                                  // gq_m2l_tc.cu
void gq_m2l_tc(gq_geom *g, const double2 *M, double2 *L);
void gq_m2l_tc_build(gq_geom *g);
int gq_m2l_tc_error(gq_geom *g);
bool gq_w_tc_supported(const gq_geom *g);
void gq_tensor_paths_impl(gq_geom *g, int *m2l_tc, int *m2qbxl_tc);
void gq_w_tc_build(gq_geom *g);
void gq_w_centres_tc(gq_geom *g, const RootInfo &R, const double2 *M, const double *logt, double2 *Q);
struct gq_mlp;
int gq_mlp_param_count();                                                                   // gq_learned.cu
gq_mlp *gq_mlp_new(gq_ctx *ctx, uint64_t seed);
void gq_mlp_free(gq_mlp *M);
gq_ctx *gq_mlp_ctx(const gq_mlp *M);
void gq_mlp_weights_impl(gq_mlp *M, float *get, const float *set);
void gq_mlp_loss_grad_impl(gq_mlp *M, const float *X, const float *Y, int n, bool dev, float *loss, float *grad);
double gq_mlp_train_impl(gq_mlp *M, const float *X, const float *Y, int n, bool dev, int epochs, int B, float lr,
                         uint64_t seed);
void gq_mlp_predict_impl(gq_mlp *M, const float *X, int n, bool xdev, float *Y, bool ydev);
void gq_centre_features_impl(gq_geom *g, float *feat_dev);
void gq_set_centre_orders_impl(gq_geom *g, const int *q_dev);
void gq_learned_orders_impl(gq_geom *g, gq_mlp *M, double eps, double margin, double margin_fmm, int q_ref,
                            int p_ref, int q_bound, int p_bound, int *p_out, int *q_out);
struct gq_batch;
gq_batch *gq_batch_new(gq_ctx *ctx, int n, gq_geom *const *geoms);                       // gq_batch.cu
void gq_batch_free(gq_batch *b);
void gq_batch_eval_impl(gq_batch *b, int kernel, int ndens, const double *const *dens, double *const *out);
int gq_batch_streams(const gq_batch *b);
void gq_batch_config_impl(gq_batch *b, int mode, long long wait_ns, int stall_geom);
int gq_batch_persistent_tile(const gq_batch *b);
int gq_batch_persistent_ctas_impl(const gq_batch *b);
gq_ctx *gq_batch_ctx(const gq_batch *b);
int gq_batch_size(const gq_batch *b);
gq_geom *gq_batch_geom(const gq_batch *b, int i);
int gq_gmres_impl(gq_geom *g, const double *rhs_dev, double tol, int maxit, int restart, double *mu_dev,
                  double *resid);                                                           // gq_gmres.cu
void gq_batch_gmres_impl(gq_batch *b, const double *const *rhs_dev, double tol, int maxit, int restart,
                         double *const *mu_dev, int *iters, double *resid);

#define GQ_LAUNCH(ctx, kern, grid, block, smem, ...)                     \
    do {                                                                 \
        kern<<<(grid), (block), (smem), (ctx)->stream>>>(__VA_ARGS__);   \
        GQ_CHECK_LAUNCH();                                               \
        (ctx)->launches++;                                               \
    } while (0)

// ------------------------------------------------------------------ device helpers
__host__ __device__ inline uint64_t gq_spread_bits(uint64_t x) {
    // insert a zero bit above each of the low 32 bits
    x &= 0xffffffffull;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
// Morton key: x bits on even positions, y bits on odd positions
__host__ __device__ inline uint64_t gq_morton(uint64_t ix, uint64_t iy) {
    return gq_spread_bits(ix) | (gq_spread_bits(iy) << 1);
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cinv(double2 a) {
    double d = 1.0 / (a.x * a.x + a.y * a.y);
    return make_double2(a.x * d, -a.y * d);
}
