// gq_api.cu -- the extern "C" boundary declared in include/gigaqbx.h.
#include <math.h>
#include <string.h>

#include <new>

#include "gq_internal.cuh"

void gq_form_centres(gq_geom *g);
void gq_tables_release(gq_geom *g);

namespace {

gq_status fail(gq_ctx *ctx, const gq_error &e) {
    if (ctx) ctx->last_error = e.msg;
    return e.code;
}

template <class F>
gq_status guarded(gq_ctx *ctx, F &&f) {
    try {
        f();
        return GQ_OK;
    } catch (const gq_error &e) {
        return fail(ctx, e);
    } catch (const std::bad_alloc &) {
        return fail(ctx, gq_error{GQ_ERR_NOMEM, "host allocation failed"});
    } catch (...) {
        return fail(ctx, gq_error{GQ_ERR_CUDA, "unexpected failure"});
    }
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// flags[0]: some on[i] outside [-1, nbase); flags[1]: some on[i] != i
__global__ void k_check_targets(int n, const int *__restrict__ on, int nbase, int *__restrict__ flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false, notbase = false;
    if (i < n) {
        int v = on[i];
        bad = v < -1 || v >= nbase;
        notbase = v != i;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1);
    if (__any_sync(0xffffffffu, notbase) && (threadIdx.x & 31) == 0) atomicOr(&flags[1], 1);
}

template <class T>
void upload(gq_ctx *ctx, dbuf<T> &dst, const T *src, size_t n) {
    GQ_REQUIRE(src != nullptr || n == 0, GQ_ERR_INVALID, "null input array");
    dst.alloc(n);
    if (n) GQ_CUDA(cudaMemcpyAsync(dst.p, src, sizeof(T) * n, cudaMemcpyDefault, ctx->stream));
}

// Lagrange interpolation matrix from the nb base reference nodes to the nu
// quadrature reference nodes of a panel: I[j][i] = prod_{k != i} (u_j - b_k) / (b_i - b_k)
std::vector<double> lagrange_matrix(const double *rb, int nb, const double *ru, int nu) {
    std::vector<double> I((size_t)nu * nb);
    for (int j = 0; j < nu; ++j)
        for (int i = 0; i < nb; ++i) {
            double v = 1.0;
            for (int k = 0; k < nb; ++k)
                if (k != i) v *= (ru[j] - rb[k]) / (rb[i] - rb[k]);
            I[(size_t)j * nb + i] = v;
        }
    return I;
}

void resolve_orders(gq_params &p) {
    if (p.p_fmm <= 0 || p.p_qbx <= 0) {
        GQ_REQUIRE(p.eps > 0 && p.eps < 1, GQ_ERR_INVALID, "orders of 0 need 0 < eps < 1");
        // FMM order: the idealised FMM error (1/2)^(p+1) <= eps (Sec. 4.1, 5.1)
        int k = (int)ceil(log2(1.0 / p.eps)) - 1;
        if (p.p_fmm <= 0) p.p_fmm = k < 1 ? 1 : (k > GQ_MAX_PFMM ? GQ_MAX_PFMM : k);
        // QBX order: truncation error ~ 10^(-2.06 - 1.26 q) measured with Green's identity on
        // starfish curves with centres half a panel length off the curve; q with error <= eps/2
        int q = (int)ceil((log10(2.0 / p.eps) - 2.06) / 1.26);
        if (p.p_qbx <= 0) p.p_qbx = q < 1 ? 1 : (q > GQ_MAX_PQBX ? GQ_MAX_PQBX : q);
    }
    GQ_REQUIRE(p.p_qbx >= 1 && p.p_qbx <= GQ_MAX_PQBX, GQ_ERR_INVALID, "p_qbx must be in [1, 16]");
    GQ_REQUIRE(p.p_fmm >= 1 && p.p_fmm <= GQ_MAX_PFMM, GQ_ERR_INVALID, "p_fmm must be in [1, 30]");
    GQ_REQUIRE(p.n_max >= 1, GQ_ERR_INVALID, "n_max must be >= 1");
    GQ_REQUIRE(p.tf_den > 0 && p.tf_num >= 0 && p.tf_num < p.tf_den, GQ_ERR_INVALID, "need 0 <= t_f < 1");
    GQ_REQUIRE(p.max_level >= 1 && p.max_level <= GQ_KEYBITS, GQ_ERR_INVALID, "max_level must be in [1, 30]");
    GQ_REQUIRE(p.radius_factor > 0, GQ_ERR_INVALID, "radius_factor must be > 0");
    GQ_REQUIRE(p.assoc_slack >= 0, GQ_ERR_INVALID, "assoc_slack must be >= 0");
    GQ_REQUIRE(p.w3_demote >= 1, GQ_ERR_INVALID, "w3_demote must be >= 1");
    GQ_REQUIRE(p.precision == GQ_PREC_FP64 || p.precision == GQ_PREC_MIXED || p.precision == GQ_PREC_MIXED_FMM,
               GQ_ERR_INVALID, "unknown precision");
    GQ_REQUIRE(p.m2l == GQ_M2L_AUTO || p.m2l == GQ_M2L_FP64, GQ_ERR_INVALID, "unknown m2l mode");
    GQ_REQUIRE(p.level_restrict == 0 || p.level_restrict == 1, GQ_ERR_INVALID, "level_restrict must be 0 or 1");
    GQ_REQUIRE(p.tcr_shape == 0 || p.tcr_shape == 1, GQ_ERR_INVALID, "tcr_shape must be 0 (square) or 1 (disk)");
}

}  // namespace

extern "C" {

gq_status gq_params_default(gq_params *out) {
    if (!out) return GQ_ERR_INVALID;
    memset(out, 0, sizeof(*out));
    out->p_qbx = 5;
    out->p_fmm = 10;
    out->n_max = 32;
    out->tf_num = 9;
    out->tf_den = 10;
    out->w3_demote = 15;
    out->max_level = 30;
    out->radius_factor = 0.5;
    out->assoc_slack = 1.2;
    out->eps = 0.0;
    out->precision = GQ_PREC_FP64;
    out->m2l = GQ_M2L_AUTO;
    out->level_restrict = 0;
    out->tcr_shape = 0;
    return GQ_OK;
}

gq_status gq_params_resolve(const gq_params *in, gq_params *out) {
    if (!in || !out) return GQ_ERR_INVALID;
    gq_params p = *in;
    try {
        resolve_orders(p);
    } catch (const gq_error &e) {
        return e.code;
    }
    *out = p;
    return GQ_OK;
}

gq_status gq_create(int device, void *cuda_stream, gq_ctx **out) {
    if (!out) return GQ_ERR_INVALID;
    *out = nullptr;
    gq_ctx *ctx = new (std::nothrow) gq_ctx;
    if (!ctx) return GQ_ERR_NOMEM;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        delete ctx;
        return GQ_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return GQ_ERR_CUDA;
    }
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    *out = ctx;
    return GQ_OK;
}

gq_status gq_destroy(gq_ctx *ctx) {
    if (!ctx) return GQ_ERR_INVALID;
    delete ctx;
    return GQ_OK;
}

const char *gq_last_error(const gq_ctx *ctx) { return ctx ? ctx->last_error.c_str() : "null context"; }

gq_status gq_set_stream(gq_ctx *ctx, void *cuda_stream) {
    if (!ctx) return GQ_ERR_INVALID;
    ctx->stream = (cudaStream_t)cuda_stream;
    return GQ_OK;
}

gq_status gq_geometry_create(gq_ctx *ctx, const gq_geometry_desc *d, const gq_params *params, gq_geom **out) {
    if (!ctx || !d || !params || !out) return GQ_ERR_INVALID;
    *out = nullptr;
    gq_geom *g = nullptr;
    gq_status s = guarded(ctx, [&] {
        GQ_CUDA(cudaSetDevice(ctx->device));
        GQ_REQUIRE(d->npanels > 0 && d->nb > 0 && d->nu > 0, GQ_ERR_INVALID, "empty geometry");
        GQ_REQUIRE((long long)d->npanels * d->nu < (1ll << 28), GQ_ERR_UNSUPPORTED, "too many quadrature nodes");
        g = new gq_geom;
        g->ctx = ctx;
        g->prm = *params;
        resolve_orders(g->prm);
        g->npanels = d->npanels;
        g->nb = d->nb;
        g->nu = d->nu;
        g->nbase = d->npanels * d->nb;
        g->nsrc = d->npanels * d->nu;
        // reference nodes are needed on the host for the interpolation matrix
        std::vector<double> rb(d->nb), ru(d->nu);
        GQ_CUDA(cudaMemcpy(rb.data(), d->ref_b, sizeof(double) * d->nb, cudaMemcpyDefault));
        GQ_CUDA(cudaMemcpy(ru.data(), d->ref_u, sizeof(double) * d->nu, cudaMemcpyDefault));
        std::vector<double> I = lagrange_matrix(rb.data(), d->nb, ru.data(), d->nu);
        upload(ctx, g->interp, I.data(), I.size());
        upload(ctx, g->base_xy, d->base_xy, 2 * (size_t)g->nbase);
        upload(ctx, g->base_n, d->base_n, 2 * (size_t)g->nbase);
        upload(ctx, g->up_xy, d->up_xy, 2 * (size_t)g->nsrc);
        upload(ctx, g->up_n, d->up_n, 2 * (size_t)g->nsrc);
        upload(ctx, g->up_w, d->up_w, (size_t)g->nsrc);
        upload(ctx, g->panel_len, d->panel_len, (size_t)g->npanels);
        gq_form_centres(g);
        GQ_CUDA(cudaStreamSynchronize(ctx->stream));
    });
    if (s != GQ_OK) {
        delete g;
        return s;
    }
    *out = g;
    return GQ_OK;
}

gq_status gq_geometry_destroy(gq_geom *g) {
    if (!g) return GQ_ERR_INVALID;
    cudaStreamSynchronize(g->ctx->stream);
    if (g->s2) {
        cudaStreamSynchronize(g->s2);
        cudaStreamDestroy(g->s2);
        cudaEventDestroy(g->ev_str);
        cudaEventDestroy(g->ev_near);
    }
    gq_tables_release(g);
    delete g;
    return GQ_OK;
}

gq_status gq_geometry_params(const gq_geom *g, gq_params *out) {
    if (!g || !out) return GQ_ERR_INVALID;
    *out = g->prm;
    return GQ_OK;
}

gq_status gq_targets_set(gq_geom *g, int n, const double *xy, const int *on_surface_node) {
    if (!g || n < 0 || (n > 0 && (!xy || !on_surface_node))) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        upload(g->ctx, g->tgt_xy, xy, 2 * (size_t)n);
        upload(g->ctx, g->tgt_on, on_surface_node, (size_t)n);
        // range check and "the base nodes in order" test on the device
        dbuf<int> flags;
        flags.alloc(2);
        GQ_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), g->ctx->stream));
        if (n) GQ_LAUNCH(g->ctx, k_check_targets, gq_blocks(n, 256), 256, 0, n, (const int *)g->tgt_on.p, g->nbase,
                         flags.p);
        int hf[2] = {0, 0};
        GQ_CUDA(cudaMemcpyAsync(hf, flags.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, g->ctx->stream));
        GQ_CUDA(cudaStreamSynchronize(g->ctx->stream));
        if (hf[0] != 0) {   // the target arrays were replaced: the geometry has no valid targets now
            g->targets_set = false;
            g->built = false;
            g->have_eval = false;
            gq_tables_release(g);
            throw gq_error{GQ_ERR_INVALID, "on_surface_node out of range"};
        }
        g->nt = n;
        g->targets_are_base_nodes = n == g->nbase && hf[1] == 0;
        g->targets_set = true;
        g->built = false;
        g->have_eval = false;
        gq_tables_release(g);
    });
}

gq_status gq_build(gq_geom *g) {
    if (!g) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_CUDA(cudaSetDevice(g->ctx->device));
        gq_tables_release(g);
        g->mixed_ready = false;
        g->split_ready = false;
        g->tc_ready = false;
        g->wtc_ready = false;
        gq_form_centres(g);
        gq_build_all(g);
        if (gq_m2l_tc_supported(g)) gq_m2l_tc_build(g);   // tiles of the tensor-core M2L
        if (gq_w_tc_supported(g)) gq_w_tc_build(g);       // pairs of the tensor-core M2QBXL
        GQ_CUDA(cudaStreamSynchronize(g->ctx->stream));
        GQ_REQUIRE(gq_scan_error_take() == 0, GQ_ERR_TIMEOUT, "gq_build: a prefix scan's bounded wait gave up");
        g->built = true;
    });
}

gq_status gq_eval(gq_geom *g, int kernel, const double *density_base, double *out, gq_stats *stats) {
    if (!g || !density_base || (!out && g->nt > 0)) return GQ_ERR_INVALID;
    if (kernel != GQ_S && kernel != GQ_D && kernel != GQ_SP) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_REQUIRE(g->built, GQ_ERR_STATE, "gq_eval before gq_build");
        cudaStream_t st = g->ctx->stream;
        const double *dens = density_base;
        if (!is_device_ptr(density_base)) {
            g->dens_dev.alloc(g->nbase);
            GQ_CUDA(cudaMemcpyAsync(g->dens_dev.p, density_base, sizeof(double) * g->nbase, cudaMemcpyDefault, st));
            dens = g->dens_dev.p;
        }
        bool out_dev = is_device_ptr(out);
        double *o = out;
        if (!out_dev) {
            g->out_dev.alloc(g->nt);
            o = g->out_dev.p;
        }
        if (stats) memset(stats, 0, sizeof(*stats));
        gq_eval_all(g, kernel, dens, o, stats);
        if (!out_dev && g->nt) {
            GQ_CUDA(cudaMemcpyAsync(out, o, sizeof(double) * g->nt, cudaMemcpyDefault, st));
            GQ_CUDA(cudaStreamSynchronize(st));
            {
            int tce = gq_m2l_tc_error(g);
            GQ_REQUIRE(tce != 2, GQ_ERR_UNSUPPORTED, "tensor-core M2L: a List 2 entry outside the offset window");
            GQ_REQUIRE(tce == 0, GQ_ERR_TIMEOUT, "tensor-core M2L: a bounded wait gave up");
        }
        }
    });
}

gq_status gq_apply(gq_geom *g, int kernel, double identity, const double *mu, double *out) {
    if (!g || !mu || !out) return GQ_ERR_INVALID;
    if (kernel != GQ_S && kernel != GQ_D && kernel != GQ_SP) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_REQUIRE(g->built, GQ_ERR_STATE, "gq_apply before gq_build");
        cudaStream_t st = g->ctx->stream;
        const double *dens = mu;
        if (!is_device_ptr(mu)) {
            g->dens_dev.alloc(g->nbase);
            GQ_CUDA(cudaMemcpyAsync(g->dens_dev.p, mu, sizeof(double) * g->nbase, cudaMemcpyDefault, st));
            dens = g->dens_dev.p;
        }
        bool out_dev = is_device_ptr(out);
        double *o = out;
        dbuf<double> stage;
        if (!out_dev) {
            stage.alloc(g->nbase);
            o = stage.p;
        }
        gq_eval_all(g, kernel, dens, o, nullptr, nullptr, &identity);
        if (!out_dev) {
            GQ_CUDA(cudaMemcpyAsync(out, o, sizeof(double) * g->nbase, cudaMemcpyDefault, st));
            GQ_CUDA(cudaStreamSynchronize(st));
        }
    });
}

gq_status gq_eval_noalloc(gq_geom *g, int kernel, const double *density_dev, double *out_dev) {
    if (!g || !density_dev || (!out_dev && g->nt > 0)) return GQ_ERR_INVALID;
    if (kernel != GQ_S && kernel != GQ_D && kernel != GQ_SP) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_REQUIRE(g->built, GQ_ERR_STATE, "gq_eval_noalloc before gq_build");
        GQ_REQUIRE(is_device_ptr(density_dev), GQ_ERR_INVALID, "gq_eval_noalloc: density must be device memory");
        GQ_REQUIRE(g->nt == 0 || is_device_ptr(out_dev), GQ_ERR_INVALID, "gq_eval_noalloc: out must be device memory");
        gq_eval_noalloc_impl(g, kernel, density_dev, out_dev);
    });
}

gq_status gq_gmres(gq_geom *g, const double *rhs, double tol, int maxit, int restart, double *mu, int *iters,
                   double *resid) {
    if (!g || !rhs || !mu || !(tol > 0) || maxit < 1 || restart < 1 || restart > 1000) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_REQUIRE(g->built, GQ_ERR_STATE, "gq_gmres before gq_build");
        cudaStream_t st = g->ctx->stream;
        dbuf<double> b, x;
        const double *bd = rhs;
        if (!is_device_ptr(rhs)) {
            b.alloc(g->nbase);
            GQ_CUDA(cudaMemcpyAsync(b.p, rhs, sizeof(double) * g->nbase, cudaMemcpyDefault, st));
            bd = b.p;
        }
        bool mu_dev = is_device_ptr(mu);
        double *xd = mu;
        if (!mu_dev) {
            x.alloc(g->nbase);
            xd = x.p;
        }
        double rr = 0;
        int it = gq_gmres_impl(g, bd, tol, maxit, restart, xd, &rr);
        if (!mu_dev) GQ_CUDA(cudaMemcpyAsync(mu, xd, sizeof(double) * g->nbase, cudaMemcpyDefault, st));
        GQ_CUDA(cudaStreamSynchronize(st));
        if (iters) *iters = it;
        if (resid) *resid = rr;
    });
}

gq_status gq_batch_create(gq_ctx *ctx, int ngeom, gq_geom *const *geoms, gq_batch **out) {
    if (!ctx || ngeom < 1 || !geoms || !out) return GQ_ERR_INVALID;
    *out = nullptr;
    return guarded(ctx, [&] {
        for (int i = 0; i < ngeom; ++i) {
            GQ_REQUIRE(geoms[i] != nullptr, GQ_ERR_INVALID, "gq_batch_create: null geometry");
            GQ_REQUIRE(geoms[i]->built, GQ_ERR_STATE, "gq_batch_create: geometry not built");
            GQ_REQUIRE(geoms[i]->ctx->device == ctx->device, GQ_ERR_INVALID, "gq_batch_create: other device");
        }
        *out = gq_batch_new(ctx, ngeom, geoms);
    });
}

gq_status gq_batch_destroy(gq_batch *b) {
    if (!b) return GQ_ERR_INVALID;
    gq_batch_free(b);
    return GQ_OK;
}

gq_status gq_batch_eval(gq_batch *b, int kernel, int ndens, const double *const *dens, double *const *out) {
    if (!b || ndens < 1 || !dens || !out) return GQ_ERR_INVALID;
    if (kernel != GQ_S && kernel != GQ_D && kernel != GQ_SP) return GQ_ERR_INVALID;
    gq_ctx *ctx = gq_batch_ctx(b);
    return guarded(ctx, [&] {
        GQ_CUDA(cudaSetDevice(ctx->device));
        gq_batch_eval_impl(b, kernel, ndens, dens, out);
    });
}

gq_status gq_batch_gmres(gq_batch *b, const double *const *rhs, double tol, int maxit, int restart,
                         double *const *mu, int *iters, double *resid) {
    if (!b || !rhs || !mu || !(tol > 0) || maxit < 1 || restart < 1 || restart > 1000) return GQ_ERR_INVALID;
    gq_ctx *ctx = gq_batch_ctx(b);
    return guarded(ctx, [&] {
        GQ_CUDA(cudaSetDevice(ctx->device));
        for (int i = 0; i < gq_batch_size(b); ++i) {
            gq_geom *g = gq_batch_geom(b, i);
            GQ_REQUIRE(g->built && g->targets_are_base_nodes, GQ_ERR_STATE,
                       "gq_batch_gmres needs every geometry built with the base nodes as targets");
            GQ_REQUIRE(rhs[i] && mu[i] && is_device_ptr(rhs[i]) && is_device_ptr(mu[i]), GQ_ERR_INVALID,
                       "gq_batch_gmres: rhs and mu must be device arrays");
        }
        gq_batch_gmres_impl(b, rhs, tol, maxit, restart, mu, iters, resid);
    });
}

gq_status gq_batch_streams(const gq_batch *b, int *streams) {
    if (!b || !streams) return GQ_ERR_INVALID;
    *streams = gq_batch_streams(b);
    return GQ_OK;
}

gq_status gq_batch_mode(gq_batch *b, int mode) {
    if (!b || mode < 0 || mode > 2) return GQ_ERR_INVALID;
    return guarded(gq_batch_ctx(b), [&] { gq_batch_config_impl(b, mode, 0, -1); });
}

gq_status gq_batch_persistent(const gq_batch *b, int *tile) {
    if (!b || !tile) return GQ_ERR_INVALID;
    *tile = gq_batch_persistent_tile(b);
    return GQ_OK;
}

gq_status gq_batch_persistent_ctas(const gq_batch *b, int *ctas) {
    if (!b || !ctas) return GQ_ERR_INVALID;
    return guarded(gq_batch_ctx(b), [&] { *ctas = gq_batch_persistent_ctas_impl(b); });
}

gq_status gq_batch_wait_test(gq_batch *b, int64_t wait_ns, int stall_geom) {
    if (!b || wait_ns <= 0 || stall_geom < -1 || stall_geom >= gq_batch_size(b)) return GQ_ERR_INVALID;
    return guarded(gq_batch_ctx(b), [&] { gq_batch_config_impl(b, 0, (long long)wait_ns, stall_geom); });
}

gq_status gq_centre_features(gq_geom *g, float *features) {
    if (!g || !features) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_REQUIRE(g->built, GQ_ERR_STATE, "gq_centre_features before gq_build");
        GQ_REQUIRE(g->nb >= 2, GQ_ERR_UNSUPPORTED, "features need at least two base nodes per panel");
        if (is_device_ptr(features)) {
            gq_centre_features_impl(g, features);
        } else {
            dbuf<float> f;
            f.alloc((size_t)g->nc * 32);
            gq_centre_features_impl(g, f.p);
            GQ_CUDA(cudaMemcpy(features, f.p, sizeof(float) * g->nc * 32, cudaMemcpyDeviceToHost));
        }
    });
}

gq_status gq_mlp_create(gq_ctx *ctx, uint64_t seed, gq_mlp **out) {
    if (!ctx || !out) return GQ_ERR_INVALID;
    *out = nullptr;
    return guarded(ctx, [&] { *out = gq_mlp_new(ctx, seed); });
}

gq_status gq_mlp_destroy(gq_mlp *m) {
    if (!m) return GQ_ERR_INVALID;
    gq_mlp_free(m);
    return GQ_OK;
}

gq_status gq_mlp_weights(gq_mlp *m, float *get, const float *set, int *count) {
    if (!m) return GQ_ERR_INVALID;
    gq_ctx *ctx = gq_mlp_ctx(m);
    if (count) *count = gq_mlp_param_count();
    return guarded(ctx, [&] { gq_mlp_weights_impl(m, get, set); });
}

gq_status gq_mlp_loss_grad(gq_mlp *m, const float *X, const float *Y, int n, float *loss, float *grad) {
    if (!m || !X || !Y || n < 1) return GQ_ERR_INVALID;
    gq_ctx *ctx = gq_mlp_ctx(m);
    return guarded(ctx, [&] {
        bool dev = is_device_ptr(X) && is_device_ptr(Y);
        gq_mlp_loss_grad_impl(m, X, Y, n, dev, loss, grad);
    });
}

gq_status gq_mlp_train(gq_mlp *m, const float *X, const float *Y, int n, int epochs, int batch, float lr,
                       uint64_t seed, float *final_loss) {
    if (!m || !X || !Y || n < 1 || epochs < 1 || batch < 1 || !(lr > 0)) return GQ_ERR_INVALID;
    gq_ctx *ctx = gq_mlp_ctx(m);
    return guarded(ctx, [&] {
        bool dev = is_device_ptr(X) && is_device_ptr(Y);
        double l = gq_mlp_train_impl(m, X, Y, n, dev, epochs, batch, lr, seed);
        if (final_loss) *final_loss = (float)l;
    });
}

gq_status gq_mlp_predict(gq_mlp *m, const float *X, int n, float *Y) {
    if (!m || !X || !Y || n < 0) return GQ_ERR_INVALID;
    gq_ctx *ctx = gq_mlp_ctx(m);
    return guarded(ctx, [&] { gq_mlp_predict_impl(m, X, n, is_device_ptr(X), Y, is_device_ptr(Y)); });
}

gq_status gq_learned_orders(gq_geom *g, gq_mlp *m, double eps, double margin_qbx, double margin_fmm, int q_ref,
                            int p_ref, int p_bound, int *p_fmm, int *q_max) {
    if (!g || !m || !(eps > 0 && eps < 1) || q_ref > GQ_MAX_PQBX || p_ref < 1 || p_bound < 1 ||
        p_bound > GQ_MAX_PFMM)
        return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_REQUIRE(g->built, GQ_ERR_STATE, "gq_learned_orders before gq_build");
        int p = 0, q = 0;
        gq_learned_orders_impl(g, m, eps, margin_qbx, margin_fmm, q_ref, p_ref, GQ_MAX_PQBX, p_bound, &p, &q);
        if (p_fmm) *p_fmm = p;
        if (q_max) *q_max = q;
    });
}

gq_status gq_set_centre_orders(gq_geom *g, const int *q) {
    if (!g || !q) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        GQ_REQUIRE(g->built, GQ_ERR_STATE, "gq_set_centre_orders before gq_build");
        std::vector<int> h(g->nc);
        GQ_CUDA(cudaMemcpy(h.data(), q, sizeof(int) * g->nc, cudaMemcpyDefault));
        for (int v : h) GQ_REQUIRE(v >= 1 && v <= GQ_MAX_PQBX, GQ_ERR_INVALID, "centre order outside [1, 16]");
        dbuf<int> d;
        d.alloc(g->nc);
        GQ_CUDA(cudaMemcpy(d.p, h.data(), sizeof(int) * g->nc, cudaMemcpyHostToDevice));
        gq_set_centre_orders_impl(g, d.p);
    });
}

gq_status gq_set_orders(gq_geom *g, int p_qbx, int p_fmm) {
    if (!g || p_qbx < 1 || p_qbx > GQ_MAX_PQBX || p_fmm < 1 || p_fmm > GQ_MAX_PFMM) return GQ_ERR_INVALID;
    g->prm.p_qbx = p_qbx;
    g->prm.p_fmm = p_fmm;
    g->has_qc = false;
    g->have_eval = false;
    return GQ_OK;
}

gq_status gq_tree_info_get(gq_geom *g, gq_tree_info *out) {
    if (!g || !out) return GQ_ERR_INVALID;
    if (!g->built) return GQ_ERR_STATE;
    out->nbox = g->nbox;
    out->nlevels = g->nlev;
    out->ncentres = g->nc;
    out->npoint_targets = g->npt;
    out->ntargets = g->nt;
    out->nsources = g->nsrc;
    for (int i = 0; i < 6; ++i) out->list_size[i] = g->list_size[i];
    return GQ_OK;
}

gq_status gq_export_root(gq_geom *g, double out[4]) {
    if (!g || !out) return GQ_ERR_INVALID;
    if (!g->built) return GQ_ERR_STATE;
    out[0] = g->root.lo_x;
    out[1] = g->root.lo_y;
    out[2] = g->root.H;
    out[3] = g->root.u;
    return GQ_OK;
}

gq_status gq_export_boxes(gq_geom *g, int *level, int64_t *ix, int64_t *iy, int *parent, int *nsrc, int *nctr,
                          int *ntgt, int *sub_src, int *sub_tgt) {
    if (!g) return GQ_ERR_INVALID;
    if (!g->built) return GQ_ERR_STATE;
    return guarded(g->ctx, [&] {
        int n = g->nbox;
        std::vector<int> a(n), b(n), c(n), d(n), e(n);
        auto get = [&](const int *src, int *dst) {
            if (dst) GQ_CUDA(cudaMemcpy(dst, src, sizeof(int) * n, cudaMemcpyDeviceToHost));
        };
        get(g->blev, level);
        get(g->bparent, parent);
        get(g->sub_src, sub_src);
        get(g->sub_tgt, sub_tgt);
        GQ_CUDA(cudaMemcpy(a.data(), g->bix.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        GQ_CUDA(cudaMemcpy(b.data(), g->biy.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        if (ix) for (int i = 0; i < n; ++i) ix[i] = a[i];
        if (iy) for (int i = 0; i < n; ++i) iy[i] = b[i];
        std::vector<int> sb(n), se(n), cb(n), ce(n), pb(n), pe(n);
        GQ_CUDA(cudaMemcpy(sb.data(), g->src_beg.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        GQ_CUDA(cudaMemcpy(se.data(), g->src_end.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        GQ_CUDA(cudaMemcpy(cb.data(), g->ctr_beg.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        GQ_CUDA(cudaMemcpy(ce.data(), g->ctr_end.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        GQ_CUDA(cudaMemcpy(pb.data(), g->pt_beg.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        GQ_CUDA(cudaMemcpy(pe.data(), g->pt_end.p, sizeof(int) * n, cudaMemcpyDeviceToHost));
        for (int i = 0; i < n; ++i) {
            if (nsrc) nsrc[i] = se[i] - sb[i];
            if (nctr) nctr[i] = ce[i] - cb[i];
            if (ntgt) ntgt[i] = pe[i] - pb[i];
        }
    });
}

gq_status gq_export_list(gq_geom *g, int which, int *off, int *idx) {
    if (!g || which < 0 || which > 5 || !off) return GQ_ERR_INVALID;
    if (!g->built) return GQ_ERR_STATE;
    return guarded(g->ctx, [&] {
        GQ_CUDA(cudaMemcpy(off, g->list_off[which].p, sizeof(int) * (g->nbox + 1), cudaMemcpyDeviceToHost));
        if (idx && g->list_size[which])
            GQ_CUDA(cudaMemcpy(idx, g->list_idx[which].p, sizeof(int) * g->list_size[which], cudaMemcpyDeviceToHost));
    });
}

gq_status gq_export_centres(gq_geom *g, double *xy, double *r, int *level) {
    if (!g) return GQ_ERR_INVALID;
    return guarded(g->ctx, [&] {
        if (xy) GQ_CUDA(cudaMemcpy(xy, g->c_xy.p, sizeof(double) * 2 * g->nc, cudaMemcpyDeviceToHost));
        if (r) GQ_CUDA(cudaMemcpy(r, g->c_r.p, sizeof(double) * g->nc, cudaMemcpyDeviceToHost));
        if (level) {
            GQ_REQUIRE(g->built, GQ_ERR_STATE, "centre levels need gq_build");
            GQ_CUDA(cudaMemcpy(level, g->c_lc.p, sizeof(int) * g->nc, cudaMemcpyDeviceToHost));
        }
    });
}

gq_status gq_export_assoc(gq_geom *g, int *kind, int *ctr) {
    if (!g) return GQ_ERR_INVALID;
    if (!g->built) return GQ_ERR_STATE;
    return guarded(g->ctx, [&] {
        if (kind && g->nt) GQ_CUDA(cudaMemcpy(kind, g->t_kind.p, sizeof(int) * g->nt, cudaMemcpyDeviceToHost));
        if (ctr && g->nt) GQ_CUDA(cudaMemcpy(ctr, g->t_ctr.p, sizeof(int) * g->nt, cudaMemcpyDeviceToHost));
    });
}

gq_status gq_export_owners(gq_geom *g, int *src_owner, int *ctr_owner, int *tgt_owner) {
    if (!g) return GQ_ERR_INVALID;
    if (!g->built) return GQ_ERR_STATE;
    return guarded(g->ctx, [&] {
        if (src_owner) {
            std::vector<int> perm(g->nsrc), own(g->nsrc);
            GQ_CUDA(cudaMemcpy(perm.data(), g->src_perm.p, sizeof(int) * g->nsrc, cudaMemcpyDeviceToHost));
            GQ_CUDA(cudaMemcpy(own.data(), g->src_owner.p, sizeof(int) * g->nsrc, cudaMemcpyDeviceToHost));
            for (int j = 0; j < g->nsrc; ++j) src_owner[perm[j]] = own[j];
        }
        if (ctr_owner) {
            std::vector<int> perm(g->nc), own(g->nc);
            GQ_CUDA(cudaMemcpy(perm.data(), g->ctr_perm.p, sizeof(int) * g->nc, cudaMemcpyDeviceToHost));
            GQ_CUDA(cudaMemcpy(own.data(), g->ctr_owner.p, sizeof(int) * g->nc, cudaMemcpyDeviceToHost));
            for (int j = 0; j < g->nc; ++j) ctr_owner[perm[j]] = own[j];
        }
        if (tgt_owner) {
            for (int t = 0; t < g->nt; ++t) tgt_owner[t] = -1;
            std::vector<int> perm(g->npt), own(g->npt);
            if (g->npt) {
                GQ_CUDA(cudaMemcpy(perm.data(), g->pt_perm.p, sizeof(int) * g->npt, cudaMemcpyDeviceToHost));
                GQ_CUDA(cudaMemcpy(own.data(), g->pt_owner.p, sizeof(int) * g->npt, cudaMemcpyDeviceToHost));
            }
            for (int j = 0; j < g->npt; ++j) tgt_owner[perm[j]] = own[j];
        }
    });
}

gq_status gq_context_launches(const gq_ctx *ctx, int64_t *out) {
    if (!ctx || !out) return GQ_ERR_INVALID;
    *out = ctx->launches;
    return GQ_OK;
}

gq_status gq_probe_fma_peak(gq_ctx *ctx, int what, double *tflops) {
    if (!ctx || !tflops || what < 0 || what > 3) return GQ_ERR_INVALID;
    return guarded(ctx, [&] { *tflops = gq_probe_fma(ctx, what); });
}

gq_status gq_memory_cached(int64_t *bytes) {
    if (!bytes) return GQ_ERR_INVALID;
    *bytes = (int64_t)gq_dev_cached_bytes();
    return GQ_OK;
}

gq_status gq_memory_release(void) {
    gq_dev_release_cache();
    return GQ_OK;
}

gq_status gq_probe_umma(gq_ctx *ctx, int K, const uint16_t *a, const uint16_t *b, int swap, float *d) {
    if (!ctx || !a || !b || !d) return GQ_ERR_INVALID;
    return guarded(ctx, [&] {
        GQ_CUDA(cudaSetDevice(ctx->device));
        gq_probe_umma_impl(ctx, K, a, b, swap, d);
    });
}

gq_status gq_tensor_paths(gq_geom *g, int *m2l_tc, int *m2qbxl_tc) {
    if (!g || !m2l_tc || !m2qbxl_tc) return GQ_ERR_INVALID;
    if (!g->built) return GQ_ERR_STATE;
    return guarded(g->ctx, [&] {
        GQ_CUDA(cudaSetDevice(g->ctx->device));
        gq_tensor_paths_impl(g, m2l_tc, m2qbxl_tc);
    });
}

gq_status gq_lists_check(gq_geom *g, int row_cap, int *passes) {
    if (!g) return GQ_ERR_INVALID;
    if (row_cap >= 0) g->list_row_cap = row_cap;
    if (passes) *passes = g->lists_fill_passes;
    return GQ_OK;
}

gq_status gq_probe_math(gq_ctx *ctx, int fn, int n, const double *x, double *y) {
    if (!ctx || fn < 0 || fn > 5 || n < 0 || (n > 0 && (!x || !y))) return GQ_ERR_INVALID;
    return guarded(ctx, [&] {
        GQ_REQUIRE(n == 0 || (is_device_ptr(x) && is_device_ptr(y)), GQ_ERR_INVALID, "gq_probe_math: device arrays");
        gq_probe_math_impl(ctx, fn, n, x, y);
    });
}

gq_status gq_export_qbx(gq_geom *g, double *coeffs) {
    if (!g || !coeffs) return GQ_ERR_INVALID;
    if (!g->have_eval) return GQ_ERR_STATE;
    return guarded(g->ctx, [&] { gq_export_qbx_impl(g, coeffs); });
}

}  // extern "C"
