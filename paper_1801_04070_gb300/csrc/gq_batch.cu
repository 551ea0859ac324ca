// gq_batch.cu -- batched evaluation of many independent geometries and many
// densities per geometry by one CUDA-graph launch.
//
// Each geometry's evaluations form one branch of the graph: the near-field QBX
// coefficients of all its densities together (gq_eval_multi), then the rest of
// the evaluation one density after another (they share the geometry's
// expansion buffers); branches are
// spread over S streams, largest first onto the least loaded stream, so small
// problems run concurrently and fill the GPU.  The graph is captured once per
// (kernel, densities, pointer set) and replayed afterwards.  S is chosen by an
// autotuner that captures the candidates S = 1, 2, 4, 8, 16 (at most the number
// of geometries), times two replays of each with CUDA events and keeps the
// fastest; the choice is cached per batch shape in memory and, when the
// environment variable GQ_AUTOTUNE_CACHE names a file, in that file.
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>

#include "gq_internal.cuh"

struct gq_batch {
    gq_ctx *ctx = nullptr;
    std::vector<gq_geom *> geoms;
    // captured graph
    cudaGraphExec_t exec = nullptr;
    int kernel = -1, ndens = 0, streams = 0;
    std::vector<const double *> dens;
    std::vector<double *> out;
    double tuned_ms = 0.0;
    int64_t kernels_per_replay = 0;
    // persistent path: the direct parts and final sums of all geometries and
    // densities in one launch after the per-geometry FMM branches
    int mode = 2;                          // 0: persistent where supported, 1: graph branches, 2: the faster
    bool persistent = false;               // the captured graph uses the persistent launch
    int tile = 1;                          // target boxes per direct item (tuned)
    int quarters = 4;                      // persistent CTAs: quarters of one per SM (tuned)
    unsigned long long wait_ns = 1000000000ull;   // bound of each dependency wait
    int stall_geom = -1;                   // test hook: that geometry's final items can never start
    gq_bplan *plan = nullptr;              // buffers and items of the persistent launch
    ~gq_batch() {
        if (plan) gq_bplan_free(plan);
    }
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, int> g_tune;   // batch shape -> stream count

std::string shape_key(const gq_batch *b, int kernel, int ndens) {
    long long ns = 0, nt = 0;
    for (auto *g : b->geoms) {
        ns += g->nsrc;
        nt += g->nt;
    }
    char buf[160];
    snprintf(buf, sizeof(buf), "g%zu_s%lld_t%lld_k%d_d%d_p%d_q%d", b->geoms.size(), ns, nt, kernel, ndens,
             b->geoms.empty() ? 0 : b->geoms[0]->prm.p_fmm, b->geoms.empty() ? 0 : b->geoms[0]->prm.p_qbx);
    return buf;
}

void load_cache_file() {
    const char *path = getenv("GQ_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    char key[200];
    int v;
    while (fscanf(f, " \"%199[^\"]\" : %d ,", key, &v) == 2) g_tune[key] = v;
    fclose(f);
}

void save_cache_file() {
    const char *path = getenv("GQ_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto &kv : g_tune) fprintf(f, "  \"%s\" : %d%s\n", kv.first.c_str(), kv.second, ++i < g_tune.size() ? " ," : "");
    fprintf(f, "}\n");
    fclose(f);
}

// the ndens densities of one geometry (consecutive arrays), the direct part of
// their QBX coefficients formed together (gq_eval_multi)
void eval_densities(gq_geom *g, int kernel, int ndens, const double *dens, double *out) {
    std::vector<const double *> d(ndens);
    std::vector<double *> o(ndens);
    for (int j = 0; j < ndens; ++j) {
        d[j] = dens + (size_t)j * g->nbase;
        o[j] = out + (size_t)j * g->nt;
    }
    gq_eval_multi(g, kernel, ndens, d.data(), o.data());
}

// work estimate used to balance branches: quadrature nodes + targets + boxes
double cost_of(const gq_geom *g) { return (double)g->nsrc + 2.0 * g->nt + 16.0 * g->nbox; }

// capture all evaluations on `S` streams into an executable graph
cudaGraphExec_t capture(gq_batch *b, int kernel, int ndens, const double *const *dens, double *const *out, int S,
                        int64_t *kernels) {
    cudaStream_t origin;
    GQ_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
    std::vector<cudaStream_t> st(S);
    std::vector<gq_ctx> sctx(S);
    for (int s = 0; s < S; ++s) {
        GQ_CUDA(cudaStreamCreateWithFlags(&st[s], cudaStreamNonBlocking));
        sctx[s].device = b->ctx->device;
        sctx[s].stream = st[s];
    }
    // largest first onto the least loaded stream
    std::vector<int> order(b->geoms.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int a, int c) { return cost_of(b->geoms[a]) > cost_of(b->geoms[c]); });
    std::vector<double> load(S, 0.0);
    std::vector<int> assign(b->geoms.size());
    for (int i : order) {
        int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        assign[i] = s;
        load[s] += cost_of(b->geoms[i]) * ndens;
    }
    cudaGraph_t graph = nullptr;
    cudaEvent_t fork;
    std::vector<cudaEvent_t> joins(S);
    GQ_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int s = 0; s < S; ++s) GQ_CUDA(cudaEventCreateWithFlags(&joins[s], cudaEventDisableTiming));
    std::vector<gq_ctx *> saved(b->geoms.size());
    GQ_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
    try {
        GQ_CUDA(cudaEventRecord(fork, origin));
        for (int s = 0; s < S; ++s) GQ_CUDA(cudaStreamWaitEvent(st[s], fork, 0));
        for (size_t i = 0; i < b->geoms.size(); ++i) {
            gq_geom *g = b->geoms[i];
            saved[i] = g->ctx;
            g->ctx = &sctx[assign[i]];
            eval_densities(g, kernel, ndens, dens[i], out[i]);
            g->ctx = saved[i];
        }
        for (int s = 0; s < S; ++s) {
            GQ_CUDA(cudaEventRecord(joins[s], st[s]));
            GQ_CUDA(cudaStreamWaitEvent(origin, joins[s], 0));
        }
        GQ_CUDA(cudaStreamEndCapture(origin, &graph));
    } catch (...) {
        for (size_t i = 0; i < b->geoms.size(); ++i)
            if (saved[i]) b->geoms[i]->ctx = saved[i];
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(origin, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        throw;
    }
    int64_t launched = 0;
    for (auto &c : sctx) launched += c.launches;
    *kernels = launched;   // kernel nodes recorded into the graph
    cudaGraphExec_t exec = nullptr;
    GQ_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    cudaEventDestroy(fork);
    for (auto e : joins) cudaEventDestroy(e);
    for (auto s : st) cudaStreamDestroy(s);
    cudaStreamDestroy(origin);
    return exec;
}

// Persistent variant: branch i records geometry i's strengths and FMM passes
// (gq_bplan_fmm); after the join, one persistent launch on the origin stream
// does every direct part and final sum (gq_bplan_persistent) with `quarters`
// quarters of a CTA per SM.
cudaGraphExec_t capture_persistent(gq_batch *b, gq_bplan *P, int S, int quarters, int64_t *kernels) {
    cudaStream_t origin;
    GQ_CUDA(cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking));
    std::vector<cudaStream_t> st(S);
    std::vector<gq_ctx> sctx(S);
    for (int s = 0; s < S; ++s) {
        GQ_CUDA(cudaStreamCreateWithFlags(&st[s], cudaStreamNonBlocking));
        sctx[s].device = b->ctx->device;
        sctx[s].stream = st[s];
    }
    gq_ctx octx;
    octx.device = b->ctx->device;
    octx.stream = origin;
    std::vector<int> order(b->geoms.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::sort(order.begin(), order.end(), [&](int a, int c) { return cost_of(b->geoms[a]) > cost_of(b->geoms[c]); });
    std::vector<double> load(S, 0.0);
    std::vector<int> assign(b->geoms.size());
    for (int i : order) {
        int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        assign[i] = s;
        load[s] += cost_of(b->geoms[i]);
    }
    int sms = 0;
    GQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx->device));
    cudaGraph_t graph = nullptr;
    cudaEvent_t fork;
    std::vector<cudaEvent_t> joins(S);
    GQ_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int s = 0; s < S; ++s) GQ_CUDA(cudaEventCreateWithFlags(&joins[s], cudaEventDisableTiming));
    std::vector<gq_ctx *> saved(b->geoms.size(), nullptr);
    GQ_CUDA(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
    try {
        GQ_CUDA(cudaEventRecord(fork, origin));
        for (int s = 0; s < S; ++s) GQ_CUDA(cudaStreamWaitEvent(st[s], fork, 0));
        for (size_t i = 0; i < b->geoms.size(); ++i) {
            gq_geom *g = b->geoms[i];
            saved[i] = g->ctx;
            g->ctx = &sctx[assign[i]];
            gq_bplan_fmm(P, (int)i);
            g->ctx = saved[i];
        }
        for (int s = 0; s < S; ++s) {
            GQ_CUDA(cudaEventRecord(joins[s], st[s]));
            GQ_CUDA(cudaStreamWaitEvent(origin, joins[s], 0));
        }
        gq_bplan_persistent(P, &octx, std::max(1, sms * quarters / 4), b->wait_ns);
        GQ_CUDA(cudaStreamEndCapture(origin, &graph));
    } catch (...) {
        for (size_t i = 0; i < b->geoms.size(); ++i)
            if (saved[i]) b->geoms[i]->ctx = saved[i];
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(origin, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        throw;
    }
    int64_t launched = octx.launches;
    for (auto &c : sctx) launched += c.launches;
    *kernels = launched;
    cudaGraphExec_t exec = nullptr;
    GQ_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    cudaGraphDestroy(graph);
    cudaEventDestroy(fork);
    for (auto e : joins) cudaEventDestroy(e);
    for (auto x : st) cudaStreamDestroy(x);
    cudaStreamDestroy(origin);
    return exec;
}

gq_bplan *plan_for(gq_batch *b, int kernel, int ndens, const double *const *dens, double *const *out, int tile) {
    if (!b->plan)
        b->plan = gq_bplan_new(b->ctx, kernel, ndens, b->geoms, dens, out, tile, b->stall_geom);
    else if (gq_bplan_tile(b->plan) != tile)
        gq_bplan_retile(b->plan, tile);
    return b->plan;
}

double time_replays(gq_batch *b, cudaGraphExec_t exec) {
    cudaStream_t st = b->ctx->stream;
    cudaEvent_t e0, e1;
    GQ_CUDA(cudaEventCreate(&e0));
    GQ_CUDA(cudaEventCreate(&e1));
    GQ_CUDA(cudaGraphLaunch(exec, st));
    GQ_CUDA(cudaEventRecord(e0, st));
    for (int r = 0; r < 2; ++r) GQ_CUDA(cudaGraphLaunch(exec, st));
    GQ_CUDA(cudaEventRecord(e1, st));
    GQ_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    GQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ms / 2.0;
}

}  // namespace

gq_batch *gq_batch_new(gq_ctx *ctx, int n, gq_geom *const *geoms) {
    gq_batch *b = new gq_batch;
    b->ctx = ctx;
    b->geoms.assign(geoms, geoms + n);
    return b;
}

void gq_batch_free(gq_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
}

static void drop_capture(gq_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    if (b->plan) gq_bplan_free(b->plan);
    b->plan = nullptr;
}

void gq_batch_config_impl(gq_batch *b, int mode, long long wait_ns, int stall_geom) {
    drop_capture(b);
    b->mode = mode;
    if (wait_ns > 0) b->wait_ns = (unsigned long long)wait_ns;
    b->stall_geom = stall_geom;
}

int gq_batch_persistent_tile(const gq_batch *b) { return b->persistent ? b->tile : 0; }
int gq_batch_persistent_ctas_impl(const gq_batch *b) {
    int sms = 0;
    GQ_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->ctx->device));
    return b->persistent ? std::max(1, sms * b->quarters / 4) : 0;
}

void gq_batch_eval_impl(gq_batch *b, int kernel, int ndens, const double *const *dens, double *const *out) {
    gq_ctx *ctx = b->ctx;
    size_t n = b->geoms.size();
    bool same = b->exec && b->kernel == kernel && b->ndens == ndens && b->dens.size() == n;
    for (size_t i = 0; same && i < n; ++i) same = b->dens[i] == dens[i] && b->out[i] == out[i];
    if (!same) {
        drop_capture(b);
        // eager pass: sizes every buffer and table so that capture allocates nothing
        for (size_t i = 0; i < n; ++i) {
            gq_geom *g = b->geoms[i];
            gq_ctx *saved = g->ctx;
            g->ctx = ctx;
            eval_densities(g, kernel, ndens, dens[i], out[i]);
            g->ctx = saved;
        }
        GQ_CUDA(cudaStreamSynchronize(ctx->stream));
        // candidates: the persistent launch (mode 0, or mode 2 where supported)
        // and the graph branches (mode 1, mode 2, or where the persistent
        // launch is not supported)
        const bool can_p = b->mode != 1 && gq_bplan_supported(b->geoms, kernel);
        const bool try_g = b->mode != 0 || !can_p;
        std::string key = std::string(b->mode == 2 ? "A" : (can_p ? "P" : "")) + shape_key(b, kernel, ndens);
        int S = 0, tile = 1, quarters = 4;
        bool pers = can_p && !try_g;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            if (g_tune.empty()) load_cache_file();
            auto it = g_tune.find(key);
            if (it != g_tune.end()) {
                S = it->second % 100;
                tile = (it->second / 100) % 100;
                pers = can_p && (!try_g || (it->second / 10000) % 10 == 1);
                quarters = it->second / 100000 ? it->second / 100000 : 4;
            }
        }
        auto time_config = [&](bool p, int streams, int t, int qq) {
            int64_t kn = 0;
            cudaGraphExec_t ex = p ? capture_persistent(b, plan_for(b, kernel, ndens, dens, out, t), streams, qq, &kn)
                                   : capture(b, kernel, ndens, dens, out, streams, &kn);
            double ms = time_replays(b, ex);
            cudaGraphExecDestroy(ex);
            return ms;
        };
        if (S <= 0 || tile <= 0) {
            // per path: streams for the per-geometry branches first, then (the
            // persistent launch) the target boxes per direct item with those
            // streams, then its CTA count; the faster path wins
            double best = 1e300;
            for (int path = 0; path < 2; ++path) {
                const bool p = path == 0;
                if (p ? !can_p : !try_g) continue;
                double pbest = 1e300;
                int pS = 1, pt = 1, pq = 4;
                for (int cand : {1, 2, 4, 8, 16}) {
                    if (cand > (int)n && cand != 1) break;
                    double ms = time_config(p, cand, 1, 4);
                    if (ms < pbest) {
                        pbest = ms;
                        pS = cand;
                    }
                }
                if (p) {
                    for (int t : {2, 4}) {
                        double ms = time_config(p, pS, t, 4);
                        if (ms < pbest) {
                            pbest = ms;
                            pt = t;
                        }
                    }
                    for (int qq : {3, 2}) {
                        double ms = time_config(p, pS, pt, qq);
                        if (ms < pbest) {
                            pbest = ms;
                            pq = qq;
                        }
                    }
                }
                {   // each path's winner also serves a later call in mode 0 or 1
                    std::lock_guard<std::mutex> lk(g_tune_mu);
                    g_tune[std::string(p ? "P" : "") + shape_key(b, kernel, ndens)] =
                        pq * 100000 + (p ? 10000 : 0) + pt * 100 + pS;
                }
                if (pbest < best) {
                    best = pbest;
                    S = pS;
                    tile = pt;
                    quarters = pq;
                    pers = p;
                }
            }
            b->tuned_ms = best;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune[key] = quarters * 100000 + (pers ? 10000 : 0) + tile * 100 + S;
            save_cache_file();
        }
        b->persistent = pers;
        if (b->plan) {   // the tuning replays of the persistent launch ran its waits
            const int e = gq_bplan_error(b->plan);
            if (!pers) {
                gq_bplan_free(b->plan);
                b->plan = nullptr;
            }
            GQ_REQUIRE(e == 0, GQ_ERR_TIMEOUT, "batched evaluation: a bounded dependency wait gave up");
        }
        b->exec = b->persistent ? capture_persistent(b, plan_for(b, kernel, ndens, dens, out, tile), S, quarters,
                                                     &b->kernels_per_replay)
                                : capture(b, kernel, ndens, dens, out, S, &b->kernels_per_replay);
        b->tile = tile;
        b->quarters = quarters;
        b->kernel = kernel;
        b->ndens = ndens;
        b->streams = S;
        b->dens.assign(dens, dens + n);
        b->out.assign(out, out + n);
    }
    GQ_CUDA(cudaGraphLaunch(b->exec, ctx->stream));
    ctx->launches += b->kernels_per_replay;
    if (b->persistent)
        GQ_REQUIRE(gq_bplan_error(b->plan) == 0, GQ_ERR_TIMEOUT,
                   "batched evaluation: a bounded dependency wait gave up");
}

int gq_batch_streams(const gq_batch *b) { return b->streams; }
int gq_batch_size(const gq_batch *b) { return (int)b->geoms.size(); }
gq_geom *gq_batch_geom(const gq_batch *b, int i) { return b->geoms[i]; }
gq_ctx *gq_batch_ctx(const gq_batch *b) { return b->ctx; }
