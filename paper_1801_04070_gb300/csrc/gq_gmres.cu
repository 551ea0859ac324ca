// gq_gmres.cu -- exterior Neumann problem (Sec. 1): represent u = S mu and
// solve the second-kind equation  -mu/2 + S' mu = g  for mu at the base
// nodes by restarted GMRES.  The operator is applied with the GIGAQBX
// evaluation of S' (two-sided QBX at the base nodes, i.e. the principal
// value); Arnoldi vectors, dot products and updates are FP64 device
// kernels (classical Gram-Schmidt applied twice), the small Hessenberg
// least-squares problem is solved on the host with Givens rotations.
#include <math.h>

#include <vector>

#include "gq_internal.cuh"

namespace {

constexpr int kT = 256;

// out = a x + b y
__global__ void k_axpby(int n, double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                        double *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

// out[i] = <V_i, w> for i < k (one block per basis vector, deterministic order)
__global__ void k_multidot(int n, int k, const double *__restrict__ V, const double *__restrict__ w,
                           double *__restrict__ out) {
    int i = blockIdx.x;
    if (i >= k) return;
    const double *v = V + (size_t)i * n;
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) s += v[j] * w[j];
    __shared__ double sh[1024];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[i] = sh[0];
}

// w -= sum_i h_i V_i
__global__ void k_subtract_basis(int n, int k, const double *__restrict__ V, const double *__restrict__ h,
                                 double *__restrict__ w) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = w[j];
    for (int i = 0; i < k; ++i) s -= h[i] * V[(size_t)i * n + j];
    w[j] = s;
}

// x += sum_i y_i V_i
__global__ void k_add_basis(int n, int k, const double *__restrict__ V, const double *__restrict__ y,
                            double *__restrict__ x) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = x[j];
    for (int i = 0; i < k; ++i) s += y[i] * V[(size_t)i * n + j];
    x[j] = s;
}

__global__ void k_scale(int n, double a, double *__restrict__ x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= a;
}

struct Solver {
    gq_geom *g;
    int n;
    dbuf<double> hdev;
    void apply(const double *v, double *out) {   // out = -v/2 + S' v at the base nodes (gq_apply)
        const double minus_half = -0.5;
        gq_eval_all(g, GQ_SP, v, out, nullptr, nullptr, &minus_half);
    }
    std::vector<double> dots(const double *V, int k, const double *w) {
        GQ_LAUNCH(g->ctx, k_multidot, k, 1024, 0, n, k, V, w, hdev.p);
        std::vector<double> h(k);
        GQ_CUDA(cudaMemcpyAsync(h.data(), hdev.p, sizeof(double) * k, cudaMemcpyDeviceToHost, g->ctx->stream));
        GQ_CUDA(cudaStreamSynchronize(g->ctx->stream));
        return h;
    }
    double norm(const double *w) { return sqrt(dots(w, 1, w)[0]); }
};

}  // namespace

// returns iterations; mu (device) holds the solution, *resid the relative residual estimate
int gq_gmres_impl(gq_geom *g, const double *rhs_dev, double tol, int maxit, int restart, double *mu_dev,
                  double *resid) {
    gq_ctx *ctx = g->ctx;
    cudaStream_t st = ctx->stream;
    const int n = g->nbase, m = restart;
    Solver S;
    S.g = g;
    S.n = n;
    S.hdev.alloc(m + 2);
    dbuf<double> V, w, r;
    V.alloc((size_t)(m + 1) * n);
    w.alloc(n);
    r.alloc(n);
    GQ_CUDA(cudaMemsetAsync(mu_dev, 0, sizeof(double) * n, st));
    double bnorm = S.norm(rhs_dev);
    if (bnorm == 0.0) {
        *resid = 0.0;
        return 0;
    }
    int it = 0;
    double rel = 1.0;
    while (it < maxit) {
        // r = b - A mu
        S.apply(mu_dev, r.p);
        GQ_LAUNCH(ctx, k_axpby, gq_blocks(n, kT), kT, 0, n, 1.0, rhs_dev, -1.0, (const double *)r.p, r.p);
        double beta = S.norm(r.p);
        rel = beta / bnorm;
        if (rel <= tol) break;
        GQ_LAUNCH(ctx, k_axpby, gq_blocks(n, kT), kT, 0, n, 1.0 / beta, (const double *)r.p, 0.0,
                  (const double *)r.p, V.p);
        std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), e(m + 1, 0.0);
        e[0] = beta;
        int j = 0;
        for (; j < m && it < maxit; ++j, ++it) {
            double *vj = V.p + (size_t)j * n, *vn = V.p + (size_t)(j + 1) * n;
            S.apply(vj, w.p);
            std::vector<double> h(j + 1, 0.0);
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                std::vector<double> c = S.dots(V.p, j + 1, w.p);
                GQ_CUDA(cudaMemcpyAsync(S.hdev.p, c.data(), sizeof(double) * (j + 1), cudaMemcpyHostToDevice, st));
                GQ_LAUNCH(ctx, k_subtract_basis, gq_blocks(n, kT), kT, 0, n, j + 1, (const double *)V.p,
                          (const double *)S.hdev.p, w.p);
                for (int i = 0; i <= j; ++i) h[i] += c[i];
            }
            double hn = S.norm(w.p);
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i];
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0) GQ_LAUNCH(ctx, k_axpby, gq_blocks(n, kT), kT, 0, n, 1.0 / hn, (const double *)w.p, 0.0,
                                  (const double *)w.p, vn);
            // apply the previous rotations to the new column, then form a new one
            for (int i = 0; i < j; ++i) {
                double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            double den = hypot(a, b);
            cs[j] = den > 0 ? a / den : 1.0;
            sn[j] = den > 0 ? b / den : 0.0;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            e[j + 1] = -sn[j] * e[j];
            e[j] = cs[j] * e[j];
            rel = fabs(e[j + 1]) / bnorm;
            if (rel <= tol || hn == 0.0) {
                ++j;
                ++it;
                break;
            }
        }
        // back substitution for the j coefficients, then mu += V y
        std::vector<double> y(j, 0.0);
        for (int i = j - 1; i >= 0; --i) {
            double s = e[i];
            for (int k = i + 1; k < j; ++k) s -= H[(size_t)i * m + k] * y[k];
            y[i] = s / H[(size_t)i * m + i];
        }
        if (j > 0) {
            GQ_CUDA(cudaMemcpyAsync(S.hdev.p, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, st));
            GQ_LAUNCH(ctx, k_add_basis, gq_blocks(n, kT), kT, 0, n, j, (const double *)V.p, (const double *)S.hdev.p,
                      mu_dev);
        }
        GQ_CUDA(cudaStreamSynchronize(st));
        if (rel <= tol) break;
    }
    // true residual of the returned solution
    S.apply(mu_dev, r.p);
    GQ_LAUNCH(ctx, k_axpby, gq_blocks(n, kT), kT, 0, n, 1.0, rhs_dev, -1.0, (const double *)r.p, r.p);
    *resid = S.norm(r.p) / bnorm;
    return it;
}

// ------------------------------------------------------------------ batched GMRES
// The same restarted GMRES on every geometry of a batch in lockstep: each
// Arnoldi step applies S' to all geometries' current basis vectors with one
// replay of the batch's CUDA graph, and the orthogonalisation runs on the
// concatenated vectors (one block per (basis vector, geometry) for the dot
// products, one thread per element for the updates), with each geometry's
// Hessenberg matrix and rotations on the host.  Per geometry the arithmetic
// is that of gq_gmres (same reductions in the same order), so the solutions
// agree with one solve after another.  A geometry that has converged keeps
// riding along in the graph replays; its vectors are no longer updated.
namespace {

__global__ void k_multidot_seg(const long long *__restrict__ off, int k, long long N, const double *__restrict__ V,
                               const double *__restrict__ w, double *__restrict__ out) {
    int kk = blockIdx.x, i = blockIdx.y;
    long long o = off[i];
    int n = (int)(off[i + 1] - o);
    const double *v = V + (size_t)kk * N + o;
    const double *ww = w + o;
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) s += v[j] * ww[j];
    __shared__ double sh[1024];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) sh[threadIdx.x] += sh[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[(size_t)i * k + kk] = sh[0];
}

__global__ void k_subtract_seg(long long N, int k, const double *__restrict__ V, const double *__restrict__ h,
                               const int *__restrict__ seg, double *__restrict__ w) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double *hi = h + (size_t)seg[j] * k;
    double s = w[j];
    for (int i = 0; i < k; ++i) s -= hi[i] * V[(size_t)i * N + j];
    w[j] = s;
}

__global__ void k_axpby_seg(long long N, const double *__restrict__ a, const double *__restrict__ x,
                            const double *__restrict__ b, const double *__restrict__ y, const int *__restrict__ seg,
                            double *__restrict__ out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    int i = seg[j];
    out[j] = a[i] * x[j] + b[i] * y[j];
}

__global__ void k_add_basis_seg(long long N, int kmax, const double *__restrict__ V, const double *__restrict__ y,
                                const int *__restrict__ cnt, const int *__restrict__ seg, double *__restrict__ x) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    int g = seg[j];
    const double *yi = y + (size_t)g * kmax;
    double s = x[j];
    for (int i = 0; i < cnt[g]; ++i) s += yi[i] * V[(size_t)i * N + j];
    x[j] = s;
}

__global__ void k_fill_seg(const long long *__restrict__ off, int *__restrict__ seg) {
    int i = blockIdx.y;
    long long o = off[i], e = off[i + 1];
    for (long long j = o + (long long)blockIdx.x * blockDim.x + threadIdx.x; j < e; j += (long long)gridDim.x * blockDim.x)
        seg[j] = i;
}

int blocks_ll(long long n) { return (int)((n + kT - 1) / kT); }

struct BatchSolver {
    gq_batch *b;
    gq_ctx *ctx;
    int G;
    long long N;
    std::vector<long long> off;
    dbuf<long long> off_d;
    dbuf<int> seg;
    dbuf<double> X, Y, hdev, sa, sb;
    std::vector<const double *> xin;
    std::vector<double *> yout;

    void apply(const double *v, double *out) {   // out = -v/2 + S' v, every geometry
        GQ_CUDA(cudaMemcpyAsync(X.p, v, sizeof(double) * N, cudaMemcpyDeviceToDevice, ctx->stream));
        gq_batch_eval_impl(b, GQ_SP, 1, xin.data(), yout.data());
        GQ_LAUNCH(ctx, k_axpby, blocks_ll(N), kT, 0, (int)N, -0.5, v, 1.0, (const double *)Y.p, out);
    }
    // [G][k] dot products of V_0..V_{k-1} with w
    std::vector<double> dots(const double *V, int k, const double *w) {
        GQ_LAUNCH(ctx, k_multidot_seg, dim3(k, G), 1024, 0, (const long long *)off_d.p, k, N, V, w, hdev.p);
        std::vector<double> h((size_t)G * k);
        GQ_CUDA(cudaMemcpyAsync(h.data(), hdev.p, sizeof(double) * G * k, cudaMemcpyDeviceToHost, ctx->stream));
        GQ_CUDA(cudaStreamSynchronize(ctx->stream));
        return h;
    }
    std::vector<double> norms(const double *w) {
        std::vector<double> h = dots(w, 1, w);
        for (auto &x : h) x = sqrt(x);
        return h;
    }
    // out = a_i x + b_i y per geometry
    void axpby(const std::vector<double> &a, const double *x, const std::vector<double> &bb, const double *y,
               double *out) {
        GQ_CUDA(cudaMemcpyAsync(sa.p, a.data(), sizeof(double) * G, cudaMemcpyHostToDevice, ctx->stream));
        GQ_CUDA(cudaMemcpyAsync(sb.p, bb.data(), sizeof(double) * G, cudaMemcpyHostToDevice, ctx->stream));
        GQ_LAUNCH(ctx, k_axpby_seg, blocks_ll(N), kT, 0, N, (const double *)sa.p, x, (const double *)sb.p, y,
                  (const int *)seg.p, out);
    }
};

}  // namespace

void gq_batch_gmres_impl(gq_batch *b, const double *const *rhs_dev, double tol, int maxit, int restart,
                         double *const *mu_dev, int *iters, double *resid) {
    BatchSolver S;
    S.b = b;
    S.ctx = gq_batch_ctx(b);
    gq_ctx *ctx = S.ctx;
    cudaStream_t st = ctx->stream;
    const int G = gq_batch_size(b), m = restart;
    S.G = G;
    S.off.assign(G + 1, 0);
    for (int i = 0; i < G; ++i) S.off[i + 1] = S.off[i] + gq_batch_geom(b, i)->nbase;
    const long long N = S.off[G];
    S.N = N;
    GQ_REQUIRE(N < (1LL << 31), GQ_ERR_UNSUPPORTED, "gq_batch_gmres: more than 2^31 unknowns in one batch");
    S.off_d.alloc(G + 1);
    GQ_CUDA(cudaMemcpyAsync(S.off_d.p, S.off.data(), sizeof(long long) * (G + 1), cudaMemcpyHostToDevice, st));
    S.seg.alloc(N);
    GQ_LAUNCH(ctx, k_fill_seg, dim3(64, G), kT, 0, (const long long *)S.off_d.p, S.seg.p);
    S.X.alloc(N);
    S.Y.alloc(N);
    S.hdev.alloc((size_t)G * (m + 2));
    S.sa.alloc(G);
    S.sb.alloc(G);
    for (int i = 0; i < G; ++i) {
        S.xin.push_back(S.X.p + S.off[i]);
        S.yout.push_back(S.Y.p + S.off[i]);
    }
    dbuf<double> V, w, r, B, MU;
    V.alloc((size_t)(m + 1) * N);
    w.alloc(N);
    r.alloc(N);
    B.alloc(N);
    MU.alloc(N);
    for (int i = 0; i < G; ++i)
        GQ_CUDA(cudaMemcpyAsync(B.p + S.off[i], rhs_dev[i], sizeof(double) * (S.off[i + 1] - S.off[i]),
                                cudaMemcpyDeviceToDevice, st));
    GQ_CUDA(cudaMemsetAsync(MU.p, 0, sizeof(double) * N, st));
    std::vector<double> bnorm = S.norms(B.p);
    std::vector<int> it(G, 0);
    std::vector<double> rel(G, 1.0);
    std::vector<char> conv(G, 0);
    for (int i = 0; i < G; ++i)
        if (bnorm[i] == 0.0) {
            conv[i] = 1;
            rel[i] = 0.0;
        }
    auto unconverged = [&] {
        for (int i = 0; i < G; ++i)
            if (!conv[i] && it[i] < maxit) return true;
        return false;
    };
    const std::vector<double> ones(G, 1.0), minus(G, -1.0), zeros(G, 0.0);
    while (unconverged()) {
        // r = b - A mu
        S.apply(MU.p, r.p);
        S.axpby(ones, B.p, minus, r.p, r.p);
        std::vector<double> beta = S.norms(r.p);
        std::vector<char> run(G, 0);
        std::vector<double> sc(G, 0.0);
        for (int i = 0; i < G; ++i) {
            if (conv[i] || it[i] >= maxit) continue;
            rel[i] = beta[i] / bnorm[i];
            if (rel[i] <= tol) {
                conv[i] = 1;
                continue;
            }
            run[i] = 1;
            sc[i] = 1.0 / beta[i];
        }
        bool any = false;
        for (int i = 0; i < G; ++i) any |= run[i] != 0;
        if (!any) break;
        S.axpby(sc, r.p, zeros, r.p, V.p);
        std::vector<std::vector<double>> H(G, std::vector<double>((size_t)(m + 1) * m, 0.0)), cs(G, std::vector<double>(m)),
            sn(G, std::vector<double>(m)), e(G, std::vector<double>(m + 1, 0.0));
        std::vector<int> cnt(G, 0);
        for (int i = 0; i < G; ++i) e[i][0] = beta[i];
        for (int j = 0; j < m; ++j) {
            bool live = false;
            for (int i = 0; i < G; ++i) live |= run[i] != 0;
            if (!live) break;
            double *vj = V.p + (size_t)j * N, *vn = V.p + (size_t)(j + 1) * N;
            S.apply(vj, w.p);
            std::vector<double> h((size_t)G * (j + 1), 0.0);
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                std::vector<double> c = S.dots(V.p, j + 1, w.p);
                GQ_CUDA(cudaMemcpyAsync(S.hdev.p, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice, st));
                GQ_LAUNCH(ctx, k_subtract_seg, blocks_ll(N), kT, 0, N, j + 1, (const double *)V.p,
                          (const double *)S.hdev.p, (const int *)S.seg.p, w.p);
                for (size_t x = 0; x < c.size(); ++x) h[x] += c[x];
            }
            std::vector<double> hn = S.norms(w.p);
            std::vector<double> inv(G, 0.0);
            for (int i = 0; i < G; ++i)
                if (run[i] && hn[i] > 0) inv[i] = 1.0 / hn[i];
            S.axpby(inv, w.p, zeros, w.p, vn);
            for (int i = 0; i < G; ++i) {
                if (!run[i]) continue;
                std::vector<double> &Hi = H[i];
                for (int k = 0; k <= j; ++k) Hi[(size_t)k * m + j] = h[(size_t)i * (j + 1) + k];
                Hi[(size_t)(j + 1) * m + j] = hn[i];
                for (int k = 0; k < j; ++k) {
                    double a = Hi[(size_t)k * m + j], bb = Hi[(size_t)(k + 1) * m + j];
                    Hi[(size_t)k * m + j] = cs[i][k] * a + sn[i][k] * bb;
                    Hi[(size_t)(k + 1) * m + j] = -sn[i][k] * a + cs[i][k] * bb;
                }
                double a = Hi[(size_t)j * m + j], bb = Hi[(size_t)(j + 1) * m + j];
                double den = hypot(a, bb);
                cs[i][j] = den > 0 ? a / den : 1.0;
                sn[i][j] = den > 0 ? bb / den : 0.0;
                Hi[(size_t)j * m + j] = den;
                Hi[(size_t)(j + 1) * m + j] = 0.0;
                e[i][j + 1] = -sn[i][j] * e[i][j];
                e[i][j] = cs[i][j] * e[i][j];
                rel[i] = fabs(e[i][j + 1]) / bnorm[i];
                cnt[i] = j + 1;
                ++it[i];
                if (rel[i] <= tol || hn[i] == 0.0 || it[i] >= maxit) run[i] = 0;
            }
        }
        // back substitution per geometry, then mu += V y
        std::vector<double> y((size_t)G * m, 0.0);
        for (int i = 0; i < G; ++i) {
            int j = cnt[i];
            for (int k = j - 1; k >= 0; --k) {
                double s = e[i][k];
                for (int l = k + 1; l < j; ++l) s -= H[i][(size_t)k * m + l] * y[(size_t)i * m + l];
                y[(size_t)i * m + k] = s / H[i][(size_t)k * m + k];
            }
        }
        dbuf<double> yd;
        dbuf<int> cd;
        yd.alloc(y.size());
        cd.alloc(G);
        GQ_CUDA(cudaMemcpyAsync(yd.p, y.data(), sizeof(double) * y.size(), cudaMemcpyHostToDevice, st));
        GQ_CUDA(cudaMemcpyAsync(cd.p, cnt.data(), sizeof(int) * G, cudaMemcpyHostToDevice, st));
        GQ_LAUNCH(ctx, k_add_basis_seg, blocks_ll(N), kT, 0, N, m, (const double *)V.p, (const double *)yd.p,
                  (const int *)cd.p, (const int *)S.seg.p, MU.p);
        GQ_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < G; ++i)
            if (cnt[i] > 0 && rel[i] <= tol) conv[i] = 1;
    }
    // true residuals of the returned solutions
    S.apply(MU.p, r.p);
    S.axpby(ones, B.p, minus, r.p, r.p);
    std::vector<double> rn = S.norms(r.p);
    for (int i = 0; i < G; ++i) {
        GQ_CUDA(cudaMemcpyAsync(mu_dev[i], MU.p + S.off[i], sizeof(double) * (S.off[i + 1] - S.off[i]),
                                cudaMemcpyDeviceToDevice, st));
        if (iters) iters[i] = it[i];
        if (resid) resid[i] = bnorm[i] > 0 ? rn[i] / bnorm[i] : 0.0;
    }
    GQ_CUDA(cudaStreamSynchronize(st));
}
