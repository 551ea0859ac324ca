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
    dbuf<double> tmp, hdev;
    void apply(const double *v, double *out) {   // out = -v/2 + S' v
        gq_eval_all(g, GQ_SP, v, tmp.p, nullptr);
        GQ_LAUNCH(g->ctx, k_axpby, gq_blocks(n, kT), kT, 0, n, -0.5, v, 1.0, (const double *)tmp.p, out);
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
    S.tmp.alloc(n);
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
