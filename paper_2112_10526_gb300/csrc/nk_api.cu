// C ABI of libnk (declared in include/nk.h): argument checks, workspace
// planning, and the orchestration of one VMC + SR step (NetKet 3, Sec. 4.1)
// out of the kernels in k_rbm.cu and k_linalg.cu.

#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/nk.h"
#include "nk_internal.h"


namespace {

thread_local std::string g_err;

nk_status fail(nk_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

nk_status cuda_fail(cudaError_t e, const char *where) {
    return fail(e == cudaErrorMemoryAllocation ? NK_ERR_OOM : NK_ERR_CUDA, "%s: %s", where,
                cudaGetErrorString(e));
}

#define NK_CU(call, where)                                       \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail(e_, where);      \
    } while (0)

// Scoped switch to the context's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            ok = false;
            return;
        }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Plan-only mode (this thread): entry points check arguments, count their
// workspace into ctx->plan_bytes and return without touching the device.
thread_local bool g_plan_only = false;

bool is_device_ptr(const void *p) {
    if (g_plan_only) return p != nullptr;
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define NK_DEV(ptr, name)                                                                  \
    do {                                                                                   \
        if (!is_device_ptr(ptr))                                                           \
            return fail(NK_ERR_INVALID_ARG, "%s must be a device pointer (got %p)", name, \
                        (const void *)(ptr));                                              \
    } while (0)

// Workspace carving: the same sequence of take() calls runs once to count
// bytes (base = null) and once to hand out pointers.
struct Carver {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
};

nk_status ensure_ws(nk_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->ws_size) return NK_OK;
    if (ctx->ws) {
        cudaError_t e = cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_size = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    size_t want = bytes + bytes / 8 + (1 << 20);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NK_ERR_OOM, "workspace of %zu bytes: %s", want, cudaGetErrorString(e));
    }
    ctx->ws = static_cast<char *>(p);
    ctx->ws_size = want;
    return NK_OK;
}

template <class Body>
nk_status with_workspace(nk_ctx *ctx, Body body) {
    Carver count{nullptr};
    nk_status st = body(count, false);
    if (st != NK_OK) return st;
    if (g_plan_only) {
        ctx->plan_bytes = count.off > ctx->plan_bytes ? count.off : ctx->plan_bytes;
        return NK_OK;
    }
    st = ensure_ws(ctx, count.off);
    if (st != NK_OK) return st;
    Carver real{ctx->ws};
    return body(real, true);
}

inline int64_t n_params(int N, int M) { return (int64_t)N + M + (int64_t)M * N; }

nk_status check_rbm(const nk_rbm *rbm) {
    if (!rbm) return fail(NK_ERR_INVALID_ARG, "rbm is NULL");
    if (rbm->N < 1 || rbm->N > 4096) return fail(NK_ERR_INVALID_ARG, "N=%d out of [1, 4096]", rbm->N);
    if (rbm->M < 1 || rbm->M > 8192) return fail(NK_ERR_INVALID_ARG, "M=%d out of [1, 8192]", rbm->M);
    NK_DEV(rbm->params, "rbm->params");
    return NK_OK;
}

nk_status check_precision(int32_t p) {
    if (p != NK_F64 && p != NK_MIXED) return fail(NK_ERR_INVALID_ARG, "precision %d unknown", p);
    return NK_OK;
}

nk_status check_ham(const nk_ham *h, int N) {
    if (!h) return fail(NK_ERR_INVALID_ARG, "ham is NULL");
    if (h->kind != NK_TFIM && h->kind != NK_HEIS)
        return fail(NK_ERR_INVALID_ARG, "ham->kind %d unknown", h->kind);
    if (h->n_edges < 1 || h->n_edges > 65536)
        return fail(NK_ERR_INVALID_ARG, "ham->n_edges=%d out of [1, 65536]", h->n_edges);
    if (h->n_edges2 < 0 || h->n_edges2 > h->n_edges)
        return fail(NK_ERR_INVALID_ARG, "ham->n_edges2=%d out of [0, n_edges]", h->n_edges2);
    NK_DEV(h->edges, "ham->edges");
    (void)N;
    return NK_OK;
}

template <typename R>
void carve_tables(Carver &c, nk::Tables<R> &t, const nk_rbm *rbm, int E, const int32_t *edges,
                  bool site, bool edge) {
    const int N = rbm->N, M = rbm->M;
    t.N = N;
    t.M = M;
    t.E = E;
    t.a = rbm->params;
    t.b = rbm->params + N;
    t.W = rbm->params + N + M;
    t.edges = edges;
    t.Wt = c.take<double>((size_t)N * M);
    t.tau_site = site ? c.take<R>((size_t)N * M) : nullptr;
    t.tau_siteT = site ? c.take<R>((size_t)N * M) : nullptr;
    t.K_site = site ? c.take<R>(N) : nullptr;
    t.tau_edge = edge ? c.take<R>((size_t)E * M) : nullptr;
    t.tau_edgeT = edge ? c.take<R>((size_t)E * M) : nullptr;
    t.K_edge = edge ? c.take<R>(E) : nullptr;
}

__global__ void k_cg_init(const double *rr, double *ff, double *rr_keep, int *done, int *iters) {
    *ff = *rr;
    *rr_keep = *rr;
    *done = (*rr == 0.0) ? 1 : 0;
    *iters = 0;
}

__global__ void k_add_u64(int n, const unsigned long long *src, unsigned long long *dst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] += src[i];
}

// ------------------------------------------------------------ SR solves ---

struct SolveWs {
    // shared
    double *U, *w, *partial, *dotp, *tmp;
    // CG
    double *x, *r, *p, *Ap, *sc;  // sc: rr, rr_new, pAp, ff, rr_keep
    int *flags;                   // done, iters
    // Cholesky
    double *dJ, *S, *mean, *ones;
    int *info;  // [0] breakdown pivot, [1] tensor-core time-out code
    double *K, *rowmean;
    // SVD solvers: eigenvectors, eigenvalues, their largest, Jacobi workspace
    double *V, *ev, *evmax, *z, *gpart;
    void *eig;
    int *kept;
    void *tc;   // tensor-core slices and inverted diagonal blocks (NK_MIXED)
    void *tcm;  // tensor-core Jacobian-product workspace (NK_MIXED)
    int *colexpT;     // NK_MIXED CG: column exponents of tanh(theta), [M + 1]
    void *colexp_ws;
    void *opA, *opT;  // NK_MIXED CG: the +-1 product operands, built once per solve
    void *thl;        // NK_MIXED CG: tanh(theta) as FP32 pairs, built once per solve
    bool ops_ready;   // opA / opT / thl hold the operands of the samples being solved for
    const int *skip;  // NK_MIXED CG: its converged flag (the products then do nothing)
    int *tcerr; // sticky tensor-core error word of the context
};

size_t tcm_bytes(int N, int M, int64_t B) {
    size_t a = nk::tc_jvp_ws_bytes(N, M, B), b = nk::tc_vjp_ws_bytes(N, M, B), c = nk::tc_theta_ws_bytes(N, M, B);
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

void carve_solve(Carver &c, SolveWs &w, int N, int M, int64_t Ns, int solver, int precision) {
    const int64_t Np = n_params(N, M);
    w = SolveWs{};
    w.partial = c.take<double>(nk::vjp_partial_doubles(N, M, Ns));
    w.dotp = c.take<double>(nk::dot_partial_doubles(Np > Ns ? Np : Ns) + 8);
    w.sc = c.take<double>(8);
    w.flags = c.take<int>(4);
    if (precision == NK_MIXED) w.tcm = c.take<char>(tcm_bytes(N, M, Ns));
    if (solver == NK_SOLVER_CG) {
        w.U = c.take<double>((size_t)Ns * (M + 1));
        w.w = c.take<double>(Ns);
        w.x = c.take<double>(Np);
        w.r = c.take<double>(Np);
        w.p = c.take<double>(Np);
        w.Ap = c.take<double>(Np);
        if (precision == NK_MIXED) {
            w.colexpT = c.take<int>(M + 1);
            w.colexp_ws = c.take<char>(nk::tc_colexp_ws_bytes(M, Ns));
            w.opA = c.take<char>(nk::tc_jvp_operand_bytes(N, Ns));
            w.opT = c.take<char>(nk::tc_vjp_operand_bytes(N, Ns));
            w.thl = c.take<char>(nk::tc_split_t_bytes(M, Ns));
        }
    } else if (solver == NK_SOLVER_CHOLESKY) {
        w.dJ = c.take<double>((size_t)Ns * Np);
        w.S = c.take<double>((size_t)Np * Np);
        w.mean = c.take<double>(Np);
        w.ones = c.take<double>(Ns);
        w.info = c.take<int>(2);
        if (precision == NK_MIXED) w.tc = c.take<char>(nk::tc_chol_ws_bytes(Np));
    } else if (solver == NK_SOLVER_SVD || solver == NK_SOLVER_SVD_SAMPLESPACE) {
        const bool ss = solver == NK_SOLVER_SVD_SAMPLESPACE;
        const int64_t n = ss ? Ns : Np;
        if (ss) {
            w.U = c.take<double>((size_t)Ns * (M + 1));
            w.w = c.take<double>(Ns);
            w.rowmean = c.take<double>(2 * Ns + 1);
            w.tmp = c.take<double>(Np);
            if (precision == NK_MIXED) w.tc = c.take<char>(nk::tc_chol_ws_bytes(Ns));
        } else {
            w.dJ = c.take<double>((size_t)Ns * Np);
            w.mean = c.take<double>(Np);
            w.ones = c.take<double>(Ns);
            if (precision == NK_MIXED) w.tc = c.take<char>(nk::tc_chol_ws_bytes(Np));
        }
        w.K = c.take<double>((size_t)n * n);
        w.V = c.take<double>((size_t)n * n);
        w.ev = c.take<double>(n);
        w.evmax = c.take<double>(4);
        w.z = c.take<double>(n);
        w.gpart = c.take<double>(nk::gemv_t_partial_doubles(n, n));
        w.eig = c.take<char>(nk::eig_ws_bytes(n));
        w.kept = c.take<int>(4);
        w.info = c.take<int>(2);
    } else {
        w.U = c.take<double>((size_t)Ns * (M + 1));
        w.w = c.take<double>(Ns);
        w.K = c.take<double>((size_t)Ns * Ns);
        w.rowmean = c.take<double>(2 * Ns + 1);  // row means, grand mean, centring coefficients
        w.tmp = c.take<double>(Np);
        w.info = c.take<int>(2);
        if (precision == NK_MIXED) w.tc = c.take<char>(nk::tc_chol_ws_bytes(Ns));
    }
}

// (G + eps I) v for the on-the-fly QGT (App. B.3).
// Accuracy of the NK_MIXED Jacobian products, in 8-bit slices per operand
// row: 4 in CG matvecs (at least 2^-32 of the row maximum; run as 3 FP16
// slices of 11 bits, 2^-33), 7 (FP64 level) where the sample-space solve
// subtracts nearly equal vectors.
constexpr int kMatvecSlices = 4, kExactSlices = 7;
// Jacobi sweeps of the SVD solvers: stop at a relative off-diagonal norm of
// 1e-14 (the rounding level of FP64 rotations), at most 60 sweeps.
constexpr int kMaxJacobiSweeps = 60;
constexpr double kJacobiTol = 1e-14;

cudaError_t jvp_any(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *v, SolveWs &w,
                    double *out, int precision, int slices, cudaStream_t st) {
    if (precision == NK_MIXED)
        return nk::launch_jvp_tc(N, M, Ns, s, T, v, out, slices, w.tcerr, w.tcm, st, w.ops_ready ? w.opA : nullptr,
                                 w.ops_ready ? w.thl : nullptr, w.ops_ready ? w.skip : nullptr);
    return nk::launch_jvp(N, M, Ns, s, T, v, w.U, out, st);
}

cudaError_t vjp_any(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *g, double scale,
                    const double *shift, SolveWs &w, double *out, int precision, int slices, cudaStream_t st,
                    const int *colexpT = nullptr) {
    if (precision == NK_MIXED)
        return nk::launch_vjp_tc(N, M, Ns, s, T, g, scale, shift, out, slices, w.tcerr, w.tcm, st, colexpT,
                                 w.ops_ready ? w.opT : nullptr, w.ops_ready ? w.thl : nullptr,
                                 w.ops_ready ? w.skip : nullptr);
    return nk::launch_vjp(N, M, Ns, s, T, g, scale, shift, w.partial, out, st);
}

// (G + eps I) v for the on-the-fly QGT (App. B.3).
// NK_MIXED CG passes the column exponents of T (colexpT) for the J^T g slices.
cudaError_t qgt_onthefly(int N, int M, int64_t Ns, const int8_t *s, const double *T,
                         const double *v, double eps, SolveWs &w, double *out, cudaStream_t st,
                         int precision = NK_F64, const int *colexpT = nullptr) {
    cudaError_t e = jvp_any(N, M, Ns, s, T, v, w, w.w, precision, kMatvecSlices, st);
    if (e != cudaSuccess) return e;
    e = nk::launch_center(Ns, w.w, w.dotp, 1.0 / (double)Ns, st);
    if (e != cudaSuccess) return e;
    e = vjp_any(N, M, Ns, s, T, w.w, 1.0, nullptr, w, out, precision, kMatvecSlices, st, colexpT);
    if (e != cudaSuccess) return e;
    return nk::launch_axpby(n_params(N, M), eps, v, 1.0, out, st);
}

// Reads the factorisation status words back (synchronises the stream).
nk_status check_factor(nk_ctx *ctx, const int *info, cudaStream_t st) {
    NK_CU(cudaMemcpyAsync(ctx->host_flags + 2, info, 2 * sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    NK_CU(cudaStreamSynchronize(st), "status");
    if (ctx->host_flags[3])
        return fail(NK_ERR_TIMEOUT, "a tensor-core product timed out (code %d)", ctx->host_flags[3]);
    if (ctx->host_flags[2])
        return fail(NK_ERR_CUDA, "Cholesky pivot %d not positive", ctx->host_flags[2]);
    return NK_OK;
}

// Cyclic Jacobi sweeps on the full symmetric K [n][n] (diagonalised in
// place; V <- V J from the identity) until the relative off-diagonal norm is
// at the rounding level or kMaxJacobiSweeps: one cooperative launch, whose
// sweep count and final norm are read back once (synchronises the stream).
// norms: 2 device doubles of scratch.
nk_status jacobi_eigen(nk_ctx *ctx, double *K, double *V, int64_t n, void *eig_ws, double *norms, cudaStream_t st,
                       int *sweeps_out, double *rel_out) {
    NK_CU(nk::launch_symmetrize_lower(n, K, st), "eig");
    NK_CU(nk::launch_identity(n, V, st), "eig");
    NK_CU(nk::launch_jacobi_coop(K, V, n, kMaxJacobiSweeps, kJacobiTol, eig_ws, norms, st), "eig sweeps");
    NK_CU(cudaMemcpyAsync(ctx->host_vals, norms, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "eig sweeps");
    NK_CU(cudaStreamSynchronize(st), "eig sweeps");
    *sweeps_out = (int)ctx->host_vals[0];
    *rel_out = ctx->host_vals[1];
    return NK_OK;
}

nk_status run_solve(nk_ctx *ctx, int N, int M, int64_t Ns, const int8_t *s, const double *T,
                    const double *F, int solver, double eps, double tol, int maxiter,
                    SolveWs &w, double *delta, int *host_info, double *host_resid,
                    cudaStream_t st, int precision = NK_F64, bool sync_check = false) {
    const bool tc = precision == NK_MIXED;
    const int64_t Np = n_params(N, M);
    const nk::CholStreams cs{ctx->side, ctx->aux, ctx->ev[0], ctx->ev[1], ctx->ev[2], ctx->ev[3]};
    if (host_info) host_info[0] = 0, host_info[1] = 1;
    if (host_resid) *host_resid = 0.0;
    if (solver == NK_SOLVER_CG) {
        double *rr = w.sc, *rr_new = w.sc + 1, *pAp = w.sc + 2, *ff = w.sc + 3, *rr_keep = w.sc + 4;
        int *done = w.flags, *iters = w.flags + 1;
        if (tc) {
            NK_CU(nk::launch_colexp_t(M, Ns, T, w.colexpT, w.colexp_ws, st), "cg exponents");
            NK_CU(nk::launch_jacobian_operands(N, Ns, s, w.opA, w.opT, st), "cg operands");
            NK_CU(nk::launch_split_t(M, Ns, T, w.thl, st), "cg operands");
        }
        // the operands stay valid for this solve's samples only
        struct OpsReady {
            SolveWs &w;
            ~OpsReady() {
                w.ops_ready = false;
                w.skip = nullptr;
            }
        } ops_guard{w};
        w.ops_ready = tc;
        // the iterations after convergence, up to the next poll, skip the
        // products (their results are discarded by the update kernels)
        w.skip = tc ? done : nullptr;
        NK_CU(nk::launch_fill(Np, 0.0, w.x, st), "cg init");
        NK_CU(nk::launch_axpby(Np, 1.0, F, 0.0, w.r, st), "cg init");
        NK_CU(nk::launch_axpby(Np, 1.0, F, 0.0, w.p, st), "cg init");
        NK_CU(nk::launch_dot(Np, w.r, w.r, w.dotp, rr, st), "cg init");
        (k_cg_init<<<1, 1, 0, st>>>(rr, ff, rr_keep, done, iters), nk::note_launch());
        NK_CU(cudaGetLastError(), "cg init");
        int it = 0;
        bool converged = false;
        while (it < maxiter) {
            NK_CU(qgt_onthefly(N, M, Ns, s, T, w.p, eps, w, w.Ap, st, precision, tc ? w.colexpT : nullptr),
                  "cg matvec");
            NK_CU(nk::launch_dot(Np, w.p, w.Ap, w.dotp, pAp, st), "cg dot");
            NK_CU(nk::launch_cg_update_xr(Np, rr_keep, pAp, w.p, w.Ap, w.x, w.r, done, st), "cg xr");
            NK_CU(nk::launch_dot(Np, w.r, w.r, w.dotp, rr_new, st), "cg dot");
            NK_CU(nk::launch_cg_update_p(Np, rr_new, rr_keep, w.r, w.p, done, st), "cg p");
            NK_CU(nk::launch_cg_check(rr_new, ff, tol, done, iters, rr_keep, st), "cg check");
            ++it;
            if (it % 8 == 0 || it == maxiter) {
                NK_CU(cudaMemcpyAsync(ctx->host_flags, w.flags, 2 * sizeof(int),
                                      cudaMemcpyDeviceToHost, st),
                      "cg poll");
                NK_CU(cudaStreamSynchronize(st), "cg poll");
                if (ctx->host_flags[0]) {
                    converged = true;
                    break;
                }
            }
        }
        NK_CU(nk::launch_axpby(Np, 1.0, w.x, 0.0, delta, st), "cg out");
        NK_CU(cudaMemcpyAsync(ctx->host_flags, w.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, st),
              "cg out");
        NK_CU(cudaMemcpyAsync(ctx->host_vals, w.sc, 5 * sizeof(double), cudaMemcpyDeviceToHost, st),
              "cg out");
        NK_CU(cudaStreamSynchronize(st), "cg out");
        converged = ctx->host_flags[0] != 0;
        const double res = ctx->host_vals[3] > 0 ? std::sqrt(ctx->host_vals[4] / ctx->host_vals[3]) : 0.0;
        if (host_info) host_info[0] = ctx->host_flags[1], host_info[1] = converged ? 1 : 0;
        if (host_resid) *host_resid = res;
        if (!converged)
            return fail(NK_ERR_NOT_CONVERGED, "CG did not reach %g in %d iterations (residual %g)",
                        tol, maxiter, res);
        return NK_OK;
    }
    if (solver == NK_SOLVER_SVD || solver == NK_SOLVER_SVD_SAMPLESPACE) {
        const bool ss = solver == NK_SOLVER_SVD_SAMPLESPACE;
        const int64_t n = ss ? Ns : Np;
        const double rcond = tol > 0.0 ? tol : 1e-12;
        NK_CU(cudaMemsetAsync(w.info, 0, 2 * sizeof(int), st), "svd");
        if (ss) {
            // the centred sample-space Gram X X^T, X = dJ / sqrt(Ns), no shift
            if (tc) {
                NK_CU(nk::launch_gram_tc(N, M, Ns, s, T, 7, w.K, w.info + 1, w.tc, st), "svd gram");
                NK_CU(nk::launch_center_gram(Ns, w.K, w.rowmean, 0.0, st), "svd gram");
            } else {
                NK_CU(nk::launch_gram_samplespace(N, M, Ns, s, T, 0.0, w.K, w.rowmean, st), "svd gram");
            }
        } else {
            // the dense S + eps I from the centred Jacobian
            NK_CU(nk::launch_fill(Ns, 1.0, w.ones, st), "svd mean");
            NK_CU(nk::launch_vjp(N, M, Ns, s, T, w.ones, 1.0 / (double)Ns, nullptr, w.partial, w.mean, st),
                  "svd mean");
            NK_CU(nk::launch_jacobian_rows(N, M, s, T, 0, Ns, w.mean, w.dJ, st), "svd dJ");
            if (tc)
                NK_CU(nk::launch_gram_cols_tc(w.dJ, Ns, Np, 1.0 / (double)Ns, eps, w.K, w.info + 1, w.tc, st),
                      "svd S");
            else
                NK_CU(nk::launch_syrk_t(w.dJ, Ns, Np, 1.0 / (double)Ns, eps, w.K, st), "svd S");
        }
        int sweeps = 0;
        double rel = 0.0;
        nk_status js = jacobi_eigen(ctx, w.K, w.V, n, w.eig, w.evmax + 2, st, &sweeps, &rel);
        if (js != NK_OK) return js;
        const bool converged = rel <= kJacobiTol;
        NK_CU(nk::launch_eig_diag(n, w.K, w.ev, w.evmax, st), "svd eigenvalues");
        NK_CU(cudaMemsetAsync(w.kept, 0, sizeof(int), st), "svd");
        if (ss) {
            // y = X F, z = U^T y / lambda^2 (kept), y = U z, delta = X^T y
            const double isq = 1.0 / std::sqrt((double)Ns);
            NK_CU(jvp_any(N, M, Ns, s, T, F, w, w.w, precision, kExactSlices, st), "svd XF");
            NK_CU(nk::launch_center(Ns, w.w, w.dotp, isq, st), "svd XF");
            NK_CU(nk::launch_gemv_t(w.V, n, n, w.w, 1.0, w.gpart, w.z, st), "svd U^T y");
            NK_CU(nk::launch_spectral_filter(n, w.ev, w.evmax, rcond, 2, w.z, w.kept, st), "svd filter");
            NK_CU(nk::launch_gemv_rows(w.V, n, n, w.z, w.w, st), "svd U z");
            NK_CU(nk::launch_center(Ns, w.w, w.dotp, isq, st), "svd X^T y");
            NK_CU(vjp_any(N, M, Ns, s, T, w.w, 1.0, nullptr, w, delta, precision, kExactSlices, st), "svd X^T y");
        } else {
            // delta = V diag(1 / lambda, kept) V^T F
            NK_CU(nk::launch_gemv_t(w.V, n, n, F, 1.0, w.gpart, w.z, st), "svd V^T F");
            NK_CU(nk::launch_spectral_filter(n, w.ev, w.evmax, rcond, 1, w.z, w.kept, st), "svd filter");
            NK_CU(nk::launch_gemv_rows(w.V, n, n, w.z, delta, st), "svd V z");
        }
        if (host_info) host_info[0] = sweeps, host_info[1] = converged ? 1 : 0;
        if (host_resid) *host_resid = rel;
        if (tc) {
            nk_status f = check_factor(ctx, w.info, st);
            if (f != NK_OK) return f;
        }
        if (!converged)
            return fail(NK_ERR_NOT_CONVERGED, "Jacobi sweeps left a relative off-diagonal norm %g after %d sweeps",
                        rel, sweeps);
        return NK_OK;
    }
    if (solver == NK_SOLVER_CHOLESKY) {
        NK_CU(nk::launch_fill(Ns, 1.0, w.ones, st), "chol");
        NK_CU(nk::launch_vjp(N, M, Ns, s, T, w.ones, 1.0 / (double)Ns, nullptr, w.partial, w.mean, st),
              "chol mean");
        NK_CU(nk::launch_jacobian_rows(N, M, s, T, 0, Ns, w.mean, w.dJ, st), "chol dJ");
        NK_CU(cudaMemsetAsync(w.info, 0, 2 * sizeof(int), st), "chol");
        if (tc)
            NK_CU(nk::launch_gram_cols_tc(w.dJ, Ns, Np, 1.0 / (double)Ns, eps, w.S, w.info + 1, w.tc, st),
                  "chol gram");
        else
            NK_CU(nk::launch_syrk_t(w.dJ, Ns, Np, 1.0 / (double)Ns, eps, w.S, st), "chol syrk");
        if (tc)
            NK_CU(nk::launch_cholesky_tc(w.S, Np, w.info, w.info + 1, w.tc, st, &cs),
                  "chol factor");
        else
            NK_CU(nk::launch_cholesky(w.S, Np, w.info, st), "chol factor");
        NK_CU(nk::launch_axpby(Np, 1.0, F, 0.0, delta, st), "chol");
        if (tc)
            NK_CU(nk::launch_cholesky_solve_tc(w.S, Np, w.tc, delta, w.info + 1, st), "chol solve");
        else
            NK_CU(nk::launch_cholesky_solve(w.S, Np, delta, st), "chol solve");
        return sync_check ? check_factor(ctx, w.info, st) : NK_OK;
    }
    // sample space: delta = (F - X^T (X X^T + eps I)^{-1} X F) / eps, X = dJ / sqrt(Ns)
    const double isq = 1.0 / std::sqrt((double)Ns);
    NK_CU(cudaMemsetAsync(w.info, 0, 2 * sizeof(int), st), "ss");
    if (tc) {
        NK_CU(nk::launch_gram_tc(N, M, Ns, s, T, 7, w.K, w.info + 1, w.tc, st), "ss gram");
        NK_CU(nk::launch_center_gram(Ns, w.K, w.rowmean, eps, st), "ss gram");
        NK_CU(nk::launch_cholesky_tc(w.K, Ns, w.info, w.info + 1, w.tc, st, &cs),
              "ss factor");
    } else {
        NK_CU(nk::launch_gram_samplespace(N, M, Ns, s, T, eps, w.K, w.rowmean, st), "ss gram");
        NK_CU(nk::launch_cholesky(w.K, Ns, w.info, st), "ss factor");
    }
    NK_CU(jvp_any(N, M, Ns, s, T, F, w, w.w, precision, kExactSlices, st), "ss XF");
    NK_CU(nk::launch_center(Ns, w.w, w.dotp, isq, st), "ss XF");
    if (tc)
        NK_CU(nk::launch_cholesky_solve_tc(w.K, Ns, w.tc, w.w, w.info + 1, st), "ss solve");
    else
        NK_CU(nk::launch_cholesky_solve(w.K, Ns, w.w, st), "ss solve");
    NK_CU(nk::launch_center(Ns, w.w, w.dotp, isq, st), "ss Xty");
    NK_CU(vjp_any(N, M, Ns, s, T, w.w, 1.0, nullptr, w, w.tmp, precision, kExactSlices, st), "ss Xty");
    NK_CU(nk::launch_axpby(Np, 1.0 / eps, F, 0.0, delta, st), "ss delta");
    NK_CU(nk::launch_axpby(Np, -1.0 / eps, w.tmp, 1.0, delta, st), "ss delta");
    return sync_check ? check_factor(ctx, w.info, st) : NK_OK;
}

// Metropolis sweeps.  NK_F64 rebuilds theta inside the sweep kernel; NK_MIXED
// runs one sweep per launch, each preceded by the FP64-exact tensor-core
// theta of all chains.
template <typename R>
nk_status run_sweeps(nk_ctx *ctx, const nk::Tables<R> &t, const nk::SweepArgs &a, bool mixed, double *theta,
                     void *tcm, cudaStream_t st) {
    if (!mixed) {
        NK_CU(nk::launch_sweep(t, a, st), "sweep");
        return NK_OK;
    }
    const int total = a.n_discard + a.n_samples;
    for (int w = 0; w < total; ++w) {
        NK_CU(nk::launch_theta_tc(t.N, t.M, t.b, t.W, a.s, a.C, theta, ctx->tc_err, tcm, st), "theta");
        nk::SweepArgs b = a;
        b.sweep0 = a.sweep0 + w;
        b.n_discard = w < a.n_discard ? 1 : 0;
        b.n_samples = w < a.n_discard ? 0 : 1;
        b.theta_in = theta;
        b.out_stride = a.n_samples;
        b.out_offset = w < a.n_discard ? 0 : w - a.n_discard;
        b.dec_stride = total;
        b.dec_offset = w;
        NK_CU(nk::launch_sweep(t, b, st), "sweep");
    }
    return NK_OK;
}

// T = tanh(theta) of a batch: FP64 CUDA-core GEMM (NK_F64) or the FP64-exact
// tensor-core product (NK_MIXED, needs tcm).
nk_status batch_T(nk_ctx *ctx, const nk_rbm *rbm, const int8_t *s, int64_t B, double *T, bool mixed, void *tcm,
                  cudaStream_t st) {
    const int N = rbm->N, M = rbm->M;
    const double *b = rbm->params + N, *W = rbm->params + N + M;
    if (!mixed) {
        NK_CU(nk::launch_theta_tanh(N, M, b, W, s, B, T, st), "theta");
        return NK_OK;
    }
    NK_CU(nk::launch_theta_tc(N, M, b, W, s, B, T, ctx->tc_err, tcm, st), "theta");
    NK_CU(nk::launch_tanh_inplace(B * M, T, st), "tanh");
    return NK_OK;
}

// The sampling half of a VMC step, shared by the plain and the symmetric
// RBM: the flip-ratio tables of `rbm`, the sweeps of the chains (rule and
// its edge count already mapped), T = tanh theta of every sample, the local
// energies and their statistics (mean, variance, error) in st3.
struct StepBufs {
    int8_t *samples;
    double *eloc, *T, *st3, *theta;
    unsigned long long *acc;
    void *tcm;
};

template <typename R>
void carve_step(Carver &c, nk::Tables<R> &t, StepBufs &b, const nk_rbm *rbm, const nk_ham *ham, int C,
                int64_t Ns, bool site, bool edge, bool mixed, int8_t *samples_out, double *eloc_out) {
    const int N = rbm->N, M = rbm->M;
    carve_tables(c, t, rbm, ham->n_edges, ham->edges, site, edge);
    b.samples = samples_out ? samples_out : c.take<int8_t>((size_t)Ns * N);
    b.eloc = eloc_out ? eloc_out : c.take<double>(Ns);
    b.T = c.take<double>((size_t)Ns * M);
    b.st3 = c.take<double>(4);
    b.acc = c.take<unsigned long long>(C);
    const int64_t TB = Ns > C ? Ns : C;
    b.theta = mixed ? c.take<double>((size_t)TB * M) : nullptr;
    b.tcm = mixed ? c.take<char>(tcm_bytes(N, M, TB)) : nullptr;
}

// NK_MIXED sweeps that leave the theta of every sample behind.  The theta of
// the chains after a sampling sweep is the theta of that sweep's samples, so
// the tensor-core product before each sweep writes it straight into those
// samples' rows of the batch's theta buffer (row stride n_samples M), and one
// more product after the last sweep gives the last samples' theta.  The
// product over the whole batch that the local energies would otherwise need
// is not run.  (Running the local energies of each sweep's samples on a
// second stream beside the next sweep was measured too: the two kernels
// slowed each other down and the step gained nothing beyond this.)
template <typename R>
nk_status run_sweeps_theta(nk_ctx *ctx, const nk::Tables<R> &t, const nk::Tables<R> &ts, const nk::SweepArgs &a,
                           const StepBufs &b, cudaStream_t st) {
    const int N = t.N, M = t.M, C = a.C;
    const int nd = a.n_discard, ns = a.n_samples, total = nd + ns;
    for (int w = 0; w <= total; ++w) {
        // the chains now hold sample q = w - 1 - nd (q < 0: still discarding;
        // sample 0's rows serve as scratch until its own theta arrives)
        const int q = w - 1 - nd;
        double *th = b.theta + (size_t)(q > 0 ? q : 0) * M;
        NK_CU(nk::launch_theta_tc(N, M, t.b, t.W, a.s, C, th, ctx->tc_err, b.tcm, st, (int64_t)ns * M), "theta");
        if (w == total) break;
        nk::SweepArgs sa = a;
        sa.sweep0 = a.sweep0 + w;
        sa.n_discard = w < nd ? 1 : 0;
        sa.n_samples = w < nd ? 0 : 1;
        sa.theta_in = th;
        sa.theta_ld = (int64_t)ns * M;
        sa.out_stride = ns;
        sa.out_offset = w < nd ? 0 : w - nd;
        sa.dec_stride = total;
        sa.dec_offset = w;
        NK_CU(nk::launch_sweep(ts, sa, st), "sweep");
    }
    return NK_OK;
}

template <typename R>
nk_status run_sample_measure(nk_ctx *ctx, const nk::Tables<R> &t, const StepBufs &b, const nk_ham *ham,
                             const nk_chains *chains, const nk_sr_cfg *cfg, int rule, int E_rule, bool site,
                             bool edge, bool mixed, cudaStream_t st) {
    const int N = t.N, M = t.M, C = chains->C;
    const int64_t Ns = (int64_t)C * cfg->n_samples;
    NK_CU(nk::launch_tables(t, site, edge, st), "tables");
    NK_CU(cudaMemsetAsync(b.acc, 0, sizeof(unsigned long long) * C, st), "memset");
    nk::SweepArgs a{};
    a.N = N;
    a.M = M;
    a.E = E_rule;
    a.C = C;
    a.rule = rule;
    a.edges = ham->edges;
    a.s = chains->s;
    a.sweep0 = chains->sweeps_done;
    a.n_discard = cfg->n_discard;
    a.n_samples = cfg->n_samples;
    a.seed = cfg->seed;
    a.stream_id = cfg->stream_id;
    a.samples = b.samples;
    a.logpsi = nullptr;
    a.n_accepted = b.acc;
    a.decisions = nullptr;
    nk::Tables<R> ts = t;  // the rule's edges: a prefix of the Hamiltonian's
    ts.E = E_rule;
    nk_status sw = mixed ? run_sweeps_theta(ctx, t, ts, a, b, st) : run_sweeps(ctx, ts, a, false, nullptr, nullptr, st);
    if (sw != NK_OK) return sw;
    nk::ElocArgs ea = nk::eloc_args(ham, b.samples, Ns, b.eloc, b.T, b.theta);
    NK_CU(nk::launch_eloc(t, ea, st), "local energy");
    NK_CU(nk::launch_stats(b.eloc, Ns, C, b.st3, st), "stats");
    return NK_OK;
}

nk_status check_solver(int solver, double eps, double tol, int maxiter) {
    if (solver != NK_SOLVER_CG && solver != NK_SOLVER_CHOLESKY && solver != NK_SOLVER_CHOLESKY_SAMPLESPACE &&
        solver != NK_SOLVER_SVD && solver != NK_SOLVER_SVD_SAMPLESPACE)
        return fail(NK_ERR_INVALID_ARG, "solver %d unknown", solver);
    if ((solver == NK_SOLVER_SVD || solver == NK_SOLVER_SVD_SAMPLESPACE) && !(tol >= 0.0 && tol < 1.0))
        return fail(NK_ERR_INVALID_ARG, "the SVD cutoff rcond must be in [0, 1)");
    if (!(eps > 0.0) && solver == NK_SOLVER_CHOLESKY_SAMPLESPACE)
        return fail(NK_ERR_INVALID_ARG, "the sample-space solve needs diag_shift > 0");
    if (!(eps >= 0.0)) return fail(NK_ERR_INVALID_ARG, "diag_shift must be >= 0");
    if (solver == NK_SOLVER_CG && (maxiter < 1 || !(tol > 0.0)))
        return fail(NK_ERR_INVALID_ARG, "CG needs cg_maxiter >= 1 and cg_tol > 0");
    return NK_OK;
}

// The SVD solvers hold two n x n FP64 matrices (n = Np or Ns).
nk_status check_svd_size(int solver, int N, int M, int64_t Ns) {
    const int64_t n = solver == NK_SOLVER_SVD ? n_params(N, M) : Ns;
    if ((solver == NK_SOLVER_SVD || solver == NK_SOLVER_SVD_SAMPLESPACE) && n > 8192)
        return fail(NK_ERR_INVALID_ARG, "the SVD solvers need %s <= 8192 (got %lld)",
                    solver == NK_SOLVER_SVD ? "Np" : "Ns", (long long)n);
    return NK_OK;
}

}  // namespace

namespace nk {
// Lets other translation units of the library report through nk_last_error.
nk_status report_error(nk_status code, const char *msg) { return fail(code, "%s", msg); }
void set_plan_only(bool on) { g_plan_only = on; }
}  // namespace nk

// =================================================================== ABI ===

extern "C" {

int32_t nk_version(void) { return 100; }

nk_status nk_ctx_error(nk_ctx *ctx, int32_t *code, void *stream) {
    if (!ctx || !code) return fail(NK_ERR_INVALID_ARG, "ctx or code is NULL");
    DeviceGuard g(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    NK_CU(cudaMemcpyAsync(ctx->host_flags + 4, ctx->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st), "ctx error");
    NK_CU(cudaMemsetAsync(ctx->tc_err, 0, sizeof(int), st), "ctx error");
    NK_CU(cudaStreamSynchronize(st), "ctx error");
    *code = ctx->host_flags[4];
    return NK_OK;
}

const char *nk_last_error(void) { return g_err.c_str(); }

nk_status nk_ctx_create(int32_t device, nk_ctx **out) {
    if (!out) return fail(NK_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(NK_ERR_INVALID_ARG, "device %d of %d", device, n);
    DeviceGuard g(device);
    if (!g.ok) return fail(NK_ERR_CUDA, "cannot select device %d", device);
    nk_ctx *c = new nk_ctx{};
    c->device = device;
    e = cudaMallocHost(&c->host_flags, 8 * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&c->host_vals, 8 * sizeof(double));
    int lo_prio = 0, hi_prio = 0;
    if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi_prio);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&c->aux, cudaStreamNonBlocking, hi_prio);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&c->ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&c->tc_err, 256);
    if (e == cudaSuccess) e = cudaMemset(c->tc_err, 0, 256);
    if (e != cudaSuccess) {
        if (c->host_flags) cudaFreeHost(c->host_flags);
        if (c->host_vals) cudaFreeHost(c->host_vals);
        if (c->side) cudaStreamDestroy(c->side);
        if (c->aux) cudaStreamDestroy(c->aux);
        for (int i = 0; i < 4; ++i)
            if (c->ev[i]) cudaEventDestroy(c->ev[i]);
        if (c->tc_err) cudaFree(c->tc_err);
        delete c;
        return cuda_fail(e, "context resources");
    }
    *out = c;
    return NK_OK;
}

nk_status nk_ctx_destroy(nk_ctx *ctx) {
    if (!ctx) return NK_OK;
    DeviceGuard g(ctx->device);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->host_flags) cudaFreeHost(ctx->host_flags);
    if (ctx->host_vals) cudaFreeHost(ctx->host_vals);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    for (int i = 0; i < 4; ++i)
        if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
    if (ctx->tc_err) cudaFree(ctx->tc_err);
    delete ctx;
    return NK_OK;
}

nk_status nk_rbm_logpsi(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                        int64_t B, double *logpsi_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if (B < 0) return fail(NK_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return NK_OK;
    NK_DEV(s, "s");
    NK_DEV(logpsi_out, "logpsi_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = rbm->N, M = rbm->M;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        nk::Tables<double> t{};
        carve_tables(c, t, rbm, 0, nullptr, false, false);
        const bool mixed = precision == NK_MIXED;
        double *theta = mixed ? c.take<double>((size_t)B * M) : nullptr;
        void *tcm = mixed ? c.take<char>(nk::tc_theta_ws_bytes(N, M, B)) : nullptr;
        if (!run) return NK_OK;
        if (mixed) {
            NK_CU(nk::launch_theta_tc(N, M, t.b, t.W, s, B, theta, ctx->tc_err, tcm, st), "theta");
            NK_CU(nk::launch_logpsi_theta(N, M, t.a, theta, s, B, logpsi_out, st), "logpsi");
            return NK_OK;
        }
        NK_CU(nk::launch_tables(t, false, false, st), "tables");
        NK_CU(nk::launch_logpsi(N, M, t.a, t.b, t.Wt, s, B, logpsi_out, st), "logpsi");
        return NK_OK;
    });
}

nk_status nk_chains_init(nk_ctx *ctx, int32_t N, int32_t C, int32_t rule, uint64_t seed,
                         uint32_t stream_id, int8_t *s_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    if (N < 1 || N > 4096) return fail(NK_ERR_INVALID_ARG, "N=%d out of [1, 4096]", N);
    if (C < 0) return fail(NK_ERR_INVALID_ARG, "C < 0");
    if (rule != NK_RULE_LOCAL && rule != NK_RULE_EXCHANGE && rule != NK_RULE_HAMILTONIAN)
        return fail(NK_ERR_INVALID_ARG, "rule %d unknown", rule);
    if (rule != NK_RULE_LOCAL && (N % 2))
        return fail(NK_ERR_INVALID_ARG, "S_z = 0 initial states need an even N");
    if (C == 0) return NK_OK;
    NK_DEV(s_out, "s_out");
    NK_CU(nk::launch_chain_init(N, C, rule, seed, stream_id, s_out, (cudaStream_t)stream),
          "chain init");
    return NK_OK;
}

nk_status nk_metropolis_sweep(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, int32_t rule,
                              int32_t n_edges, const int32_t *edges, int32_t C, int8_t *s,
                              int64_t sweep0, int32_t n_discard, int32_t n_samples, uint64_t seed,
                              uint32_t stream_id, int8_t *samples_out, double *logpsi_out,
                              uint64_t *n_accepted, uint8_t *decisions_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if (rule != NK_RULE_LOCAL && rule != NK_RULE_EXCHANGE && rule != NK_RULE_HAMILTONIAN)
        return fail(NK_ERR_INVALID_ARG, "rule %d unknown", rule);
    if (C < 0 || n_discard < 0 || n_samples < 0 || sweep0 < 0)
        return fail(NK_ERR_INVALID_ARG, "negative C, n_discard, n_samples or sweep0");
    if (C == 0 || n_discard + n_samples == 0) return NK_OK;
    const bool pair = rule != NK_RULE_LOCAL;  // moves along edges
    if (pair) {
        if (n_edges < 1 || n_edges > 65536)
            return fail(NK_ERR_INVALID_ARG, "exchange and Hamiltonian rules need 1 <= n_edges <= 65536");
        NK_DEV(edges, "edges");
    }
    NK_DEV(s, "s");
    if (n_samples > 0) NK_DEV(samples_out, "samples_out");
    if (logpsi_out) NK_DEV(logpsi_out, "logpsi_out");
    if (n_accepted) NK_DEV(n_accepted, "n_accepted");
    if (decisions_out) NK_DEV(decisions_out, "decisions_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int E = pair ? n_edges : 0;
    nk::SweepArgs a{};
    a.N = rbm->N;
    a.M = rbm->M;
    a.E = E;
    a.C = C;
    a.rule = rule;
    a.edges = edges;
    a.s = s;
    a.sweep0 = sweep0;
    a.n_discard = n_discard;
    a.n_samples = n_samples;
    a.seed = seed;
    a.stream_id = stream_id;
    a.samples = samples_out;
    a.logpsi = logpsi_out;
    a.n_accepted = reinterpret_cast<unsigned long long *>(n_accepted);
    a.decisions = decisions_out;
    auto body = [&](auto tag, Carver &c, bool run) -> nk_status {
        using R = decltype(tag);
        nk::Tables<R> t{};
        carve_tables(c, t, rbm, E, edges, !pair, pair);
        const bool mixed = precision == NK_MIXED;
        double *theta = mixed ? c.take<double>((size_t)C * rbm->M) : nullptr;
        void *tcm = mixed ? c.take<char>(nk::tc_theta_ws_bytes(rbm->N, rbm->M, C)) : nullptr;
        if (!run) return NK_OK;
        NK_CU(nk::launch_tables(t, !pair, pair, st), "tables");
        return run_sweeps(ctx, t, a, mixed, theta, tcm, st);
    };
    if (precision == NK_F64)
        return with_workspace(ctx, [&](Carver &c, bool run) { return body(double{}, c, run); });
    return with_workspace(ctx, [&](Carver &c, bool run) { return body(float{}, c, run); });
}

nk_status nk_local_energy(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const nk_ham *ham,
                          const int8_t *s, int64_t Ns, double *eloc_out, double *t_out,
                          void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if ((st0 = check_ham(ham, rbm->N)) != NK_OK) return st0;
    if (Ns < 0) return fail(NK_ERR_INVALID_ARG, "Ns < 0");
    if (Ns == 0) return NK_OK;
    NK_DEV(s, "s");
    NK_DEV(eloc_out, "eloc_out");
    if (t_out) NK_DEV(t_out, "t_out");
    cudaStream_t st = (cudaStream_t)stream;
    nk::ElocArgs a = nk::eloc_args(ham, s, Ns, eloc_out, t_out);
    const bool site = ham->kind == NK_TFIM, edge = ham->kind == NK_HEIS;
    auto body = [&](auto tag, Carver &c, bool run) -> nk_status {
        using R = decltype(tag);
        nk::Tables<R> t{};
        carve_tables(c, t, rbm, ham->n_edges, ham->edges, site, edge);
        const bool mixed = precision == NK_MIXED;
        double *theta = mixed ? c.take<double>((size_t)Ns * rbm->M) : nullptr;
        void *tcm = mixed ? c.take<char>(nk::tc_theta_ws_bytes(rbm->N, rbm->M, Ns)) : nullptr;
        if (!run) return NK_OK;
        NK_CU(nk::launch_tables(t, site, edge, st), "tables");
        nk::ElocArgs am = a;
        if (mixed) {
            NK_CU(nk::launch_theta_tc(rbm->N, rbm->M, t.b, t.W, s, Ns, theta, ctx->tc_err, tcm, st), "theta");
            am.theta_in = theta;
        }
        NK_CU(nk::launch_eloc(t, am, st), "local energy");
        return NK_OK;
    };
    if (precision == NK_F64)
        return with_workspace(ctx, [&](Carver &c, bool run) { return body(double{}, c, run); });
    return with_workspace(ctx, [&](Carver &c, bool run) { return body(float{}, c, run); });
}

nk_status nk_stats(nk_ctx *ctx, const double *eloc, int64_t Ns, int32_t n_chains, double *out,
                   void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    if (Ns < 1) return fail(NK_ERR_INVALID_ARG, "Ns must be >= 1");
    NK_DEV(eloc, "eloc");
    NK_DEV(out, "out");
    NK_CU(nk::launch_stats(eloc, Ns, n_chains, out, (cudaStream_t)stream), "stats");
    return NK_OK;
}

nk_status nk_jacobian(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                      int64_t Ns, int32_t centered, int64_t row0, int64_t rows, double *O_out,
                      void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if (Ns < 1 || row0 < 0 || rows < 0 || row0 + rows > Ns)
        return fail(NK_ERR_INVALID_ARG, "rows [%lld, %lld) outside [0, %lld)", (long long)row0,
                    (long long)(row0 + rows), (long long)Ns);
    if (rows == 0) return NK_OK;
    NK_DEV(s, "s");
    NK_DEV(O_out, "O_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = rbm->N, M = rbm->M;
    const int64_t Np = n_params(N, M);
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        double *T = c.take<double>((size_t)(centered ? Ns : rows) * M);
        double *mean = centered ? c.take<double>(Np) : nullptr;
        double *ones = centered ? c.take<double>(Ns) : nullptr;
        double *partial = centered ? c.take<double>(nk::vjp_partial_doubles(N, M, Ns)) : nullptr;
        if (!run) return NK_OK;
        const double *b = rbm->params + N, *W = rbm->params + N + M;
        if (centered) {
            NK_CU(nk::launch_theta_tanh(N, M, b, W, s, Ns, T, st), "theta");
            NK_CU(nk::launch_fill(Ns, 1.0, ones, st), "ones");
            NK_CU(nk::launch_vjp(N, M, Ns, s, T, ones, 1.0 / (double)Ns, nullptr, partial, mean, st),
                  "mean");
            NK_CU(nk::launch_jacobian_rows(N, M, s, T, row0, rows, mean, O_out, st), "jacobian");
        } else {
            NK_CU(nk::launch_theta_tanh(N, M, b, W, s + (size_t)row0 * N, rows, T, st), "theta");
            NK_CU(nk::launch_jacobian_rows(N, M, s + (size_t)row0 * N, T, 0, rows, nullptr, O_out, st),
                  "jacobian");
        }
        (void)Np;
        return NK_OK;
    });
}

nk_status nk_vjp(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s, int64_t Ns,
                 const double *gvec, double *out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if (Ns < 1) return fail(NK_ERR_INVALID_ARG, "Ns must be >= 1");
    NK_DEV(s, "s");
    NK_DEV(gvec, "g");
    NK_DEV(out, "out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = rbm->N, M = rbm->M;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        double *T = c.take<double>((size_t)Ns * M);
        SolveWs w{};
        w.partial = c.take<double>(nk::vjp_partial_doubles(N, M, Ns));
        const bool mixed = precision == NK_MIXED;
        w.tcm = mixed ? c.take<char>(tcm_bytes(N, M, Ns)) : nullptr;
        w.tcerr = ctx->tc_err;
        if (!run) return NK_OK;
        nk_status bt = batch_T(ctx, rbm, s, Ns, T, mixed, w.tcm, st);
        if (bt != NK_OK) return bt;
        NK_CU(vjp_any(N, M, Ns, s, T, gvec, 1.0, nullptr, w, out, precision, kMatvecSlices, st), "vjp");
        return NK_OK;
    });
}

nk_status nk_jvp(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s, int64_t Ns,
                 const double *v, double *out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if (Ns < 1) return fail(NK_ERR_INVALID_ARG, "Ns must be >= 1");
    NK_DEV(s, "s");
    NK_DEV(v, "v");
    NK_DEV(out, "out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = rbm->N, M = rbm->M;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        double *T = c.take<double>((size_t)Ns * M);
        SolveWs w{};
        w.U = c.take<double>((size_t)Ns * (M + 1));
        const bool mixed = precision == NK_MIXED;
        w.tcm = mixed ? c.take<char>(tcm_bytes(N, M, Ns)) : nullptr;
        w.tcerr = ctx->tc_err;
        if (!run) return NK_OK;
        nk_status bt = batch_T(ctx, rbm, s, Ns, T, mixed, w.tcm, st);
        if (bt != NK_OK) return bt;
        NK_CU(jvp_any(N, M, Ns, s, T, v, w, out, precision, kMatvecSlices, st), "jvp");
        return NK_OK;
    });
}

nk_status nk_force(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                   int64_t Ns, const double *eloc, double *F_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if (Ns < 1) return fail(NK_ERR_INVALID_ARG, "Ns must be >= 1");
    NK_DEV(s, "s");
    NK_DEV(eloc, "eloc");
    NK_DEV(F_out, "F_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = rbm->N, M = rbm->M;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        double *T = c.take<double>((size_t)Ns * M);
        SolveWs w{};
        w.partial = c.take<double>(nk::vjp_partial_doubles(N, M, Ns));
        double *st3 = c.take<double>(4);
        double *gv = c.take<double>(Ns);
        const bool mixed = precision == NK_MIXED;
        w.tcm = mixed ? c.take<char>(tcm_bytes(N, M, Ns)) : nullptr;
        w.tcerr = ctx->tc_err;
        if (!run) return NK_OK;
        nk_status bt = batch_T(ctx, rbm, s, Ns, T, mixed, w.tcm, st);
        if (bt != NK_OK) return bt;
        NK_CU(nk::launch_stats(eloc, Ns, 1, st3, st), "stats");
        NK_CU(nk::launch_make_force_g(Ns, eloc, st3, gv, st), "force g");
        NK_CU(vjp_any(N, M, Ns, s, T, gv, 1.0, nullptr, w, F_out, precision, kExactSlices, st), "vjp");
        return NK_OK;
    });
}

nk_status nk_qgt_matvec(nk_ctx *ctx, const nk_qgt *q, double diag_shift, const double *v,
                        double *out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    if (!q) return fail(NK_ERR_INVALID_ARG, "qgt is NULL");
    DeviceGuard g(ctx->device);
    if (q->Ns < 1) return fail(NK_ERR_INVALID_ARG, "Ns must be >= 1");
    NK_DEV(v, "v");
    NK_DEV(out, "out");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t Ns = q->Ns;
    if (q->kind == NK_QGT_JACOBIAN) {
        if (q->Np < 1) return fail(NK_ERR_INVALID_ARG, "Np must be >= 1");
        NK_DEV(q->dJ, "qgt->dJ");
        const int64_t Np = q->Np;
        return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
            double *w = c.take<double>(Ns);
            double *partial = c.take<double>(nk::gemv_t_partial_doubles(Ns, Np));
            if (!run) return NK_OK;
            NK_CU(nk::launch_gemv_rows(q->dJ, Ns, Np, v, w, st), "dJ v");
            NK_CU(nk::launch_gemv_t(q->dJ, Ns, Np, w, 1.0 / (double)Ns, partial, out, st), "dJ^T w");
            NK_CU(nk::launch_axpby(Np, diag_shift, v, 1.0, out, st), "shift");
            return NK_OK;
        });
    }
    if (q->kind != NK_QGT_ONTHEFLY) return fail(NK_ERR_INVALID_ARG, "qgt->kind %d unknown", q->kind);
    nk_status st0 = check_rbm(q->rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(q->precision)) != NK_OK) return st0;
    NK_DEV(q->s, "qgt->s");
    const nk_rbm *rbm = q->rbm;
    const int N = rbm->N, M = rbm->M;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        double *T = c.take<double>((size_t)Ns * M);
        SolveWs w{};
        w.partial = c.take<double>(nk::vjp_partial_doubles(N, M, Ns));
        w.dotp = c.take<double>(nk::dot_partial_doubles(Ns) + 8);
        w.U = c.take<double>((size_t)Ns * (M + 1));
        w.w = c.take<double>(Ns);
        const bool mixed = q->precision == NK_MIXED;
        w.tcm = mixed ? c.take<char>(tcm_bytes(N, M, Ns)) : nullptr;
        w.tcerr = ctx->tc_err;
        if (!run) return NK_OK;
        nk_status bt = batch_T(ctx, rbm, q->s, Ns, T, mixed, w.tcm, st);
        if (bt != NK_OK) return bt;
        NK_CU(qgt_onthefly(N, M, Ns, q->s, T, v, diag_shift, w, out, st, q->precision), "qgt matvec");
        return NK_OK;
    });
}

nk_status nk_tc_gemm(nk_ctx *ctx, int64_t rows, int64_t cols, int32_t k, const double *A, int64_t lda,
                     const double *B, int64_t ldb, int32_t slices, int32_t mode, int32_t lower,
                     double *C, int64_t ldc, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    if (rows < 0 || cols < 0 || k < 1 || k > 64 || slices < 1 || slices > 7 || mode < 0 || mode > 2)
        return fail(NK_ERR_INVALID_ARG, "need rows, cols >= 0, 1 <= k <= 64, 1 <= slices <= 7, 0 <= mode <= 2");
    if (lda < k || ldb < k || ldc < cols) return fail(NK_ERR_INVALID_ARG, "leading dimension too small");
    if (rows == 0 || cols == 0) return NK_OK;
    NK_DEV(A, "A");
    NK_DEV(B, "B");
    NK_DEV(C, "C");
    cudaStream_t st = (cudaStream_t)stream;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        __nv_bfloat16 *as = c.take<__nv_bfloat16>(nk::slice_elems(rows, slices));
        __nv_bfloat16 *bs = c.take<__nv_bfloat16>(nk::slice_elems(cols, slices));
        int *ea = c.take<int>(rows), *eb = c.take<int>(cols), *err = c.take<int>(2);
        if (!run) return NK_OK;
        NK_CU(cudaMemsetAsync(err, 0, 2 * sizeof(int), st), "tc gemm");
        NK_CU(nk::launch_slice_rows(A, lda, rows, k, slices, as, ea, st), "slice A");
        NK_CU(nk::launch_slice_rows(B, ldb, cols, k, slices, bs, eb, st), "slice B");
        NK_CU(nk::launch_ozaki_gemm(as, ea, rows, bs, eb, cols, slices, C, ldc, mode, lower != 0, err + 1, st),
              "tc gemm");
        return check_factor(ctx, err, st);
    });
}

nk_status nk_sr_solve(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                      int64_t Ns, const double *F, int32_t solver, double diag_shift,
                      double cg_tol, int32_t cg_maxiter, double *delta_out, int32_t *info_out,
                      double *resid_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if ((st0 = check_solver(solver, diag_shift, cg_tol, cg_maxiter)) != NK_OK) return st0;
    if (Ns < 1) return fail(NK_ERR_INVALID_ARG, "Ns must be >= 1");
    if ((st0 = check_svd_size(solver, rbm->N, rbm->M, Ns)) != NK_OK) return st0;
    NK_DEV(s, "s");
    NK_DEV(F, "F");
    NK_DEV(delta_out, "delta_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = rbm->N, M = rbm->M;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        double *T = c.take<double>((size_t)Ns * M);
        SolveWs w;
        carve_solve(c, w, N, M, Ns, solver, precision);
        w.tcerr = ctx->tc_err;
        if (!run) return NK_OK;
        nk_status bt = batch_T(ctx, rbm, s, Ns, T, precision == NK_MIXED, w.tcm, st);
        if (bt != NK_OK) return bt;
        return run_solve(ctx, N, M, Ns, s, T, F, solver, diag_shift, cg_tol, cg_maxiter, w,
                         delta_out, info_out, resid_out, st, precision, precision == NK_MIXED);
    });
}

nk_status nk_sr_step(nk_ctx *ctx, nk_rbm *rbm, const nk_ham *ham, nk_chains *chains,
                     const nk_sr_cfg *cfg, nk_sr_stats *stats_out, int8_t *samples_out,
                     double *eloc_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_rbm(rbm);
    if (st0 != NK_OK) return st0;
    if (!cfg || !chains) return fail(NK_ERR_INVALID_ARG, "cfg or chains is NULL");
    if ((st0 = check_precision(cfg->precision)) != NK_OK) return st0;
    if ((st0 = check_ham(ham, rbm->N)) != NK_OK) return st0;
    const bool svd_solver = cfg->solver == NK_SOLVER_SVD || cfg->solver == NK_SOLVER_SVD_SAMPLESPACE;
    if ((st0 = check_solver(cfg->solver, cfg->diag_shift, svd_solver ? cfg->svd_rcond : cfg->cg_tol,
                            cfg->cg_maxiter)) != NK_OK)
        return st0;
    if (cfg->rule != NK_RULE_LOCAL && cfg->rule != NK_RULE_EXCHANGE && cfg->rule != NK_RULE_HAMILTONIAN)
        return fail(NK_ERR_INVALID_ARG, "rule %d unknown", cfg->rule);
    if (chains->C < 1 || cfg->n_samples < 1 || cfg->n_discard < 0 || chains->sweeps_done < 0)
        return fail(NK_ERR_INVALID_ARG, "need C >= 1, n_samples >= 1, n_discard >= 0");
    if ((st0 = check_svd_size(cfg->solver, rbm->N, rbm->M, (int64_t)chains->C * cfg->n_samples)) != NK_OK)
        return st0;
    NK_DEV(chains->s, "chains->s");
    if (chains->n_accepted) NK_DEV(chains->n_accepted, "chains->n_accepted");
    if (stats_out) NK_DEV(stats_out, "stats_out");
    if (samples_out) NK_DEV(samples_out, "samples_out");
    if (eloc_out) NK_DEV(eloc_out, "eloc_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = rbm->N, M = rbm->M, C = chains->C, E = ham->n_edges;
    const int64_t Ns = (int64_t)C * cfg->n_samples, Np = n_params(N, M);
    // The Hamiltonian rule of the Ising model draws one of the N single flips
    // uniformly: the local rule.  For NK_HEIS it moves along the edges with a
    // nonzero coupling (the next-nearest class drops out when J2 = 0).
    const int rule = nk::effective_rule(cfg->rule, ham->kind);
    const int E_rule = rule == NK_RULE_HAMILTONIAN && ham->J2 == 0.0 ? E - ham->n_edges2 : E;
    const bool site = rule == NK_RULE_LOCAL || ham->kind == NK_TFIM;
    const bool edge = rule != NK_RULE_LOCAL || ham->kind == NK_HEIS;

    auto body = [&](auto tag, Carver &c, bool run) -> nk_status {
        using R = decltype(tag);
        const bool mixed = cfg->precision == NK_MIXED;
        nk::Tables<R> t{};
        StepBufs sb{};
        carve_step(c, t, sb, rbm, ham, C, Ns, site, edge, mixed, samples_out, eloc_out);
        double *gv = c.take<double>(Ns);
        double *F = c.take<double>(Np);
        double *delta = c.take<double>(Np);
        double *nrm = c.take<double>(2);
        SolveWs w;
        carve_solve(c, w, N, M, Ns, cfg->solver, cfg->precision);
        w.tcerr = ctx->tc_err;
        if (!run) return NK_OK;
        nk_status sm = run_sample_measure(ctx, t, sb, ham, chains, cfg, rule, E_rule, site, edge, mixed, st);
        if (sm != NK_OK) return sm;
        int8_t *samples = sb.samples;
        double *eloc = sb.eloc, *T = sb.T, *st3 = sb.st3;
        unsigned long long *acc = sb.acc;
        NK_CU(nk::launch_make_force_g(Ns, eloc, st3, gv, st), "force g");
        NK_CU(vjp_any(N, M, Ns, samples, T, gv, 1.0, nullptr, w, F, cfg->precision, kExactSlices, st), "force");
        int info[2] = {0, 0};
        double resid = 0.0;
        const bool svd = cfg->solver == NK_SOLVER_SVD || cfg->solver == NK_SOLVER_SVD_SAMPLESPACE;
        nk_status ss = run_solve(ctx, N, M, Ns, samples, T, F, cfg->solver, cfg->diag_shift,
                                 svd ? cfg->svd_rcond : cfg->cg_tol, cfg->cg_maxiter, w, delta, info, &resid, st,
                                 cfg->precision, false);
        if (ss != NK_OK && ss != NK_ERR_NOT_CONVERGED) return ss;
        NK_CU(nk::launch_dot(Np, F, F, w.dotp, nrm, st), "norm");
        NK_CU(nk::launch_dot(Np, delta, delta, w.dotp, nrm + 1, st), "norm");
        NK_CU(nk::launch_sgd(Np, cfg->lr, delta, rbm->params, st), "update");
        if (stats_out) {
            const double nprop = (double)C * (cfg->n_discard + cfg->n_samples) * N;
            const bool cg = cfg->solver == NK_SOLVER_CG;
            NK_CU(nk::launch_write_sr_stats(st3, acc, C, nprop, cg ? w.sc + 3 : nrm, nrm + 1,
                                            cg ? w.flags + 1 : nullptr, cg ? w.sc + 4 : nullptr,
                                            cg ? nullptr : w.info, stats_out, st),
                  "stats out");
        }
        if (chains->n_accepted) {
            (k_add_u64<<<(C + 255) / 256, 256, 0, st>>>(
                C, acc, reinterpret_cast<unsigned long long *>(chains->n_accepted)), nk::note_launch());
            NK_CU(cudaGetLastError(), "acc");
        }
        chains->sweeps_done += cfg->n_discard + cfg->n_samples;
        return ss;
    };
    if (cfg->precision == NK_F64)
        return with_workspace(ctx, [&](Carver &c, bool run) { return body(double{}, c, run); });
    return with_workspace(ctx, [&](Carver &c, bool run) { return body(float{}, c, run); });
}

}  // extern "C"

// ------------------------------------------------------ symmetric RBM ---

namespace {

nk_status check_symm(const nk_rbm_symm *m) {
    if (!m) return fail(NK_ERR_INVALID_ARG, "symmetric RBM is NULL");
    if (m->N < 1 || m->N > 4096) return fail(NK_ERR_INVALID_ARG, "N=%d out of [1, 4096]", m->N);
    if (m->alpha < 1 || m->n_group < 1 || (int64_t)m->alpha * m->n_group > 8192)
        return fail(NK_ERR_INVALID_ARG, "alpha=%d, n_group=%d: need alpha >= 1, n_group >= 1, alpha n_group <= 8192",
                    m->alpha, m->n_group);
    NK_DEV(m->perms, "symm->perms");
    NK_DEV(m->params, "symm->params");
    return NK_OK;
}

inline int64_t symm_params(const nk_rbm_symm *m) { return 1 + m->alpha + (int64_t)m->alpha * m->N; }

// int offset, in the context's 256-byte device status block (tc_err), of the
// flag of the permutation check
constexpr int kPermsFlag = 16;

// Checks that every row of perms is a permutation of [0, N) (reads one flag
// back: synchronises the stream), then writes the expanded plain-RBM
// parameters.
nk_status symm_expand_checked(nk_ctx *ctx, const nk_rbm_symm *m, double *plain, cudaStream_t st) {
    int *flag = ctx->tc_err + kPermsFlag;
    NK_CU(cudaMemsetAsync(flag, 0, sizeof(int), st), "perms");
    NK_CU(nk::launch_symm_check_perms(m->N, m->n_group, m->perms, flag, st), "perms");
    NK_CU(cudaMemcpyAsync(ctx->host_flags + 5, flag, sizeof(int), cudaMemcpyDeviceToHost, st), "perms");
    NK_CU(cudaStreamSynchronize(st), "perms");
    if (ctx->host_flags[5])
        return fail(NK_ERR_INVALID_ARG, "symm->perms: a row is not a permutation of [0, %d)", m->N);
    NK_CU(nk::launch_symm_expand(m->N, m->alpha, m->n_group, m->perms, m->params, plain, st), "expand");
    return NK_OK;
}

}  // namespace

extern "C" {

nk_status nk_symm_expand(nk_ctx *ctx, const nk_rbm_symm *symm, double *plain_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_symm(symm);
    if (st0 != NK_OK) return st0;
    NK_DEV(plain_out, "plain_out");
    if (g_plan_only) return NK_OK;
    return symm_expand_checked(ctx, symm, plain_out, (cudaStream_t)stream);
}

nk_status nk_symm_jacobian(nk_ctx *ctx, const nk_rbm_symm *symm, int32_t precision, const int8_t *s, int64_t Ns,
                           double *O_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_symm(symm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_precision(precision)) != NK_OK) return st0;
    if (Ns < 0) return fail(NK_ERR_INVALID_ARG, "Ns < 0");
    if (Ns == 0) return NK_OK;
    NK_DEV(s, "s");
    NK_DEV(O_out, "O_out");
    if (nk::symm_jacobian_smem(symm->N, symm->alpha, symm->n_group) > 227 * 1024)
        return fail(NK_ERR_INVALID_ARG, "alpha n_group too large for one sample's activations in shared memory");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = symm->N, M = symm->alpha * symm->n_group;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        double *plain = c.take<double>((size_t)n_params(N, M));
        double *T = c.take<double>((size_t)Ns * M);
        const bool mixed = precision == NK_MIXED;
        void *tcm = mixed ? c.take<char>(nk::tc_theta_ws_bytes(N, M, Ns)) : nullptr;
        if (!run) return NK_OK;
        nk_status e = symm_expand_checked(ctx, symm, plain, st);
        if (e != NK_OK) return e;
        nk_rbm r{N, M, plain};
        if ((e = batch_T(ctx, &r, s, Ns, T, mixed, tcm, st)) != NK_OK) return e;
        NK_CU(nk::launch_symm_jacobian(N, symm->alpha, symm->n_group, symm->perms, s, T, Ns, O_out, st),
              "symmetric jacobian");
        return NK_OK;
    });
}

nk_status nk_symm_sr_step(nk_ctx *ctx, nk_rbm_symm *symm, const nk_ham *ham, nk_chains *chains,
                          const nk_sr_cfg *cfg, nk_sr_stats *stats_out, int8_t *samples_out, double *eloc_out,
                          void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_symm(symm);
    if (st0 != NK_OK) return st0;
    if (!cfg || !chains) return fail(NK_ERR_INVALID_ARG, "cfg or chains is NULL");
    if ((st0 = check_precision(cfg->precision)) != NK_OK) return st0;
    if ((st0 = check_ham(ham, symm->N)) != NK_OK) return st0;
    if (cfg->solver != NK_SOLVER_CHOLESKY)
        return fail(NK_ERR_UNIMPLEMENTED,
                    "the symmetric RBM solves its 1 + alpha + alpha N parameters by the dense Cholesky only");
    if ((st0 = check_solver(cfg->solver, cfg->diag_shift, cfg->cg_tol, cfg->cg_maxiter)) != NK_OK) return st0;
    if (cfg->rule != NK_RULE_LOCAL && cfg->rule != NK_RULE_EXCHANGE && cfg->rule != NK_RULE_HAMILTONIAN)
        return fail(NK_ERR_INVALID_ARG, "rule %d unknown", cfg->rule);
    if (chains->C < 1 || cfg->n_samples < 1 || cfg->n_discard < 0 || chains->sweeps_done < 0)
        return fail(NK_ERR_INVALID_ARG, "need C >= 1, n_samples >= 1, n_discard >= 0");
    if (nk::symm_jacobian_smem(symm->N, symm->alpha, symm->n_group) > 227 * 1024)
        return fail(NK_ERR_INVALID_ARG, "alpha n_group too large for one sample's activations in shared memory");
    NK_DEV(chains->s, "chains->s");
    if (chains->n_accepted) NK_DEV(chains->n_accepted, "chains->n_accepted");
    if (stats_out) NK_DEV(stats_out, "stats_out");
    if (samples_out) NK_DEV(samples_out, "samples_out");
    if (eloc_out) NK_DEV(eloc_out, "eloc_out");
    cudaStream_t st = (cudaStream_t)stream;
    const int N = symm->N, alpha = symm->alpha, G = symm->n_group, M = alpha * G, C = chains->C,
              E = ham->n_edges;
    const int64_t Ns = (int64_t)C * cfg->n_samples, Np = symm_params(symm);
    const int rule = nk::effective_rule(cfg->rule, ham->kind);
    const int E_rule = rule == NK_RULE_HAMILTONIAN && ham->J2 == 0.0 ? E - ham->n_edges2 : E;
    const bool site = rule == NK_RULE_LOCAL || ham->kind == NK_TFIM;
    const bool edge = rule != NK_RULE_LOCAL || ham->kind == NK_HEIS;
    const bool mixed = cfg->precision == NK_MIXED;
    const nk::CholStreams cs{ctx->side, ctx->aux, ctx->ev[0], ctx->ev[1], ctx->ev[2], ctx->ev[3]};

    auto body = [&](auto tag, Carver &c, bool run) -> nk_status {
        using R = decltype(tag);
        double *plain = c.take<double>((size_t)n_params(N, M));
        nk_rbm r{N, M, plain};
        nk::Tables<R> t{};
        StepBufs sb{};
        carve_step(c, t, sb, &r, ham, C, Ns, site, edge, mixed, samples_out, eloc_out);
        double *O = c.take<double>((size_t)Ns * Np);
        double *ones = c.take<double>(Ns);
        double *mean = c.take<double>(Np);
        double *partial = c.take<double>(nk::gemv_t_partial_doubles(Ns, Np));
        double *gv = c.take<double>(Ns);
        double *F = c.take<double>(Np);
        double *S = c.take<double>((size_t)Np * Np);
        double *nrm = c.take<double>(2);
        double *dotp = c.take<double>(nk::dot_partial_doubles(Np) + 8);
        int *info = c.take<int>(2);
        void *tc = mixed ? c.take<char>(nk::tc_chol_ws_bytes(Np)) : nullptr;
        if (!run) return NK_OK;
        nk_status e = symm_expand_checked(ctx, symm, plain, st);
        if (e != NK_OK) return e;
        e = run_sample_measure(ctx, t, sb, ham, chains, cfg, rule, E_rule, site, edge, mixed, st);
        if (e != NK_OK) return e;
        // the Jacobian in the symmetric parameters, centred
        NK_CU(nk::launch_symm_jacobian(N, alpha, G, symm->perms, sb.samples, sb.T, Ns, O, st), "jacobian");
        NK_CU(nk::launch_fill(Ns, 1.0, ones, st), "mean");
        NK_CU(nk::launch_gemv_t(O, Ns, Np, ones, 1.0 / (double)Ns, partial, mean, st), "mean");
        NK_CU(nk::launch_sub_colmean(Ns, Np, mean, O, st), "centre");
        // force F = (2/Ns) dJ^T (E_loc - mean E_loc)
        NK_CU(nk::launch_make_force_g(Ns, sb.eloc, sb.st3, gv, st), "force g");
        NK_CU(nk::launch_gemv_t(O, Ns, Np, gv, 1.0, partial, F, st), "force");
        // S + eps I = dJ^T dJ / Ns + eps I, Cholesky, two triangular solves
        NK_CU(cudaMemsetAsync(info, 0, 2 * sizeof(int), st), "chol");
        if (mixed) {
            NK_CU(nk::launch_gram_cols_tc(O, Ns, Np, 1.0 / (double)Ns, cfg->diag_shift, S, info + 1, tc, st), "gram");
            NK_CU(nk::launch_cholesky_tc(S, Np, info, info + 1, tc, st, &cs), "factor");
        } else {
            NK_CU(nk::launch_syrk_t(O, Ns, Np, 1.0 / (double)Ns, cfg->diag_shift, S, st), "syrk");
            NK_CU(nk::launch_cholesky(S, Np, info, st), "factor");
        }
        NK_CU(nk::launch_axpby(Np, 1.0, F, 0.0, mean, st), "solve");  // mean <- F, solved in place
        if (mixed)
            NK_CU(nk::launch_cholesky_solve_tc(S, Np, tc, mean, info + 1, st), "solve");
        else
            NK_CU(nk::launch_cholesky_solve(S, Np, mean, st), "solve");
        NK_CU(nk::launch_dot(Np, F, F, dotp, nrm, st), "norm");
        NK_CU(nk::launch_dot(Np, mean, mean, dotp, nrm + 1, st), "norm");
        NK_CU(nk::launch_sgd(Np, cfg->lr, mean, symm->params, st), "update");
        if (stats_out) {
            const double nprop = (double)C * (cfg->n_discard + cfg->n_samples) * N;
            NK_CU(nk::launch_write_sr_stats(sb.st3, sb.acc, C, nprop, nrm, nrm + 1, nullptr, nullptr, info,
                                            stats_out, st),
                  "stats out");
        }
        if (chains->n_accepted) {
            (k_add_u64<<<(C + 255) / 256, 256, 0, st>>>(
                C, sb.acc, reinterpret_cast<unsigned long long *>(chains->n_accepted)), nk::note_launch());
            NK_CU(cudaGetLastError(), "acc");
        }
        chains->sweeps_done += cfg->n_discard + cfg->n_samples;
        return mixed ? check_factor(ctx, info, st) : NK_OK;
    };
    if (!mixed) return with_workspace(ctx, [&](Carver &c, bool run) { return body(double{}, c, run); });
    return with_workspace(ctx, [&](Carver &c, bool run) { return body(float{}, c, run); });
}

}  // extern "C"

// ------------------------------------------ complex RBM and time evolution ---

namespace {

nk_status check_crbm(const nk_crbm *r) {
    if (!r) return fail(NK_ERR_INVALID_ARG, "complex RBM is NULL");
    if (r->N < 1 || r->N > 4096) return fail(NK_ERR_INVALID_ARG, "N=%d out of [1, 4096]", r->N);
    if (r->M < 1 || r->M > 4096) return fail(NK_ERR_INVALID_ARG, "M=%d out of [1, 4096]", r->M);
    NK_DEV(r->params, "rbm->params");
    if (reinterpret_cast<uintptr_t>(r->params) % 16)
        return fail(NK_ERR_INVALID_ARG, "rbm->params must be 16-byte aligned (complex pairs)");
    if (4 * nk::crbm_smem_per_warp(r->N, r->M) > 227 * 1024)
        return fail(NK_ERR_INVALID_ARG, "N, M too large for the activations of 4 chains in shared memory");
    return NK_OK;
}

nk_status check_complex_out(const double *p, const char *name) {
    NK_DEV(p, name);
    if (reinterpret_cast<uintptr_t>(p) % 16) return fail(NK_ERR_INVALID_ARG, "%s must be 16-byte aligned", name);
    return NK_OK;
}

// One slope of the t-VMC equation of motion at parameters p: sample, local
// energies and their statistics, the realified centred Jacobian R, the force
// R^T g = [Re f; Im f], the real embedding of G + eps I and its solve for
// gamma f.  x: the slope, realified [Re; Im] (2 Np doubles).
struct TdvpWs {
    int8_t *samples;
    double *eloc, *stats4, *O, *mean, *R, *g, *F, *rhs, *S, *V, *ev, *evmax, *z, *gpart, *partial;
    void *eig;
    int *info, *kept;
    unsigned long long *acc;
};

nk_status tdvp_slope(nk_ctx *ctx, int N, int M, const double *p, const nk_ham *ham, nk_chains *chains,
                     const nk_tdvp_cfg *cfg, int n_discard, TdvpWs &w, double *x, cudaStream_t st) {
    const int C = chains->C;
    const int64_t Ns = (int64_t)C * cfg->n_samples, Np = n_params(N, M), n = 2 * Np;
    NK_CU(nk::launch_crbm_sweep(N, M, p, cfg->rule, ham->n_edges, ham->edges, C, chains->s, chains->sweeps_done,
                                n_discard, cfg->n_samples, cfg->seed, cfg->stream_id, w.samples, w.acc, st),
          "sweep");
    chains->sweeps_done += n_discard + cfg->n_samples;
    NK_CU(nk::launch_crbm_eloc(N, M, p, ham, w.samples, Ns, w.eloc, st), "local energy");
    NK_CU(nk::launch_cstats(Ns, w.eloc, w.stats4, st), "stats");
    NK_CU(nk::launch_crbm_jacobian(N, M, p, w.samples, Ns, w.O, st), "jacobian");
    NK_CU(nk::launch_crealify(Ns, Np, w.O, w.mean, w.R, st), "realify");
    NK_CU(nk::launch_cforce_g(Ns, w.eloc, w.stats4, w.g, st), "force g");
    NK_CU(nk::launch_gemv_t(w.R, 2 * Ns, n, w.g, 1.0, w.partial, w.F, st), "force");
    NK_CU(nk::launch_tdvp_rhs(Np, w.F, cfg->real_time, w.rhs, st), "rhs");
    NK_CU(nk::launch_syrk_t(w.R, 2 * Ns, n, 1.0 / (double)Ns, cfg->diag_shift, w.S, st), "qgt");
    if (cfg->solver == NK_SOLVER_CHOLESKY) {
        NK_CU(cudaMemsetAsync(w.info, 0, 2 * sizeof(int), st), "chol");
        NK_CU(nk::launch_cholesky(w.S, n, w.info, st), "chol");
        NK_CU(nk::launch_axpby(n, 1.0, w.rhs, 0.0, x, st), "chol");
        NK_CU(nk::launch_cholesky_solve(w.S, n, x, st), "chol solve");
        return check_factor(ctx, w.info, st);
    }
    int sweeps = 0;
    double rel = 0.0;
    nk_status js = jacobi_eigen(ctx, w.S, w.V, n, w.eig, w.evmax + 2, st, &sweeps, &rel);
    if (js != NK_OK) return js;
    if (rel > kJacobiTol)
        return fail(NK_ERR_NOT_CONVERGED, "Jacobi sweeps left a relative off-diagonal norm %g", rel);
    NK_CU(nk::launch_eig_diag(n, w.S, w.ev, w.evmax, st), "eigenvalues");
    NK_CU(nk::launch_gemv_t(w.V, n, n, w.rhs, 1.0, w.gpart, w.z, st), "V^T rhs");
    NK_CU(nk::launch_spectral_filter(n, w.ev, w.evmax, cfg->rcond > 0.0 ? cfg->rcond : 1e-12, 1, w.z, w.kept, st),
          "filter");
    NK_CU(nk::launch_gemv_rows(w.V, n, n, w.z, x, st), "V z");
    return NK_OK;
}

}  // namespace

extern "C" {

nk_status nk_crbm_logpsi(nk_ctx *ctx, const nk_crbm *rbm, const int8_t *s, int64_t B, double *out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_crbm(rbm);
    if (st0 != NK_OK) return st0;
    if (B < 0) return fail(NK_ERR_INVALID_ARG, "B < 0");
    if (B == 0) return NK_OK;
    NK_DEV(s, "s");
    if ((st0 = check_complex_out(out, "out")) != NK_OK) return st0;
    if (g_plan_only) return NK_OK;
    NK_CU(nk::launch_crbm_logpsi(rbm->N, rbm->M, rbm->params, s, B, out, (cudaStream_t)stream), "logpsi");
    return NK_OK;
}

nk_status nk_crbm_metropolis(nk_ctx *ctx, const nk_crbm *rbm, int32_t rule, int32_t n_edges, const int32_t *edges,
                             int32_t C, int8_t *s, int64_t sweep0, int32_t n_discard, int32_t n_samples,
                             uint64_t seed, uint32_t stream_id, int8_t *samples_out, uint64_t *n_accepted,
                             void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_crbm(rbm);
    if (st0 != NK_OK) return st0;
    if (rule != NK_RULE_LOCAL && rule != NK_RULE_EXCHANGE)
        return fail(NK_ERR_INVALID_ARG, "rule %d: the complex RBM samples with the local or exchange rule", rule);
    if (C < 0 || n_discard < 0 || n_samples < 1 || sweep0 < 0)
        return fail(NK_ERR_INVALID_ARG, "need C >= 0, n_discard >= 0, n_samples >= 1, sweep0 >= 0");
    if (rule == NK_RULE_EXCHANGE) {
        if (n_edges < 1 || n_edges > 65536) return fail(NK_ERR_INVALID_ARG, "n_edges out of [1, 65536]");
        NK_DEV(edges, "edges");
    }
    if (C == 0) return NK_OK;
    NK_DEV(s, "s");
    NK_DEV(samples_out, "samples_out");
    if (n_accepted) NK_DEV(n_accepted, "n_accepted");
    if (g_plan_only) return NK_OK;
    NK_CU(nk::launch_crbm_sweep(rbm->N, rbm->M, rbm->params, rule, n_edges, edges, C, s, sweep0, n_discard,
                                n_samples, seed, stream_id, samples_out,
                                reinterpret_cast<unsigned long long *>(n_accepted), (cudaStream_t)stream),
          "sweep");
    return NK_OK;
}

nk_status nk_crbm_local_energy(nk_ctx *ctx, const nk_crbm *rbm, const nk_ham *ham, const int8_t *s, int64_t Ns,
                               double *eloc_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_crbm(rbm);
    if (st0 != NK_OK) return st0;
    if ((st0 = check_ham(ham, rbm->N)) != NK_OK) return st0;
    if (Ns < 0) return fail(NK_ERR_INVALID_ARG, "Ns < 0");
    if (Ns == 0) return NK_OK;
    NK_DEV(s, "s");
    if ((st0 = check_complex_out(eloc_out, "eloc_out")) != NK_OK) return st0;
    if (g_plan_only) return NK_OK;
    NK_CU(nk::launch_crbm_eloc(rbm->N, rbm->M, rbm->params, ham, s, Ns, eloc_out, (cudaStream_t)stream),
          "local energy");
    return NK_OK;
}

nk_status nk_crbm_jacobian(nk_ctx *ctx, const nk_crbm *rbm, const int8_t *s, int64_t Ns, double *O_out,
                           void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_crbm(rbm);
    if (st0 != NK_OK) return st0;
    if (Ns < 0) return fail(NK_ERR_INVALID_ARG, "Ns < 0");
    if (Ns == 0) return NK_OK;
    NK_DEV(s, "s");
    if ((st0 = check_complex_out(O_out, "O_out")) != NK_OK) return st0;
    if (g_plan_only) return NK_OK;
    NK_CU(nk::launch_crbm_jacobian(rbm->N, rbm->M, rbm->params, s, Ns, O_out, (cudaStream_t)stream), "jacobian");
    return NK_OK;
}

nk_status nk_tdvp_step(nk_ctx *ctx, nk_crbm *rbm, const nk_ham *ham, nk_chains *chains, const nk_tdvp_cfg *cfg,
                       nk_tdvp_stats *stats_out, double *theta_dot_out, void *stream) {
    if (!ctx) return fail(NK_ERR_INVALID_ARG, "ctx is NULL");
    DeviceGuard g(ctx->device);
    nk_status st0 = check_crbm(rbm);
    if (st0 != NK_OK) return st0;
    if (!cfg || !chains) return fail(NK_ERR_INVALID_ARG, "cfg or chains is NULL");
    if ((st0 = check_ham(ham, rbm->N)) != NK_OK) return st0;
    if (cfg->rule != NK_RULE_LOCAL && cfg->rule != NK_RULE_EXCHANGE)
        return fail(NK_ERR_INVALID_ARG, "rule %d: the local or exchange rule", cfg->rule);
    if (cfg->integrator != NK_TDVP_EULER && cfg->integrator != NK_TDVP_HEUN)
        return fail(NK_ERR_INVALID_ARG, "integrator %d unknown", cfg->integrator);
    if (cfg->solver != NK_SOLVER_CHOLESKY && cfg->solver != NK_SOLVER_SVD)
        return fail(NK_ERR_INVALID_ARG, "solver %d: NK_SOLVER_CHOLESKY or NK_SOLVER_SVD", cfg->solver);
    if (cfg->solver == NK_SOLVER_CHOLESKY && !(cfg->diag_shift > 0.0))
        return fail(NK_ERR_INVALID_ARG, "the Cholesky solve needs diag_shift > 0");
    if (!(cfg->diag_shift >= 0.0) || !(cfg->rcond >= 0.0 && cfg->rcond < 1.0) || !std::isfinite(cfg->dt))
        return fail(NK_ERR_INVALID_ARG, "need diag_shift >= 0, 0 <= rcond < 1 and a finite dt");
    if (chains->C < 1 || cfg->n_samples < 1 || cfg->n_discard < 0 || chains->sweeps_done < 0)
        return fail(NK_ERR_INVALID_ARG, "need C >= 1, n_samples >= 1, n_discard >= 0");
    const int N = rbm->N, M = rbm->M, C = chains->C;
    const int64_t Ns = (int64_t)C * cfg->n_samples, Np = n_params(N, M), n = 2 * Np;
    if (cfg->solver == NK_SOLVER_SVD && n > 8192)
        return fail(NK_ERR_INVALID_ARG, "the SVD solve needs 2 Np <= 8192 (got %lld)", (long long)n);
    if (cfg->rule == NK_RULE_EXCHANGE && ham->n_edges < 1) return fail(NK_ERR_INVALID_ARG, "no edges");
    NK_DEV(chains->s, "chains->s");
    if (chains->n_accepted) NK_DEV(chains->n_accepted, "chains->n_accepted");
    if (stats_out) NK_DEV(stats_out, "stats_out");
    if (theta_dot_out && (st0 = check_complex_out(theta_dot_out, "theta_dot_out")) != NK_OK) return st0;
    cudaStream_t st = (cudaStream_t)stream;
    const bool svd = cfg->solver == NK_SOLVER_SVD;
    return with_workspace(ctx, [&](Carver &c, bool run) -> nk_status {
        TdvpWs w{};
        w.samples = c.take<int8_t>((size_t)Ns * N);
        w.eloc = c.take<double>(2 * Ns);
        w.stats4 = c.take<double>(4);
        w.O = c.take<double>((size_t)2 * Ns * Np);
        w.mean = c.take<double>(2 * Np);
        w.R = c.take<double>((size_t)4 * Ns * Np);
        w.g = c.take<double>(2 * Ns);
        w.F = c.take<double>(n);
        w.rhs = c.take<double>(n);
        w.S = c.take<double>((size_t)n * n);
        w.partial = c.take<double>(nk::gemv_t_partial_doubles(2 * Ns, n));
        w.info = c.take<int>(2);
        w.acc = c.take<unsigned long long>(C);
        if (svd) {
            w.V = c.take<double>((size_t)n * n);
            w.ev = c.take<double>(n);
            w.evmax = c.take<double>(4);
            w.z = c.take<double>(n);
            w.gpart = c.take<double>(nk::gemv_t_partial_doubles(n, n));
            w.eig = c.take<char>(nk::eig_ws_bytes(n));
            w.kept = c.take<int>(4);
        }
        double *k1 = c.take<double>(n);
        double *k2 = c.take<double>(n);
        double *ptmp = c.take<double>(2 * Np);
        if (!run) return NK_OK;
        NK_CU(cudaMemsetAsync(w.acc, 0, sizeof(unsigned long long) * C, st), "acc");
        nk_status e = tdvp_slope(ctx, N, M, rbm->params, ham, chains, cfg, cfg->n_discard, w, k1, st);
        if (e != NK_OK) return e;
        if (stats_out)
            NK_CU(cudaMemcpyAsync(stats_out, w.stats4, 4 * sizeof(double), cudaMemcpyDeviceToDevice, st), "stats");
        if (theta_dot_out) NK_CU(nk::launch_caxpy_realified(Np, nullptr, 1.0, k1, theta_dot_out, st), "theta dot");
        if (cfg->integrator == NK_TDVP_EULER) {
            NK_CU(nk::launch_caxpy_realified(Np, rbm->params, cfg->dt, k1, rbm->params, st), "euler");
        } else {
            NK_CU(nk::launch_caxpy_realified(Np, rbm->params, cfg->dt, k1, ptmp, st), "heun");
            e = tdvp_slope(ctx, N, M, ptmp, ham, chains, cfg, 0, w, k2, st);
            if (e != NK_OK) return e;
            NK_CU(nk::launch_caxpy_realified(Np, rbm->params, 0.5 * cfg->dt, k1, rbm->params, st), "heun");
            NK_CU(nk::launch_caxpy_realified(Np, rbm->params, 0.5 * cfg->dt, k2, rbm->params, st), "heun");
        }
        if (chains->n_accepted) {
            (k_add_u64<<<(C + 255) / 256, 256, 0, st>>>(
                C, w.acc, reinterpret_cast<unsigned long long *>(chains->n_accepted)), nk::note_launch());
            NK_CU(cudaGetLastError(), "acc");
        }
        return NK_OK;
    });
}

}  // extern "C"
