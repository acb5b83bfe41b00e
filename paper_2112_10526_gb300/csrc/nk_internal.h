// Internal launch interface between the C ABI (nk_api.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/nk.h"

// The context behind the opaque nk_ctx handle.
struct nk_ctx {
    int device;
    char *ws;
    size_t ws_size;
    int *host_flags;    // pinned: [0] done, [1] iterations, [2..3] factor status, [4] tc error,
                        // [5] permutation check
    double *host_vals;  // pinned
    cudaStream_t side;  // high-priority stream for the Cholesky look-ahead
    cudaStream_t aux;   // high-priority stream for work beside the panel chain
    cudaEvent_t ev[4];
    int *tc_err;        // device, 256 bytes: [0] sticky code of the first tensor-core
                        // time-out; [16] flag of the symmetric RBM's permutation check
    size_t plan_bytes;  // workspace counted by plan-only calls
};

namespace nk {

// Plan-only mode for the calling thread (see nk_api.cu).
void set_plan_only(bool on);

// Kernel timing hooks (prof.cu).  prof_begin returns a slot (or -1 when
// timing is off); prof_end closes it and adds `work` (the method's
// algorithmic work: ratio terms, or the flops of the FP64 operation) and
// `executed` (what the hardware ran, e.g. BF16 slice-product flops; < 0:
// equal to work) to the class.
int prof_begin(int cls, cudaStream_t st);
// Sets the message returned by nk_last_error on this thread; returns code.
nk_status report_error(nk_status code, const char *msg);
// Process-wide count of kernel launches issued by the library.
void note_launch(long long n = 1);
// Raises the dynamic shared-memory limit of a kernel to the device's opt-in
// maximum, once per (kernel, device).  The limit is process-wide state, so a
// per-launch value would race between host threads launching the same kernel
// with different sizes; a constant maximum does not (occupancy follows the
// size given at launch, not this limit).
cudaError_t allow_max_dynamic_smem(const void *func);
void prof_end(int slot, cudaStream_t st, double work, double executed = -1.0);

// Per-parameter tables of the flip-ratio identity (see k_rbm.cu).  All
// pointers are device workspace.  R = double (NK_F64) or float (NK_MIXED).
template <typename R>
struct Tables {
    int N, M, E;
    const double *a, *b, *W;  // views of the parameter vector
    double *Wt;               // [N][M] transposed W (FP64, coalesced theta rebuild)
    R *tau_site;              // [N][M]  tanh(2 W_ji)
    R *tau_siteT;             // [M][N]
    R *K_site;                // [N]     sum_j ln cosh(2 W_ji)
    const int32_t *edges;     // [E][2]
    R *tau_edge;              // [E][M]  tanh(2 (W_ji - W_jk))
    R *tau_edgeT;             // [M][E]
    R *K_edge;                // [E]
};

template <typename R>
cudaError_t launch_tables(const Tables<R> &t, bool need_site, bool need_edge, cudaStream_t st);

cudaError_t launch_logpsi(int N, int M, const double *a, const double *b, const double *Wt,
                          const int8_t *s, int64_t B, double *out, cudaStream_t st);

cudaError_t launch_logpsi_theta(int N, int M, const double *a, const double *theta, const int8_t *s, int64_t B,
                                double *out, cudaStream_t st);
cudaError_t launch_tanh_inplace(int64_t n, double *x, cudaStream_t st);

cudaError_t launch_chain_init(int N, int C, int rule, uint64_t seed, uint32_t stream_id,
                              int8_t *s, cudaStream_t st);

struct SweepArgs {
    int N, M, E, C, rule;
    const int32_t *edges;
    int8_t *s;
    int64_t sweep0;
    int n_discard, n_samples;
    uint64_t seed;
    uint32_t stream_id;
    int8_t *samples;
    double *logpsi;
    unsigned long long *n_accepted;
    uint8_t *decisions;
    // Optional, for one-sweep launches: theta of every chain at the start of
    // the sweep ([C][M], FP64) instead of the in-kernel rebuild; the output
    // rows are c * out_stride + out_offset + sample, the decision rows
    // c * dec_stride + dec_offset + sweep.
    const double *theta_in;
    int out_stride, out_offset, dec_stride, dec_offset;
    int64_t theta_ld;  // row stride of theta_in in doubles (0: M)
};

template <typename R>
cudaError_t launch_sweep(const Tables<R> &t, const SweepArgs &a, cudaStream_t st);

struct ElocArgs {
    int kind;
    double J, h;
    int marshall;
    const int8_t *s;
    int64_t Ns;
    double *eloc;
    double *t_out;            // [Ns][M] or null
    const double *theta_in;   // [Ns][M] precomputed theta, or null (rebuilt in the kernel)
    double J2;                // coupling of the last E2 edges (next-nearest neighbours)
    int E2;
};

// The rule NK_RULE_HAMILTONIAN becomes for a Hamiltonian kind: the Ising
// model's connected configurations are the N single flips, drawn uniformly,
// which is the local rule.
inline int effective_rule(int rule, int ham_kind) {
    return rule == NK_RULE_HAMILTONIAN && ham_kind == NK_TFIM ? NK_RULE_LOCAL : rule;
}

// Local-energy arguments of a Hamiltonian descriptor.
inline ElocArgs eloc_args(const nk_ham *h, const int8_t *s, int64_t Ns, double *eloc, double *t_out,
                          const double *theta_in = nullptr) {
    ElocArgs a{h->kind, h->J, h->h, h->marshall, s, Ns, eloc, t_out, theta_in};
    a.J2 = h->J2;
    a.E2 = h->n_edges2;
    return a;
}

template <typename R>
cudaError_t launch_eloc(const Tables<R> &t, const ElocArgs &a, cudaStream_t st);

// T[k][j] = tanh(b_j + sum_i W_ji s_ki) for a batch (FP64 tiled GEMM).
cudaError_t launch_theta_tanh(int N, int M, const double *b, const double *W, const int8_t *s,
                              int64_t B, double *T, cudaStream_t st);

// ---- linear algebra (k_linalg.cu) -----------------------------------------

cudaError_t launch_stats(const double *e, int64_t Ns, int n_chains, double *out, cudaStream_t st);

// out = J^T g, with J given by samples s [Ns,N] and T = tanh theta [Ns,M].
// partial: workspace of vjp_partial_doubles(...) doubles.
size_t vjp_partial_doubles(int N, int M, int64_t Ns);
cudaError_t launch_vjp(int N, int M, int64_t Ns, const int8_t *s, const double *T,
                       const double *g, double g_scale, const double *g_shift, double *partial,
                       double *out, cudaStream_t st);

// out = J v.  U: workspace [Ns][M+1] doubles.
cudaError_t launch_jvp(int N, int M, int64_t Ns, const int8_t *s, const double *T,
                       const double *v, double *U, double *out, cudaStream_t st);

cudaError_t launch_jacobian_rows(int N, int M, const int8_t *s, const double *T, int64_t row0,
                                 int64_t rows, const double *mean, double *O, cudaStream_t st);

// Dense QGT products on a stored centred Jacobian dJ [Ns][Np].
cudaError_t launch_gemv_rows(const double *A, int64_t rows, int64_t cols, const double *x,
                             double *y, cudaStream_t st);
size_t gemv_t_partial_doubles(int64_t rows, int64_t cols);
cudaError_t launch_gemv_t(const double *A, int64_t rows, int64_t cols, const double *x,
                          double scale, double *partial, double *y, cudaStream_t st);

// S = dJ^T dJ / Ns + eps I  [Np][Np] (lower triangle filled, full written).
cudaError_t launch_syrk_t(const double *A, int64_t rows, int64_t cols, double scale, double eps,
                          double *C, cudaStream_t st);

// Sample-space Gram K = P (S S^T + T T^T + (T T^T) o (S S^T)) P / Ns + eps I
// (rowmean: 2 Ns + 1 doubles of scratch).
cudaError_t launch_gram_samplespace(int N, int M, int64_t Ns, const int8_t *s, const double *T,
                                    double eps, double *K, double *rowmean, cudaStream_t st);

// Row means, grand mean and K <- P K P / Ns + eps I for a full symmetric K
// (lower triangle written); rowmean holds 2 Ns + 1 doubles of scratch.
cudaError_t launch_center_gram(int64_t Ns, double *K, double *rowmean, double eps, cudaStream_t st);

// In-place lower Cholesky of an n x n matrix (lda = n); info: device int.
cudaError_t launch_cholesky(double *A, int64_t n, int *info, cudaStream_t st);
// Solve L L^T x = b in place (b -> x).
cudaError_t launch_cholesky_solve(const double *L, int64_t n, double *b, cudaStream_t st);

// ---- tensor-core products (k_tc.cu) ---------------------------------------
// FP64 rows -> S BF16 integer slices [S][rows][64] + row exponents.
size_t slice_elems(int64_t rows, int S);
cudaError_t launch_slice_rows(const double *A, int64_t lda, int64_t rows, int kcols, int S,
                              __nv_bfloat16 *out, int *expo, cudaStream_t st);
// C (mode 0: =, 1: -=, 2: +=) A B^T from slices, 128 x 32 tiles, K <= 64.
cudaError_t launch_ozaki_gemm(const __nv_bfloat16 *Asl, const int *expA, int64_t rows,
                              const __nv_bfloat16 *Bsl, const int *expB, int64_t cols, int S, double *C,
                              int64_t ldc, int mode, bool lower, int *err, cudaStream_t st);
size_t tc_chol_ws_bytes(int64_t n);
// Streams of the panel look-ahead: `side` carries the panel chain, `aux`
// the slicing of a panel beside its diagonal block; the events join them.
struct CholStreams {
    cudaStream_t side, aux;
    cudaEvent_t ev_wide, ev_panel, ev_fork, ev_join;
};
// cs null: everything on st.
cudaError_t launch_cholesky_tc(double *A, int64_t n, int *info, int *err, void *ws, cudaStream_t st,
                               const CholStreams *cs = nullptr);
// Forward and backward solves with the factor of launch_cholesky_tc (one
// cooperative launch each); err receives 6 / 7 if a block-row wait timed out.
cudaError_t launch_cholesky_solve_tc(const double *L, int64_t n, const void *ws, double *b, int *err,
                                     cudaStream_t st);
cudaError_t launch_gram_tc(int N, int M, int64_t Ns, const int8_t *s, const double *T, int S, double *K,
                           int *err, void *ws, cudaStream_t st);
// Lower triangle of C = scale X^T X + eps I (X [rows][ncols]) by 7-slice
// tensor-core products, 64 rows of X per pass; ws as for launch_cholesky_tc(ncols).
cudaError_t launch_gram_cols_tc(const double *X, int64_t rows, int64_t ncols, double scale, double eps, double *C,
                                int *err, void *ws, cudaStream_t st);


// ---- tensor-core products with the configurations (k_sgemm.cu) -------------
size_t tc_theta_ws_bytes(int N, int M, int64_t B);
// theta [B][M] = S W^T + b, exact to 2^-56 of max|W_j| (7 slices); row r of
// theta at theta + r * ldtheta (0: M).
cudaError_t launch_theta_tc(int N, int M, const double *b, const double *W, const int8_t *s, int64_t B,
                            double *theta, int *err, void *ws, cudaStream_t st, int64_t ldtheta = 0);
// The +-1 operands of the two Jacobian products depend on the samples only:
// a solve that repeats the products (CG) builds them once.  opA: [S, 1] as
// BF16 [Ns][pad8(N + 1)] (J v); opT: [S, 1]^T as BF16 [N + 1][pad8(Ns)] (J^T g).
size_t tc_jvp_operand_bytes(int N, int64_t Ns);
size_t tc_vjp_operand_bytes(int N, int64_t Ns);
cudaError_t launch_jacobian_operands(int N, int64_t Ns, const int8_t *s, void *opA, void *opT, cudaStream_t st);
// t' = [tanh(theta), 1] as FP32 pairs (hi, lo) in the tile order of the
// persistent J v kernel (k_tc4); fixed during a solve, so CG builds it once.
size_t tc_split_t_bytes(int M, int64_t Ns);
cudaError_t launch_split_t(int M, int64_t Ns, const double *T, void *Thl, cudaStream_t st);
size_t tc_jvp_ws_bytes(int N, int M, int64_t Ns);
// opA (optional): the prebuilt J v operand of launch_jacobian_operands;
// Thl (optional): the pairs of launch_split_t for T (else built in ws);
// skip (optional, device int): the product kernel does nothing while *skip
// is set (the converged flag of a CG whose loop still runs to its next poll).
cudaError_t launch_jvp_tc(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *v,
                          double *out, int SB, int *err, void *ws, cudaStream_t st, const void *opA = nullptr,
                          const void *Thl = nullptr, const int *skip = nullptr);
size_t tc_vjp_ws_bytes(int N, int M, int64_t Ns);
// colexpT (optional, [M + 1], from launch_colexp_t): the column exponents of
// tanh(theta), so that the slices of (T' o g')^T take their exponents from
// the bound max_k |t'_kj| max_k |g'_k| instead of a pass over T.  opT
// (optional): the prebuilt J^T g operand of launch_jacobian_operands.  Thl
// and skip as for launch_jvp_tc (the 3-slice path slices (T' o g')^T from
// the FP32 pairs of T; without Thl or colexpT it builds them in ws).
cudaError_t launch_vjp_tc(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *g,
                          double scale, const double *shift, double *out, int SB, int *err, void *ws,
                          cudaStream_t st, const int *colexpT = nullptr, const void *opT = nullptr,
                          const void *Thl = nullptr, const int *skip = nullptr);
size_t tc_colexp_ws_bytes(int M, int64_t Ns);
cudaError_t launch_colexp_t(int M, int64_t Ns, const double *T, int *colexpT, void *ws, cudaStream_t st);

// vector helpers
cudaError_t launch_axpby(int64_t n, double alpha, const double *x, double beta, double *y,
                         cudaStream_t st);  // y = alpha x + beta y
size_t dot_partial_doubles(int64_t n);
cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *partial, double *out,
                       cudaStream_t st);
cudaError_t launch_center(int64_t n, double *x, double *partial, double scale, cudaStream_t st);
cudaError_t launch_fill(int64_t n, double v, double *x, cudaStream_t st);

// CG step kernels (scalars live in device memory).
cudaError_t launch_cg_update_xr(int64_t n, const double *rr, const double *pAp, const double *p,
                                const double *Ap, double *x, double *r, const int *done,
                                cudaStream_t st);
cudaError_t launch_cg_update_p(int64_t n, const double *rr_new, const double *rr_old,
                               const double *r, double *p, const int *done, cudaStream_t st);
cudaError_t launch_cg_check(const double *rr, const double *ff, double tol, int *done,
                            int *iters, double *rr_keep, cudaStream_t st);

// Symmetric RBM (k_symm.cu): perms [G][N] device; err |= 1 when a row is not
// a permutation of [0, N); expanded plain-RBM parameters [N + M + M N],
// M = alpha G; uncentred symmetric Jacobian rows O [Ns][1 + alpha + alpha N]
// from t = tanh theta of the expanded units [Ns][M]; O -= column means.
cudaError_t launch_symm_check_perms(int N, int G, const int32_t *perms, int *err, cudaStream_t st);
cudaError_t launch_symm_expand(int N, int alpha, int G, const int32_t *perms, const double *p, double *out,
                               cudaStream_t st);
size_t symm_jacobian_smem(int N, int alpha, int G);
cudaError_t launch_symm_jacobian(int N, int alpha, int G, const int32_t *perms, const int8_t *s, const double *T,
                                 int64_t Ns, double *O, cudaStream_t st);
cudaError_t launch_sub_colmean(int64_t rows, int64_t cols, const double *mean, double *O, cudaStream_t st);

// Symmetric eigensolver (k_eig.cu): cyclic two-sided Jacobi sweeps with the
// round-robin parallel ordering on a full symmetric A [n][n] (diagonalised
// in place) and V [n][n] (V <- V J; start from the identity: columns are the
// eigenvectors); ws of eig_ws_bytes(n).  w = diag A, wmax = max w.  The filter: z_k <- z_k /
// w_k^power for w_k > rcond wmax, else 0; kept counts the kept ones.
size_t eig_ws_bytes(int64_t n);
cudaError_t launch_symmetrize_lower(int64_t n, double *A, cudaStream_t st);
cudaError_t launch_identity(int64_t n, double *V, cudaStream_t st);
// All sweeps in one cooperative launch, until the relative off-diagonal
// norm is <= tol or max_sweeps; out2 = (sweeps taken, final norm).
cudaError_t launch_jacobi_coop(double *A, double *V, int64_t n, int max_sweeps, double tol, void *ws, double *out2,
                               cudaStream_t st);
cudaError_t launch_eig_diag(int64_t n, const double *A, double *w, double *wmax, cudaStream_t st);
cudaError_t launch_spectral_filter(int64_t n, const double *w, const double *wmax, double rcond, int power,
                                   double *z, int *kept, cudaStream_t st);

// Complex holomorphic RBM (k_complex.cu); complex arrays are interleaved
// (re, im) doubles, 16-byte aligned.  Shared memory per warp of the one-
// warp-per-chain kernels: crbm_smem_per_warp (4 warps per block).
size_t crbm_smem_per_warp(int N, int M);
cudaError_t launch_crbm_logpsi(int N, int M, const double *p, const int8_t *s, int64_t B, double *out,
                               cudaStream_t st);
cudaError_t launch_crbm_sweep(int N, int M, const double *p, int rule, int E, const int32_t *edges, int C, int8_t *s,
                              int64_t sweep0, int n_discard, int n_samples, uint64_t seed, uint32_t stream_id,
                              int8_t *samples, unsigned long long *n_accepted, cudaStream_t st);
cudaError_t launch_crbm_eloc(int N, int M, const double *p, const nk_ham *ham, const int8_t *s, int64_t Ns,
                             double *eloc, cudaStream_t st);
cudaError_t launch_crbm_jacobian(int N, int M, const double *p, const int8_t *s, int64_t Ns, double *O,
                                 cudaStream_t st);
// mean: complex [cols] scratch; R [2 rows][2 cols] the realified centred O.
cudaError_t launch_crealify(int64_t rows, int64_t cols, const double *O, double *mean, double *R, cudaStream_t st);
// out4 = [Re mean, Im mean, variance, error] of complex local energies.
cudaError_t launch_cstats(int64_t Ns, const double *e, double *out4, cudaStream_t st);
cudaError_t launch_cforce_g(int64_t Ns, const double *e, const double *stats4, double *g, cudaStream_t st);
cudaError_t launch_tdvp_rhs(int64_t n, const double *f, int real_time, double *rhs, cudaStream_t st);
cudaError_t launch_caxpy_realified(int64_t n, const double *base, double h, const double *x, double *out,
                                   cudaStream_t st);

// params -= lr * delta; norms into stats.
cudaError_t launch_sgd(int64_t n, double lr, const double *delta, double *params,
                       cudaStream_t st);
cudaError_t launch_make_force_g(int64_t Ns, const double *eloc, const double *stats,
                                double *g, cudaStream_t st);
cudaError_t launch_write_sr_stats(const double *stats3, const unsigned long long *acc, int C,
                                  double n_proposals, const double *ff, const double *dd,
                                  const int *cg_iters, const double *cg_rr, const int *status,
                                  nk_sr_stats *out, cudaStream_t st);

}  // namespace nk
