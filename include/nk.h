/*
 * nk.h -- C ABI of libnk.so, the GB300 (sm_103a) hot path of variational
 * Monte Carlo with a restricted Boltzmann machine, after the NetKet 3 paper
 * (F. Vicentini et al., arXiv:2112.10526).
 *
 * One VMC step: Metropolis sampling of |psi|^2 (Sec. 3.4), local energies
 * (Sec. 3.3, Eq. eq:local-estimator), log-derivatives (Eq.
 * eq:log-derivative-O), force (Eqs. eq:force VMC, eq:gradE:real), the
 * quantum geometric tensor (Sec. 3.5, App. B) and the stochastic
 * reconfiguration solve (Eq. eq:stochastic-reconfiguration) followed by the
 * SGD update (Sec. 4.1).
 *
 * Conventions for every call:
 *   - Return value: NK_OK (0) or a negative NK_ERR_* code.  The message of
 *     the last failure on the calling host thread is nk_last_error().
 *   - Array arguments are DEVICE pointers owned by the caller, contiguous,
 *     row-major, unless a comment says "host".  The library never frees them.
 *   - Configurations are int8 with values -1/+1, layout [batch, N].
 *   - RBM parameters are one float64 device vector
 *         theta = [ a (N) ; b (M) ; W (M x N, row-major) ],  Np = N + M + M N,
 *     with ln psi(s) = sum_i a_i s_i + sum_j ln cosh(b_j + sum_i W_ji s_i)
 *     (the RBM of Sec. 3.2, Table tab:nk.models).
 *   - Every call is asynchronous on the given CUDA stream (cudaStream_t
 *     passed as void*, NULL = legacy default stream) and does not
 *     synchronise it, except nk_sr_step with the CG solver, which reads the
 *     residual back every few iterations (documented there).
 *   - Workspace is allocated inside the nk_ctx and grows on demand
 *     (cudaMalloc, which synchronises the device).  A context is not
 *     thread-safe: use one per host thread.  Calls on one context must not
 *     overlap on different streams (they share the workspace).
 *   - precision: NK_F64 computes everything in FP64 on CUDA cores.
 *     NK_MIXED keeps the Metropolis chains and local-energy ratios in FP32,
 *     rebuilds the hidden activations from scratch at every sweep with an
 *     FP64-exact tensor-core product (configurations x W cut into 7 BF16
 *     integer slices, FP32 accumulation), runs the Jacobian products on the
 *     tensor cores (in CG matvecs 3 FP16 slices of 11-bit digits, 33 bits of
 *     each operand row; 7 BF16 slices where the sample-space solve needs
 *     FP64-level products) and keeps FP64 for sample means, centring,
 *     the SR factorisation (tensor-core products at FP64 level) and update.
 */
#ifndef NK_H
#define NK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t nk_status;
#define NK_OK 0
#define NK_ERR_INVALID_ARG (-1)
#define NK_ERR_CUDA (-2)
#define NK_ERR_OOM (-3)
#define NK_ERR_TIMEOUT (-4)
#define NK_ERR_NOT_CONVERGED (-5) /* result still written */
#define NK_ERR_UNIMPLEMENTED (-6)

#define NK_F64 0
#define NK_MIXED 1

#define NK_RULE_LOCAL 0    /* MetropolisLocal: flip one spin (Sec. 3.4) */
#define NK_RULE_EXCHANGE 1 /* MetropolisExchange: swap an edge (Sec. 3.4) */
#define NK_RULE_HAMILTONIAN 2 /* MetropolisHamiltonian: move along an off-diagonal
                                 element of H (Sec. 3.4), with the Hastings
                                 correction of the asymmetric proposal */

#define NK_TFIM 0 /* H = J sum_<ik> sz sz + J2 sum_<<ik>> sz sz - h sum_i sx (Eq. eq:tf-ising-hamiltonian) */
#define NK_HEIS 1 /* H = J sum_<ik> sigma.sigma + J2 sum_<<ik>> sigma.sigma (Eq. eq: j1 j2 heisenberg) */

#define NK_SOLVER_CHOLESKY 0             /* dense (S + eps I) in parameter space */
#define NK_SOLVER_CHOLESKY_SAMPLESPACE 1 /* same solution via an Ns x Ns factor */
#define NK_SOLVER_CG 2                   /* CG on on-the-fly QGT products */
#define NK_SOLVER_SVD 3                  /* pseudo-inverse of the dense (S + eps I) in parameter
                                            space, eigenvalues below rcond x the largest dropped */
#define NK_SOLVER_SVD_SAMPLESPACE 4      /* the same truncated solve (eps = 0) from the
                                            eigenpairs of the Ns x Ns sample-space Gram */

#define NK_QGT_ONTHEFLY 0 /* QGTOnTheFly (App. B.3) */
#define NK_QGT_JACOBIAN 1 /* QGTJacobianDense on a stored centred Jacobian (App. B.2) */

typedef struct nk_ctx nk_ctx;

typedef struct {
    int32_t N;      /* visible units = lattice sites, >= 1 */
    int32_t M;      /* hidden units (alpha N), >= 1 */
    double *params; /* device [Np]; only nk_sr_step writes it */
} nk_rbm;

typedef struct {
    int32_t kind;          /* NK_TFIM or NK_HEIS */
    double J;              /* coupling of the nearest-neighbour edges <ik> */
    double h;              /* transverse field (NK_TFIM) */
    int32_t marshall;      /* NK_HEIS: 1 = Marshall sign folded in: off-diagonal
                              element -2J on every nearest-neighbour edge (each
                              must join the two sublattices of a bipartite
                              lattice) and +2 J2 on every next-nearest one (each
                              must stay inside one sublattice); 0 = +2J, +2 J2 */
    int32_t n_edges;       /* E >= 1, both classes */
    const int32_t *edges;  /* device [E, 2], site indices in [0, N); the
                              nearest-neighbour edges first */
    double J2;             /* coupling of the next-nearest-neighbour edges <<ik>> */
    int32_t n_edges2;      /* the last n_edges2 of the E edges are next-nearest
                              neighbours, 0 <= n_edges2 <= E (0: J2 unused; a
                              zero-initialised tail gives the nearest-neighbour
                              model).  nk_sr_step's exchange rule draws from all
                              E edges (d_max = 2 of the J1-J2 example, Sec. 7) */
} nk_ham;

/* Context: device ordinal, workspace, cached per-parameter tables. */
nk_status nk_ctx_create(int32_t device, nk_ctx **out /* host */);
nk_status nk_ctx_destroy(nk_ctx *ctx);
/* Message of the last failure on this host thread ("" if none); valid until
 * the next failing call on this thread. */
const char *nk_last_error(void);
/* Library version (major*10000 + minor*100 + patch). */
int32_t nk_version(void);
/*
 * Sticky status of the context's tensor-core products (NK_MIXED paths):
 * waits for the context's work on `stream` and returns in *code 0, or the
 * code of the last bounded wait that timed out since the last call (the
 * results of that call are invalid): 3-5 the S-GEMM (producer, MMA issuer,
 * epilogue), 6 / 7 the forward / backward triangular solve, 12-16 the
 * FP64-accurate product (producer, A slices, B slices, accumulator buffer,
 * epilogue).  Resets the word.
 */
nk_status nk_ctx_error(nk_ctx *ctx, int32_t *code /* host */, void *stream);

/*
 * ln psi(s) for a batch of configurations (Eq. eq:mapping: the model maps
 * (theta, s) to ln psi_theta(s); the batched evaluation of Sec. 3.2).
 *   s          [B, N] int8 +-1
 *   logpsi_out [B] float64
 * B = 0 is a no-op.
 */
nk_status nk_rbm_logpsi(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                        int64_t B, double *logpsi_out, void *stream);

/*
 * Random initial chain states (random_state of Sec. 2.1), from the Philox
 * stream (key (seed, 0), counter (index, chain, stream_id, 1)).
 *   rule NK_RULE_LOCAL: i.i.d. spins; NK_RULE_EXCHANGE and
 *   NK_RULE_HAMILTONIAN: S_z = 0 (N even).
 *   s_out [C, N] int8.
 */
nk_status nk_chains_init(nk_ctx *ctx, int32_t N, int32_t C, int32_t rule, uint64_t seed,
                         uint32_t stream_id, int8_t *s_out, void *stream);

/*
 * Metropolis-Hastings sweeps (Sec. 3.4: P_acc = min(1, |psi(s')/psi(s)|^2)
 * for the symmetric local and exchange proposals, times g(s|s')/g(s'|s)
 * for the Hamiltonian rule).  One sweep is N
 * proposals per chain.  Proposal p of sweep w uses the Philox4x64-10 block
 * with key (seed, 0) and counter ((sweep0 + w) N + p, chain, stream_id, 0):
 * the site (local) or edge (exchange) is floor(hi32(y0) * n / 2^32), the
 * uniform is u = ((y1 >> 11) + 0.5) 2^-53, and the move is accepted iff
 * ln u < 2 (ln psi(s') - ln psi(s)).  An exchange proposal on an edge with
 * equal spins is not a move.  NK_RULE_HAMILTONIAN is the rule of a
 * Heisenberg-type Hamiltonian on `edges`: the configurations connected to s
 * are the swaps across its n(s) antiparallel edges, s' is the r-th of them
 * in edge order, r = floor(hi32(y0) n(s) / 2^32), and the move is accepted
 * iff ln u < 2 (ln psi(s') - ln psi(s)) + ln n(s) - ln n(s') (n(s) = 0: not
 * a move).  Hidden activations theta = b + W s are rebuilt
 * from scratch (FP64) at the start of every sweep and updated incrementally
 * on every accepted move.
 *   s            [C, N] in/out chain states
 *   n_edges/edges  device [E, 2] edge list (exchange and Hamiltonian rules;
 *                else 0/NULL)
 *   samples_out  [C, n_samples, N]: the state after each of the n_samples
 *                sweeps that follow n_discard discarded sweeps
 *   logpsi_out   [C, n_samples] float64 or NULL
 *   n_accepted   [C] uint64, incremented by accepted moves, or NULL
 *   decisions_out [C, n_discard + n_samples, N] uint8 or NULL: per proposal
 *                0 rejected, 1 accepted, 2 not a move (for replay checks)
 * Limits: N <= 4096, M <= 8192.  C = 0 is a no-op.
 */
nk_status nk_metropolis_sweep(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, int32_t rule,
                              int32_t n_edges, const int32_t *edges, int32_t C, int8_t *s,
                              int64_t sweep0, int32_t n_discard, int32_t n_samples, uint64_t seed,
                              uint32_t stream_id, int8_t *samples_out, double *logpsi_out,
                              uint64_t *n_accepted, uint8_t *decisions_out, void *stream);

/*
 * Local energies E_loc(s) = sum_s' H_ss' psi(s')/psi(s)
 * (Eq. eq:local-estimator) through single-flip (NK_TFIM) and pair-flip
 * (NK_HEIS) amplitude ratios.
 *   s [Ns, N];  eloc_out [Ns] float64;  t_out [Ns, M] float64 tanh(theta)
 *   of every sample as a by-product, or NULL.
 */
nk_status nk_local_energy(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const nk_ham *ham,
                          const int8_t *s, int64_t Ns, double *eloc_out, double *t_out,
                          void *stream);

/*
 * Local energies as nk_local_energy, for callers that cannot let a library
 * allocate device memory (their HBM is owned by another allocator, or they
 * cannot afford cudaMalloc's device-wide synchronisation).  The paper has no
 * counterpart; this is a property of the library, not of the method.
 * No context and no allocation: the flip-ratio tables live in one fixed
 * __device__ array of NK_NOALLOC_SCRATCH_BYTES compiled into libnk.so, held
 * by every GPU that loads the library until the process exits.  Sizes whose
 * tables do not fit (about 8 (3 N M + N) bytes for NK_TFIM, 8 (N M + 2 E M
 * + E) for NK_HEIS in FP64, half the tau part in NK_MIXED) return
 * NK_ERR_INVALID_ARG.
 *   NK_F64: the same kernels on the same tables as nk_local_energy, so the
 *   results are bit-identical.  NK_MIXED: there is no room for the batch's
 *   hidden activations, so the local-energy kernel rebuilds theta = b + W s
 *   per sample in FP64 instead of taking the tensor-core product; the
 *   results agree with nk_local_energy within the mixed tolerance (1e-4
 *   relative per sample), not bit for bit.
 * The first call on each device, with it current, looks up the array's
 * device address; the address is cached per device and CUDA context and
 * looked up again when the context changes (after cudaDeviceReset, say).
 * Make the first call, and the first after a reset, before any stream
 * capture.  All calls share the array: calls that overlap on the GPU race,
 * so serialise them.  Runs on the current device; every array must be
 * memory of that device (or managed memory), else NK_ERR_INVALID_ARG.
 * Arguments as nk_local_energy.
 */
#define NK_NOALLOC_SCRATCH_BYTES (8u << 20)
nk_status nk_local_energy_noalloc(const nk_rbm *rbm, int32_t precision, const nk_ham *ham,
                                  const int8_t *s, int64_t Ns, double *eloc_out, double *t_out,
                                  void *stream);

/*
 * Sample statistics of the local energy (Sec. 3.3): out[0] = mean,
 * out[1] = variance (1/Ns normalisation), out[2] = standard error of the
 * mean (from the n_chains chain means when each chain holds >= 2 samples
 * stored chain-major, else sqrt(variance/Ns)).  out: device float64 [3].
 */
nk_status nk_stats(nk_ctx *ctx, const double *eloc, int64_t Ns, int32_t n_chains, double *out,
                   void *stream);

/*
 * Rows [row0, row0 + rows) of the Jacobian J_kl = O_l(s_k) (Eq.
 * eq:log-derivative-O, App. B.1): O_a = s, O_b = tanh theta,
 * O_W = tanh theta s^T, theta recomputed from s.  With centered = 1 the
 * column means over all Ns samples are subtracted (the centred Jacobian of
 * App. B.2).  O_out [rows, Np] float64.
 */
nk_status nk_jacobian(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                      int64_t Ns, int32_t centered, int64_t row0, int64_t rows, double *O_out,
                      void *stream);

/* Vector-Jacobian product out = J^T g (App. B.1), g [Ns], out [Np].  With
 * NK_MIXED both products run on the tensor cores with the sliced operand
 * (v, or T o g) cut into 3 FP16 slices of 11-bit digits per row (a 33-bit
 * grid on each row's largest entry, about 2^-33 relative) and exact FP32
 * accumulation; nk_vjp builds the FP32 pairs of tanh(theta) it slices from
 * in the context workspace. */
nk_status nk_vjp(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s, int64_t Ns,
                 const double *g, double *out, void *stream);

/* Jacobian-vector product out = J v (App. B.1), v [Np], out [Ns]. */
nk_status nk_jvp(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s, int64_t Ns,
                 const double *v, double *out, void *stream);

/*
 * Force f = 2 Re Cov[O, E_loc] = (2/Ns) J^T (E_loc - mean E_loc)
 * (Eqs. eq:force VMC and eq:gradE:real).  F_out [Np].
 */
nk_status nk_force(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                   int64_t Ns, const double *eloc, double *F_out, void *stream);

typedef struct {
    int32_t kind;        /* NK_QGT_ONTHEFLY or NK_QGT_JACOBIAN */
    const nk_rbm *rbm;   /* ONTHEFLY: the model and its samples */
    int32_t precision;
    const int8_t *s;     /* ONTHEFLY: [Ns, N] */
    const double *dJ;    /* JACOBIAN: centred Jacobian [Ns, Np] (nk_jacobian, centered=1) */
    int64_t Ns;
    int32_t Np;          /* JACOBIAN: number of parameters */
} nk_qgt;

/*
 * out = (G + diag_shift I) v with G = (1/Ns) J^T dJ (Sec. 3.5, App. B.2 /
 * B.3): ONTHEFLY computes w = J v / Ns, dw = w - <w>, J^T dw; JACOBIAN
 * computes dJ^T (dJ v) / Ns.  v, out [Np].
 */
nk_status nk_qgt_matvec(nk_ctx *ctx, const nk_qgt *qgt, double diag_shift, const double *v,
                        double *out, void *stream);

/*
 * FP64-accurate dense product on the tensor cores: C (op)= A B^T with
 * A [rows, k] (row stride lda), B [cols, k] (ldb), k <= 64, C [rows, cols]
 * (ldc); op by mode: 0 '=', 1 '-=', 2 '+='; lower = 1 touches only entries
 * with column <= row.  Each operand row is scaled by a power of two and cut
 * into `slices` (1..7) 8-bit integer slices; the slice products run as BF16
 * tcgen05 MMAs with exact FP32 accumulation and are recombined in FP64
 * (slices = 7: FP64-level accuracy; 3: about FP32).  This is the building
 * block of the NK_MIXED Cholesky and sample-space Gram (the dense products
 * G = dJ^T dJ / Ns of App. B.2 and the factorisation of Sec. 3.5).  The call
 * synchronises the stream and returns NK_ERR_TIMEOUT if a product timed out.
 */
nk_status nk_tc_gemm(nk_ctx *ctx, int64_t rows, int64_t cols, int32_t k, const double *A, int64_t lda,
                     const double *B, int64_t ldb, int32_t slices, int32_t mode, int32_t lower,
                     double *C, int64_t ldc, void *stream);

/*
 * Solve (G + diag_shift I) delta = F for the QGT of the given samples
 * (Eq. eq:stochastic-reconfiguration, real case; Sec. 3.5 "Solving linear
 * systems").  solver: NK_SOLVER_CHOLESKY (dense Np x Np FP64 Cholesky),
 * NK_SOLVER_CHOLESKY_SAMPLESPACE (FP64 Cholesky of the Ns x Ns matrix
 * dJ dJ^T / Ns + diag_shift I and delta = (F - dJ^T y / sqrt(Ns)) /
 * diag_shift, equal in exact arithmetic), NK_SOLVER_CG (unpreconditioned
 * conjugate gradients, x0 = 0, stops at ||r|| <= cg_tol ||F|| or cg_maxiter;
 * reads the residual back to the host every 8 iterations, which
 * synchronises the stream), NK_SOLVER_SVD (the pseudo-inverse of the dense
 * Np x Np matrix S + diag_shift I, keeping the eigenvalues above rcond times
 * the largest) and NK_SOLVER_SVD_SAMPLESPACE (the same truncated solve at
 * diag_shift = 0 from the eigenpairs (lambda_k, u_k) of X X^T, X = dJ /
 * sqrt(Ns): delta = X^T sum_{lambda_k > rcond max lambda} u_k lambda_k^-2
 * u_k^T X F).  For the two SVD solvers cg_tol is rcond (0: 1e-12); their
 * eigendecomposition is cyclic Jacobi in FP64 on CUDA cores, which reads
 * its convergence back once per sweep (synchronises the stream); n = Np or
 * Ns at most 8192.  With NK_MIXED the Cholesky factorisations run their
 * panel and trailing products on the tensor cores at FP64-level accuracy
 * (see nk_tc_gemm), and so do the Gram matrices; the call then synchronises
 * the stream and returns NK_ERR_CUDA on a failed factorisation
 * (NK_ERR_TIMEOUT on a tensor-core time-out).
 *   info_out host int32[2] or NULL: iterations (CG) or Jacobi sweeps (SVD),
 *   converged flag.
 *   resid_out host double or NULL: final relative residual (CG), or the
 *   relative off-diagonal norm left by the sweeps (SVD).
 */
nk_status nk_sr_solve(nk_ctx *ctx, const nk_rbm *rbm, int32_t precision, const int8_t *s,
                      int64_t Ns, const double *F, int32_t solver, double diag_shift,
                      double cg_tol, int32_t cg_maxiter, double *delta_out, int32_t *info_out,
                      double *resid_out, void *stream);

typedef struct {
    int32_t C;          /* chains */
    int8_t *s;          /* device [C, N] chain states, in/out */
    int64_t sweeps_done;/* host: sweeps already run by these chains; advanced by nk_sr_step */
    uint64_t *n_accepted; /* device [C] or NULL */
} nk_chains;

typedef struct {
    int32_t rule;        /* NK_RULE_*; in nk_sr_step NK_RULE_HAMILTONIAN is the
                            local rule for NK_TFIM (its connected configurations
                            are the N single flips) and swaps across the
                            Hamiltonian's edges for NK_HEIS, without the
                            next-nearest class when J2 = 0 */
    int32_t precision;   /* NK_F64 or NK_MIXED */
    int32_t solver;      /* NK_SOLVER_* */
    int32_t n_discard;   /* sweeps discarded before sampling */
    int32_t n_samples;   /* samples (sweeps) per chain */
    int32_t cg_maxiter;
    double diag_shift;   /* eps */
    double lr;           /* eta */
    double cg_tol;
    uint64_t seed;
    uint32_t stream_id;
    double svd_rcond;    /* NK_SOLVER_SVD*: relative cutoff of the eigenvalues (0: 1e-12) */
} nk_sr_cfg;

/* Diagnostics of one step, written to DEVICE memory (float64 fields). */
typedef struct {
    double energy;       /* mean E_loc */
    double variance;
    double error;        /* standard error of the mean */
    double acceptance;   /* accepted / proposed moves in this step */
    double cg_iters;
    double cg_residual;
    double f_norm;       /* ||F|| */
    double delta_norm;   /* ||delta|| */
    double solver_status; /* 0 = ok; k > 0: the Cholesky pivot k (1-based) was not
                             positive; -1 / -2: a tensor-core product timed out
                             waiting for its operands / its MMAs */
} nk_sr_stats;

/*
 * One VMC iteration with stochastic reconfiguration (Sec. 4.1): sample
 * n_samples states per chain after n_discard sweeps, local energies,
 * statistics, force, SR solve, and theta <- theta - lr delta (rbm->params
 * updated in place).
 *   chains: states advanced in place; chains->sweeps_done advanced (host).
 *   stats_out: device nk_sr_stats or NULL.
 *   samples_out [C*n_samples, N], eloc_out [C*n_samples]: optional device
 *   outputs of this step's samples and local energies (NULL = internal).
 */
nk_status nk_sr_step(nk_ctx *ctx, nk_rbm *rbm, const nk_ham *ham, nk_chains *chains,
                     const nk_sr_cfg *cfg, nk_sr_stats *stats_out, int8_t *samples_out,
                     double *eloc_out, void *stream);


/* ------------------------------------------------------ symmetric RBM ---
 * RBMSymm (Sec. 5, "fully symmetric RBMs"): a permutation group G of the
 * sites, given as rows perms[g][j] = pi_g(j) (each a permutation of [0, N);
 * the identity need not come first), and alpha features whose activation at
 * group element g is the embedding layer of Eq. eq: equivariant: embedding,
 *     theta_{f,g}(s) = b_f + sum_j W_{f,j} s_{pi_g(j)},
 * with ln psi(s) = a sum_j s_j + sum_{f,g} ln cosh theta_{f,g}(s).  The
 * printed form has no biases; a hidden bias per feature and one visible bias
 * (the symmetric restriction of the RBM's) are kept, and vanish at zero.
 * Parameters: one float64 device vector [a (1); b (alpha); W (alpha x N,
 * row-major)], Np = 1 + alpha + alpha N.  psi is invariant under G.
 * The model equals a plain RBM with M = alpha |G| hidden units and tied
 * parameters (unit f |G| + g: bias b_f, weight W_{f,j} on site pi_g(j), every
 * visible bias a); the sampler and the local energies run on those expanded
 * parameters.  Limits: N <= 4096, alpha |G| <= 8192.
 */
typedef struct {
    int32_t N;             /* sites */
    int32_t alpha;         /* features */
    int32_t n_group;       /* |G| */
    const int32_t *perms;  /* device [n_group, N] */
    double *params;        /* device [1 + alpha + alpha N]; only nk_symm_sr_step writes it */
} nk_rbm_symm;

/* The equal plain RBM's parameters: plain_out device [N + M + M N], M =
 * alpha n_group.  Checks first that every row of perms is a permutation of
 * [0, N) (NK_ERR_INVALID_ARG otherwise); the check reads one flag back and
 * synchronises the stream. */
nk_status nk_symm_expand(nk_ctx *ctx, const nk_rbm_symm *symm, double *plain_out, void *stream);

/* Log-derivatives in the symmetric parameters (Eq. eq:log-derivative-O by
 * the chain rule through the tying): O_a = sum_j s_j, O_{b_f} = sum_g
 * tanh theta_{f,g}, O_{W_{f,j}} = sum_g tanh theta_{f,g} s_{pi_g(j)}.
 *   s [Ns, N];  O_out [Ns, Np] float64, uncentred.
 * theta in FP64 (NK_F64) or by the FP64-exact tensor-core product (NK_MIXED);
 * the sums in FP64.  Synchronises the stream (permutation check). */
nk_status nk_symm_jacobian(nk_ctx *ctx, const nk_rbm_symm *symm, int32_t precision, const int8_t *s,
                           int64_t Ns, double *O_out, void *stream);

/* One VMC iteration with stochastic reconfiguration (Sec. 4.1) for the
 * symmetric RBM: the chains and local energies of the expanded RBM (the same
 * psi), then the centred Jacobian in the Np symmetric parameters, the force
 * F = (2/Ns) dJ^T (E_loc - mean), S = dJ^T dJ / Ns + diag_shift I, its
 * Cholesky factor, two triangular solves, and params <- params - lr delta.
 * cfg->solver must be NK_SOLVER_CHOLESKY (NK_ERR_UNIMPLEMENTED otherwise):
 * Np is small enough for the dense factor.  NK_MIXED runs the sweeps and
 * local energies in FP32 as nk_sr_step does, and builds and factors S with
 * the FP64-accurate tensor-core products.  The other arguments, and the
 * diagnostics, as nk_sr_step.  Synchronises the stream (permutation check;
 * NK_MIXED also reads the factorisation status). */
nk_status nk_symm_sr_step(nk_ctx *ctx, nk_rbm_symm *symm, const nk_ham *ham, nk_chains *chains,
                          const nk_sr_cfg *cfg, nk_sr_stats *stats_out, int8_t *samples_out, double *eloc_out,
                          void *stream);

/* ---------------------------------------- complex RBM and time evolution ---
 * The RBM of Sec. 3.2 with complex parameters a, b, W (the holomorphic ansatz
 * of the time-evolution examples, Sec. 9): ln psi(s) = a.s + sum_j
 * ln cosh(b_j + W_j.s) is complex, psi(s) need not be positive, and the map
 * theta -> ln psi(s) is holomorphic, so O_k = d ln psi / d theta_k is the
 * complex O_a = s, O_b = tanh theta, O_W = tanh theta s^T.
 * Complex arrays are interleaved (re, im) float64 pairs and must be 16-byte
 * aligned (NK_ERR_INVALID_ARG otherwise).  Parameters: [a (N); b (M); W (M x
 * N, row-major)] complex, 2 Np doubles.  Everything is FP64 on CUDA cores.
 * Limits: N <= 4096, M <= 4096.
 */
typedef struct {
    int32_t N, M;
    double *params;  /* device, 2 Np doubles; only nk_tdvp_step writes it */
} nk_crbm;

/* Complex ln psi of a batch: s [B, N]; out [B] complex (2 B doubles). */
nk_status nk_crbm_logpsi(nk_ctx *ctx, const nk_crbm *rbm, const int8_t *s, int64_t B, double *out, void *stream);

/* Metropolis-Hastings chains on |psi|^2 (Sec. 3.4), on the Philox streams and
 * proposal rules of nk_metropolis_sweep (NK_RULE_LOCAL or NK_RULE_EXCHANGE):
 * the move is accepted iff ln u < 2 Re[ln psi(s') - ln psi(s)]; each
 * log-ratio is summed term by term over the hidden units from the moved
 * activations.  s [C, N] in/out; samples_out [C, n_samples, N]; n_accepted
 * [C] or NULL. */
nk_status nk_crbm_metropolis(nk_ctx *ctx, const nk_crbm *rbm, int32_t rule, int32_t n_edges, const int32_t *edges,
                             int32_t C, int8_t *s, int64_t sweep0, int32_t n_discard, int32_t n_samples,
                             uint64_t seed, uint32_t stream_id, int8_t *samples_out, uint64_t *n_accepted,
                             void *stream);

/* Complex local energies (Eq. eq:local-estimator): eloc_out [Ns] complex. */
nk_status nk_crbm_local_energy(nk_ctx *ctx, const nk_crbm *rbm, const nk_ham *ham, const int8_t *s, int64_t Ns,
                               double *eloc_out, void *stream);

/* Complex log-derivatives: O_out [Ns, Np] complex, uncentred. */
nk_status nk_crbm_jacobian(nk_ctx *ctx, const nk_crbm *rbm, const int8_t *s, int64_t Ns, double *O_out,
                           void *stream);

#define NK_TDVP_EULER 1 /* theta(t + dt) = theta + dt k1 */
#define NK_TDVP_HEUN 2  /* k2 at theta + dt k1 on fresh samples; theta + dt (k1 + k2) / 2 */

typedef struct {
    int32_t rule;        /* NK_RULE_LOCAL or NK_RULE_EXCHANGE */
    int32_t integrator;  /* NK_TDVP_EULER or NK_TDVP_HEUN */
    int32_t real_time;   /* 1: gamma = -i (unitary dynamics); 0: gamma = -1 (imaginary time) */
    int32_t solver;      /* NK_SOLVER_CHOLESKY ((G + eps I), eps > 0) or NK_SOLVER_SVD (its
                            pseudo-inverse: eigenvalues above rcond x the largest) */
    int32_t n_discard;   /* sweeps discarded before the first slope's samples */
    int32_t n_samples;   /* samples (sweeps) per chain for each slope */
    double dt;
    double diag_shift;   /* eps */
    double rcond;        /* NK_SOLVER_SVD (0: 1e-12) */
    uint64_t seed;
    uint32_t stream_id;
} nk_tdvp_cfg;

/* Diagnostics of one time step (DEVICE float64 fields), from the first
 * slope's samples. */
typedef struct {
    double energy_re, energy_im;  /* mean E_loc */
    double variance;              /* mean |E_loc - mean|^2 */
    double error;                 /* sqrt(variance / Ns) */
} nk_tdvp_stats;

/*
 * One step of time-dependent variational Monte Carlo (Sec. 4.3): each slope
 * samples the chains (continuing them; the second slope of Heun draws the
 * sweeps after the first's, with no discards), forms the sample-mean force
 * f~ = E[O^* (E_loc - E[E_loc])] and QGT G = E[O^* O] - E[O^*] E[O] (Sec.
 * 3.5, Eq. eq:force VMC) and solves (G + eps I) theta_dot = gamma f~ (Eq.
 * eq:tvmc); then the explicit Runge-Kutta update of Eq. eq:rk-step.  The
 * Hermitian system is solved through its real embedding [[Re G, -Im G],
 * [Im G, Re G]] of order 2 Np, built as R^T R / Ns from the realified
 * centred Jacobian R (2 Ns x 2 Np): by the FP64 Cholesky, or by the cyclic
 * Jacobi eigensolver of the SVD solvers (2 Np <= 8192; synchronises the
 * stream once per sweep).
 *   rbm->params updated in place; chains advanced (sweeps_done on the host).
 *   stats_out: device nk_tdvp_stats or NULL; theta_dot_out: device [Np]
 *   complex, the first slope, or NULL.
 */
nk_status nk_tdvp_step(nk_ctx *ctx, nk_crbm *rbm, const nk_ham *ham, nk_chains *chains, const nk_tdvp_cfg *cfg,
                       nk_tdvp_stats *stats_out, double *theta_dot_out, void *stream);

/* ------------------------------------------------------------- serving ---
 * A persistent request loop on one GPU for VMC expectation values and SR
 * steps (the serving use of this library; the paper has no counterpart).
 * Requests for different lattices, RBM widths and sample counts arrive from
 * any host thread and wait in a FIFO; a scheduler thread admits the head
 * request as soon as a worker slot is free and the HBM budget has room for
 * the request's device state plus the growth of the slot's workspace
 * (nk_request_bytes: a plan-only pass of the same entry points).  Each slot
 * has its own context and stream, so admitted requests run concurrently and
 * their kernels overlap, while new requests keep being admitted as slots and
 * memory free up.  A request's parameters, chains, samples and solver
 * workspace stay on the device until it completes.  Each request draws from
 * its own Philox stream (cfg.seed, cfg.stream_id) and every reduction has a
 * fixed order, so its result does not depend on what runs beside it.
 */
#define NK_REQ_EXPECT 0  /* sample + local energies + statistics */
#define NK_REQ_SR_STEP 1 /* the same + force + SR solve + update (nk_sr_step) */

typedef struct nk_server nk_server;

typedef struct {
    int32_t kind;            /* NK_REQ_* */
    int32_t N, M;
    const double *params;    /* HOST [Np], copied by nk_server_submit */
    int32_t ham_kind;        /* NK_TFIM / NK_HEIS */
    double J, h;
    int32_t marshall;
    int32_t n_edges;
    const int32_t *edges;    /* HOST [E, 2], copied by nk_server_submit */
    int32_t n_chains;        /* chains start from nk_chains_init(cfg.seed, cfg.stream_id) */
    nk_sr_cfg cfg;           /* rule, precision, solver, sweeps, eps, lr, RNG stream */
    double J2;               /* as nk_ham: coupling of the last n_edges2 edges */
    int32_t n_edges2;        /* 0 <= n_edges2 <= n_edges (0: nearest neighbours only) */
} nk_request;

typedef struct {
    int32_t status;          /* NK_OK or the request's NK_ERR_* code */
    int32_t slot;            /* worker slot that ran it */
    double energy, variance, error, acceptance, cg_iters, solver_status;
    double queue_ms;         /* submit -> admission */
    double run_ms;           /* admission -> completion */
    double latency_ms;       /* submit -> completion */
    size_t device_bytes;     /* HBM reserved at admission */
    char message[128];       /* the failing entry point's message, or "" */
} nk_result;

typedef struct {
    int64_t submitted, completed, failed, inflight, queued;
    size_t hbm_in_use, hbm_budget;
    double p50_ms, p99_ms;   /* latency quantiles over completed requests */
} nk_server_stats;

nk_status nk_server_create(int32_t device, size_t hbm_budget, int32_t slots, nk_server **out /* host */);
/* params_out: HOST [Np] buffer that receives the updated parameters of an
 * NK_REQ_SR_STEP (written before the request is marked done), or NULL. */
nk_status nk_server_submit(nk_server *srv, const nk_request *req, double *params_out, uint64_t *id /* host */);
nk_status nk_server_poll(nk_server *srv, uint64_t id, int32_t *done /* host */, nk_result *out /* host */);
nk_status nk_server_wait(nk_server *srv, uint64_t id, nk_result *out /* host */);
nk_status nk_server_stats_get(nk_server *srv, nk_server_stats *out /* host */);
/* Drops queued requests, waits for those in flight, frees everything. */
nk_status nk_server_destroy(nk_server *srv);
/* HBM estimate used for admission: the request's device state plus the
 * context workspace its entry points would allocate (planned bytes + 1/8
 * + 1 MiB, the allocation rule of every context).  0 if the plan fails. */
size_t nk_request_bytes(const nk_request *req);

/*
 * Kernel timing for measurement tools (not part of the method).  When
 * enabled, every launch of a tracked kernel class is bracketed by CUDA
 * events recorded on the stream it is launched on, and its work is added
 * up.  nk_prof_read waits for those events and returns the total
 * milliseconds, the number of launches and the total ALGORITHMIC work since
 * the last nk_prof_enable: the method's own count (ratio terms, or the flops
 * of the FP64 operation a launch stands for, whatever precision runs it).
 * nk_prof_read_executed returns what the hardware executed for the same
 * launches: for the NK_MIXED tensor-core products the BF16 MMA flops of all
 * slice products (several times the algorithmic flops), else the same as
 * the algorithmic work.  Process-wide; thread-safe.
 */
#define NK_PROF_SWEEP 0       /* Metropolis sweeps: ratio terms (proposals x M) */
#define NK_PROF_ELOC 1        /* local energies: ratio terms (connections x M) */
#define NK_PROF_GRAM 2        /* Gram matrices: lower-triangle flops, (N + M) per entry of the
                                 sample-space Jacobian-row Gram s.s + t.t + (t.t)(s.s), 2 Ns
                                 per entry of the parameter-space S */
#define NK_PROF_CHOL_UPDATE 3 /* Cholesky products: the FP64 flops of the trailing updates
                                 (lower triangle) and, in NK_MIXED, of the panel solves run as
                                 tensor-core products with the inverted diagonal block; summed
                                 over a factorisation of order n, about n^3 / 3 */
#define NK_PROF_CHOL_PANEL 4  /* Cholesky panels: FP64 flops of the diagonal blocks (and their
                                 inverses in NK_MIXED); NK_F64 panel solves; operand slicing */
#define NK_PROF_TRSV 5        /* triangular solves: flops */
#define NK_PROF_JVP_VJP 6     /* Jacobian products J v, J^T g (2 Ns (N + 1)(M + 1) flops each)
                                 and the batched theta = b + W s (2 B N M) */
#define NK_PROF_N 8
nk_status nk_prof_enable(int32_t on);
/* Number of CUDA kernels this library has launched in this process. */
int64_t nk_launch_count(void);
nk_status nk_prof_read(int32_t cls, double *ms /* host */, int64_t *launches /* host */,
                       double *work /* host */);
nk_status nk_prof_read_executed(int32_t cls, double *executed /* host */);
/* The bracketed launches since the last nk_prof_enable, in the order they
 * were enqueued: for entry i (i < max) the class cls[i] and the start and
 * end times t0_ms[i], t1_ms[i] in milliseconds from the start of the first
 * entry (all streams on one clock: the events' device timestamps).  Waits
 * for the events.  *n_out receives the number of entries (which may exceed
 * max; only the first max are written).  All pointers HOST; cls, t0_ms and
 * t1_ms may be NULL when max is 0.  NK_ERR_INVALID_ARG for a NULL n_out or
 * a NULL array with max > 0. */
nk_status nk_prof_trace(int32_t max, int32_t *cls /* host */, double *t0_ms /* host */, double *t1_ms /* host */,
                        int32_t *n_out /* host */);

#ifdef __cplusplus
}
#endif
#endif /* NK_H */
