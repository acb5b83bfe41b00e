/*
 * Plain FP64 CPU oracle for the RBM variational Monte Carlo hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * called from tests/, from __graft_entry__.smoke() and from the CPU-baseline
 * leg of bench.py.  The product library never links, loads or calls it, and
 * it shares no code, header, table or constant with the CUDA path.
 *
 * Everything here is deliberately slow and written as the definitions read:
 * full FP64, one configuration at a time, no blocking, no identities.
 * Configurations (and Metropolis chains) are independent of one another, so
 * when the file is compiled with OpenMP the loop over them may be split over
 * host threads (OMP_NUM_THREADS); each one is still computed by one thread
 * in the order written here, so the results do not depend on the thread
 * count.
 *
 * Parameter vector layout (NetKet 3, Sec. 3.2 "Defining the variational
 * ansatz", Table "tab:nk.models", RBM entry):
 *     theta = [ a (N) ; b (M) ; W (M x N, row-major) ]
 *     ln psi(s) = sum_i a_i s_i + sum_j ln cosh( b_j + sum_i W_ji s_i )
 * Configurations are int8 in {-1,+1}, row-major [batch, N].
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_LN2
#define M_LN2 0.69314718055994530942
#endif

/* ln cosh(x).  For moderate |x| this is the definition itself; for large |x|
 * cosh overflows, so the algebraically equal |x| - ln 2 + log1p(e^{-2|x|}) is
 * used there. */
static double oc_lncosh(double x)
{
    double ax = fabs(x);
    if (ax < 20.0) return log(cosh(x));
    return ax - M_LN2 + log1p(exp(-2.0 * ax));
}

/* Hidden activations theta_j = b_j + sum_i W_ji s_i (the dense layer of the
 * RBM, Sec. 3.2). */
static void oc_hidden(int N, int M, const double *params, const int8_t *s,
                      double *theta)
{
    const double *b = params + N;
    const double *W = params + N + M;
    for (int j = 0; j < M; ++j) {
        double acc = b[j];
        for (int i = 0; i < N; ++i) acc += W[(size_t)j * N + i] * (double)s[i];
        theta[j] = acc;
    }
}

/* ln psi(s) for one configuration (RBM entry of Table "tab:nk.models"). */
static double oc_logpsi_one(int N, int M, const double *params,
                            const int8_t *s, double *theta_scratch)
{
    const double *a = params;
    oc_hidden(N, M, params, s, theta_scratch);
    double lp = 0.0;
    for (int i = 0; i < N; ++i) lp += a[i] * (double)s[i];
    for (int j = 0; j < M; ++j) lp += oc_lncosh(theta_scratch[j]);
    return lp;
}

void oc_logpsi(int N, int M, const double *params, const int8_t *s,
               int64_t B, double *out)
{
#pragma omp parallel
    {
        double *theta = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
#pragma omp for schedule(static)
        for (int64_t k = 0; k < B; ++k)
            out[k] = oc_logpsi_one(N, M, params, s + (size_t)k * N, theta);
        free(theta);
    }
}

/* ln psi(s') - ln psi(s) when the sites in `sites` (n of them) are flipped,
 * given theta = b + W s.  theta' = theta - 2 sum_{i in sites} W_:i s_i is the
 * new dense-layer output; the difference of ln cosh is taken term by term
 * (no product or tanh identity). */
static double oc_log_ratio(int N, int M, const double *params, const int8_t *s,
                           const double *theta, const int *sites, int n)
{
    const double *a = params;
    const double *W = params + N + M;
    double d = 0.0;
    for (int q = 0; q < n; ++q) d += -2.0 * a[sites[q]] * (double)s[sites[q]];
    for (int j = 0; j < M; ++j) {
        double tp = theta[j];
        for (int q = 0; q < n; ++q)
            tp -= 2.0 * W[(size_t)j * N + sites[q]] * (double)s[sites[q]];
        d += oc_lncosh(tp) - oc_lncosh(theta[j]);
    }
    return d;
}

/*
 * Local energy E_loc(s) = sum_{s'} H_{s s'} psi(s')/psi(s)
 * (Sec. 3.3 "Estimating observables", Eq. "eq:local-estimator").
 *
 * The E edges form two classes: the first E - E2 are nearest neighbours
 * <ik> with coupling J, the last E2 next-nearest neighbours <<ik>> with
 * coupling J2 (Sec. 7, Eq. "eq: j1 j2 heisenberg"; E2 = 0 is the plain
 * nearest-neighbour model).  J_e below is the coupling of edge e.
 *
 * kind 0, transverse-field Ising (Sec. 9, Eq. "eq:tf-ising-hamiltonian"):
 *     H = sum_e J_e sz_i sz_k - h sum_i sx_i
 *     diagonal: sum_e J_e s_i s_k;  connected: s^(i) (site i flipped), H = -h.
 * kind 1, Heisenberg in Pauli matrices (Sec. 7, Eq. "eq: j1 j2 heisenberg"):
 *     H = sum_e J_e (sx sx + sy sy + sz sz)
 *     diagonal: sum_e J_e s_i s_k;  connected: for each edge with s_i != s_k,
 *     s^(ik) (both flipped), H = 2 J_e.  With `marshall` set, the sign
 *     rotation prod_{i in A} sz_i of a two-sublattice lattice is folded in:
 *     it negates the element of every edge joining the two sublattices and
 *     keeps that of every edge inside one.  The nearest-neighbour edges are
 *     taken to join the sublattices and the next-nearest ones to stay inside
 *     one (the square lattice and the even ring), so the elements are -2J
 *     and +2 J2.
 * edges: int32 [E, 2].
 */
void oc_local_energy(int N, int M, const double *params, int kind, double J,
                     double J2, double h, int marshall, int E, int E2,
                     const int32_t *edges, const int8_t *s, int64_t B,
                     double *out)
{
    const int E1 = E - E2;
#pragma omp parallel
    {
    double *theta = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
#pragma omp for schedule(dynamic, 4)
    for (int64_t k = 0; k < B; ++k) {
        const int8_t *sk = s + (size_t)k * N;
        oc_hidden(N, M, params, sk, theta);
        double e = 0.0;
        for (int q = 0; q < E; ++q) {
            int i = edges[2 * q], l = edges[2 * q + 1];
            double Je = q < E1 ? J : J2;
            e += Je * (double)sk[i] * (double)sk[l];
        }
        if (kind == 0) {
            for (int i = 0; i < N; ++i) {
                int site[1] = {i};
                e += -h * exp(oc_log_ratio(N, M, params, sk, theta, site, 1));
            }
        } else {
            for (int q = 0; q < E; ++q) {
                int pair[2] = {edges[2 * q], edges[2 * q + 1]};
                if (sk[pair[0]] == sk[pair[1]]) continue;
                double hoff = q < E1 ? (marshall ? -2.0 * J : 2.0 * J) : 2.0 * J2;
                e += hoff * exp(oc_log_ratio(N, M, params, sk, theta, pair, 2));
            }
        }
        out[k] = e;
    }
    free(theta);
    }
}

/*
 * Log-derivatives O_k(s) = d ln psi(s) / d theta_k
 * (Sec. 3.3, Eq. "eq:log-derivative-O"), written out for the RBM:
 *     O_{a_i} = s_i,  O_{b_j} = tanh(theta_j),  O_{W_ji} = tanh(theta_j) s_i.
 * Output O: [B, Np] with Np = N + M + M N, the parameter layout above.
 */
void oc_jacobian(int N, int M, const double *params, const int8_t *s,
                 int64_t B, double *O)
{
    size_t Np = (size_t)N + M + (size_t)M * N;
#pragma omp parallel
    {
    double *theta = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
#pragma omp for schedule(static)
    for (int64_t k = 0; k < B; ++k) {
        const int8_t *sk = s + (size_t)k * N;
        double *row = O + (size_t)k * Np;
        oc_hidden(N, M, params, sk, theta);
        for (int i = 0; i < N; ++i) row[i] = (double)sk[i];
        for (int j = 0; j < M; ++j) {
            double t = tanh(theta[j]);
            row[N + j] = t;
            for (int i = 0; i < N; ++i)
                row[N + M + (size_t)j * N + i] = t * (double)sk[i];
        }
    }
    free(theta);
    }
}

/*
 * Selected columns of the same Jacobian: O[k][c] = O_{cols[c]}(s_k) for
 * every configuration k, with the derivatives of Eq. "eq:log-derivative-O"
 * written out as above.  theta_j is formed, by its definition
 * b_j + sum_i W_ji s_i, only for the hidden units the columns need.
 * Output O: [B, ncols].
 */
void oc_jacobian_cols(int N, int M, const double *params, const int8_t *s,
                      int64_t B, int ncols, const int64_t *cols, double *O)
{
    const double *b = params + N;
    const double *W = params + N + M;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < B; ++k) {
        const int8_t *sk = s + (size_t)k * N;
        for (int c = 0; c < ncols; ++c) {
            int64_t q = cols[c];
            double v;
            if (q < N) {
                v = (double)sk[q];
            } else {
                int64_t j = q < N + M ? q - N : (q - N - M) / N;
                double th = b[j];
                for (int i = 0; i < N; ++i) th += W[(size_t)j * N + i] * (double)sk[i];
                v = tanh(th);
                if (q >= N + M) v *= (double)sk[(q - N - M) % N];
            }
            O[(size_t)k * ncols + c] = v;
        }
    }
}

/*
 * Philox4x64-10 counter-based generator, written from its published
 * definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel
 * random numbers: as easy as 1, 2, 3", SC'11.  Ten rounds; each round takes
 * the two 64x64->128-bit products of words 0 and 2 with the round
 * multipliers, permutes and xors with the round key; the key is advanced by
 * the two Weyl constants between rounds.
 */
static void oc_mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void oc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2],
                      uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t hi0, lo0, hi1, lo1;
        oc_mulhilo64(0xD2E7470EE14C6C93ULL, x0, &hi0, &lo0);
        oc_mulhilo64(0xCA5A826395121157ULL, x2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ x1 ^ k0, n1 = lo1, n2 = hi0 ^ x3 ^ k1, n3 = lo0;
        x0 = n0; x1 = n1; x2 = n2; x3 = n3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout: (word0 = index, word1 = chain, word2 = stream id,
 * word3 = purpose: 0 = Metropolis proposal, 1 = chain initialisation);
 * key = (seed, 0). */
static void oc_draw(uint64_t index, uint64_t chain, uint64_t stream,
                    uint64_t purpose, uint64_t seed, uint64_t y[4])
{
    uint64_t c[4] = {index, chain, stream, purpose};
    uint64_t k[2] = {seed, 0};
    oc_philox4x64_10(c, k, y);
}

/* floor(hi32(y) * n / 2^32): an index in [0, n) from the top 32 bits. */
static int oc_pick(uint64_t y, int n)
{
    return (int)(((y >> 32) * (uint64_t)n) >> 32);
}

/* A uniform double in (0, 1): ((y >> 11) + 1/2) 2^-53. */
static double oc_uniform(uint64_t y)
{
    return ((double)(y >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/*
 * Random initial chain states (the Hilbert-space random_state of Sec. 2.1).
 * rule 0 (unconstrained spins): s_i = +1 iff bit (i mod 256) of the 256-bit
 *   word y0|y1|y2|y3 (y0 lowest) of block floor(i / 256) is set.
 * rules 1, 2 (total S_z = 0, N even): start from N/2 up spins followed by N/2
 *   down spins and shuffle by Fisher-Yates: for i = N-1 .. 1 swap s_i with
 *   s_j, j = pick(y0 of block i, i + 1).
 * Output s: [C, N].
 */
void oc_chain_init(int N, int C, int rule, uint64_t seed, uint32_t stream,
                   int8_t *s)
{
    uint64_t y[4];
    for (int c = 0; c < C; ++c) {
        int8_t *sc = s + (size_t)c * N;
        if (rule == 0) {
            for (int i = 0; i < N; ++i) {
                oc_draw((uint64_t)(i / 256), (uint64_t)c, stream, 1, seed, y);
                int bit = i % 256;
                uint64_t word = y[bit / 64];
                sc[i] = ((word >> (bit % 64)) & 1ULL) ? 1 : -1;
            }
        } else {
            for (int i = 0; i < N; ++i) sc[i] = (i < N / 2) ? 1 : -1;
            for (int i = N - 1; i >= 1; --i) {
                oc_draw((uint64_t)i, (uint64_t)c, stream, 1, seed, y);
                int j = oc_pick(y[0], i + 1);
                int8_t tmp = sc[i]; sc[i] = sc[j]; sc[j] = tmp;
            }
        }
    }
}

/*
 * Metropolis-Hastings chains on |psi|^2 (Sec. 3.4 "Monte Carlo samplers",
 * the acceptance probability P_acc = min(1, P(s')/P(s)) for a symmetric
 * proposal).
 *
 * One sweep is N proposals (the paper's "N_sites intermediate updates" per
 * sample in Sec. 7).  Proposal p of sweep w of this call has global index
 * q = (sweep0 + w) N + p and uses the Philox block (q, chain, stream, 0):
 *   rule 0 (MetropolisLocal): flip site i = pick(y0, N);
 *   rule 1 (MetropolisExchange): swap the spins of edge e = pick(y0, E); if
 *     they are equal the proposal leaves s unchanged and is not a move.
 *   rule 2 (MetropolisHamiltonian of a Heisenberg-type H on these edges):
 *     the configurations connected to s by an off-diagonal element are the
 *     swaps across its n(s) antiparallel edges; s' is the r-th of them in
 *     edge-list order, r = pick(y0, n(s)) (n(s) = 0: not a move).  The
 *     proposal is not symmetric, g(s'|s) = 1/n(s), so the acceptance takes
 *     the correction L(s, s') = ln g(s|s')/g(s'|s) = ln n(s) - ln n(s').
 *   u = uniform(y1); accept iff ln u < 2 [ln psi(s') - ln psi(s)] + L(s, s')
 *   (L = 0 for rules 0 and 1).
 * theta = b + W s is rebuilt from scratch at the start of every sweep and
 * moved by -2 W_:i s_i on each accepted flip.
 *
 * The first n_discard sweeps are thrown away; after each of the next
 * n_samples sweeps the state is written to samples [C, n_samples, N] and
 * ln psi of it (full evaluation) to logpsi_out [C, n_samples].
 *
 * Forced-follow replay: if `forced` is not NULL it holds, for every proposal
 * (layout [C, n_discard + n_samples, N]), the decision of another
 * implementation (0 reject, 1 accept, 2 not a move).  The chain then
 * follows the forced decision.  For every proposal this oracle writes its
 * own decision to decisions_out (same layout, may be NULL) and
 * |2 (ln psi(s') - ln psi(s)) - ln u| to margin_out (may be NULL; 0 for
 * non-moves).  n_accepted[c] counts accepted moves.
 */
/* Number of edges whose two spins differ. */
static int oc_antiparallel(int E, const int32_t *edges, const int8_t *s)
{
    int n = 0;
    for (int e = 0; e < E; ++e) n += s[edges[2 * e]] != s[edges[2 * e + 1]];
    return n;
}

void oc_metropolis(int N, int M, const double *params, int rule, int E,
                   const int32_t *edges, int C, int8_t *s, int64_t sweep0,
                   int n_discard, int n_samples, uint64_t seed, uint32_t stream,
                   int8_t *samples, double *logpsi_out, const uint8_t *forced,
                   uint8_t *decisions_out, double *margin_out,
                   int64_t *n_accepted)
{
    const double *W = params + N + M;
    int n_sweeps = n_discard + n_samples;
#pragma omp parallel
    {
    double *theta = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
    double *scratch = (double *)malloc(sizeof(double) * (size_t)(M > 0 ? M : 1));
    uint64_t y[4];
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < C; ++c) {
        int8_t *sc = s + (size_t)c * N;
        int64_t acc = 0;
        for (int w = 0; w < n_sweeps; ++w) {
            oc_hidden(N, M, params, sc, theta);
            for (int p = 0; p < N; ++p) {
                uint64_t q = (uint64_t)(sweep0 + w) * (uint64_t)N + (uint64_t)p;
                size_t slot = ((size_t)c * n_sweeps + w) * N + p;
                oc_draw(q, (uint64_t)c, stream, 0, seed, y);
                int sites[2], n;
                double corr = 0.0;
                if (rule == 0) {
                    sites[0] = oc_pick(y[0], N);
                    n = 1;
                } else if (rule == 2) {
                    int ns = oc_antiparallel(E, edges, sc);
                    if (ns == 0) {
                        if (decisions_out) decisions_out[slot] = 2;
                        if (margin_out) margin_out[slot] = 0.0;
                        continue;
                    }
                    int r = oc_pick(y[0], ns), e = 0;
                    for (;; ++e)
                        if (sc[edges[2 * e]] != sc[edges[2 * e + 1]] && r-- == 0) break;
                    sites[0] = edges[2 * e];
                    sites[1] = edges[2 * e + 1];
                    n = 2;
                    /* n(s') by counting on the swapped configuration */
                    sc[sites[0]] = (int8_t)-sc[sites[0]];
                    sc[sites[1]] = (int8_t)-sc[sites[1]];
                    int nsp = oc_antiparallel(E, edges, sc);
                    sc[sites[0]] = (int8_t)-sc[sites[0]];
                    sc[sites[1]] = (int8_t)-sc[sites[1]];
                    corr = log((double)ns) - log((double)nsp);
                } else {
                    int e = oc_pick(y[0], E);
                    sites[0] = edges[2 * e];
                    sites[1] = edges[2 * e + 1];
                    n = 2;
                    if (sc[sites[0]] == sc[sites[1]]) {
                        if (decisions_out) decisions_out[slot] = 2;
                        if (margin_out) margin_out[slot] = 0.0;
                        continue;
                    }
                }
                double d = oc_log_ratio(N, M, params, sc, theta, sites, n);
                double lu = log(oc_uniform(y[1]));
                int mine = lu < 2.0 * d + corr;
                if (decisions_out) decisions_out[slot] = (uint8_t)mine;
                if (margin_out) margin_out[slot] = fabs(2.0 * d + corr - lu);
                int take = forced ? (forced[slot] == 1) : mine;
                if (take) {
                    for (int j = 0; j < M; ++j)
                        for (int r = 0; r < n; ++r)
                            theta[j] -= 2.0 * W[(size_t)j * N + sites[r]] *
                                        (double)sc[sites[r]];
                    for (int r = 0; r < n; ++r) sc[sites[r]] = (int8_t)-sc[sites[r]];
                    ++acc;
                }
            }
            if (w >= n_discard) {
                int k = w - n_discard;
                size_t row = (size_t)c * n_samples + k;
                memcpy(samples + row * N, sc, (size_t)N);
                if (logpsi_out)
                    logpsi_out[row] = oc_logpsi_one(N, M, params, sc, scratch);
            }
        }
        if (n_accepted) n_accepted[c] = acc;
    }
    free(theta);
    free(scratch);
    }
}
