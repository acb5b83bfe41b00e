// The complex holomorphic RBM (NetKet 3, Sec. 3.2 with complex parameters)
// and the pieces of time-dependent variational Monte Carlo (Sec. 4.3):
//     ln psi(s) = a.s + sum_j ln cosh(b_j + W_j.s),  a, b, W complex,
// sampled from |psi|^2, with local energies, log-derivatives O = [s, tanh
// theta, tanh theta s^T] (holomorphic, Eq. eq:log-derivative-O) and the
// realified Jacobian whose Gram gives the real embedding of the complex QGT.
//
// Complex numbers are double2 (x = real, y = imaginary part); everything is
// FP64 on CUDA cores.  One warp per chain or sample, hidden units over the
// lanes, theta in shared memory.  Log-ratios are differences of ln cosh term
// by term on the moved activations (no tanh tables): complex ln cosh is cheap
// next to keeping the phase of a running product right.

#include <cuda_runtime.h>

#include "nk_common.cuh"
#include "nk_internal.h"

namespace nk {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cexp(double2 z) {
    const double m = exp(z.x);
    double sn, cs;
    sincos(z.y, &sn, &cs);
    return make_double2(m * cs, m * sn);
}

// ln cosh z = y + ln(1 + e^{-2y}) - ln 2 with y = z or -z, whichever has a
// non-negative real part (cosh is even), so that |e^{-2y}| <= 1.  The
// logarithm of 1 + w takes its modulus through log1p and its argument
// through atan2.
__device__ __forceinline__ double2 clncosh(double2 z) {
    const double2 y = z.x >= 0.0 ? z : make_double2(-z.x, -z.y);
    const double2 w = cexp(make_double2(-2.0 * y.x, -2.0 * y.y));
    const double re = 0.5 * log1p(2.0 * w.x + w.x * w.x + w.y * w.y);
    const double im = atan2(w.y, 1.0 + w.x);
    return make_double2(y.x + re - 0.69314718055994530942, y.y + im);
}

// tanh z = (sinh 2x + i sin 2y) / (cosh 2x + cos 2y), z = x + i y; for |x|
// > 20 it is sign(x) to within e^{-40}.
__device__ __forceinline__ double2 ctanh(double2 z) {
    if (fabs(z.x) > 20.0) return make_double2(z.x > 0.0 ? 1.0 : -1.0, 0.0);
    double s2, c2;
    sincos(2.0 * z.y, &s2, &c2);
    const double d = cosh(2.0 * z.x) + c2;
    return make_double2(sinh(2.0 * z.x) / d, s2 / d);
}

__device__ __forceinline__ double2 warp_csum(double2 v) {
    v.x = warp_sum(v.x);
    v.y = warp_sum(v.y);
    return v;
}

// parameters: interleaved complex [a (N); b (M); W (M x N)]
struct CView {
    const double2 *a, *b, *W;
};
__device__ __forceinline__ CView cview(const double *p, int N, int M) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    return CView{q, q + N, q + N + M};
}

// theta_j = b_j + sum_i W_ji s_i for this lane's units; returns sum_i a_i s_i
// (lane 0 holds it after the reduction).
__device__ __forceinline__ double2 hidden(const CView &v, int N, int M, const int8_t *sv, double2 *th, int lane) {
    for (int j = lane; j < M; j += 32) {
        double2 acc = v.b[j];
        for (int i = 0; i < N; ++i) {
            const double si = (double)sv[i];
            acc.x = fma(v.W[(size_t)j * N + i].x, si, acc.x);
            acc.y = fma(v.W[(size_t)j * N + i].y, si, acc.y);
        }
        th[j] = acc;
    }
    double2 as = make_double2(0.0, 0.0);
    for (int i = lane; i < N; i += 32) as = cadd(as, cscale(v.a[i], (double)sv[i]));
    return warp_csum(as);
}

// ln psi(s') - ln psi(s) for the n sites flipped (term by term on the moved
// activations theta_j - 2 sum W_ji s_i); warp-uniform result.
__device__ __forceinline__ double2 clog_ratio(const CView &v, int N, int M, const int8_t *sv, const double2 *th,
                                              const int *sites, int n, int lane) {
    double2 d = make_double2(0.0, 0.0);
    for (int j = lane; j < M; j += 32) {
        double2 tp = th[j];
        for (int r = 0; r < n; ++r) {
            const double s2 = 2.0 * (double)sv[sites[r]];
            const double2 w = v.W[(size_t)j * N + sites[r]];
            tp.x -= s2 * w.x;
            tp.y -= s2 * w.y;
        }
        d = cadd(d, csub(clncosh(tp), clncosh(th[j])));
    }
    d = warp_csum(d);
    for (int r = 0; r < n; ++r) d = csub(d, cscale(v.a[sites[r]], 2.0 * (double)sv[sites[r]]));
    return d;
}

// ---------------------------------------------------------------- ln psi ---

__global__ void k_crbm_logpsi(int N, int M, const double *__restrict__ p, const int8_t *__restrict__ s, int64_t B,
                              double *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const size_t wb = ((size_t)M * sizeof(double2) + (size_t)N + 15) / 16 * 16;
    double2 *th = reinterpret_cast<double2 *>(sm + warp * wb);
    int8_t *sv = reinterpret_cast<int8_t *>(th + M);
    if (k >= B) return;
    for (int i = lane; i < N; i += 32) sv[i] = s[(size_t)k * N + i];
    __syncwarp();
    const CView v = cview(p, N, M);
    double2 lp = hidden(v, N, M, sv, th, lane);
    __syncwarp();
    double2 acc = make_double2(0.0, 0.0);
    for (int j = lane; j < M; j += 32) acc = cadd(acc, clncosh(th[j]));
    acc = warp_csum(acc);
    lp = cadd(lp, acc);
    if (lane == 0) reinterpret_cast<double2 *>(out)[k] = lp;
}

// ------------------------------------------------------------ Metropolis ---
// Chains on |psi|^2 on the Philox streams of the real RBM: proposal p of
// sweep w uses the block ((sweep0 + w) N + p, chain, stream_id, 0); site or
// edge floor(hi32(y0) n / 2^32), u = ((y1 >> 11) + 1/2) 2^-53, accept iff
// ln u < 2 Re[ln psi(s') - ln psi(s)]; an exchange on equal spins is not a
// move.  theta is rebuilt from scratch at every sweep and moved on accepted
// flips.

struct CSweepArgs {
    int N, M, E, rule, C;
    const double *p;
    const int32_t *edges;
    int8_t *s;
    int64_t sweep0;
    int n_discard, n_samples;
    unsigned long long seed;
    unsigned stream_id;
    int8_t *samples;  // [C][n_samples][N]
    unsigned long long *n_accepted;
};

__global__ void __launch_bounds__(128) k_crbm_sweep(CSweepArgs A) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    const int N = A.N, M = A.M;
    const size_t wb = ((size_t)M * sizeof(double2) + (size_t)N + 15) / 16 * 16;
    double2 *th = reinterpret_cast<double2 *>(sm + warp * wb);
    int8_t *sv = reinterpret_cast<int8_t *>(th + M);
    if (c >= A.C) return;
    for (int i = lane; i < N; i += 32) sv[i] = A.s[(size_t)c * N + i];
    __syncwarp();
    const CView v = cview(A.p, N, M);
    unsigned long long acc = 0;
    for (int w = 0; w < A.n_discard + A.n_samples; ++w) {
        hidden(v, N, M, sv, th, lane);
        __syncwarp();
        const unsigned long long qbase = (unsigned long long)(A.sweep0 + w) * (unsigned long long)N;
        for (int q = 0; q < N; ++q) {
            const Philox4 y = philox4x64_10(qbase + (unsigned long long)q, (unsigned long long)c,
                                            (unsigned long long)A.stream_id, 0ULL, A.seed, 0ULL);
            int sites[2], n;
            if (A.rule == NK_RULE_LOCAL) {
                sites[0] = pick_index(y.v[0], N);
                n = 1;
            } else {
                const int e = pick_index(y.v[0], A.E);
                const int i0 = A.edges[2 * e], k0 = A.edges[2 * e + 1];
                if ((unsigned)i0 >= (unsigned)N || (unsigned)k0 >= (unsigned)N || sv[i0] == sv[k0]) continue;
                sites[0] = i0;
                sites[1] = k0;
                n = 2;
            }
            const double2 d = clog_ratio(v, N, M, sv, th, sites, n, lane);
            const double lu = log(uniform53(y.v[1]));
            if (lu < 2.0 * d.x) {
                for (int j = lane; j < M; j += 32) {
                    double2 t = th[j];
                    for (int r = 0; r < n; ++r) {
                        const double s2 = 2.0 * (double)sv[sites[r]];
                        const double2 wj = v.W[(size_t)j * N + sites[r]];
                        t.x -= s2 * wj.x;
                        t.y -= s2 * wj.y;
                    }
                    th[j] = t;
                }
                __syncwarp();
                if (lane == 0)
                    for (int r = 0; r < n; ++r) sv[sites[r]] = (int8_t)-sv[sites[r]];
                ++acc;
            }
            __syncwarp();
        }
        if (w >= A.n_discard) {
            const size_t row = (size_t)c * A.n_samples + (w - A.n_discard);
            for (int i = lane; i < N; i += 32) A.samples[row * N + i] = sv[i];
        }
        __syncwarp();
    }
    for (int i = lane; i < N; i += 32) A.s[(size_t)c * N + i] = sv[i];
    if (lane == 0 && A.n_accepted) A.n_accepted[c] += acc;
}

// ----------------------------------------------------------- local energy ---
// E_loc(s) = sum_s' H_ss' psi(s')/psi(s) (Eq. eq:local-estimator): diagonal
// sum_e J_e s_i s_k; TFIM: -h e^{dlnpsi} per single flip; Heisenberg: the
// element (+-2 J_e, Marshall sign on the nearest-neighbour class) per
// antiparallel edge.  out: complex [Ns].

struct CElocArgs {
    int N, M, E, E2, kind, marshall;
    double J, J2, h;
    const double *p;
    const int32_t *edges;
    const int8_t *s;
    int64_t Ns;
    double *eloc;
};

__global__ void __launch_bounds__(128) k_crbm_eloc(CElocArgs A) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const int N = A.N, M = A.M, E1 = A.E - A.E2;
    const size_t wb = ((size_t)M * sizeof(double2) + (size_t)N + 15) / 16 * 16;
    double2 *th = reinterpret_cast<double2 *>(sm + warp * wb);
    int8_t *sv = reinterpret_cast<int8_t *>(th + M);
    if (k >= A.Ns) return;
    for (int i = lane; i < N; i += 32) sv[i] = A.s[(size_t)k * N + i];
    __syncwarp();
    const CView v = cview(A.p, N, M);
    hidden(v, N, M, sv, th, lane);
    __syncwarp();
    double diag = 0.0;
    for (int e = lane; e < A.E; e += 32) {
        const int i = A.edges[2 * e], kk = A.edges[2 * e + 1];
        if ((unsigned)i < (unsigned)N && (unsigned)kk < (unsigned)N)
            diag += (e < E1 ? A.J : A.J2) * (double)sv[i] * (double)sv[kk];
    }
    diag = warp_sum(diag);
    double2 off = make_double2(0.0, 0.0);
    if (A.kind == NK_TFIM) {
        for (int i = 0; i < N; ++i) {
            const int site[1] = {i};
            const double2 r = cexp(clog_ratio(v, N, M, sv, th, site, 1, lane));
            off = cadd(off, cscale(r, -A.h));
        }
    } else {
        for (int e = 0; e < A.E; ++e) {
            const int i = A.edges[2 * e], kk = A.edges[2 * e + 1];
            if ((unsigned)i >= (unsigned)N || (unsigned)kk >= (unsigned)N || sv[i] == sv[kk]) continue;
            const int pair[2] = {i, kk};
            const double el = e < E1 ? (A.marshall ? -2.0 * A.J : 2.0 * A.J) : 2.0 * A.J2;
            const double2 r = cexp(clog_ratio(v, N, M, sv, th, pair, 2, lane));
            off = cadd(off, cscale(r, el));
        }
    }
    if (lane == 0) reinterpret_cast<double2 *>(A.eloc)[k] = make_double2(diag + off.x, off.y);
}

// --------------------------------------------------------------- Jacobian ---
// O [Ns][Np] complex: O_a = s, O_b = tanh theta, O_W = tanh theta s^T.
__global__ void k_crbm_jacobian(int N, int M, const double *__restrict__ p, const int8_t *__restrict__ s,
                                int64_t Ns, double *__restrict__ O) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    const size_t wb = ((size_t)M * sizeof(double2) + (size_t)N + 15) / 16 * 16;
    double2 *th = reinterpret_cast<double2 *>(sm + warp * wb);
    int8_t *sv = reinterpret_cast<int8_t *>(th + M);
    if (k >= Ns) return;
    for (int i = lane; i < N; i += 32) sv[i] = s[(size_t)k * N + i];
    __syncwarp();
    const CView v = cview(p, N, M);
    hidden(v, N, M, sv, th, lane);
    __syncwarp();
    for (int j = lane; j < M; j += 32) th[j] = ctanh(th[j]);
    __syncwarp();
    const int64_t Np = (int64_t)N + M + (int64_t)M * N;
    double2 *row = reinterpret_cast<double2 *>(O) + (size_t)k * Np;
    for (int i = lane; i < N; i += 32) row[i] = make_double2((double)sv[i], 0.0);
    for (int j = lane; j < M; j += 32) row[N + j] = th[j];
    for (int64_t q = lane; q < (int64_t)M * N; q += 32) {
        const int j = (int)(q / N), i = (int)(q % N);
        row[N + M + q] = cscale(th[j], (double)sv[i]);
    }
}

// Column means of a complex [rows][cols] matrix: one thread per column.
__global__ void k_ccolmean(int64_t rows, int64_t cols, const double2 *__restrict__ O, double2 *__restrict__ mean) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cols) return;
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t k = 0; k < rows; ++k) acc = cadd(acc, O[(size_t)k * cols + q]);
    mean[q] = cscale(acc, 1.0 / (double)rows);
}

// The realified centred Jacobian R [2 rows][2 cols]: with dO = X + i Y
// (centred), row 2k = [X_k, -Y_k], row 2k + 1 = [Y_k, X_k], so that
// R^T R = Ns [[Re G, -Im G], [Im G, Re G]] for G = dO^H dO / Ns.
__global__ void k_realify(int64_t rows, int64_t cols, const double2 *__restrict__ O, const double2 *__restrict__ mean,
                          double *__restrict__ R) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * cols) return;
    const int64_t k = idx / cols, q = idx % cols;
    const double2 d = csub(O[idx], mean[q]);
    double *r0 = R + (size_t)(2 * k) * (2 * cols), *r1 = r0 + 2 * cols;
    r0[q] = d.x;
    r0[cols + q] = -d.y;
    r1[q] = d.y;
    r1[cols + q] = d.x;
}

// The realified right-hand side of the force: g [2 Ns] with g_2k = Re(E_k -
// Ebar) / Ns, g_2k+1 = Im(E_k - Ebar) / Ns, so that R^T g = [Re f; Im f] for
// f = dO^H (E - Ebar) / Ns.  Ebar: complex mean (emean).
__global__ void k_cforce_g(int64_t Ns, const double2 *__restrict__ e, const double2 *__restrict__ emean,
                           double *__restrict__ g) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ns) return;
    const double2 d = csub(e[k], *emean);
    g[2 * k] = d.x / (double)Ns;
    g[2 * k + 1] = d.y / (double)Ns;
}

// Complex mean and variance of the local energies (one block; fixed order):
// out = [Re mean, Im mean, var = mean |E - Ebar|^2, error sqrt(var / Ns)].
__global__ void k_cstats(int64_t Ns, const double2 *__restrict__ e, double *__restrict__ out) {
    __shared__ double red[3][32];
    double sr = 0.0, si = 0.0;
    for (int64_t k = threadIdx.x; k < Ns; k += blockDim.x) {
        sr += e[k].x;
        si += e[k].y;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sr;
        red[1][threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
        double v = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
        u = warp_sum(u);
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            red[0][0] = u / (double)Ns;
            red[1][0] = v / (double)Ns;
        }
    }
    __syncthreads();
    const double mr = red[0][0], mi = red[1][0];
    __syncthreads();
    double q = 0.0;
    for (int64_t k = threadIdx.x; k < Ns; k += blockDim.x) {
        const double dr = e[k].x - mr, di = e[k].y - mi;
        q += dr * dr + di * di;
    }
    q = warp_sum(q);
    if ((threadIdx.x & 31) == 0) red[2][threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[2][threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            out[0] = mr;
            out[1] = mi;
            out[2] = v / (double)Ns;
            out[3] = sqrt(v / (double)Ns / (double)Ns);
        }
    }
}

// The TDVP right-hand side gamma f from the realified force [Re f; Im f]
// (n complex entries): gamma = -i (real time): [Im f; -Re f]; gamma = -1
// (imaginary time): [-Re f; -Im f].
__global__ void k_tdvp_rhs(int64_t n, const double *__restrict__ f, int real_time, double *__restrict__ rhs) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double fr = f[q], fi = f[n + q];
    rhs[q] = real_time ? fi : -fr;
    rhs[n + q] = real_time ? -fr : -fi;
}

// theta (interleaved complex, n entries) <- base + h x with x realified
// [Re; Im]; base == null reads as zero.
__global__ void k_caxpy_realified(int64_t n, const double *base, double h, const double *__restrict__ x,
                                  double *out) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double b0 = base ? base[2 * q] : 0.0, b1 = base ? base[2 * q + 1] : 0.0;
    out[2 * q] = b0 + h * x[q];
    out[2 * q + 1] = b1 + h * x[n + q];
}

size_t cwarp_bytes(int N, int M) { return ((size_t)M * sizeof(double2) + (size_t)N + 15) / 16 * 16; }

}  // namespace

size_t crbm_smem_per_warp(int N, int M) { return cwarp_bytes(N, M); }

cudaError_t launch_crbm_logpsi(int N, int M, const double *p, const int8_t *s, int64_t B, double *out,
                               cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const size_t smem = 4 * cwarp_bytes(N, M);
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_crbm_logpsi);
    if (e != cudaSuccess) return e;
    (k_crbm_logpsi<<<nblk(B, 4), 128, smem, st>>>(N, M, p, s, B, out), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_crbm_sweep(int N, int M, const double *p, int rule, int E, const int32_t *edges, int C, int8_t *s,
                              int64_t sweep0, int n_discard, int n_samples, uint64_t seed, uint32_t stream_id,
                              int8_t *samples, unsigned long long *n_accepted, cudaStream_t st) {
    if (C <= 0) return cudaSuccess;
    CSweepArgs a{N, M, E, rule, C, p, edges, s, sweep0, n_discard, n_samples, seed, stream_id, samples, n_accepted};
    const size_t smem = 4 * cwarp_bytes(N, M);
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_crbm_sweep);
    if (e != cudaSuccess) return e;
    const int slot = prof_begin(NK_PROF_SWEEP, st);
    (k_crbm_sweep<<<nblk(C, 4), 128, smem, st>>>(a), nk::note_launch());
    prof_end(slot, st, (double)C * (n_discard + n_samples) * N * (double)M);
    return cudaGetLastError();
}

cudaError_t launch_crbm_eloc(int N, int M, const double *p, const nk_ham *ham, const int8_t *s, int64_t Ns,
                             double *eloc, cudaStream_t st) {
    if (Ns <= 0) return cudaSuccess;
    CElocArgs a{N, M, ham->n_edges, ham->n_edges2, ham->kind, ham->marshall, ham->J, ham->J2, ham->h,
                p, ham->edges, s, Ns, eloc};
    const size_t smem = 4 * cwarp_bytes(N, M);
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_crbm_eloc);
    if (e != cudaSuccess) return e;
    const int slot = prof_begin(NK_PROF_ELOC, st);
    (k_crbm_eloc<<<nblk(Ns, 4), 128, smem, st>>>(a), nk::note_launch());
    prof_end(slot, st, (double)Ns * (ham->kind == NK_TFIM ? N : 0.5 * ham->n_edges) * (double)M);
    return cudaGetLastError();
}

cudaError_t launch_crbm_jacobian(int N, int M, const double *p, const int8_t *s, int64_t Ns, double *O,
                                 cudaStream_t st) {
    if (Ns <= 0) return cudaSuccess;
    const size_t smem = 4 * cwarp_bytes(N, M);
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_crbm_jacobian);
    if (e != cudaSuccess) return e;
    (k_crbm_jacobian<<<nblk(Ns, 4), 128, smem, st>>>(N, M, p, s, Ns, O), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_crealify(int64_t rows, int64_t cols, const double *O, double *mean, double *R, cudaStream_t st) {
    (k_ccolmean<<<nblk(cols, 128), 128, 0, st>>>(rows, cols, reinterpret_cast<const double2 *>(O),
                                                 reinterpret_cast<double2 *>(mean)), nk::note_launch());
    (k_realify<<<nblk(rows * cols, 256), 256, 0, st>>>(rows, cols, reinterpret_cast<const double2 *>(O),
                                                       reinterpret_cast<const double2 *>(mean), R), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_cstats(int64_t Ns, const double *e, double *out4, cudaStream_t st) {
    (k_cstats<<<1, 1024, 0, st>>>(Ns, reinterpret_cast<const double2 *>(e), out4), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_cforce_g(int64_t Ns, const double *e, const double *stats4, double *g, cudaStream_t st) {
    (k_cforce_g<<<nblk(Ns, 256), 256, 0, st>>>(Ns, reinterpret_cast<const double2 *>(e),
                                               reinterpret_cast<const double2 *>(stats4), g), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_tdvp_rhs(int64_t n, const double *f, int real_time, double *rhs, cudaStream_t st) {
    (k_tdvp_rhs<<<nblk(n, 256), 256, 0, st>>>(n, f, real_time, rhs), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_caxpy_realified(int64_t n, const double *base, double h, const double *x, double *out,
                                   cudaStream_t st) {
    (k_caxpy_realified<<<nblk(n, 256), 256, 0, st>>>(n, base, h, x, out), nk::note_launch());
    return cudaGetLastError();
}

}  // namespace nk
