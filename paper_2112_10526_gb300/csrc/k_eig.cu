// Symmetric eigendecomposition for the SVD solvers of the SR system (NetKet
// 3, Sec. 3.5: non-iterative solvers whose stability is controlled by
// suppressing small singular values).
//
// Cyclic two-sided Jacobi (Jacobi 1846; the symmetric Schur rotation and the
// cyclic sweep as in Golub & Van Loan, "Matrix Computations", Sec. 8.5),
// with the parallel round-robin ("tournament") ordering of Brent & Luk
// (1985): in each of the m - 1 rounds of a sweep (m = n rounded up to even)
// the indices form m / 2 disjoint pairs, so all their rotations are
// computed and applied at once: the row rotation A <- J^T A, then the column
// rotation A <- A J together with V <- V J.  A sweep rotates every pair once;
// sweeps stop when the off-diagonal part is below tol times the Frobenius
// norm.  The whole decomposition is one cooperative launch with two grid
// syncs per round.
// Everything is FP64 on CUDA cores: Jacobi's rotations keep the small
// eigenvalues to high relative accuracy, which the cutoff of the solver
// needs.

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "nk_common.cuh"
#include "nk_internal.h"

namespace nk {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Pair i of round r among m players (m even): player m - 1 stays fixed and
// meets r; the others meet (r + i) and (r - i) modulo m - 1.
__device__ __forceinline__ void round_pair(int m, int r, int i, int &p, int &q) {
    const int L = m - 1;
    if (i == 0) {
        p = r;
        q = L;
    } else {
        p = (r + i) % L;
        q = (r - i + L) % L;
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

// A[j][i] <- A[i][j] for j < i (the upper triangle from the lower).
__global__ void k_symmetrize_lower(int64_t n, double *__restrict__ A) {
    const int64_t i = blockIdx.y * 32 + threadIdx.y, j = blockIdx.x * 32 + threadIdx.x;
    if (i < n && j < i) A[(size_t)j * n + i] = A[(size_t)i * n + j];
}

__global__ void k_identity(int64_t n, double *__restrict__ V) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n * n) V[idx] = (idx / n == idx % n) ? 1.0 : 0.0;
}

__global__ void k_diag(int64_t n, const double *__restrict__ A, double *__restrict__ w) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) w[i] = A[(size_t)i * n + i];
}

// Largest eigenvalue (the cutoff's reference) by a one-block max reduction.
__global__ void k_max(int64_t n, const double *__restrict__ w, double *__restrict__ out) {
    __shared__ double red[32];
    double m = -1e308;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, w[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -1e308;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) *out = v;
    }
}

// z_k <- z_k / w_k^power for w_k > rcond max(w), else 0 (power 1: the
// parameter-space pseudo-inverse; 2: the sample-space form).
__global__ void k_spectral_filter(int64_t n, const double *__restrict__ w, const double *__restrict__ wmax,
                                  double rcond, int power, double *__restrict__ z, int *__restrict__ kept) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double cut = rcond * *wmax;
    const bool keep = w[k] > cut && w[k] > 0.0;
    z[k] = keep ? z[k] / (power == 2 ? w[k] * w[k] : w[k]) : 0.0;
    if (keep && kept) atomicAdd(kept, 1);
}

namespace cg = cooperative_groups;

// All sweeps in one cooperative launch (every CTA resident).  Per sweep the
// relative off-diagonal norm is summed from per-CTA partials in a fixed order
// (every CTA forms the same total, so all take the same decision); per
// round, phase A: CTA b rotates the rows p, q of its pairs b, b + G, ... (it
// alone touches those rows, so it computes their angles first), then a grid
// sync; phase B: every thread rotates the columns p, q of A and V of one
// (row, pair) at a time, then a grid sync.  The arithmetic of each rotation
// is the symmetric Schur rotation of Golub & Van Loan: the 2 x 2 block's
// off-diagonal entry is annihilated.
__global__ void __launch_bounds__(256) k_jacobi_coop(double *__restrict__ A, double *__restrict__ V, int64_t n,
                                                     int m, int max_sweeps, double tol, double2 *__restrict__ cs,
                                                     double2 *__restrict__ partial, double *__restrict__ out) {
    cg::grid_group grid = cg::this_grid();
    __shared__ double red[2][8];
    __shared__ double2 rot;
    const int G = gridDim.x, P = m / 2;
    const int64_t nthreads = (int64_t)G * blockDim.x, gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int sweep = 0;
    double rel = 0.0;
    for (;; ++sweep) {
        // the norms, from this CTA's rows
        double off = 0.0, dia = 0.0;
        for (int64_t row = blockIdx.x; row < n; row += G)
            for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                const double x = A[(size_t)row * n + j];
                if (j == row)
                    dia += x * x;
                else
                    off += x * x;
            }
        off = warp_sum(off);
        dia = warp_sum(dia);
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = off;
            red[1][threadIdx.x >> 5] = dia;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double u = 0.0, v = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) u += red[0][w], v += red[1][w];
            partial[blockIdx.x] = make_double2(u, v);
        }
        grid.sync();
        double u = 0.0, v = 0.0;
        for (int b = threadIdx.x; b < G; b += blockDim.x) u += partial[b].x, v += partial[b].y;
        u = warp_sum(u);
        v = warp_sum(v);
        __syncthreads();
        if ((threadIdx.x & 31) == 0) {
            red[0][threadIdx.x >> 5] = u;
            red[1][threadIdx.x >> 5] = v;
        }
        __syncthreads();
        double tot_off = 0.0, tot_dia = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot_off += red[0][w], tot_dia += red[1][w];
        rel = tot_off + tot_dia > 0.0 ? sqrt(tot_off / (tot_off + tot_dia)) : 0.0;
        grid.sync();  // every CTA has read the partials before they are rewritten
        if (rel <= tol || sweep == max_sweeps) break;
        for (int r = 0; r < m - 1; ++r) {
            for (int i = blockIdx.x; i < P; i += G) {
                int p, q;
                round_pair(m, r, i, p, q);
                if (threadIdx.x == 0) {
                    double c = 1.0, s = 0.0;
                    if (q < n) {
                        const double apq = A[(size_t)p * n + q];
                        if (apq != 0.0) {
                            const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                            const double tau = (aqq - app) / (2.0 * apq);
                            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                            c = 1.0 / sqrt(1.0 + t * t);
                            s = t * c;
                        }
                    }
                    rot = make_double2(c, s);
                    cs[i] = rot;
                }
                __syncthreads();
                const double2 rr = rot;
                if (q < n && rr.y != 0.0) {
                    double *ap = A + (size_t)p * n, *aq = A + (size_t)q * n;
                    for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
                        const double x = ap[j], y = aq[j];
                        ap[j] = rr.x * x - rr.y * y;
                        aq[j] = rr.y * x + rr.x * y;
                    }
                }
                __syncthreads();
            }
            grid.sync();
            for (int64_t idx = gtid; idx < (int64_t)P * n; idx += nthreads) {
                const int i = (int)(idx % P);
                const int64_t row = idx / P;
                int p, q;
                round_pair(m, r, i, p, q);
                const double2 rr = cs[i];
                if (q >= n || rr.y == 0.0) continue;
                double *a = A + (size_t)row * n, *vv = V + (size_t)row * n;
                const double x = a[p], y = a[q];
                a[p] = rr.x * x - rr.y * y;
                a[q] = rr.y * x + rr.x * y;
                const double vx = vv[p], vy = vv[q];
                vv[p] = rr.x * vx - rr.y * vy;
                vv[q] = rr.y * vx + rr.x * vy;
            }
            grid.sync();
        }
    }
    if (gtid == 0) {
        out[0] = (double)sweep;
        out[1] = rel;
    }
}

// The workspace: rotation (c, s) and index pair per pair of a round, and the
// per-row partial norms, each sub-array starting on a 256-byte boundary (the
// double2 arrays need 16-byte alignment for their vector loads and stores).
struct EigWs {
    double2 *cs;
    int2 *pq;
    double2 *partial;
};

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }

EigWs carve_eig(void *ws, int64_t n) {
    const int64_t m = n + (n & 1);
    char *p = static_cast<char *>(ws);
    EigWs w;
    w.cs = reinterpret_cast<double2 *>(p);
    p += align256((size_t)(m / 2) * sizeof(double2));
    w.pq = reinterpret_cast<int2 *>(p);
    p += align256((size_t)(m / 2) * sizeof(int2));
    w.partial = reinterpret_cast<double2 *>(p);
    return w;
}

}  // namespace

size_t eig_ws_bytes(int64_t n) {
    const int64_t m = n + (n & 1);
    return align256((size_t)(m / 2) * sizeof(double2)) + align256((size_t)(m / 2) * sizeof(int2)) +
           align256((size_t)n * sizeof(double2)) + 256;
}

cudaError_t launch_jacobi_coop(double *A, double *V, int64_t n, int max_sweeps, double tol, void *ws, double *out2,
                               cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_coop, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm > 8) per_sm = 8;
    int m = (int)(n + (n & 1));
    int G = sms * per_sm;
    if (G > m / 2) G = m / 2 > 0 ? m / 2 : 1;  // no more CTAs than the row phase has pairs
    if (G < 1) return cudaErrorInvalidConfiguration;
    const EigWs w = carve_eig(ws, n);
    double2 *cs = w.cs;
    double2 *partial = w.partial;  // n >= G entries (G <= m / 2 <= n)
    void *args[] = {&A, &V, &n, &m, &max_sweeps, &tol, &cs, &partial, &out2};
    e = cudaLaunchCooperativeKernel((const void *)k_jacobi_coop, dim3(G), dim3(256), args, 0, st);
    nk::note_launch();
    return e;
}

cudaError_t launch_symmetrize_lower(int64_t n, double *A, cudaStream_t st) {
    (k_symmetrize_lower<<<dim3(nblk(n, 32), nblk(n, 32)), dim3(32, 32), 0, st>>>(n, A), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_identity(int64_t n, double *V, cudaStream_t st) {
    (k_identity<<<nblk(n * n, 256), 256, 0, st>>>(n, V), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_eig_diag(int64_t n, const double *A, double *w, double *wmax, cudaStream_t st) {
    (k_diag<<<nblk(n, 256), 256, 0, st>>>(n, A, w), nk::note_launch());
    (k_max<<<1, 1024, 0, st>>>(n, w, wmax), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_spectral_filter(int64_t n, const double *w, const double *wmax, double rcond, int power,
                                   double *z, int *kept, cudaStream_t st) {
    (k_spectral_filter<<<nblk(n, 256), 256, 0, st>>>(n, w, wmax, rcond, power, z, kept), nk::note_launch());
    return cudaGetLastError();
}

}  // namespace nk
