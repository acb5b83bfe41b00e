// Symmetric eigendecomposition for the SVD solvers of the SR system (NetKet
// 3, Sec. 3.5: non-iterative solvers whose stability is controlled by
// suppressing small singular values).
//
// Cyclic two-sided Jacobi (Jacobi 1846; the symmetric Schur rotation and the
// cyclic sweep as in Golub & Van Loan, "Matrix Computations", Sec. 8.5),
// with the parallel round-robin ("tournament") ordering of Brent & Luk
// (1985): in each of the m - 1 rounds of a sweep (m = n rounded up to even)
// the indices form m / 2 disjoint pairs, so all their rotations are
// computed and applied at once.  A round is three launches: the rotation
// angles of the pairs, the row rotation A <- J^T A, and the column rotation
// A <- A J together with V <- V J.  A sweep rotates every pair once; sweeps
// stop when the off-diagonal part is below tol times the Frobenius norm.
// Everything is FP64 on CUDA cores: Jacobi's rotations keep the small
// eigenvalues to high relative accuracy, which the cutoff of the solver
// needs.

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

// Rotation (c, s) of pair i that annihilates A[p][q] (Golub & Van Loan, the
// symmetric Schur decomposition of a 2 x 2 block).  Indices >= n (the padding
// of odd n) give the identity.
__global__ void k_jacobi_angles(const double *__restrict__ A, int64_t n, int m, int r, double2 *__restrict__ cs,
                                int2 *__restrict__ pq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m / 2) return;
    int p, q;
    round_pair(m, r, i, p, q);
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
    cs[i] = make_double2(c, s);
    pq[i] = make_int2(p, q);
}

// A <- J^T A on rows p, q of every pair: [A_pj, A_qj] <- [c A_pj - s A_qj,
// s A_pj + c A_qj].  blockIdx.y = pair, x over columns.
__global__ void k_jacobi_rows(double *__restrict__ A, int64_t n, const double2 *__restrict__ cs,
                              const int2 *__restrict__ pq) {
    const int i = blockIdx.y;
    const int2 idx = pq[i];
    if (idx.y >= n) return;
    const double2 r = cs[i];
    if (r.y == 0.0) return;
    double *ap = A + (size_t)idx.x * n, *aq = A + (size_t)idx.y * n;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const double x = ap[j], y = aq[j];
        ap[j] = r.x * x - r.y * y;
        aq[j] = r.y * x + r.x * y;
    }
}

// A <- A J and V <- V J on columns p, q of every pair.  blockIdx.y = pair, x
// over rows.
__global__ void k_jacobi_cols(double *__restrict__ A, double *__restrict__ V, int64_t n,
                              const double2 *__restrict__ cs, const int2 *__restrict__ pq) {
    const int i = blockIdx.y;
    const int2 idx = pq[i];
    if (idx.y >= n) return;
    const double2 r = cs[i];
    if (r.y == 0.0) return;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        double *a = A + (size_t)row * n, *v = V + (size_t)row * n;
        const double x = a[idx.x], y = a[idx.y];
        a[idx.x] = r.x * x - r.y * y;
        a[idx.y] = r.y * x + r.x * y;
        const double vx = v[idx.x], vy = v[idx.y];
        v[idx.x] = r.x * vx - r.y * vy;
        v[idx.y] = r.y * vx + r.x * vy;
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

// partial[b] = (sum of squares off the diagonal, on the diagonal) of the
// rows of block b.
__global__ void k_offdiag_partial(const double *__restrict__ A, int64_t n, double2 *__restrict__ partial) {
    __shared__ double red[2][32];
    double off = 0.0, dia = 0.0;
    const int64_t row = blockIdx.x;
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
    if (threadIdx.x < 32) {
        double u = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
        double v = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
        u = warp_sum(u);
        v = warp_sum(v);
        if (threadIdx.x == 0) partial[row] = make_double2(u, v);
    }
}

__global__ void k_offdiag_final(int64_t n, const double2 *__restrict__ partial, double *__restrict__ out) {
    __shared__ double red[2][32];
    double off = 0.0, dia = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        off += partial[i].x;
        dia += partial[i].y;
    }
    off = warp_sum(off);
    dia = warp_sum(dia);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = off;
        red[1][threadIdx.x >> 5] = dia;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double u = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
        double v = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
        u = warp_sum(u);
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            out[0] = u;
            out[1] = v;
        }
    }
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

cudaError_t launch_jacobi_sweep(double *A, double *V, int64_t n, void *ws, cudaStream_t st) {
    const int m = (int)(n + (n & 1));
    const EigWs w = carve_eig(ws, n);
    double2 *cs = w.cs;
    int2 *pq = w.pq;
    const unsigned tx = (unsigned)(n < 256 ? 128 : 256);
    const unsigned gx = (unsigned)((n + tx - 1) / tx);
    for (int r = 0; r < m - 1; ++r) {
        (k_jacobi_angles<<<nblk(m / 2, 128), 128, 0, st>>>(A, n, m, r, cs, pq), nk::note_launch());
        (k_jacobi_rows<<<dim3(gx, (unsigned)(m / 2)), tx, 0, st>>>(A, n, cs, pq), nk::note_launch());
        (k_jacobi_cols<<<dim3(gx, (unsigned)(m / 2)), tx, 0, st>>>(A, V, n, cs, pq), nk::note_launch());
    }
    return cudaGetLastError();
}

cudaError_t launch_symmetrize_lower(int64_t n, double *A, cudaStream_t st) {
    (k_symmetrize_lower<<<dim3(nblk(n, 32), nblk(n, 32)), dim3(32, 32), 0, st>>>(n, A), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_identity(int64_t n, double *V, cudaStream_t st) {
    (k_identity<<<nblk(n * n, 256), 256, 0, st>>>(n, V), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_offdiag_norms(const double *A, int64_t n, void *ws, double *out2, cudaStream_t st) {
    double2 *partial = carve_eig(ws, n).partial;
    (k_offdiag_partial<<<(unsigned)n, 256, 0, st>>>(A, n, partial), nk::note_launch());
    (k_offdiag_final<<<1, 1024, 0, st>>>(n, partial, out2), nk::note_launch());
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
