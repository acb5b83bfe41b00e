// FP64 linear algebra of the VMC step: sample statistics, Jacobian products
// (vjp / jvp, App. B.1), the stored centred Jacobian, QGT products and
// Gram matrices (App. B.2 / B.3), blocked Cholesky and triangular solves
// (Sec. 3.5, direct solver), and the CG / SGD vector kernels.
//
// Every reduction runs in a fixed order (split-K partials summed in split
// order, tree reductions with a fixed shape), so results are bitwise
// reproducible from run to run.

#include <cuda_runtime.h>

#include "nk_common.cuh"
#include "nk_internal.h"

namespace nk {

namespace {

// ------------------------------------------------------ tile GEMM engine ---
// C(m, n) = sum_{k in split} A(m, k) B(n, k): 64 x 64 tile per block, 256
// threads with 4 x 4 outputs, K staged 16 at a time in shared memory.  The
// loaders say whether k (kContig = true) or m/n is the contiguous index in
// memory so that the staging loads coalesce either way.

template <class LA, class LB, class EP>
__global__ void __launch_bounds__(256) k_gemm64(int64_t Md, int64_t Nd, int64_t Kd, int64_t kchunk,
                                                LA la, LB lb, EP ep) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    if (!ep.active(m0, n0)) return;
    const int split = blockIdx.z;
    const int64_t kb = (int64_t)split * kchunk;
    const int64_t ke = kb + kchunk < Kd ? kb + kchunk : Kd;
    double acc[4][4] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            int kk, r;
            if (LA::kContig) {
                kk = e & 15;
                r = e >> 4;
            } else {
                r = e & 63;
                kk = e >> 6;
            }
            const int64_t k = k0 + kk;
            As[kk][r] = (m0 + r < Md && k < ke) ? la(m0 + r, k) : 0.0;
            if (LB::kContig) {
                kk = e & 15;
                r = e >> 4;
            } else {
                r = e & 63;
                kk = e >> 6;
            }
            const int64_t k2 = k0 + kk;
            Bs[kk][r] = (n0 + r < Nd && k2 < ke) ? lb(n0 + r, k2) : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                av[u] = As[kk][ty * 4 + u];
                bv[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t m = m0 + ty * 4 + u;
        if (m >= Md) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t n = n0 + tx * 4 + v;
            if (n < Nd) ep(m, n, split, acc[u][v]);
        }
    }
}

template <class LA, class LB, class EP>
cudaError_t gemm64(int64_t Md, int64_t Nd, int64_t Kd, int splits, LA la, LB lb, EP ep,
                   cudaStream_t st) {
    if (Md <= 0 || Nd <= 0) return cudaSuccess;
    if (splits < 1) splits = 1;
    int64_t kchunk = (Kd + splits - 1) / splits;
    kchunk = (kchunk + 15) / 16 * 16;
    if (kchunk < 16) kchunk = 16;
    dim3 grid((unsigned)((Nd + 63) / 64), (unsigned)((Md + 63) / 64), (unsigned)splits);
    (k_gemm64<<<grid, 256, 0, st>>>(Md, Nd, Kd, kchunk, la, lb, ep), nk::note_launch());
    return cudaGetLastError();
}

// -------------------------------------------------------- vjp: J^T g -------
// Augmented GEMM P[j][i] = sum_k A'(k, j) g_k B'(k, i) with A' = [T, 1] and
// B' = [S, 1]: P[j<M][i<N] is the W block, P[j][N] the b block and P[M][i]
// the a block of J^T g.

struct VjpA {
    static constexpr bool kContig = false;
    const double *T, *g, *shift;
    double scale;
    int M;
    __device__ double operator()(int64_t j, int64_t k) const {
        const double gk = scale * (g[k] - (shift ? *shift : 0.0));
        return (j < M ? T[(size_t)k * M + j] : 1.0) * gk;
    }
};

struct AugS_kn {  // B'(i, k) = s_ki (i < N) or 1, i contiguous
    static constexpr bool kContig = false;
    const int8_t *s;
    int N;
    __device__ double operator()(int64_t i, int64_t k) const {
        return i < N ? (double)s[(size_t)k * N + i] : 1.0;
    }
};

struct EpPartial {
    double *P;
    int64_t ld, plane;
    __device__ bool active(int64_t, int64_t) const { return true; }
    __device__ void operator()(int64_t m, int64_t n, int split, double v) const {
        P[(size_t)split * plane + (size_t)m * ld + n] = v;
    }
};

__global__ void k_vjp_reduce(int N, int M, int splits, const double *__restrict__ P,
                             double *__restrict__ out) {
    const int64_t plane = (int64_t)(M + 1) * (N + 1);
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= plane) return;
    const int j = (int)(idx / (N + 1)), i = (int)(idx % (N + 1));
    if (j == M && i == N) return;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += P[(size_t)sp * plane + idx];
    if (j == M)
        out[i] = s;
    else if (i == N)
        out[N + j] = s;
    else
        out[N + M + (size_t)j * N + i] = s;
}

int vjp_splits(int N, int M, int64_t Ns) {
    const int64_t tiles = ((M + 1 + 63) / 64) * ((N + 1 + 63) / 64);
    int64_t sp = (1216 + tiles - 1) / tiles;  // ~8 blocks per SM on 152 SMs
    const int64_t maxsp = (Ns + 255) / 256;   // at least 256 samples per split
    if (sp > maxsp) sp = maxsp;
    if (sp < 1) sp = 1;
    return (int)sp;
}

// --------------------------------------------------------- jvp: J v --------
// U[k][j] = sum_i B'(k, i) V'(j, i) with V' = [[V_W, v_b], [v_a, 0]], then
// w_k = sum_j A'(k, j) U[k][j].

struct AugS_k {  // A(k, i) = s_ki or 1, i (the K index) contiguous
    static constexpr bool kContig = true;
    const int8_t *s;
    int N;
    __device__ double operator()(int64_t k, int64_t i) const {
        return i < N ? (double)s[(size_t)k * N + i] : 1.0;
    }
};

struct VAug {
    static constexpr bool kContig = true;
    const double *v;
    int N, M;
    __device__ double operator()(int64_t j, int64_t i) const {
        if (j < M) return i < N ? v[N + M + (size_t)j * N + i] : v[N + j];
        return i < N ? v[i] : 0.0;
    }
};

struct EpStore {
    double *C;
    int64_t ld;
    __device__ bool active(int64_t, int64_t) const { return true; }
    __device__ void operator()(int64_t m, int64_t n, int, double v) const {
        C[(size_t)m * ld + n] = v;
    }
};

__global__ void k_rowdot_aug(int M, int64_t Ns, const double *__restrict__ T,
                             const double *__restrict__ U, double *__restrict__ w) {
    const int lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= Ns) return;
    double acc = 0.0;
    for (int j = lane; j <= M; j += 32)
        acc += (j < M ? T[(size_t)k * M + j] : 1.0) * U[(size_t)k * (M + 1) + j];
    acc = warp_sum(acc);
    if (lane == 0) w[k] = acc;
}

// ------------------------------------------------------- Jacobian rows -----

__global__ void k_jacobian_rows(int N, int M, const int8_t *__restrict__ s,
                                const double *__restrict__ T, int64_t row0, int64_t rows,
                                const double *__restrict__ mean, double *__restrict__ O) {
    const int64_t Np = (int64_t)N + M + (int64_t)M * N;
    const int64_t r = blockIdx.y;
    if (r >= rows) return;
    const int64_t k = row0 + r;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < Np;
         p += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (p < N)
            v = (double)s[(size_t)k * N + p];
        else if (p < N + M)
            v = T[(size_t)k * M + (p - N)];
        else {
            const int64_t q = p - N - M;
            const int64_t j = q / N, i = q % N;
            v = T[(size_t)k * M + j] * (double)s[(size_t)k * N + i];
        }
        if (mean) v -= mean[p];
        O[(size_t)r * Np + p] = v;
    }
}

// ------------------------------------------------------------- GEMV -------

__global__ void k_gemv_rows(const double *__restrict__ A, int64_t rows, int64_t cols,
                            const double *__restrict__ x, double *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    double acc = 0.0;
    for (int64_t c = lane; c < cols; c += 32) acc += A[(size_t)r * cols + c] * x[c];
    acc = warp_sum(acc);
    if (lane == 0) y[r] = acc;
}

constexpr int kGemvTRows = 256;

// partial[b][c] = sum over rows of chunk b of A[r][c] x[r]
__global__ void k_gemv_t_partial(const double *__restrict__ A, int64_t rows, int64_t cols,
                                 const double *__restrict__ x, double *__restrict__ partial) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * kGemvTRows;
    if (c >= cols) return;
    const int64_t r1 = r0 + kGemvTRows < rows ? r0 + kGemvTRows : rows;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) acc += A[(size_t)r * cols + c] * x[r];
    partial[(size_t)blockIdx.y * cols + c] = acc;
}

__global__ void k_sum_partials(int64_t cols, int nparts, const double *__restrict__ partial,
                               double scale, double *__restrict__ y) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double acc = 0.0;
    for (int b = 0; b < nparts; ++b) acc += partial[(size_t)b * cols + c];
    y[c] = scale * acc;
}

// ----------------------------------------------------------- SYRK (J^T J) --

struct ColMajorA {  // A(p, k) = dJ[k][p], p contiguous
    static constexpr bool kContig = false;
    const double *A;
    int64_t ld;
    __device__ double operator()(int64_t p, int64_t k) const { return A[(size_t)k * ld + p]; }
};

struct EpSyrk {
    double *C;
    int64_t n;
    double scale, eps;
    __device__ bool active(int64_t m0, int64_t n0) const { return n0 <= m0 + 63; }
    __device__ void operator()(int64_t m, int64_t q, int, double v) const {
        if (q > m) return;
        const double r = v * scale + (m == q ? eps : 0.0);
        C[(size_t)m * n + q] = r;
        C[(size_t)q * n + m] = r;
    }
};

// ---------------------------------------------------- sample-space Gram ---
// K_raw[k][l] = g_s + g_t + g_t g_s with g_s = s_k.s_l (exact integer) and
// g_t = t_k.t_l (FP64): the Gram of the Jacobian rows O_k = [s_k, t_k,
// t_k (x) s_k] without forming them.

__global__ void __launch_bounds__(256) k_gram_raw(int N, int M, int64_t Ns,
                                                  const int8_t *__restrict__ s,
                                                  const double *__restrict__ T,
                                                  double *__restrict__ K) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    if (n0 > m0 + 63) return;  // lower triangle of tiles only
    int gs[4][4] = {};
    double gt[4][4] = {};
    for (int i0 = 0; i0 < N; i0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            const int kk = e & 15, r = e >> 4;
            const int i = i0 + kk;
            As[kk][r] = (m0 + r < Ns && i < N) ? (double)s[(size_t)(m0 + r) * N + i] : 0.0;
            Bs[kk][r] = (n0 + r < Ns && i < N) ? (double)s[(size_t)(n0 + r) * N + i] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    gs[u][v] += (int)As[kk][ty * 4 + u] * (int)Bs[kk][tx * 4 + v];
        __syncthreads();
    }
    for (int j0 = 0; j0 < M; j0 += 16) {
        for (int e = threadIdx.x; e < 1024; e += 256) {
            const int kk = e & 15, r = e >> 4;
            const int j = j0 + kk;
            As[kk][r] = (m0 + r < Ns && j < M) ? T[(size_t)(m0 + r) * M + j] : 0.0;
            Bs[kk][r] = (n0 + r < Ns && j < M) ? T[(size_t)(n0 + r) * M + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                av[u] = As[kk][ty * 4 + u];
                bv[u] = Bs[kk][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) gt[u][v] = fma(av[u], bv[v], gt[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int64_t k = m0 + ty * 4 + u;
        if (k >= Ns) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int64_t l = n0 + tx * 4 + v;
            if (l >= Ns || l > k) continue;
            const double g = (double)gs[u][v] + gt[u][v] + gt[u][v] * (double)gs[u][v];
            K[(size_t)k * Ns + l] = g;
            K[(size_t)l * Ns + k] = g;
        }
    }
}

__global__ void k_row_mean(int64_t n, const double *__restrict__ K, double *__restrict__ r) {
    const int lane = threadIdx.x & 31;
    const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    double acc = 0.0;
    for (int64_t c = lane; c < n; c += 32) acc += K[(size_t)row * n + c];
    acc = warp_sum(acc);
    if (lane == 0) r[row] = acc / (double)n;
}

// Single block: rbar = mean(r) into r[n].
__global__ void k_mean_into(int64_t n, double *__restrict__ r) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int64_t c = threadIdx.x; c < n; c += blockDim.x) acc += r[c];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) r[n] = v / (double)n;
    }
}

// K_kl <- (K_kl - r_k - r_l + rbar) / n (+ eps on the diagonal), written
// as fma(K_kl - r_l, 1/n, (rbar - r_k) / n): two FP64 operations per entry
// (the FP64 pipe bounds this kernel, not HBM).  Rows in blockIdx.y (grid-
// stride), 256 columns per block in blockIdx.x; lower_only leaves the part
// above the diagonal untouched.
__global__ void k_double_center(int64_t n, double *__restrict__ K, const double *__restrict__ r,
                                const double *__restrict__ bk, double inv_n, double eps, int lower_only) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t k = blockIdx.y; k < n; k += gridDim.y) {
        if (lower_only && (int64_t)blockIdx.x * blockDim.x > k) continue;  // block-uniform
        if (l >= n || (lower_only && l > k)) continue;
        double v = fma(K[(size_t)k * n + l] - r[l], inv_n, bk[k]);
        if (k == l) v += eps;
        K[(size_t)k * n + l] = v;
    }
}

// bk[k] = (rbar - r_k) / n, the per-row part of the double centring.
__global__ void k_center_rows(int64_t n, const double *__restrict__ r, double inv_n, double *__restrict__ bk) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) bk[k] = (r[n] - r[k]) * inv_n;
}


// ------------------------------------------------------------- Cholesky ---

constexpr int kNB = 64;

// Factor the kb x kb diagonal block at (k, k) in shared memory.
__global__ void k_potrf_diag(double *__restrict__ A, int64_t n, int64_t k, int kb,
                             int *__restrict__ info) {
    __shared__ double L[kNB][kNB + 1];
    const int t = threadIdx.x;
    for (int r = 0; r < kb; ++r)
        if (t < kb) L[r][t] = A[(size_t)(k + r) * n + k + t];
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
        if (t == 0) {
            double d = L[c][c];
            if (!(d > 0.0)) {
                if (info) atomicCAS(info, 0, (int)(k + c + 1));  // the first failure
                d = 1e-300;
            }
            L[c][c] = sqrt(d);
        }
        __syncthreads();
        if (t > c && t < kb) L[t][c] /= L[c][c];
        __syncthreads();
        if (t > c && t < kb) {
            const double ltc = L[t][c];
            for (int q = c + 1; q <= t; ++q) L[t][q] -= ltc * L[q][c];
        }
        __syncthreads();
    }
    for (int r = 0; r < kb; ++r)
        if (t <= r && t < kb) A[(size_t)(k + r) * n + k + t] = L[r][t];
}

// Rows below the diagonal block: A[r, k:k+kb] <- A[r, k:k+kb] L_kk^{-T}.
__global__ void k_trsm_panel(double *__restrict__ A, int64_t n, int64_t k, int kb) {
    __shared__ double L[kNB][kNB + 1];
    __shared__ double X[kNB][kNB + 1];
    const int t = threadIdx.x;
    const int64_t r0 = k + kb + (int64_t)blockIdx.x * kNB;
    for (int r = 0; r < kb; ++r)
        if (t < kb) L[r][t] = A[(size_t)(k + r) * n + k + t];
    for (int r = 0; r < kNB; ++r) {
        const int64_t row = r0 + r;
        if (t < kb) X[r][t] = row < n ? A[(size_t)row * n + k + t] : 0.0;
    }
    __syncthreads();
    const int64_t row = r0 + t;
    if (row < n) {
        for (int c = 0; c < kb; ++c) {
            double v = X[t][c];
            for (int j = 0; j < c; ++j) v -= X[t][j] * L[c][j];
            X[t][c] = v / L[c][c];
        }
    }
    __syncthreads();
    for (int r = 0; r < kNB; ++r) {
        const int64_t rr = r0 + r;
        if (rr < n && t < kb) A[(size_t)rr * n + k + t] = X[r][t];
    }
}

struct PanelLoad {  // L(r, c) = A[(off + r) n + k + c], c contiguous
    static constexpr bool kContig = true;
    const double *A;
    int64_t n, off, k;
    __device__ double operator()(int64_t r, int64_t c) const {
        return A[(size_t)(off + r) * n + k + c];
    }
};

struct EpTrailing {
    double *A;
    int64_t n, off;
    __device__ bool active(int64_t m0, int64_t n0) const { return n0 <= m0 + 63; }
    __device__ void operator()(int64_t r, int64_t q, int, double v) const {
        if (q > r) return;
        A[(size_t)(off + r) * n + off + q] -= v;
    }
};

// Forward substitution on the diagonal block: y_k = L_kk^{-1} b_k.
__global__ void k_trsv_diag_lower(const double *__restrict__ A, int64_t n, int64_t k, int kb,
                                  double *__restrict__ b) {
    __shared__ double y[kNB];
    const int t = threadIdx.x;
    if (t < kb) y[t] = b[k + t];
    __syncthreads();
    for (int c = 0; c < kb; ++c) {
        if (t == 0) y[c] /= A[(size_t)(k + c) * n + k + c];
        __syncthreads();
        if (t > c && t < kb) y[t] -= A[(size_t)(k + t) * n + k + c] * y[c];
        __syncthreads();
    }
    if (t < kb) b[k + t] = y[t];
}

// b[r] -= sum_{c in block} L[r][k + c] y[k + c] for rows r >= k + kb.
__global__ void k_trsv_update_lower(const double *__restrict__ A, int64_t n, int64_t k, int kb,
                                    double *__restrict__ b) {
    const int lane = threadIdx.x & 31;
    const int64_t r = k + kb + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    double acc = 0.0;
    for (int c = lane; c < kb; c += 32) acc += A[(size_t)r * n + k + c] * b[k + c];
    acc = warp_sum(acc);
    if (lane == 0) b[r] -= acc;
}

// Back substitution on the diagonal block: x_k = L_kk^{-T} y_k.
__global__ void k_trsv_diag_upper(const double *__restrict__ A, int64_t n, int64_t k, int kb,
                                  double *__restrict__ b) {
    __shared__ double x[kNB];
    const int t = threadIdx.x;
    if (t < kb) x[t] = b[k + t];
    __syncthreads();
    for (int c = kb - 1; c >= 0; --c) {
        if (t == 0) x[c] /= A[(size_t)(k + c) * n + k + c];
        __syncthreads();
        if (t < c) x[t] -= A[(size_t)(k + c) * n + k + t] * x[c];
        __syncthreads();
    }
    if (t < kb) b[k + t] = x[t];
}

// b[r] -= sum_{c in block} L[k + c][r] x[k + c] for rows r < k.
__global__ void k_trsv_update_upper(const double *__restrict__ A, int64_t n, int64_t k, int kb,
                                    double *__restrict__ b) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= k) return;
    double acc = 0.0;
    for (int c = 0; c < kb; ++c) acc += A[(size_t)(k + c) * n + r] * b[k + c];
    b[r] -= acc;
}

// ------------------------------------------------------------ statistics ---

// Block-wide compensated sum (Neumaier per thread, TwoSum tree); every
// thread returns the total.
__device__ double block_comp_sum(double s, double c) {
    __shared__ double ss[1024], cc[1024];
    const int t = threadIdx.x;
    ss[t] = s;
    cc[t] = c;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if (t < w) {
            double r, e;
            two_sum(ss[t], ss[t + w], r, e);
            ss[t] = r;
            cc[t] = cc[t] + cc[t + w] + e;
        }
        __syncthreads();
    }
    const double out = ss[0] + cc[0];
    __syncthreads();
    return out;
}

__device__ __forceinline__ void neumaier_add(double &s, double &c, double x) {
    double r, e;
    two_sum(s, x, r, e);
    s = r;
    c += e;
}

__global__ void __launch_bounds__(1024) k_stats(const double *__restrict__ e, int64_t Ns,
                                                int n_chains, double *__restrict__ out) {
    double s = 0.0, c = 0.0;
    for (int64_t k = threadIdx.x; k < Ns; k += blockDim.x) neumaier_add(s, c, e[k]);
    const double mean = block_comp_sum(s, c) / (double)Ns;
    s = 0.0;
    c = 0.0;
    for (int64_t k = threadIdx.x; k < Ns; k += blockDim.x) {
        const double d = e[k] - mean;
        neumaier_add(s, c, d * d);
    }
    const double var = block_comp_sum(s, c) / (double)Ns;
    double err;
    const int64_t per = n_chains > 0 ? Ns / n_chains : 0;
    if (n_chains > 1 && per >= 2 && per * n_chains == Ns) {
        // chain means, their mean and variance
        s = 0.0;
        c = 0.0;
        for (int64_t ch = threadIdx.x; ch < n_chains; ch += blockDim.x) {
            double a = 0.0, ac = 0.0;
            for (int64_t q = 0; q < per; ++q) neumaier_add(a, ac, e[ch * per + q]);
            neumaier_add(s, c, (a + ac) / (double)per);
        }
        const double cm = block_comp_sum(s, c) / (double)n_chains;
        s = 0.0;
        c = 0.0;
        for (int64_t ch = threadIdx.x; ch < n_chains; ch += blockDim.x) {
            double a = 0.0, ac = 0.0;
            for (int64_t q = 0; q < per; ++q) neumaier_add(a, ac, e[ch * per + q]);
            const double d = (a + ac) / (double)per - cm;
            neumaier_add(s, c, d * d);
        }
        const double vcm = block_comp_sum(s, c) / (double)n_chains;
        err = sqrt(vcm / (double)n_chains);
    } else {
        err = sqrt(var / (double)Ns);
    }
    if (threadIdx.x == 0) {
        out[0] = mean;
        out[1] = var;
        out[2] = err;
    }
}

// -------------------------------------------------------------- vectors ---

__global__ void k_axpby(int64_t n, double alpha, const double *__restrict__ x, double beta,
                        double *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = beta == 0.0 ? alpha * x[i] : alpha * x[i] + beta * y[i];
}

constexpr int kDotBlock = 256;

int dot_blocks(int64_t n) {
    int64_t b = (n + kDotBlock * 8 - 1) / (kDotBlock * 8);
    if (b > 1024) b = 1024;
    if (b < 1) b = 1;
    return (int)b;
}

__global__ void k_dot_partial(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                              double *__restrict__ partial) {
    __shared__ double red[kDotBlock / 32];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        acc += x[i] * (y ? y[i] : 1.0);
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < kDotBlock / 32 ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__global__ void k_dot_final(int nb, const double *__restrict__ partial, double scale,
                            double *__restrict__ out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) *out = v * scale;
    }
}

__global__ void k_sub_scalar_scale(int64_t n, double *__restrict__ x, const double *__restrict__ m,
                                   double scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (x[i] - *m) * scale;
}

__global__ void k_fill(int64_t n, double v, double *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

__global__ void k_cg_xr(int64_t n, const double *__restrict__ rr, const double *__restrict__ pAp,
                        const double *__restrict__ p, const double *__restrict__ Ap,
                        double *__restrict__ x, double *__restrict__ r, const int *__restrict__ done) {
    if (*done) return;
    const double alpha = *rr / *pAp;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        x[i] += alpha * p[i];
        r[i] -= alpha * Ap[i];
    }
}

__global__ void k_cg_p(int64_t n, const double *__restrict__ rr_new,
                       const double *__restrict__ rr_old, const double *__restrict__ r,
                       double *__restrict__ p, const int *__restrict__ done) {
    if (*done) return;
    const double beta = *rr_new / *rr_old;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = r[i] + beta * p[i];
}

// Counts the iteration just taken (unless already converged), tests the
// residual and keeps rr_keep = rr for the next iteration.
__global__ void k_cg_check(const double *__restrict__ rr, const double *__restrict__ ff, double tol,
                           int *__restrict__ done, int *__restrict__ iters,
                           double *__restrict__ rr_keep) {
    if (*done) return;
    *iters += 1;
    *rr_keep = *rr;
    if (*rr <= tol * tol * *ff) *done = 1;
}

__global__ void k_sgd(int64_t n, double lr, const double *__restrict__ d, double *__restrict__ p) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] -= lr * d[i];
}

__global__ void k_force_g(int64_t Ns, const double *__restrict__ e, const double *__restrict__ st,
                          double *__restrict__ g) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < Ns) g[k] = 2.0 * (e[k] - st[0]) / (double)Ns;
}

__global__ void k_write_sr_stats(const double *__restrict__ st3, const unsigned long long *acc, int C,
                                 double n_proposals, const double *__restrict__ ff,
                                 const double *__restrict__ dd, const int *__restrict__ it,
                                 const double *__restrict__ rr, const int *__restrict__ status,
                                 nk_sr_stats *__restrict__ out) {
    __shared__ unsigned long long red[256];
    unsigned long long a = 0;
    for (int c = threadIdx.x; c < C; c += blockDim.x) a += acc[c];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->energy = st3[0];
        out->variance = st3[1];
        out->error = st3[2];
        out->acceptance = n_proposals > 0 ? (double)red[0] / n_proposals : 0.0;
        out->cg_iters = it ? (double)*it : 0.0;
        out->cg_residual = (rr && ff && *ff > 0) ? sqrt(*rr / *ff) : 0.0;
        out->f_norm = ff ? sqrt(*ff) : 0.0;
        out->delta_norm = dd ? sqrt(*dd) : 0.0;
        // status[0]: Cholesky breakdown pivot, status[1]: tensor-core time-out
        out->solver_status = status ? (status[1] ? -(double)status[1] : (double)status[0]) : 0.0;
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// r holds n + 1 row means (the last the grand mean) followed by room for n
// per-row coefficients.
void launch_double_center(int64_t n, double *K, double *r, double eps, bool lower_only, cudaStream_t st) {
    double *bk = r + n + 1;
    (k_center_rows<<<nblk(n, 256), 256, 0, st>>>(n, r, 1.0 / (double)n, bk), nk::note_launch());
    const dim3 grid(nblk(n, 256), (unsigned)(n < 65535 ? n : 65535));
    (k_double_center<<<grid, 256, 0, st>>>(n, K, r, bk, 1.0 / (double)n, eps, lower_only ? 1 : 0),
     nk::note_launch());
}

}  // namespace

// ============================================================ launchers ====

cudaError_t launch_stats(const double *e, int64_t Ns, int n_chains, double *out, cudaStream_t st) {
    (k_stats<<<1, 1024, 0, st>>>(e, Ns, n_chains, out), nk::note_launch());
    return cudaGetLastError();
}

size_t vjp_partial_doubles(int N, int M, int64_t Ns) {
    return (size_t)vjp_splits(N, M, Ns) * (size_t)(M + 1) * (size_t)(N + 1);
}

cudaError_t launch_vjp(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *g,
                       double g_scale, const double *g_shift, double *partial, double *out,
                       cudaStream_t st) {
    const int sp = vjp_splits(N, M, Ns);
    VjpA la{T, g, g_shift, g_scale, M};
    AugS_kn lb{s, N};
    const int64_t plane = (int64_t)(M + 1) * (N + 1);
    EpPartial ep{partial, N + 1, plane};
    const int slot = prof_begin(NK_PROF_JVP_VJP, st);
    cudaError_t err = gemm64(M + 1, N + 1, Ns, sp, la, lb, ep, st);
    if (err != cudaSuccess) return err;
    (k_vjp_reduce<<<nblk(plane, 256), 256, 0, st>>>(N, M, sp, partial, out), nk::note_launch());
    prof_end(slot, st, 2.0 * (double)Ns * (N + 1) * (double)(M + 1));
    return cudaGetLastError();
}

cudaError_t launch_jvp(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *v,
                       double *U, double *out, cudaStream_t st) {
    AugS_k la{s, N};
    VAug lb{v, N, M};
    EpStore ep{U, M + 1};
    const int slot = prof_begin(NK_PROF_JVP_VJP, st);
    cudaError_t err = gemm64(Ns, M + 1, N + 1, 1, la, lb, ep, st);
    if (err != cudaSuccess) return err;
    (k_rowdot_aug<<<nblk(Ns, 8), 256, 0, st>>>(M, Ns, T, U, out), nk::note_launch());
    prof_end(slot, st, 2.0 * (double)Ns * (N + 1) * (double)(M + 1) + 2.0 * (double)Ns * (M + 1));
    return cudaGetLastError();
}


cudaError_t launch_jacobian_rows(int N, int M, const int8_t *s, const double *T, int64_t row0,
                                 int64_t rows, const double *mean, double *O, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int64_t Np = (int64_t)N + M + (int64_t)M * N;
    int64_t gx = (Np + 255) / 256;
    if (gx > 64) gx = 64;
    for (int64_t r = 0; r < rows; r += 65535) {
        const int64_t rr = rows - r < 65535 ? rows - r : 65535;
        dim3 grid((unsigned)gx, (unsigned)rr);
        (k_jacobian_rows<<<grid, 256, 0, st>>>(N, M, s, T, row0 + r, rr, mean,
                                              O + (size_t)r * Np), nk::note_launch());
    }
    return cudaGetLastError();
}

cudaError_t launch_gemv_rows(const double *A, int64_t rows, int64_t cols, const double *x,
                             double *y, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    (k_gemv_rows<<<nblk(rows, 8), 256, 0, st>>>(A, rows, cols, x, y), nk::note_launch());
    return cudaGetLastError();
}

size_t gemv_t_partial_doubles(int64_t rows, int64_t cols) {
    return (size_t)((rows + kGemvTRows - 1) / kGemvTRows) * (size_t)cols;
}

cudaError_t launch_gemv_t(const double *A, int64_t rows, int64_t cols, const double *x,
                          double scale, double *partial, double *y, cudaStream_t st) {
    const int64_t nb = (rows + kGemvTRows - 1) / kGemvTRows;
    for (int64_t b0 = 0; b0 < nb; b0 += 65535) {
        const int64_t bb = nb - b0 < 65535 ? nb - b0 : 65535;
        dim3 grid(nblk(cols, 256), (unsigned)bb);
        (k_gemv_t_partial<<<grid, 256, 0, st>>>(A + (size_t)b0 * kGemvTRows * cols,
                                               rows - b0 * kGemvTRows, cols, x + b0 * kGemvTRows,
                                               partial + (size_t)b0 * cols), nk::note_launch());
    }
    (k_sum_partials<<<nblk(cols, 256), 256, 0, st>>>(cols, (int)nb, partial, scale, y), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_syrk_t(const double *A, int64_t rows, int64_t cols, double scale, double eps,
                          double *C, cudaStream_t st) {
    ColMajorA la{A, cols};
    EpSyrk ep{C, cols, scale, eps};
    return gemm64(cols, cols, rows, 1, la, la, ep, st);
}

cudaError_t launch_gram_samplespace(int N, int M, int64_t Ns, const int8_t *s, const double *T,
                                    double eps, double *K, double *rowmean, cudaStream_t st) {
    dim3 grid((unsigned)((Ns + 63) / 64), (unsigned)((Ns + 63) / 64));
    const int slot = prof_begin(NK_PROF_GRAM, st);
    (k_gram_raw<<<grid, 256, 0, st>>>(N, M, Ns, s, T, K), nk::note_launch());
    prof_end(slot, st, (double)Ns * (Ns + 1) * (double)(N + M));
    (k_row_mean<<<nblk(Ns, 8), 256, 0, st>>>(Ns, K, rowmean), nk::note_launch());
    (k_mean_into<<<1, 1024, 0, st>>>(Ns, rowmean), nk::note_launch());
    launch_double_center(Ns, K, rowmean, eps, false, st);
    return cudaGetLastError();
}

// The tensor-core Cholesky reads only the lower triangle.
cudaError_t launch_center_gram(int64_t Ns, double *K, double *rowmean, double eps, cudaStream_t st) {
    (k_row_mean<<<nblk(Ns, 8), 256, 0, st>>>(Ns, K, rowmean), nk::note_launch());
    (k_mean_into<<<1, 1024, 0, st>>>(Ns, rowmean), nk::note_launch());
    launch_double_center(Ns, K, rowmean, eps, true, st);
    return cudaGetLastError();
}

cudaError_t launch_cholesky(double *A, int64_t n, int *info, cudaStream_t st) {
    for (int64_t k = 0; k < n; k += kNB) {
        const int kb = (int)(n - k < kNB ? n - k : kNB);
        const int64_t rest = n - k - kb;
        int slot = prof_begin(NK_PROF_CHOL_PANEL, st);
        (k_potrf_diag<<<1, kNB, 0, st>>>(A, n, k, kb, info), nk::note_launch());
        if (rest > 0) (k_trsm_panel<<<nblk(rest, kNB), kNB, 0, st>>>(A, n, k, kb), nk::note_launch());
        prof_end(slot, st, (double)kb * kb * kb / 3.0 + (double)rest * kb * kb);
        if (rest > 0) {
            PanelLoad pl{A, n, k + kb, k};
            EpTrailing ep{A, n, k + kb};
            slot = prof_begin(NK_PROF_CHOL_UPDATE, st);
            cudaError_t err = gemm64(rest, rest, kb, 1, pl, pl, ep, st);
            prof_end(slot, st, (double)kb * rest * (double)(rest + 1));
            if (err != cudaSuccess) return err;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_cholesky_solve(const double *L, int64_t n, double *b, cudaStream_t st) {
    const int slot = prof_begin(NK_PROF_TRSV, st);
    for (int64_t k = 0; k < n; k += kNB) {
        const int kb = (int)(n - k < kNB ? n - k : kNB);
        (k_trsv_diag_lower<<<1, kNB, 0, st>>>(L, n, k, kb, b), nk::note_launch());
        const int64_t rest = n - k - kb;
        if (rest > 0) (k_trsv_update_lower<<<nblk(rest, 8), 256, 0, st>>>(L, n, k, kb, b), nk::note_launch());
    }
    const int64_t last = ((n - 1) / kNB) * kNB;
    for (int64_t k = last; k >= 0; k -= kNB) {
        const int kb = (int)(n - k < kNB ? n - k : kNB);
        (k_trsv_diag_upper<<<1, kNB, 0, st>>>(L, n, k, kb, b), nk::note_launch());
        if (k > 0) (k_trsv_update_upper<<<nblk(k, 256), 256, 0, st>>>(L, n, k, kb, b), nk::note_launch());
    }
    prof_end(slot, st, 2.0 * (double)n * (double)n);
    return cudaGetLastError();
}

cudaError_t launch_axpby(int64_t n, double alpha, const double *x, double beta, double *y,
                         cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    (k_axpby<<<nblk(n, 256), 256, 0, st>>>(n, alpha, x, beta, y), nk::note_launch());
    return cudaGetLastError();
}

size_t dot_partial_doubles(int64_t n) { return (size_t)dot_blocks(n); }

cudaError_t launch_dot(int64_t n, const double *x, const double *y, double *partial, double *out,
                       cudaStream_t st) {
    const int nb = dot_blocks(n);
    (k_dot_partial<<<nb, kDotBlock, 0, st>>>(n, x, y, partial), nk::note_launch());
    (k_dot_final<<<1, 1024, 0, st>>>(nb, partial, 1.0, out), nk::note_launch());
    return cudaGetLastError();
}

// x <- (x - mean(x)) * scale; partial holds dot_partial_doubles(n) + 1 doubles.
cudaError_t launch_center(int64_t n, double *x, double *partial, double scale, cudaStream_t st) {
    const int nb = dot_blocks(n);
    (k_dot_partial<<<nb, kDotBlock, 0, st>>>(n, x, nullptr, partial), nk::note_launch());
    (k_dot_final<<<1, 1024, 0, st>>>(nb, partial, 1.0 / (double)n, partial + nb), nk::note_launch());
    (k_sub_scalar_scale<<<nblk(n, 256), 256, 0, st>>>(n, x, partial + nb, scale), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_fill(int64_t n, double v, double *x, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    (k_fill<<<nblk(n, 256), 256, 0, st>>>(n, v, x), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_cg_update_xr(int64_t n, const double *rr, const double *pAp, const double *p,
                                const double *Ap, double *x, double *r, const int *done,
                                cudaStream_t st) {
    (k_cg_xr<<<nblk(n, 256), 256, 0, st>>>(n, rr, pAp, p, Ap, x, r, done), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_cg_update_p(int64_t n, const double *rr_new, const double *rr_old,
                               const double *r, double *p, const int *done, cudaStream_t st) {
    (k_cg_p<<<nblk(n, 256), 256, 0, st>>>(n, rr_new, rr_old, r, p, done), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_cg_check(const double *rr, const double *ff, double tol, int *done, int *iters,
                            double *rr_keep, cudaStream_t st) {
    (k_cg_check<<<1, 1, 0, st>>>(rr, ff, tol, done, iters, rr_keep), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_sgd(int64_t n, double lr, const double *delta, double *params,
                       cudaStream_t st) {
    (k_sgd<<<nblk(n, 256), 256, 0, st>>>(n, lr, delta, params), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_make_force_g(int64_t Ns, const double *eloc, const double *stats, double *g,
                                cudaStream_t st) {
    (k_force_g<<<nblk(Ns, 256), 256, 0, st>>>(Ns, eloc, stats, g), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_write_sr_stats(const double *stats3, const unsigned long long *acc, int C,
                                  double n_proposals, const double *ff, const double *dd,
                                  const int *cg_iters, const double *cg_rr, const int *status,
                                  nk_sr_stats *out, cudaStream_t st) {
    (k_write_sr_stats<<<1, 256, 0, st>>>(stats3, acc, C, n_proposals, ff, dd, cg_iters, cg_rr, status, out), nk::note_launch());
    return cudaGetLastError();
}

}  // namespace nk
