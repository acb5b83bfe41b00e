// The symmetric RBM (RBMSymm, NetKet 3 Sec. 5): a permutation group G of
// the sites acts on the configurations, and feature f at group element g has
// the activation
//     theta_{f,g}(s) = b_f + sum_j W_{f,j} s_{pi_g(j)}
// (the embedding layer, Eq. eq: equivariant: embedding), with
//     ln psi(s) = a sum_j s_j + sum_{f,g} ln cosh theta_{f,g}(s).
// Parameters [a (1); b (alpha); W (alpha x N)], Np = 1 + alpha + alpha N.
//
// The model is a plain RBM with M = alpha |G| hidden units and tied
// parameters: unit f |G| + g has bias b_f and weight W_{f,j} on site pi_g(j),
// every visible bias equals a.  The sampler and the local energies run on
// those expanded parameters; the log-derivatives in the symmetric parameters
// follow by the chain rule (a sum over the units each parameter ties):
//     O_a = sum_j s_j,  O_{b_f} = sum_g t_{f,g},
//     O_{W_{f,j}} = sum_g t_{f,g} s_{pi_g(j)},   t = tanh theta.

#include <cuda_runtime.h>

#include "nk_common.cuh"
#include "nk_internal.h"

namespace nk {

namespace {

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// err |= 1 if a row of perms is not a permutation of [0, N).  One block per
// group element; a bitmap of the sites seen in shared memory.
__global__ void k_check_perms(int N, int G, const int32_t *__restrict__ perms, int *__restrict__ err) {
    extern __shared__ unsigned int seen[];
    const int g = blockIdx.x;
    const int words = (N + 31) / 32;
    for (int w = threadIdx.x; w < words; w += blockDim.x) seen[w] = 0u;
    __syncthreads();
    bool bad = false;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const int v = perms[(size_t)g * N + j];
        if ((unsigned)v >= (unsigned)N) {
            bad = true;
            continue;
        }
        const unsigned int bit = 1u << (v & 31);
        if (atomicOr(&seen[v >> 5], bit) & bit) bad = true;  // a site hit twice
    }
    if (bad) atomicOr(err, 1);
}

// Expanded plain-RBM parameters [a_i = a (N); b_{fG+g} = b_f (M); W (M x N)]
// with W[(f G + g) N + pi_g(j)] = W_{f,j}: one thread per (f, g, j); every
// entry of a row is written once because pi_g is a permutation (checked
// before), and indices are bounds-checked all the same.
__global__ void k_symm_expand(int N, int alpha, int G, const int32_t *__restrict__ perms,
                              const double *__restrict__ p, double *__restrict__ out) {
    const int64_t M = (int64_t)alpha * G;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const double a = p[0];
    if (idx < N) out[idx] = a;
    if (idx < M) out[N + idx] = p[1 + idx / G];
    if (idx >= M * N) return;
    const int64_t unit = idx / N;
    const int j = (int)(idx % N);
    const int f = (int)(unit / G), g = (int)(unit % G);
    const int site = perms[(size_t)g * N + j];
    if ((unsigned)site < (unsigned)N) out[N + M + (size_t)unit * N + site] = p[1 + alpha + (size_t)f * N + j];
}

// Rows of the symmetric Jacobian: O [Ns][1 + alpha + alpha N] from the
// samples and t = tanh theta of the expanded units ([Ns][alpha G]).  One
// block per sample: s and t staged in shared memory; thread (f, j) sums its
// G terms in group order.
__global__ void k_symm_jacobian(int N, int alpha, int G, const int32_t *__restrict__ perms,
                                const int8_t *__restrict__ s, const double *__restrict__ T, int64_t Ns,
                                double *__restrict__ O) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int64_t k = blockIdx.x;
    if (k >= Ns) return;
    const int M = alpha * G;
    double *t = reinterpret_cast<double *>(sm);
    int8_t *sv = reinterpret_cast<int8_t *>(sm + (size_t)M * sizeof(double));
    for (int j = threadIdx.x; j < N; j += blockDim.x) sv[j] = s[(size_t)k * N + j];
    for (int u = threadIdx.x; u < M; u += blockDim.x) t[u] = T[(size_t)k * M + u];
    __syncthreads();
    const int64_t Np = 1 + alpha + (int64_t)alpha * N;
    double *row = O + (size_t)k * Np;
    if (threadIdx.x < 32) {
        double acc = 0.0;
        for (int j = threadIdx.x; j < N; j += 32) acc += (double)sv[j];
        acc = warp_sum(acc);
        if (threadIdx.x == 0) row[0] = acc;
    }
    for (int f = threadIdx.x; f < alpha; f += blockDim.x) {
        double acc = 0.0;
        for (int g = 0; g < G; ++g) acc += t[f * G + g];
        row[1 + f] = acc;
    }
    for (int64_t q = threadIdx.x; q < (int64_t)alpha * N; q += blockDim.x) {
        const int f = (int)(q / N), j = (int)(q % N);
        double acc = 0.0;
        for (int g = 0; g < G; ++g) {
            const int site = perms[(size_t)g * N + j];
            if ((unsigned)site < (unsigned)N) acc = fma(t[f * G + g], (double)sv[site], acc);
        }
        row[1 + alpha + q] = acc;
    }
}

// dJ[k][q] = O[k][q] - mean[q], in place.
__global__ void k_sub_colmean(int64_t rows, int64_t cols, const double *__restrict__ mean, double *__restrict__ O) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < rows * cols) O[idx] -= mean[idx % cols];
}

}  // namespace

cudaError_t launch_symm_check_perms(int N, int G, const int32_t *perms, int *err, cudaStream_t st) {
    const size_t smem = (size_t)((N + 31) / 32) * sizeof(unsigned int);
    (k_check_perms<<<G, 256, smem, st>>>(N, G, perms, err), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_symm_expand(int N, int alpha, int G, const int32_t *perms, const double *p, double *out,
                               cudaStream_t st) {
    const int64_t M = (int64_t)alpha * G;
    const int64_t n = M * N > M ? M * N : M;
    (k_symm_expand<<<nblk(n > N ? n : N, 256), 256, 0, st>>>(N, alpha, G, perms, p, out), nk::note_launch());
    return cudaGetLastError();
}

size_t symm_jacobian_smem(int N, int alpha, int G) {
    return (size_t)alpha * G * sizeof(double) + (size_t)(N + 15) / 16 * 16;
}

cudaError_t launch_symm_jacobian(int N, int alpha, int G, const int32_t *perms, const int8_t *s, const double *T,
                                 int64_t Ns, double *O, cudaStream_t st) {
    if (Ns <= 0) return cudaSuccess;
    const size_t smem = symm_jacobian_smem(N, alpha, G);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_symm_jacobian);
    if (e != cudaSuccess) return e;
    for (int64_t k0 = 0; k0 < Ns; k0 += 65535) {
        const int64_t kb = Ns - k0 < 65535 ? Ns - k0 : 65535;
        const int64_t Np = 1 + alpha + (int64_t)alpha * N;
        (k_symm_jacobian<<<(unsigned)kb, 256, smem, st>>>(N, alpha, G, perms, s + (size_t)k0 * N,
                                                          T + (size_t)k0 * alpha * G, kb, O + (size_t)k0 * Np),
         nk::note_launch());
    }
    return cudaGetLastError();
}

cudaError_t launch_sub_colmean(int64_t rows, int64_t cols, const double *mean, double *O, cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    (k_sub_colmean<<<nblk(rows * cols, 256), 256, 0, st>>>(rows, cols, mean, O), nk::note_launch());
    return cudaGetLastError();
}

}  // namespace nk
