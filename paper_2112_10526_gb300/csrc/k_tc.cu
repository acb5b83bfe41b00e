// Tensor-core (tcgen05) products for the dense contractions of the SR solve.
//
// FP64-accurate GEMM by integer splitting (the Ozaki scheme: Ozaki, Ogita,
// Oishi, Rump, Numer. Algorithms 59 (2012); Ootomo, Ozaki, Yokota,
// IJHPCA 2024).  Every row r of an FP64 operand (K <= 64 columns) is scaled
// by its own power of two 2^-e_r (max |a_rk| < 2^e_r) and cut into S slices
// of 8-bit integers alpha_s in [-255, 255]:
//     a_rk = 2^e_r sum_{s=1..S} alpha_s,rk 2^{-8s} + (remainder < 2^{e_r - 8S}).
// Integers of at most 8 bits are exact in BF16, their products exact in the
// FP32 accumulator of kind::f16 MMAs, and a sum of up to four slice products
// over K = 64 stays below 2^24, so the partial products
//     D_g = sum_{s+t=g} sum_k alpha_s,ik beta_t,jk      (g = 2 .. S+1)
// are exact integers for g <= 5 (the levels that carry the leading bits) and
// carry a relative error 2^-24 x 2^{-8g} < 2^-70 beyond.  The epilogue
// recombines C_ij = 2^{e_i + f_j} sum_g 2^{-8g} D_g in FP64.  With S = 7 the
// dropped terms are below 2^-56 of K max|a| max|b|: FP64-level accuracy.
// S = 3 gives about FP32 accuracy (24 bits per operand).
//
// Kernel shape: one 128 x 64 output tile per CTA, K = 64.  Thread 0 loads the
// S slices of the A rows (128 x 64) and of the B rows (64 x 64) with TMA
// (3-D tensor maps [S][rows][64] BF16, 128-byte swizzle) onto one mbarrier,
// then issues the S(S+1)/2 x 4 tcgen05.mma (M = 128, N = 64, K = 16) into
// S accumulators of 64 TMEM columns each, and commits to a second mbarrier;
// the four warps then read their 32 TMEM lanes (= tile rows) and update C.
// Every wait is bounded by the global timer; on time-out the kernel records
// an error code, frees its TMEM and returns.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "nk_common.cuh"
#include "nk_internal.h"
#include "tc_ptx.cuh"

namespace nk {

namespace {

constexpr int kTileM = 128;
constexpr int kTileN = 64;
constexpr int kTileK = 64;
constexpr int kMaxSlices = 7;
constexpr uint32_t kTmemCols = 512;
constexpr int kABytes = kTileM * kTileK * 2;  // one slice of the A tile
constexpr int kBBytes = kTileN * kTileK * 2;  // one slice of the B tile

// ---------------------------------------------------------------- slicing ---

// One warp per row: the first kcols (<= 64) entries of row r of A (row
// stride lda) -> S BF16 integer slices out[s][r][0..63] (zero beyond kcols)
// and the row exponent e_r (max |a_rk| < 2^e_r).  The slices are the bytes,
// from the top, of the fixed-point magnitude floor(|a| 2^(8S - e_r)), with the
// sign of a: exactly the digits of repeated multiply-by-256-and-truncate,
// taken from the FP64 bit pattern with integer shifts only.
__global__ void k_slice_rows(const double *__restrict__ A, int64_t lda, int64_t rows, int kcols, int S,
                             __nv_bfloat16 *__restrict__ out, int *__restrict__ expo) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const double x0 = lane < kcols ? A[(size_t)r * lda + lane] : 0.0;
    const double x1 = lane + 32 < kcols ? A[(size_t)r * lda + lane + 32] : 0.0;
    int b0, b1;
    unsigned long long m0, m1;
    bool n0, n1;
    split_bits(x0, b0, m0, n0);
    split_bits(x1, b1, m1, n1);
    // |x| < 2^(biased - 1022) for nonzero x; the row exponent is the largest
    int ex = -100000;
    if (m0) ex = b0 - 1022;
    if (m1) ex = max(ex, b1 - 1022);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, off));
    const int e = ex == -100000 ? 0 : ex;
    // fixed point Y = floor(|x| 2^(8S - e)) = mant 2^(biased - 1075 + 8S - e) < 2^(8S)
    auto fixp = [&](int biased, unsigned long long mant) -> unsigned long long {
        if (!mant) return 0ULL;
        const int sh = biased - 1075 + 8 * S - e;
        if (sh >= 0) return mant << sh;  // sh <= 3 here
        if (sh <= -64) return 0ULL;
        return mant >> (-sh);
    };
    const unsigned long long y0 = fixp(b0, m0), y1 = fixp(b1, m1);
    for (int q = 0; q < S; ++q) {
        const int sh = 8 * (S - 1 - q);
        const int d0 = (int)((y0 >> sh) & 0xFFULL), d1 = (int)((y1 >> sh) & 0xFFULL);
        __nv_bfloat16 *o = out + ((size_t)q * rows + r) * kTileK;
        o[lane] = __int2bfloat16_rn(n0 ? -d0 : d0);
        o[lane + 32] = __int2bfloat16_rn(n1 ? -d1 : d1);
    }
    if (lane == 0) expo[r] = e;
}

// ------------------------------------------------------------- the GEMM ---

struct OzArgs {
    int64_t rows, cols;   // output rows (A rows) and columns (B rows)
    int S;
    const int *expA, *expB;
    double *C;
    int64_t ldc;
    int mode;             // 0: C = R, 1: C -= R, 2: C += R
    int lower;            // only entries with col <= row (tiles above are skipped)
    int *err;
};

constexpr int kOzThreads = 256;
constexpr int kOutLd = kTileN + 1;  // staged output tile [128][65] doubles

__global__ void __launch_bounds__(kOzThreads, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const int64_t m0 = (int64_t)blockIdx.y * kTileM;
    const int64_t n0 = (int64_t)blockIdx.x * kTileN;
    if (a.lower && n0 > m0 + kTileM - 1) return;
    // 1024-byte aligned operand area (128-byte swizzle atoms)
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *ops = smem_raw + ((1024 - (base & 1023)) & 1023);
    unsigned char *sA = ops;                                  // [S][128][64] bf16
    unsigned char *sB = ops + (size_t)kMaxSlices * kABytes;   // [S][64][64] bf16
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + (size_t)kMaxSlices * kBBytes);  // [0] tma, [1] mma
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.S;

    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (threadIdx.x == 0) {
        mbar_expect_tx(&bars[0], (uint32_t)S * (kABytes + kBBytes));
        for (int s = 0; s < S; ++s) {
            tma_load_3d(sA + (size_t)s * kABytes, &mapA, &bars[0], 0, (int)m0, s);
            tma_load_3d(sB + (size_t)s * kBBytes, &mapB, &bars[0], 0, (int)n0, s);
        }
        if (!mbar_wait(&bars[0], 0)) {
            *abort_flag = 1;
            atomicExch(a.err, 1);
        } else {
            tc_fence_after();
            const uint32_t idesc = idesc_bf16(kTileM, kTileN);
            for (int g = 2; g <= S + 1; ++g) {
                const uint32_t dcol = tmem + (uint32_t)((g - 2) * kTileN);
                bool first = true;
                for (int s = 1; s < g; ++s) {
                    const int t = g - s;
                    if (s > S || t > S) continue;
                    const uint64_t da = sw128_desc(sA + (size_t)(s - 1) * kABytes);
                    const uint64_t db = sw128_desc(sB + (size_t)(t - 1) * kBBytes);
#pragma unroll
                    for (int kk = 0; kk < kTileK / 16; ++kk) {
                        // advance 16 BF16 = 32 bytes along K inside the swizzle atom
                        umma_bf16(dcol, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), idesc,
                                  first ? 0u : 1u);
                        first = false;
                    }
                }
            }
            umma_commit(&bars[1]);
        }
    }
    __syncthreads();
    if (!*abort_flag) {
        // one waiter per warp, so that the .sync.aligned TMEM loads below are
        // executed by whole warps
        int ok = 1;
        if (lane == 0) ok = mbar_wait(&bars[1], 0) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.err, 2);
                *abort_flag = 2;
            }
        } else {
            tc_fence_after();
            // Warp w reads TMEM lanes 32 (w % 4) .. +31 (= tile rows) and the
            // column half w / 4; results go to a staged tile in the operand
            // area, which the MMAs no longer read.
            const int rloc = (warp & 3) * 32 + lane;
            const int64_t row = m0 + rloc;
            const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16);
            const int ei = row < a.rows ? a.expA[row] : 0;
            double *tile = reinterpret_cast<double *>(sA);
            for (int c0 = (warp >> 2) * 32; c0 < (warp >> 2) * 32 + 32; c0 += 16) {
                // V = sum_g D_g 2^(8 (8 - g)) = hi 2^32 + lo, exactly, in integers
                long long hi[16], lo[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) hi[j] = lo[j] = 0;
                for (int g = 2; g <= S + 1; ++g) {
                    uint32_t r[16];
                    tmem_ld16(lane_base + (uint32_t)((g - 2) * kTileN + c0), r);
                    tmem_wait_ld();
                    if (g <= 4) {
                        const int sh = 8 * (4 - g);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            hi[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
                    } else {
                        const int sh = 8 * (8 - g);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            lo[j] += (long long)__float2int_rn(__uint_as_float(r[j])) << sh;
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int64_t col = n0 + c0 + j;
                    const int fj = col < a.cols ? a.expB[col] : 0;
                    tile[rloc * kOutLd + c0 + j] = fixed_to_double(hi[j], lo[j], ei + fj - 64);
                }
            }
        }
    }
    __syncthreads();
    if (!*abort_flag) {
        // coalesced update of C: consecutive threads take consecutive columns
        const double *tile = reinterpret_cast<const double *>(sA);
        const int cx = threadIdx.x & 63, ry = threadIdx.x >> 6;
        const int64_t col = n0 + cx;
        constexpr int kStep = kOzThreads / 64, kBatch = 8;
        if (col < a.cols) {
            for (int rb = ry; rb < kTileM; rb += kStep * kBatch) {
                // all loads of a batch first, so that they are in flight together
                double cv[kBatch];
                bool on[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int rl = rb + kStep * u;
                    const int64_t row = m0 + rl;
                    on[u] = rl < kTileM && row < a.rows && !(a.lower && col > row);
                    cv[u] = (on[u] && a.mode != 0) ? a.C[(size_t)row * a.ldc + col] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    if (!on[u]) continue;
                    const int rl = rb + kStep * u;
                    const double v = tile[rl * kOutLd + cx];
                    a.C[(size_t)(m0 + rl) * a.ldc + col] = a.mode == 0 ? v : (a.mode == 1 ? cv[u] - v : cv[u] + v);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// ------------------------------------------------- Cholesky building blocks ---

constexpr int kNB = 64;

// Factor the kb x kb diagonal block at (k, k) in place (lower) and write its
// inverse, a lower-triangular 64 x 64 block (zero above the diagonal and
// beyond kb), to Linv.  256 threads; per column one thread takes the square
// root and its reciprocal, the others scale and update with independent
// FMAs.  The inverse is built right-looking (row k of X = L^-1 is final once
// scaled; it is then eliminated from the rows below).
constexpr int kPotrfThreads = 256;
constexpr int kLd = kNB + 1;

__global__ void __launch_bounds__(kPotrfThreads) k_potrf_inv(double *__restrict__ A, int64_t n, int64_t k, int kb,
                                                             int *__restrict__ info, double *__restrict__ Linv) {
    extern __shared__ double psm[];
    double *L = psm;                 // [64][65]
    double *X = psm + kNB * kLd;     // [64][65]
    double *rd = X + kNB * kLd;      // [64] reciprocal diagonal
    const int t = threadIdx.x;
    for (int e = t; e < kNB * kNB; e += kPotrfThreads) {
        const int r = e >> 6, c = e & 63;
        L[r * kLd + c] = (r < kb && c < kb) ? A[(size_t)(k + r) * n + k + c] : 0.0;
        X[r * kLd + c] = (r == c) ? 1.0 : 0.0;
    }
    __syncthreads();
    const int ry = t >> 6, cx = t & 63;
    for (int c = 0; c < kb; ++c) {
        if (t == 0) {
            double d = L[c * kLd + c];
            if (!(d > 0.0)) {
                if (info) atomicExch(info, (int)(k + c + 1));
                d = 1e-300;
            }
            const double lcc = sqrt(d);
            L[c * kLd + c] = lcc;
            rd[c] = 1.0 / lcc;
        }
        __syncthreads();
        const double inv = rd[c];
        for (int r = c + 1 + t; r < kb; r += kPotrfThreads) L[r * kLd + c] *= inv;
        __syncthreads();
        const int q = c + 1 + cx;
        if (q < kb) {
            const double lqc = L[q * kLd + c];
            for (int r = q + ((ry - (q - c - 1)) & 3); r < kb; r += 4) L[r * kLd + q] -= L[r * kLd + c] * lqc;
        }
        __syncthreads();  // the next pivot reads this update
    }
    for (int kk = 0; kk < kb; ++kk) {
        const double inv = rd[kk];
        if (t <= kk) X[kk * kLd + t] *= inv;
        __syncthreads();
        // rows i > kk, columns j <= kk:  X[i][j] -= L[i][kk] X[kk][j]
        if (cx <= kk) {
            const double xk = X[kk * kLd + cx];
            for (int i = kk + 1 + ry; i < kb; i += 4) X[i * kLd + cx] -= L[i * kLd + kk] * xk;
        }
        __syncthreads();
    }
    for (int e = t; e < kNB * kNB; e += kPotrfThreads) {
        const int r = e >> 6, c = e & 63;
        if (r < kb && c <= r) A[(size_t)(k + r) * n + k + c] = L[r * kLd + c];
        Linv[(size_t)r * kNB + c] = (r < kb && c <= r) ? X[r * kLd + c] : 0.0;
    }
}

constexpr size_t kPotrfSmem = (size_t)(2 * kNB * kLd + kNB) * sizeof(double);

// y_k = Linv_k b_k (forward step of L y = b on block k).
__global__ void k_trsv_inv_lower(const double *__restrict__ Linv, int64_t k, int kb, double *__restrict__ b) {
    __shared__ double v[kNB];
    const int t = threadIdx.x;
    v[t] = t < kb ? b[k + t] : 0.0;
    __syncthreads();
    double acc = 0.0;
    for (int c = 0; c <= t && c < kb; ++c) acc += Linv[(size_t)t * kNB + c] * v[c];
    if (t < kb) b[k + t] = acc;
}

// x_k = Linv_k^T y_k (backward step of L^T x = y on block k).
__global__ void k_trsv_inv_upper(const double *__restrict__ Linv, int64_t k, int kb, double *__restrict__ b) {
    __shared__ double v[kNB];
    const int t = threadIdx.x;
    v[t] = t < kb ? b[k + t] : 0.0;
    __syncthreads();
    double acc = 0.0;
    for (int c = t; c < kb; ++c) acc += Linv[(size_t)c * kNB + t] * v[c];
    if (t < kb) b[k + t] = acc;
}

__global__ void k_trsv_sub_lower(const double *__restrict__ A, int64_t n, int64_t k, int kb,
                                 double *__restrict__ b) {
    const int lane = threadIdx.x & 31;
    const int64_t r = k + kb + (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= n) return;
    double acc = 0.0;
    for (int c = lane; c < kb; c += 32) acc += A[(size_t)r * n + k + c] * b[k + c];
    acc = warp_sum(acc);
    if (lane == 0) b[r] -= acc;
}

__global__ void k_trsv_sub_upper(const double *__restrict__ A, int64_t n, int64_t k, int kb,
                                 double *__restrict__ b) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= k) return;
    double acc = 0.0;
    for (int c = 0; c < kb; ++c) acc += A[(size_t)(k + c) * n + r] * b[k + c];
    b[r] -= acc;
}

// Lower triangle of K holds g_t = t_k . t_l; replace it (both triangles) by
// the Gram of the Jacobian rows g_s + g_t + g_t g_s with g_s = s_k . s_l
// (exact integer dot products of the +-1 configurations).
__global__ void __launch_bounds__(256) k_gram_combine(int N, int64_t Ns, const int8_t *__restrict__ s,
                                                      double *__restrict__ K) {
    __shared__ __align__(16) int8_t sa[64][132];
    __shared__ __align__(16) int8_t sb[64][132];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * 64, n0 = (int64_t)blockIdx.x * 64;
    if (n0 > m0 + 63) return;
    int gs[4][4] = {};
    for (int i0 = 0; i0 < N; i0 += 128) {
        for (int e = threadIdx.x; e < 64 * 128; e += 256) {
            const int r = e >> 7, c = e & 127;
            const int i = i0 + c;
            sa[r][c] = (m0 + r < Ns && i < N) ? s[(size_t)(m0 + r) * N + i] : (int8_t)0;
            sb[r][c] = (n0 + r < Ns && i < N) ? s[(size_t)(n0 + r) * N + i] : (int8_t)0;
        }
        __syncthreads();
        for (int c = 0; c < 128; c += 4) {
            int av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                av[u] = *reinterpret_cast<const int *>(&sa[ty * 4 + u][c]);
                bv[u] = *reinterpret_cast<const int *>(&sb[tx * 4 + u][c]);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) gs[u][v] = __dp4a(av[u], bv[v], gs[u][v]);
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
            const double gt = K[(size_t)k * Ns + l];
            const double g = (double)gs[u][v] + gt + gt * (double)gs[u][v];
            K[(size_t)k * Ns + l] = g;
            K[(size_t)l * Ns + k] = g;
        }
    }
}

size_t ozaki_smem_bytes() {
    return 1024 + (size_t)kMaxSlices * (kABytes + kBBytes) + 2 * sizeof(uint64_t) + 2 * sizeof(uint32_t) + 16;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ============================================================ launchers ====

size_t slice_elems(int64_t rows, int S) { return (size_t)S * (size_t)rows * kTileK; }

cudaError_t launch_slice_rows(const double *A, int64_t lda, int64_t rows, int kcols, int S,
                              __nv_bfloat16 *out, int *expo, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (kcols < 1 || kcols > kTileK || S < 1 || S > kMaxSlices) return cudaErrorInvalidValue;
    (k_slice_rows<<<nblk(rows, 8), 256, 0, st>>>(A, lda, rows, kcols, S, out, expo), nk::note_launch());
    return cudaGetLastError();
}

// R = A B^T (FP64-accurate to the slice count), applied to C by mode.
// A and B are given by their slices (rows x 64, as written by
// launch_slice_rows) and row exponents.
cudaError_t launch_ozaki_gemm_strided(const __nv_bfloat16 *Asl, const int *expA, int64_t rows, int64_t a_stride,
                                      const __nv_bfloat16 *Bsl, const int *expB, int64_t cols, int64_t b_stride,
                                      int S, double *C, int64_t ldc, int mode, bool lower, int *err,
                                      cudaStream_t st) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if (S < 1 || S > kMaxSlices) return cudaErrorInvalidValue;
    if (rows > (1LL << 31) - kTileM || cols > (1LL << 31) - kTileN) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_slice_map(&ma, Asl, rows, S, kTileM, a_stride) || !make_slice_map(&mb, Bsl, cols, S, kTileN, b_stride))
        return cudaErrorInvalidValue;
    cudaError_t attr_err = cudaFuncSetAttribute(k_ozaki_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)ozaki_smem_bytes());
    if (attr_err != cudaSuccess) return attr_err;
    OzArgs a{rows, cols, S, expA, expB, C, ldc, mode, lower ? 1 : 0, err};
    dim3 grid(nblk(cols, kTileN), nblk(rows, kTileM));
    (k_ozaki_gemm<<<grid, kOzThreads, ozaki_smem_bytes(), st>>>(ma, mb, a), nk::note_launch());
    return cudaGetLastError();
}

// BF16 MMA flops a launch executes: active tiles x S(S+1)/2 slice products x
// 2 x 128 x 64 x 64.
double ozaki_mma_flops(int64_t rows, int64_t cols, int S, bool lower) {
    const int64_t tm = (rows + kTileM - 1) / kTileM, tn = (cols + kTileN - 1) / kTileN;
    int64_t tiles = 0;
    for (int64_t i = 0; i < tm; ++i) {
        const int64_t m0 = i * kTileM;
        tiles += lower ? (m0 + kTileM - 1) / kTileN + 1 < tn ? (m0 + kTileM - 1) / kTileN + 1 : tn : tn;
    }
    return (double)tiles * (S * (S + 1) / 2) * 2.0 * kTileM * kTileN * kTileK;
}

cudaError_t launch_ozaki_gemm(const __nv_bfloat16 *Asl, const int *expA, int64_t rows,
                              const __nv_bfloat16 *Bsl, const int *expB, int64_t cols, int S, double *C,
                              int64_t ldc, int mode, bool lower, int *err, cudaStream_t st) {
    return launch_ozaki_gemm_strided(Asl, expA, rows, rows, Bsl, expB, cols, cols, S, C, ldc, mode, lower, err, st);
}

size_t tc_chol_ws_bytes(int64_t n) {
    const int64_t nb = (n + kNB - 1) / kNB;
    return 2 * slice_elems(n, kMaxSlices) * 2 + slice_elems(kNB, kMaxSlices) * 2 + (size_t)(2 * n + kNB) * 4 +
           (size_t)nb * kNB * kNB * 8 + 8 * 256;
}

namespace {
struct TcWs {
    __nv_bfloat16 *Asl, *Bsl, *Asl2;
    int *expA, *expB, *expA2;
    double *Linv;
};
TcWs carve_tc(void *ws, int64_t n) {
    char *p = static_cast<char *>(ws);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) & ~size_t(255);
        return q;
    };
    TcWs w;
    w.Asl = reinterpret_cast<__nv_bfloat16 *>(take(slice_elems(n, kMaxSlices) * 2));
    w.Bsl = reinterpret_cast<__nv_bfloat16 *>(take(slice_elems(kNB, kMaxSlices) * 2));
    w.expA = reinterpret_cast<int *>(take((size_t)n * 4));
    w.expB = reinterpret_cast<int *>(take((size_t)kNB * 4));
    w.Linv = reinterpret_cast<double *>(take((size_t)((n + kNB - 1) / kNB) * kNB * kNB * 8));
    w.Asl2 = reinterpret_cast<__nv_bfloat16 *>(take(slice_elems(n, kMaxSlices) * 2));
    w.expA2 = reinterpret_cast<int *>(take((size_t)n * 4));
    return w;
}
}  // namespace

// Blocked right-looking Cholesky with tensor-core (Ozaki, 7 slices) panel
// solves and trailing updates, and a look-ahead of one panel: after panel k
// the main stream first updates only block column k + 1 ("narrow" update),
// then the side stream factors panel k + 1 (diagonal block, its inverse, the
// panel product and its slices) while the main stream applies panel k to the
// rest of the trailing matrix ("wide" update).  Panel slices alternate
// between two buffers.  The inverted diagonal blocks stay in the workspace
// for launch_cholesky_solve_tc.
namespace {

// Factor panel k (columns k0 .. k0 + kb - 1) whose block column is up to date:
// diagonal block + inverse, L_panel = A_panel L_kk^-T, slices of L_panel.
cudaError_t panel_step(double *A, int64_t n, int64_t k0, int *info, int *err, TcWs &w, __nv_bfloat16 *Lsl,
                       int *Lexp, cudaStream_t st) {
    const int S = kMaxSlices;
    const int kb = (int)(n - k0 < kNB ? n - k0 : kNB);
    const int64_t rest = n - k0 - kb;
    double *Linv = w.Linv + (size_t)(k0 / kNB) * kNB * kNB;
    const int slot = prof_begin(NK_PROF_CHOL_PANEL, st);
    (k_potrf_inv<<<1, kPotrfThreads, kPotrfSmem, st>>>(A, n, k0, kb, info, Linv), nk::note_launch());
    cudaError_t e = cudaSuccess;
    if (rest > 0) {
        double *panel = A + (size_t)(k0 + kb) * n + k0;
        e = launch_slice_rows(Linv, kNB, kb, kb, S, w.Bsl, w.expB, st);
        if (e == cudaSuccess) e = launch_slice_rows(panel, n, rest, kb, S, Lsl, Lexp, st);
        if (e == cudaSuccess)
            e = launch_ozaki_gemm(Lsl, Lexp, rest, w.Bsl, w.expB, kb, S, panel, n, 0, false, err, st);
        if (e == cudaSuccess) e = launch_slice_rows(panel, n, rest, kb, S, Lsl, Lexp, st);
    }
    prof_end(slot, st, (double)kb * kb * kb / 3.0 + 2.0 * (double)rest * kb * kb);
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t launch_cholesky_tc(double *A, int64_t n, int *info, int *err, void *ws, cudaStream_t st,
                               cudaStream_t side, cudaEvent_t ev_narrow, cudaEvent_t ev_panel) {
    TcWs w = carve_tc(ws, n);
    const int S = kMaxSlices;
    cudaError_t e = cudaFuncSetAttribute(k_potrf_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPotrfSmem);
    if (e != cudaSuccess) return e;
    __nv_bfloat16 *buf[2] = {w.Asl, w.Asl2};
    int *bexp[2] = {w.expA, w.expA2};
    const int64_t nb = (n + kNB - 1) / kNB;
    e = panel_step(A, n, 0, info, err, w, buf[0], bexp[0], st);
    if (e != cudaSuccess) return e;
    for (int64_t k = 0; k + 1 < nb; ++k) {
        const int64_t k0 = k * kNB;
        const int64_t rest = n - k0 - kNB;         // rows of panel k below its diagonal block
        const int kb1 = (int)(rest < kNB ? rest : kNB);  // width of block column k + 1
        __nv_bfloat16 *Lk = buf[k & 1];
        int *Le = bexp[k & 1];
        double *C1 = A + (size_t)(k0 + kNB) * n + (k0 + kNB);
        int slot = prof_begin(NK_PROF_CHOL_UPDATE, st);
        // narrow: block column k + 1 (all rows below panel k)
        e = launch_ozaki_gemm_strided(Lk, Le, rest, rest, Lk, Le, kb1, rest, S, C1, n, 1, true, err, st);
        prof_end(slot, st, ozaki_mma_flops(rest, kb1, S, true));
        if (e != cudaSuccess) return e;
        if (side) {
            e = cudaEventRecord(ev_narrow, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_narrow, 0);
            if (e != cudaSuccess) return e;
        }
        cudaStream_t ps = side ? side : st;
        e = panel_step(A, n, k0 + kNB, info, err, w, buf[(k + 1) & 1], bexp[(k + 1) & 1], ps);
        if (e != cudaSuccess) return e;
        if (side) {
            e = cudaEventRecord(ev_panel, side);
            if (e != cudaSuccess) return e;
        }
        // wide: everything right of block column k + 1
        const int64_t rest2 = rest - kb1;
        if (rest2 > 0) {
            slot = prof_begin(NK_PROF_CHOL_UPDATE, st);
            e = launch_ozaki_gemm_strided(Lk + (size_t)kb1 * kTileK, Le + kb1, rest2, rest, Lk + (size_t)kb1 * kTileK,
                                          Le + kb1, rest2, rest, S, C1 + (size_t)kb1 * n + kb1, n, 1, true, err, st);
            prof_end(slot, st, ozaki_mma_flops(rest2, rest2, S, true));
            if (e != cudaSuccess) return e;
        }
        if (side) {
            e = cudaStreamWaitEvent(st, ev_panel, 0);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_cholesky_solve_tc(const double *L, int64_t n, const void *ws, double *b, cudaStream_t st) {
    TcWs w = carve_tc(const_cast<void *>(ws), n);
    const int slot = prof_begin(NK_PROF_TRSV, st);
    for (int64_t k = 0; k < n; k += kNB) {
        const int kb = (int)(n - k < kNB ? n - k : kNB);
        const double *Linv = w.Linv + (size_t)(k / kNB) * kNB * kNB;
        (k_trsv_inv_lower<<<1, kNB, 0, st>>>(Linv, k, kb, b), nk::note_launch());
        const int64_t rest = n - k - kb;
        if (rest > 0) (k_trsv_sub_lower<<<nblk(rest, 8), 256, 0, st>>>(L, n, k, kb, b), nk::note_launch());
    }
    const int64_t last = ((n - 1) / kNB) * kNB;
    for (int64_t k = last; k >= 0; k -= kNB) {
        const int kb = (int)(n - k < kNB ? n - k : kNB);
        const double *Linv = w.Linv + (size_t)(k / kNB) * kNB * kNB;
        (k_trsv_inv_upper<<<1, kNB, 0, st>>>(Linv, k, kb, b), nk::note_launch());
        if (k > 0) (k_trsv_sub_upper<<<nblk(k, 256), 256, 0, st>>>(L, n, k, kb, b), nk::note_launch());
    }
    prof_end(slot, st, 2.0 * (double)n * (double)n);
    return cudaGetLastError();
}

// Lower triangle of K = T T^T by tensor cores with S slices per 64-column
// chunk of T [Ns][M], then the Jacobian-row Gram s.s + t.t + (t.t)(s.s)
// written to both triangles.
cudaError_t launch_gram_tc(int N, int M, int64_t Ns, const int8_t *s, const double *T, int S, double *K,
                           int *err, void *ws, cudaStream_t st) {
    TcWs w = carve_tc(ws, Ns);
    const int slot = prof_begin(NK_PROF_GRAM, st);
    for (int c = 0; c < M; c += kTileK) {
        const int kc = M - c < kTileK ? M - c : kTileK;
        cudaError_t e = launch_slice_rows(T + c, M, Ns, kc, S, w.Asl, w.expA, st);
        if (e == cudaSuccess)
            e = launch_ozaki_gemm(w.Asl, w.expA, Ns, w.Asl, w.expA, Ns, S, K, Ns, c == 0 ? 0 : 2, true, err, st);
        if (e != cudaSuccess) return e;
    }
    dim3 grid(nblk(Ns, 64), nblk(Ns, 64));
    (k_gram_combine<<<grid, 256, 0, st>>>(N, Ns, s, K), nk::note_launch());
    prof_end(slot, st, (double)Ns * (Ns + 1) * (double)(N + M));
    return cudaGetLastError();
}

}  // namespace nk
