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
// Kernel shape: a CTA per strip of up to eight 128 x 32 output tiles (K =
// 64): TMA brings the S slices of the A rows (once per strip) and of the B
// rows (3-D tensor maps [S][rows][64] BF16, 128-byte swizzle), one thread
// issues S x 4 tcgen05.mma (M = 128, K = 16, A slice s against B slices
// 1 .. S+1-s side by side: N = 32 (S+1-s)) into S accumulators of 32 TMEM
// columns, double-buffered, and sixteen warps drain the other buffer and
// update C.  Every wait is bounded by the global timer; on time-out the
// kernel records an error code, lets its copies and MMAs in flight finish,
// frees its TMEM and returns.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "nk_common.cuh"
#include "nk_internal.h"
#include "tc_ptx.cuh"

namespace nk {

namespace {

constexpr int kTileM = 128;
constexpr int kTileK = 64;
constexpr int kMaxSlices = 7;
constexpr uint32_t kTmemCols = 512;
constexpr int kABytes = kTileM * kTileK * 2;  // one slice of the A tile

// ---------------------------------------------------------------- slicing ---

// One warp per row: the first kcols (<= 64) entries of row r of A (row
// stride lda) -> S BF16 integer slices out[s][r][0..63] (zero beyond kcols)
// and the row exponent e_r (max |a_rk| < 2^e_r).  The slices are the bytes,
// from the top, of the fixed-point magnitude floor(|a| 2^(8S - e_r)), with the
// sign of a: exactly the digits of repeated multiply-by-256-and-truncate,
// taken from the FP64 bit pattern with integer shifts only.
// The warp's row r, with lane l holding columns l (x0) and l + 32 (x1), as S
// slices out[q][r][0..63] (plane stride `rows` rows) and the row exponent.
__device__ __forceinline__ void slice_row_warp(double x0, double x1, int lane, int64_t rows, int64_t r, int S,
                                               __nv_bfloat16 *__restrict__ out, int *__restrict__ expo) {
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

__global__ void k_slice_rows(const double *__restrict__ A, int64_t lda, int64_t rows, int kcols, int S,
                             __nv_bfloat16 *__restrict__ out, int *__restrict__ expo) {
    const int lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const double x0 = lane < kcols ? A[(size_t)r * lda + lane] : 0.0;
    const double x1 = lane + 32 < kcols ? A[(size_t)r * lda + lane + 32] : 0.0;
    slice_row_warp(x0, x1, lane, rows, r, S, out, expo);
}

// Columns p of rows r0 .. r0 + kr - 1 (kr <= 64) of X [.][ldx] -> S BF16
// integer slices out[s][p][0..63] (zero beyond kr) with the column exponent
// expo[p] (max over those rows): the transposed counterpart of k_slice_rows,
// same digits.  One block per 32 columns, staged through shared memory.
__global__ void __launch_bounds__(256) k_slice_cols(const double *__restrict__ X, int64_t ldx, int64_t r0, int kr,
                                                    int64_t ncols, int S, __nv_bfloat16 *__restrict__ out,
                                                    int *__restrict__ expo) {
    __shared__ double tile[kTileK][33];
    __shared__ int ex[32];
    const int tid = threadIdx.x;
    const int64_t p0 = (int64_t)blockIdx.x * 32;
    for (int idx = tid; idx < kTileK * 32; idx += 256) {
        const int r = idx >> 5, c = idx & 31;
        tile[r][c] = (r < kr && p0 + c < ncols) ? X[(size_t)(r0 + r) * ldx + p0 + c] : 0.0;
    }
    __syncthreads();
    if (tid < 32) {
        int e = -100000;
        for (int r = 0; r < kTileK; ++r) {
            int b;
            unsigned long long m;
            bool n;
            split_bits(tile[r][tid], b, m, n);
            if (m) e = max(e, b - 1022);
        }
        e = e == -100000 ? 0 : e;
        ex[tid] = e;
        if (p0 + tid < ncols) expo[p0 + tid] = e;
    }
    __syncthreads();
    for (int idx = tid; idx < kTileK * 32; idx += 256) {
        const int c = idx >> 6, r = idx & 63;
        if (p0 + c >= ncols) continue;
        int b;
        unsigned long long m;
        bool n;
        split_bits(tile[r][c], b, m, n);
        unsigned long long y = 0;
        if (m) {
            const int sh = b - 1075 + 8 * S - ex[c];
            y = sh >= 0 ? (m << sh) : (sh <= -64 ? 0ULL : (m >> (-sh)));
        }
        for (int q = 0; q < S; ++q) {
            const int d = (int)((y >> (8 * (S - 1 - q))) & 0xFFULL);
            out[((size_t)q * ncols + p0 + c) * kTileK + r] = __int2bfloat16_rn(n ? -d : d);
        }
    }
}

// C <- scale C + eps I on the lower triangle.
__global__ void k_scale_shift_lower(double *__restrict__ C, int64_t n, double scale, double eps) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t i = blockIdx.y; i < n; i += gridDim.y) {
        if (j > i || j >= n) continue;
        double v = C[(size_t)i * n + j] * scale;
        if (i == j) v += eps;
        C[(size_t)i * n + j] = v;
    }
}

// ------------------------------------------------------------- the GEMM ---
//
// Warp-specialised kernel over output strips: a CTA owns up to `chunk` (<= 8)
// consecutive 128 x 32 tiles of one tile row (a 128 x 256 strip at most), keeps the
// S slices of its 128 A rows resident, and pipelines the tiles:
//   warp 0 (one thread): TMA producer, A slices once, B slices per tile into
//     one of two buffers;
//   warp 1 (one thread): MMA issuer, S MMAs (one per A slice, against the
//     B slices side by side) x 4 K-steps per tile into one of two TMEM
//     accumulator sets (S x 32 columns each), so
//     that the MMAs of tile i+1 run while tile i is drained;
//   warps 2-17: epilogue; warp w owns tile rows 32 (w % 4) .. +31 (its TMEM
//     lane quarter) and 8 columns, loads its C entries a tile ahead, and
//     turns the S accumulators into FP64 by exact integer recombination
//     before writing C back.
// Strips (lower triangle only when `lower`) are numbered row by row.  CTAs
// are short-lived on purpose: kernels of a higher-priority stream (the
// Cholesky look-ahead) get SMs as strips retire.  mbarriers hand buffers
// between the roles; every wait is bounded by the global timer and gives up
// when another role of the CTA has aborted.

struct OzArgs {
    int64_t rows, cols;   // output rows (A rows) and columns (B rows)
    int S;
    const int *expA, *expB;
    double *C;
    int64_t ldc;
    int mode;             // 0: C = R, 1: C -= R, 2: C += R
    int lower;            // only entries with col <= row (tiles above are skipped)
    int *err;
    int64_t n_nb;         // tile columns
    int chunk;            // tiles per strip: 1, 2, 4 or 8
    int chunk_log2;
};

constexpr int kPN = 32;                      // tile columns
constexpr int kMaxChunk = 8;                 // tiles per strip at most
constexpr int kPEpiWarps = 16;
constexpr int kPThreads = 64 + 32 * kPEpiWarps;        // producer, MMA issuer, epilogue warps
constexpr int kPColsPerWarp = kPN / (kPEpiWarps / 4);  // 8
constexpr int kPBBytes = kPN * kTileK * 2;   // one slice of the B tile (4 KB)
constexpr uint32_t kPAccCols = 256;          // TMEM columns per accumulator set

__host__ __device__ inline int64_t oz_row_tiles(int64_t n_nb, bool lower, int64_t mb) {
    if (!lower) return n_nb;
    const int64_t last = (mb * kTileM + kTileM - 1) / kPN + 1;
    return last < n_nb ? last : n_nb;
}

// strips of tile row mb (a power-of-two chunk: every CTA walks the rows before
// its own, so the step is a shift, not a 64-bit division)
__host__ __device__ inline int64_t oz_row_strips(int64_t n_nb, bool lower, int64_t mb, int chunk_log2) {
    return (oz_row_tiles(n_nb, lower, mb) + ((int64_t)1 << chunk_log2) - 1) >> chunk_log2;
}

// The MMAs of one tile: level g = s + t (2 .. S+1) collects the products of
// A slice s and B slice t in TMEM columns dbase + (g - 2) 32.  The B slices
// of a tile lie back to back in shared memory ([S][32][64], 128-byte rows),
// so B slices 1 .. S+1-s read as one operand of 32 (S+1-s) rows, and a single
// MMA of that width adds A slice s times all of them to the contiguous levels
// s+1 .. S+1.  S MMAs per K-step (instead of S(S+1)/2 of width 32) read each
// A slice once; the first one of a tile (s = 1, K-step 0) initialises every
// level.  SS > 0 fixes S at compile time.
template <int SS>
__device__ __forceinline__ void issue_tile(uint32_t dbase, uint64_t da, uint64_t db,
                                           const uint32_t (&idesc)[kMaxSlices], int S_rt) {
    const int S = SS > 0 ? SS : S_rt;
    constexpr int kS = (SS > 0 ? SS : kMaxSlices);
#pragma unroll 1
    for (int kk = 0; kk < kTileK / 16; ++kk) {
#pragma unroll
        for (int sa = 1; sa <= kS; ++sa) {
            if (sa > S) continue;
            const uint32_t acc = (kk > 0 || sa > 1) ? 1u : 0u;
            // A slice sa starts (sa - 1) kABytes after slice 1 (descriptor address field in 16-byte units)
            umma_bf16(dbase + (uint32_t)((sa - 1) * kPN), da + (uint64_t)((sa - 1) * (kABytes >> 4) + kk * 2),
                      db + (uint64_t)(kk * 2), idesc[sa - 1], acc);
        }
    }
}

template <int SS>
__global__ void __launch_bounds__(kPThreads, 1)
    k_ozaki_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, OzArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *ops = smem_raw + ((1024 - (base & 1023)) & 1023);
    unsigned char *sA = ops;                                            // [S][128][64] bf16
    unsigned char *sB = ops + (size_t)kMaxSlices * kABytes;             // [2][S][32][64] bf16
    unsigned char *sE = sB + (size_t)2 * kMaxSlices * kPBBytes;         // [16 warps][32][8] fp64
    uint64_t *bars = reinterpret_cast<uint64_t *>(sE + (size_t)kPEpiWarps * 32 * kPColsPerWarp * 8);
    uint64_t *a_full = bars, *b_full = bars + 2, *b_empty = bars + 4;
    uint64_t *acc_full = bars + 6, *acc_empty = bars + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 10);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = SS > 0 ? SS : a.S;
    // strip -> tile row mb, first tile column nb0, tile count: every warp scans
    // the strips per tile row, 32 rows per round (inclusive prefix by
    // shuffles), and takes the first row whose prefix passes blockIdx.x
    int64_t mb = 0, rem = blockIdx.x;
    {
        const int64_t n_mb = (a.rows + kTileM - 1) / kTileM;
        for (int64_t base = 0; base < n_mb; base += 32) {
            const int64_t m = base + lane;
            const int64_t ns = m < n_mb ? oz_row_strips(a.n_nb, a.lower != 0, m, a.chunk_log2) : 0;
            int64_t incl = ns;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += v;
            }
            const int64_t total = __shfl_sync(0xffffffffu, incl, 31);
            if (rem < total) {  // warp-uniform
                const int l = __ffs(__ballot_sync(0xffffffffu, rem < incl)) - 1;
                mb = base + l;
                rem -= __shfl_sync(0xffffffffu, incl - ns, l);
                break;
            }
            rem -= total;
            mb = base + 32;
        }
    }
    const int64_t nb0 = rem << a.chunk_log2, in_row = oz_row_tiles(a.n_nb, a.lower != 0, mb);
    const int count = (int)(in_row - nb0 < a.chunk ? in_row - nb0 : a.chunk);
    const int64_t m0 = mb * kTileM;

    if (threadIdx.x == 0) {
        mbar_init(a_full, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&b_full[b], 1);
            mbar_init(&b_empty[b], 1);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kPEpiWarps);
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    auto fail = [&](int code) {
        *abort_flag = 1;
        atomicExch(a.err, code);
    };

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        uint32_t fills0 = 0, fills1 = 0;  // loads issued into B buffer 0 / 1
        mbar_expect_tx(a_full, (uint32_t)S * kABytes);
        for (int s = 0; s < S; ++s) tma_load_3d(sA + (size_t)s * kABytes, &mapA, a_full, 0, (int)m0, s);
        for (int i = 0; i < count && !*abort_flag; ++i) {
            const int b = i & 1;
            const uint32_t fills = b ? fills1 : fills0;
            if (fills > 0 && !mbar_wait_or_abort(&b_empty[b], (fills - 1) & 1, abort_flag)) {
                fail(12);
                break;
            }
            mbar_expect_tx(&b_full[b], (uint32_t)S * kPBBytes);
            for (int s = 0; s < S; ++s)
                tma_load_3d(sB + (size_t)(b * kMaxSlices + s) * kPBBytes, &mapB, &b_full[b], 0,
                            (int)((nb0 + i) * kPN), s);
            if (b)
                ++fills1;
            else
                ++fills0;
        }
        if (*abort_flag) {
            // let the copies in flight land before the CTA exits
            mbar_wait(a_full, 0);
            if (fills0 > 0) mbar_wait(&b_full[0], (fills0 - 1) & 1);
            if (fills1 > 0) mbar_wait(&b_full[1], (fills1 - 1) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------- MMA issuer
        int issued = 0;
        uint32_t idesc[kMaxSlices];  // A slice s + 1 meets B slices 1 .. S - s: N = 32 (S - s)
#pragma unroll
        for (int s = 0; s < kMaxSlices; ++s) idesc[s] = idesc_bf16(kTileM, kPN * (S - s > 0 ? S - s : 1));
        const uint64_t da = sw128_desc(sA), db0 = sw128_desc(sB),
                       db1 = sw128_desc(sB + (size_t)kMaxSlices * kPBBytes);
        if (!mbar_wait_or_abort(a_full, 0, abort_flag)) fail(13);
        for (int i = 0; i < count && !*abort_flag; ++i) {
            const int b = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            if (!mbar_wait_or_abort(&b_full[b], use & 1, abort_flag)) {
                fail(14);
                break;
            }
            if (use > 0 && !mbar_wait_or_abort(&acc_empty[b], (use - 1) & 1, abort_flag)) {
                fail(15);
                break;
            }
            tc_fence_after();
            if (b)
                issue_tile<SS>(tmem + kPAccCols, da, db1, idesc, S);
            else
                issue_tile<SS>(tmem, da, db0, idesc, S);
            umma_commit(&acc_full[b]);
            umma_commit(&b_empty[b]);
            ++issued;
        }
        if (*abort_flag && issued > 0) {
            // the MMAs in flight must finish before the TMEM is released
            const int last = issued - 1;
            mbar_wait(&acc_full[last & 1], (uint32_t)(last >> 1) & 1);
        }
    } else if (warp >= 2) {
        // --------------------------------------------------------- epilogue
        // Lane l turns TMEM lane 32q + l (tile row 32q + l) into FP64 for the
        // warp's 8 columns and parks the values in its shared block
        // [32 rows][8 columns] (column index XOR (row / 2) mod 8: conflict-free
        // for both access patterns); C is then read and written with lane l on
        // row 4k + l / 8, column l mod 8 (k = 0 .. 7), 64-byte row segments.
        const int q = warp & 3;                 // TMEM lane quarter = tile rows 32q .. 32q + 31
        const int c0 = ((warp - 2) >> 2) * kPColsPerWarp;  // the warp's 8 tile columns
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        double *stage = reinterpret_cast<double *>(sE) + (warp - 2) * 32 * kPColsPerWarp;
        const int64_t row = m0 + q * 32 + lane;
        const int ei = row < a.rows ? a.expA[row] : 0;
        const int rr = lane >> 3, cc = lane & 7;
        const int64_t row_c = m0 + q * 32 + rr;  // + 4k: the rows this lane reads and writes in C
        auto on = [&](int64_t r, int64_t col) { return r < a.rows && col < a.cols && !(a.lower && col > r); };
        auto load_c = [&](int i, double (&cv)[8]) {
            const int64_t col = (nb0 + i) * kPN + c0 + cc;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int64_t r = row_c + 4 * k;
                cv[k] = (a.mode != 0 && on(r, col)) ? a.C[(size_t)r * a.ldc + col] : 0.0;
            }
        };
        // column exponents (lane & 7 holds column c0 + (lane & 7)), broadcast by shuffles
        auto load_f = [&](int i) {
            const int64_t col = (nb0 + i) * kPN + c0 + cc;
            return col < a.cols ? a.expB[col] : 0;
        };
        const long long flip = a.mode == 1 ? (long long)0x8000000000000000ULL : 0LL;
        if (a.mode != 0) {
            // the strip's C entries (at most 128 x 256 FP64 per CTA) into L2 up
            // front, so that the per-tile loads below wait on L2, not on HBM
            for (int i = 0; i < count; ++i) {
                const int64_t col = (nb0 + i) * kPN + c0 + cc;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int64_t r = row_c + 4 * k;
                    if (on(r, col)) prefetch_l2(a.C + (size_t)r * a.ldc + col);
                }
            }
        }
        for (int i = 0; i < count; ++i) {
            const int b = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            // this tile's C entries and column exponents are in flight while
            // the accumulators fill and drain; C is needed only at the end
            double cv[8];
            load_c(i, cv);
            const int fj_lane = load_f(i);
            int ok = 1;
            if (lane == 0) ok = mbar_wait_or_abort(&acc_full[b], use & 1, abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) fail(16);
                break;
            }
            tc_fence_after();
#pragma unroll 1
            for (int c4 = 0; c4 < kPColsPerWarp; c4 += 2) {
                uint32_t r[kMaxSlices][2];
#pragma unroll
                for (int gi = 0; gi < kMaxSlices; ++gi)
                    if (gi < S)
                        tmem_ld2(tmem + (uint32_t)b * kPAccCols + lane_base + (uint32_t)(gi * kPN + c0 + c4), r[gi]);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    int d[kMaxSlices];
#pragma unroll
                    for (int gi = 0; gi < kMaxSlices; ++gi)
                        d[gi] = gi < S ? __float2int_rn(__uint_as_float(r[gi][j])) : 0;
                    // V 2^sc with V = sum_g D_g 2^(8 (8 - g)); C - R as C + (-R)
                    const int sc = ei + __shfl_sync(0xffffffffu, fj_lane, c4 + j) - 64;
                    const double v = __longlong_as_double(
                        __double_as_longlong(window_to_double(ozaki_window8(d), sc + 8)) ^ flip);
                    const int c = c4 + j;
                    stage[lane * 8 + (c ^ ((lane >> 1) & 7))] = v;
                }
            }
            // the accumulators are drained: hand the buffer back before the C traffic
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            const int64_t col = (nb0 + i) * kPN + c0 + cc;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int rl = 4 * k + rr;
                const double v = stage[rl * 8 + (cc ^ ((rl >> 1) & 7))];
                const int64_t r = row_c + 4 * k;
                if (on(r, col)) a.C[(size_t)r * a.ldc + col] = cv[k] + v;  // C reads as 0 in mode 0
            }
            __syncwarp();
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

// Factor the kb x kb diagonal block at (k, k) in place (lower).  One CTA of
// 256 threads holds the block in shared memory (continued by the identity
// beyond kb) and factors it column by column with a look-ahead of one:
//   * warp 0 carries the dependency chain (lanes hold rows lane and
//     lane + 32): it updates column c+1 with the finished column c in
//     registers, broadcasts the pivot d_{c+1} by shuffle, and scales column
//     c+1 by d_{c+1}^-1/2;
//   * meanwhile six warps (none on warp 0's SM sub-partition) apply column c
//     to the columns right of c+1: a_rq -= l_rc l_qc, c+2 <= q <= r, over a
//     packed table of the lower triangle ordered by column q descending
//     (entries with q >= x are its first (64 - x)(65 - x)/2), four entries
//     per thread at a time so that their FMA chains overlap.
// One barrier per column; kb^3/6 FMAs.  On this part a dependent FP64
// operation takes tens of cycles and an FP64 reciprocal square root hundreds
// (pairing columns to share one did not pay: the longer FP64 sequence per
// pair cost more), so the chain per column is one FMA, one shuffle, one
// rsqrt and one multiply, with the positivity test done on the bit pattern.
constexpr int kPotrfThreads = 256;
constexpr int kLd = kNB + 1;
constexpr int kTriEntries = kNB * (kNB - 1) / 2 + 0;  // (r, q) with 1 <= q <= r <= 63: 2016

__host__ __device__ constexpr int tri_from(int x) {  // packed entries with column q >= x (1 <= x <= 64)
    return (64 - x) * (65 - x) / 2;
}

__device__ __forceinline__ bool positive_finite(double x) {  // integer compares, off the FP64 pipe
    const long long bits = __double_as_longlong(x);
    return bits > 0 && bits < 0x7FF0000000000000LL;
}

__global__ void __launch_bounds__(kPotrfThreads) k_potrf64(double *__restrict__ A, int64_t n, int64_t k, int kb,
                                                           int *__restrict__ info) {
    __shared__ double L[kNB * kLd];
    __shared__ uint16_t tab[kTriEntries];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    for (int e = t; e < kNB * kNB; e += kPotrfThreads) {
        const int r = e >> 6, c = e & 63;
        L[r * kLd + c] = (r < kb && c <= r) ? A[(size_t)(k + r) * n + k + c] : (r == c ? 1.0 : 0.0);
    }
    // column q (1 .. 63) owns entries [(63 - q)(64 - q)/2, +64 - q): rows q .. 63
    if (t >= 1 && t < kNB) {
        const int q = t, s0 = (63 - q) * (64 - q) / 2;
        for (int r = q; r < kNB; ++r) tab[s0 + r - q] = (uint16_t)((r << 8) | q);
    }
    const int r0 = lane, r1 = lane + 32;
    // warp 0: pivot of column c from d (its updated diagonal) and the scaling
    // of the column's rows below, held as v0 (row r0) and v1 (row r1)
    auto pivot_scale = [&](int c, double d, double v0, double v1) {
        if (!positive_finite(d)) {
            if (lane == 0 && info && c < kb) atomicCAS(info, 0, (int)(k + c + 1));  // the first failure
            d = 1e-300;
        }
        const double rs = rsqrt(d);
        if (r0 >= c) L[r0 * kLd + c] = r0 == c ? d * rs : v0 * rs;
        if (r1 >= c) L[r1 * kLd + c] = r1 == c ? d * rs : v1 * rs;
    };
    __syncthreads();
    if (warp == 0) pivot_scale(0, L[0], L[r0 * kLd], L[r1 * kLd]);
    __syncthreads();
    // bulk workers: warps 1-3 and 5-7
    const int bulk_rank = warp == 0 || warp == 4 ? -1 : (warp < 4 ? warp - 1 : warp - 2) * 32 + lane;
    constexpr int kBulkThreads = 6 * 32;
    for (int c = 0; c + 1 < kNB; ++c) {
        if (warp == 0) {
            // column c+1 by the finished column c, in registers
            const double lq = L[(c + 1) * kLd + c];
            const double v0 = r0 > c ? fma(-L[r0 * kLd + c], lq, L[r0 * kLd + c + 1]) : 0.0;
            const double v1 = r1 > c ? fma(-L[r1 * kLd + c], lq, L[r1 * kLd + c + 1]) : 0.0;
            const double d = c + 1 < 32 ? __shfl_sync(0xffffffffu, v0, c + 1) : __shfl_sync(0xffffffffu, v1, c - 31);
            pivot_scale(c + 1, d, v0, v1);
        } else if (bulk_rank >= 0) {
            // four entries at a time, loads first: their FMA chains overlap (a
            // store could alias the next loads as far as the compiler knows)
            const int ne = tri_from(c + 2);
            for (int e0 = bulk_rank; e0 < ne; e0 += 4 * kBulkThreads) {
                int at[4];
                double acc[4], x[4], y[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int e = e0 + u * kBulkThreads;
                    const int rq = e < ne ? tab[e] : ((63 << 8) | 63), r = rq >> 8, q = rq & 255;
                    at[u] = e < ne ? r * kLd + q : -1;
                    acc[u] = L[r * kLd + q];
                    x[u] = L[r * kLd + c];
                    y[u] = L[q * kLd + c];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[u] = fma(-x[u], y[u], acc[u]);
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (at[u] >= 0) L[at[u]] = acc[u];
            }
        }
        __syncthreads();
    }
    for (int e = t; e < kNB * kNB; e += kPotrfThreads) {
        const int r = e >> 6, c = e & 63;
        if (r < kb && c <= r) A[(size_t)(k + r) * n + k + c] = L[r * kLd + c];
    }
}

// Linv = L^-1 for the factored kb x kb diagonal block at (k, k): a lower-
// triangular 64 x 64 block, zero above the diagonal and beyond kb, written
// row by row together with its S slices (out [S][kb][64], exponents expo[kb];
// the B operand of the panel solve).  Row i of L^-1 solves x^T L = e_i^T;
// with U'_rc = l_rc / l_cc (columns divided by their diagonal on load) it is
// x_i = 1 / l_ii and x_c = -sum_{r > c} x_r U'_rc, taken by backward
// substitution: one warp per row (16 CTAs of 4 warps, one per SM
// sub-partition, each staging only the rows its rows read), lanes holding
// columns lane and lane + 32, one shuffle and one FMA per step.  A dependent
// FP64 operation costs about as much as a shuffle on this part, so the unit
// diagonal keeps the division off the chain.  The warp then slices its row
// as k_slice_rows would.
constexpr int kTrtriWarps = 4;

__global__ void __launch_bounds__(32 * kTrtriWarps) k_trtri64(const double *__restrict__ A, int64_t n, int64_t k,
                                                              int kb, double *__restrict__ Linv, int S,
                                                              __nv_bfloat16 *__restrict__ out, int *__restrict__ expo) {
    __shared__ double U[kNB * kLd];
    __shared__ double rd[kNB];
    const int t = threadIdx.x, lane = t & 31;
    const int i = blockIdx.x * kTrtriWarps + (t >> 5);
    // row i of the inverse reads only rows 0 .. i of L
    const int rows = blockIdx.x * kTrtriWarps + kTrtriWarps;  // rows staged: 0 .. rows - 1
    for (int c = t; c < kNB; c += 32 * kTrtriWarps) rd[c] = c < kb ? 1.0 / A[(size_t)(k + c) * n + k + c] : 1.0;
    __syncthreads();
    for (int e = t; e < rows * kNB; e += 32 * kTrtriWarps) {
        const int r = e / kNB, c = e % kNB;
        U[r * kLd + c] = (r < kb && c < r) ? A[(size_t)(k + r) * n + k + c] * rd[c] : 0.0;
    }
    __syncthreads();
    double x0 = 0.0, x1 = 0.0;  // columns lane, lane + 32 of row i
    if (i < kb) {
        // acc holds -sum_{r > c} x_r U'_rc over the rows finished so far; x_c is
        // final once row c + 1 has been applied
        double acc0 = lane == i ? rd[i] : 0.0, acc1 = lane + 32 == i ? rd[i] : 0.0;
        for (int r = i; r >= 1; --r) {  // warp-uniform bounds
            const double xr = r < 32 ? __shfl_sync(0xffffffffu, acc0, r) : __shfl_sync(0xffffffffu, acc1, r - 32);
            // columns c < r take -x_r U'_rc (U' is zero on and above the diagonal)
            acc0 = fma(-xr, U[r * kLd + lane], acc0);
            if (r > 32) acc1 = fma(-xr, U[r * kLd + lane + 32], acc1);
        }
        x0 = acc0;
        x1 = acc1;
        slice_row_warp(x0, x1, lane, kb, i, S, out, expo);
    }
    Linv[(size_t)i * kNB + lane] = x0;
    Linv[(size_t)i * kNB + lane + 32] = x1;
}

// ---------------------------------------------- triangular solves with L ---
//
// One cooperative launch per direction.  CTA b owns block rows b, b + G, ...
// (64 rows each) in solve order.  For its block row i it streams the blocks
// L_ij of the rows already solved, accumulating L_ij y_j with coalesced row
// loads, then applies the inverted diagonal block and writes y_i.  There are
// no flags: the solved vector starts filled with a NaN sentinel (all bytes
// 0xFF, a pattern FP64 arithmetic does not produce), and each warp waits on
// the values themselves, so that the wait and the load of y_j are one L2
// access on the chain of dependent block rows.  Every block row waits only on
// rows that come earlier in solve order, and a CTA takes its rows in that
// order, so with all CTAs resident (cooperative launch) every wait ends; each
// wait is still bounded by the global timer and records error 6 (forward) or
// 7 (backward), after which the CTA finishes its row without waiting again.
// (A right-hand side holding a NaN with exactly the sentinel's payload would
// read as unsolved and end in that time-out error rather than in a NaN.)
constexpr int kTrsvThreads = 256;
constexpr unsigned long long kSolveSentinel = 0xFFFFFFFFFFFFFFFFULL;

__device__ __forceinline__ double ld_relaxed_f64(const double *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return __longlong_as_double((long long)v);
}

// The warp waits until both y[lane] and y[lane + 32] hold solved values
// (lanes past `valid` read nothing and give 0); false on time-out.
__device__ bool wait_solved(const double *y, int lane, int valid, double &a, double &b, int *err, int code) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0;; ++it) {
        a = lane < valid ? ld_relaxed_f64(y + lane) : 0.0;
        b = lane + 32 < valid ? ld_relaxed_f64(y + lane + 32) : 0.0;
        const bool ok = (unsigned long long)__double_as_longlong(a) != kSolveSentinel &&
                        (unsigned long long)__double_as_longlong(b) != kSolveSentinel;
        if (__all_sync(0xffffffffu, ok)) return true;
        if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) {
            if (lane == 0) atomicExch(err, code);
            return false;
        }
    }
}

// L y = b: y (sentinel-filled) receives the solution; b is read and refilled
// with the sentinel for the backward solve.
__global__ void __launch_bounds__(kTrsvThreads) k_trsv_fwd(const double *__restrict__ L, int64_t n,
                                                           const double *__restrict__ Linv, double *b, double *y,
                                                           int *err) {
    __shared__ double inv[kNB * kNB];
    __shared__ double acc[kNB];
    const int nb = (int)((n + kNB - 1) / kNB);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int i = blockIdx.x; i < nb; i += gridDim.x) {
        const int64_t r0 = (int64_t)i * kNB;
        const int kb = (int)(n - r0 < kNB ? n - r0 : kNB);
        for (int e = t; e < kNB * kNB; e += kTrsvThreads) inv[e] = Linv[(size_t)i * kNB * kNB + e];
        // warp w: rows 8w .. 8w + 7 of the block; lanes: columns lane, lane + 32
        double part[8], bi[8];  // bi: the right-hand side of the warp's rows, read early
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            part[u] = 0.0;
            bi[u] = (lane == 0 && warp * 8 + u < kb) ? b[r0 + warp * 8 + u] : 0.0;
        }
        bool live = true;
        for (int j = 0; j < i && live; ++j) {
            const int64_t c0 = (int64_t)j * kNB;  // j < i: a full block
            // the block's L entries are in flight while the warp waits for y_j
            double p0[8], p1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = warp * 8 + u;
                const double *row = L + (size_t)(r0 + (r < kb ? r : 0)) * n + c0;
                p0[u] = row[lane];
                p1[u] = row[lane + 32];
            }
            double y0, y1;
            live = wait_solved(y + c0, lane, kNB, y0, y1, err, 6);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (warp * 8 + u < kb) part[u] = fma(p0[u], y0, fma(p1[u], y1, part[u]));
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const double sum = warp_sum(part[u]);
            const int r = warp * 8 + u;
            if (lane == 0) {
                acc[r] = r < kb ? bi[u] - sum : 0.0;
                if (r < kb) b[r0 + r] = __longlong_as_double((long long)kSolveSentinel);
            }
        }
        __syncthreads();
        // y_i = Linv_i acc: four threads per row, 16 columns each, in two
        // independent FMA chains (a dependent FP64 FMA costs tens of cycles)
        {
            const int r = t >> 2, q = t & 3;
            double ya = 0.0, yb = 0.0;
#pragma unroll
            for (int c = q * 16; c < q * 16 + 16; c += 2) {
                ya = fma(inv[r * kNB + c], acc[c], ya);
                yb = fma(inv[r * kNB + c + 1], acc[c + 1], yb);
            }
            double v = ya + yb;
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            if (q == 0 && r < kb) __stcg(y + r0 + r, v);
        }
        __syncthreads();  // inv and acc are reused by the CTA's next row
    }
}

// L^T x = y: y holds the forward solution; x goes to b (sentinel-filled by
// the forward solve).  Block rows are solved from the last to the first.
__global__ void __launch_bounds__(kTrsvThreads) k_trsv_bwd(const double *__restrict__ L, int64_t n,
                                                           const double *__restrict__ Linv, double *b,
                                                           const double *y, int *err) {
    __shared__ double inv[kNB * kNB];
    __shared__ double part_s[kTrsvThreads / 32][kNB];
    __shared__ double acc[kNB];
    const int nb = (int)((n + kNB - 1) / kNB);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    for (int ii = blockIdx.x; ii < nb; ii += gridDim.x) {
        const int i = nb - 1 - ii;
        const int64_t c0 = (int64_t)i * kNB;
        const int kb = (int)(n - c0 < kNB ? n - c0 : kNB);
        for (int e = t; e < kNB * kNB; e += kTrsvThreads) inv[e] = Linv[(size_t)i * kNB * kNB + e];
        // lanes: columns lane, lane + 32 of block column i; warp w: rows w, w + 8, ... of block row j
        double p0 = 0.0, p1 = 0.0;
        const bool v0 = lane < kb, v1 = lane + 32 < kb;
        const double yi = t < kb ? y[c0 + t] : 0.0;  // the right-hand side, read early (threads < 64 use it)
        bool live = true;
        for (int j = nb - 1; j > i && live; --j) {
            const int64_t r0 = (int64_t)j * kNB;
            const int kr = (int)(n - r0 < kNB ? n - r0 : kNB);
            // the block's L entries are in flight while the warp waits for x_j
            double q0[8], q1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = warp + 8 * u;
                const double *row = L + (size_t)(r0 + (r < kr ? r : 0)) * n + c0;
                q0[u] = v0 ? row[lane] : 0.0;
                q1[u] = v1 ? row[lane + 32] : 0.0;
            }
            double xa, xb;  // x_j: lane holds rows lane, lane + 32 of block j
            live = wait_solved(b + r0, lane, kr, xa, xb, err, 7);
            // four independent chains per column, summed after
            double a0[4] = {0.0, 0.0, 0.0, 0.0}, a1[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int r = warp + 8 * u;  // < 64: its x is in lane r (xa) or r - 32 (xb)
                const double xr = r < 32 ? __shfl_sync(0xffffffffu, xa, r) : __shfl_sync(0xffffffffu, xb, r - 32);
                if (r < kr) {
                    a0[u & 3] = fma(q0[u], xr, a0[u & 3]);
                    a1[u & 3] = fma(q1[u], xr, a1[u & 3]);
                }
            }
            p0 += (a0[0] + a0[1]) + (a0[2] + a0[3]);
            p1 += (a1[0] + a1[1]) + (a1[2] + a1[3]);
        }
        part_s[warp][lane] = p0;
        part_s[warp][lane + 32] = p1;
        __syncthreads();
        if (t < kNB) {
            double sum = 0.0;
#pragma unroll
            for (int w = 0; w < kTrsvThreads / 32; ++w) sum += part_s[w][t];
            acc[t] = t < kb ? yi - sum : 0.0;
        }
        __syncthreads();
        // x_i = Linv_i^T acc: four threads per column, 16 rows each, in two
        // independent FMA chains
        {
            const int c = t >> 2, q = t & 3;
            double xa = 0.0, xb = 0.0;
#pragma unroll
            for (int r = q * 16; r < q * 16 + 16; r += 2) {
                xa = fma(inv[r * kNB + c], acc[r], xa);
                xb = fma(inv[(r + 1) * kNB + c], acc[r + 1], xb);
            }
            double x = xa + xb;
            x += __shfl_xor_sync(0xffffffffu, x, 1);
            x += __shfl_xor_sync(0xffffffffu, x, 2);
            if (q == 0 && c < kb) __stcg(b + c0 + c, x);
        }
        __syncthreads();  // inv, part_s and acc are reused by the CTA's next row
    }
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
    return 1024 + (size_t)kMaxSlices * kABytes + (size_t)2 * kMaxSlices * kPBBytes +
           (size_t)kPEpiWarps * 32 * kPColsPerWarp * sizeof(double) + 10 * sizeof(uint64_t) + 16;
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
    if (rows > (1LL << 31) - kTileM || cols > (1LL << 31) - kPN) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_slice_map(&ma, Asl, rows, S, kTileM, a_stride) || !make_slice_map(&mb, Bsl, cols, S, kPN, b_stride))
        return cudaErrorInvalidValue;
    const void *kern = S == kMaxSlices ? (const void *)k_ozaki_gemm<kMaxSlices> : (const void *)k_ozaki_gemm<0>;
    cudaError_t e = nk::allow_max_dynamic_smem(kern);
    if (e != cudaSuccess) return e;
    OzArgs a{rows, cols, S, expA, expB, C, ldc, mode, lower ? 1 : 0, err, (cols + kPN - 1) / kPN, 1, 0};
    const int64_t n_mb = (rows + kTileM - 1) / kTileM;
    // strips of up to 8 tiles amortise a CTA's A slices over its tiles; a
    // product with few tiles per SM (the panel solve and the narrow update of
    // the Cholesky, on its critical path) takes one tile per CTA instead
    int64_t tiles = 0;
    for (int64_t m = 0; m < n_mb; ++m) tiles += oz_row_tiles(a.n_nb, lower, m);
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int64_t per_sm = sms > 0 ? tiles / sms : kMaxChunk;
    while (a.chunk < kMaxChunk && 2 * a.chunk <= per_sm) {
        a.chunk *= 2;
        ++a.chunk_log2;
    }
    int64_t strips = 0;
    for (int64_t m = 0; m < n_mb; ++m) strips += oz_row_strips(a.n_nb, lower, m, a.chunk_log2);
    if (strips > (1LL << 31) - 1) return cudaErrorInvalidValue;
    if (S == kMaxSlices)
        (k_ozaki_gemm<kMaxSlices><<<(unsigned)strips, kPThreads, ozaki_smem_bytes(), st>>>(ma, mb, a),
         nk::note_launch());
    else
        (k_ozaki_gemm<0><<<(unsigned)strips, kPThreads, ozaki_smem_bytes(), st>>>(ma, mb, a), nk::note_launch());
    return cudaGetLastError();
}

// BF16 MMA flops a launch executes: active tiles x S(S+1)/2 slice products x
// 2 x 128 x 32 x 64.
double ozaki_mma_flops(int64_t rows, int64_t cols, int S, bool lower) {
    const int64_t tm = (rows + kTileM - 1) / kTileM, tn = (cols + kPN - 1) / kPN;
    int64_t tiles = 0;
    for (int64_t i = 0; i < tm; ++i) tiles += oz_row_tiles(tn, lower, i);
    return (double)tiles * (S * (S + 1) / 2) * 2.0 * kTileM * kPN * kTileK;
}

cudaError_t launch_ozaki_gemm(const __nv_bfloat16 *Asl, const int *expA, int64_t rows,
                              const __nv_bfloat16 *Bsl, const int *expB, int64_t cols, int S, double *C,
                              int64_t ldc, int mode, bool lower, int *err, cudaStream_t st) {
    return launch_ozaki_gemm_strided(Asl, expA, rows, rows, Bsl, expB, cols, cols, S, C, ldc, mode, lower, err, st);
}

size_t tc_chol_ws_bytes(int64_t n) {
    const int64_t nb = (n + kNB - 1) / kNB;
    return 2 * slice_elems(n, kMaxSlices) * 2 + slice_elems(kNB, kMaxSlices) * 2 + (size_t)(2 * n + kNB) * 4 +
           (size_t)nb * kNB * kNB * 8 + (size_t)n * 8 + 9 * 256;
}

namespace {
struct TcWs {
    __nv_bfloat16 *Asl, *Bsl, *Asl2;
    int *expA, *expB, *expA2;
    double *Linv;
    double *y;   // [n] forward-solve vector of the triangular solves
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
    w.y = reinterpret_cast<double *>(take((size_t)n * 8));
    return w;
}
}  // namespace

// Blocked right-looking Cholesky with tensor-core (Ozaki, 7 slices) panel
// solves and trailing updates, and a look-ahead of one panel: after panel k
// the side stream updates block column k + 1 alone (the "narrow" update) and
// factors panel k + 1 (diagonal block, its inverse, the panel product and its
// slices), while the main stream applies panel k to the rest of the trailing
// matrix (the "wide" update).  Panel slices alternate between two buffers.
// The inverted diagonal blocks stay in the workspace for
// launch_cholesky_solve_tc.
namespace {

// Factor panel k (columns k0 .. k0 + kb - 1) whose block column is up to date:
// diagonal block + inverse, L_panel = A_panel L_kk^-T, slices of L_panel.
// With an aux stream (cs non-null), the panel rows below the diagonal block
// are sliced there, beside the diagonal block's factorisation and inverse:
// the slicing depends only on the narrow update that precedes the panel.
cudaError_t panel_step(double *A, int64_t n, int64_t k0, int *info, int *err, TcWs &w, __nv_bfloat16 *Lsl,
                       int *Lexp, cudaStream_t st, const CholStreams *cs) {
    const int S = kMaxSlices;
    const int kb = (int)(n - k0 < kNB ? n - k0 : kNB);
    const int64_t rest = n - k0 - kb;
    double *Linv = w.Linv + (size_t)(k0 / kNB) * kNB * kNB;
    double *panel = A + (size_t)(k0 + kb) * n + k0;
    cudaError_t e = cudaSuccess;
    const bool fork = cs != nullptr && cs->aux != nullptr && rest > 0;
    if (fork) {
        e = cudaEventRecord(cs->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs->aux, cs->ev_fork, 0);
        if (e != cudaSuccess) return e;
        const int aslot = prof_begin(NK_PROF_CHOL_PANEL, cs->aux);
        e = launch_slice_rows(panel, n, rest, kb, S, Lsl, Lexp, cs->aux);
        prof_end(aslot, cs->aux, 0.0);
        if (e == cudaSuccess) e = cudaEventRecord(cs->ev_join, cs->aux);
        if (e != cudaSuccess) return e;
    }
    // timing classes: the FP64 diagonal-block kernels and the slicing count
    // as the panel, the tensor-core panel product with the trailing updates
    int slot = prof_begin(NK_PROF_CHOL_PANEL, st);
    (k_potrf64<<<1, kPotrfThreads, 0, st>>>(A, n, k0, kb, info), nk::note_launch());
    // the inverse and its slices (the B operand of the panel solve)
    (k_trtri64<<<kNB / kTrtriWarps, 32 * kTrtriWarps, 0, st>>>(A, n, k0, kb, Linv, S, w.Bsl, w.expB),
     nk::note_launch());
    if (rest > 0)
        e = fork ? cudaStreamWaitEvent(st, cs->ev_join, 0) : launch_slice_rows(panel, n, rest, kb, S, Lsl, Lexp, st);
    prof_end(slot, st, 2.0 * (double)kb * kb * kb / 3.0);
    if (rest > 0 && e == cudaSuccess) {
        slot = prof_begin(NK_PROF_CHOL_UPDATE, st);
        e = launch_ozaki_gemm(Lsl, Lexp, rest, w.Bsl, w.expB, kb, S, panel, n, 0, false, err, st);
        // the triangular solve L21 = A21 L11^-T: rest kb^2 flops in FP64
        prof_end(slot, st, (double)rest * kb * kb, ozaki_mma_flops(rest, kb, S, false));
        slot = prof_begin(NK_PROF_CHOL_PANEL, st);
        if (e == cudaSuccess) e = launch_slice_rows(panel, n, rest, kb, S, Lsl, Lexp, st);
        prof_end(slot, st, 0.0);
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

cudaError_t launch_cholesky_tc(double *A, int64_t n, int *info, int *err, void *ws, cudaStream_t st,
                               const CholStreams *cs) {
    // Step k, with panel k factored and sliced:
    //   side stream: the narrow update (block column k+1 by panel k), then
    //     panel k+1 (factor, invert, solve, slice);
    //   main stream: the wide update (everything right of block column k+1).
    // The side stream waits for the previous wide update (block column k+1
    // must have received it, and panel k+1's slice buffer is the one that
    // update read); the main stream waits for panel k+1 before the next wide
    // update.  A step then takes max(wide, narrow + panel).
    TcWs w = carve_tc(ws, n);
    const int S = kMaxSlices;
    cudaError_t e = cudaSuccess;
    __nv_bfloat16 *buf[2] = {w.Asl, w.Asl2};
    int *bexp[2] = {w.expA, w.expA2};
    const int64_t nb = (n + kNB - 1) / kNB;
    const bool two = cs != nullptr && cs->side != nullptr;
    cudaStream_t side = two ? cs->side : nullptr, ps = two ? cs->side : st;
    cudaEvent_t ev_wide = two ? cs->ev_wide : nullptr, ev_panel = two ? cs->ev_panel : nullptr;
    e = panel_step(A, n, 0, info, err, w, buf[0], bexp[0], st, cs);
    if (e != cudaSuccess) return e;
    for (int64_t k = 0; k + 1 < nb; ++k) {
        const int64_t k0 = k * kNB;
        const int64_t rest = n - k0 - kNB;         // rows of panel k below its diagonal block
        const int kb1 = (int)(rest < kNB ? rest : kNB);  // width of block column k + 1
        __nv_bfloat16 *Lk = buf[k & 1];
        int *Le = bexp[k & 1];
        double *C1 = A + (size_t)(k0 + kNB) * n + (k0 + kNB);
        if (two) {
            e = cudaEventRecord(ev_wide, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(side, ev_wide, 0);
            if (e != cudaSuccess) return e;
        }
        // narrow: block column k + 1 (all rows below panel k)
        int slot = prof_begin(NK_PROF_CHOL_UPDATE, ps);
        e = launch_ozaki_gemm_strided(Lk, Le, rest, rest, Lk, Le, kb1, rest, S, C1, n, 1, true, err, ps);
        // FP64 flops of the lower part of the rest x kb1 block column, K = kNB
        prof_end(slot, ps, 2.0 * kNB * ((double)rest * kb1 - 0.5 * (double)kb1 * (kb1 - 1)),
                 ozaki_mma_flops(rest, kb1, S, true));
        if (e != cudaSuccess) return e;
        e = panel_step(A, n, k0 + kNB, info, err, w, buf[(k + 1) & 1], bexp[(k + 1) & 1], ps, cs);
        if (e != cudaSuccess) return e;
        if (two) {
            e = cudaEventRecord(ev_panel, side);
            if (e != cudaSuccess) return e;
        }
        // wide: everything right of block column k + 1
        const int64_t rest2 = rest - kb1;
        if (rest2 > 0) {
            slot = prof_begin(NK_PROF_CHOL_UPDATE, st);
            e = launch_ozaki_gemm_strided(Lk + (size_t)kb1 * kTileK, Le + kb1, rest2, rest, Lk + (size_t)kb1 * kTileK,
                                          Le + kb1, rest2, rest, S, C1 + (size_t)kb1 * n + kb1, n, 1, true, err, st);
            // FP64 flops of the lower rest2 x rest2 trailing update, K = kNB
            prof_end(slot, st, (double)kNB * rest2 * (double)(rest2 + 1), ozaki_mma_flops(rest2, rest2, S, true));
            if (e != cudaSuccess) return e;
        }
        if (two) {
            e = cudaStreamWaitEvent(st, ev_panel, 0);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_cholesky_solve_tc(const double *L, int64_t n, const void *ws, double *b, int *err,
                                     cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    TcWs w = carve_tc(const_cast<void *>(ws), n);
    const int nb = (int)((n + kNB - 1) / kNB);
    int dev = 0, sms = 0, per_sm_f = 0, per_sm_b = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_f, k_trsv_fwd, kTrsvThreads, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_b, k_trsv_bwd, kTrsvThreads, 0);
    if (e != cudaSuccess) return e;
    // at most one CTA per SM: the resident grid needs no more, and blocks
    // rows then spread over the SMs' load bandwidth
    const int gf = std::min(nb, sms * std::min(per_sm_f, 1)), gb = std::min(nb, sms * std::min(per_sm_b, 1));
    if (gf < 1 || gb < 1) return cudaErrorLaunchOutOfResources;
    const int slot = prof_begin(NK_PROF_TRSV, st);
    e = cudaMemsetAsync(w.y, 0xFF, (size_t)n * 8, st);  // the sentinel of unsolved entries
    if (e != cudaSuccess) return e;
    const double *Linv = w.Linv;
    double *y = w.y;
    void *args[] = {(void *)&L, (void *)&n, (void *)&Linv, (void *)&b, (void *)&y, (void *)&err};
    e = cudaLaunchCooperativeKernel((const void *)k_trsv_fwd, dim3(gf), dim3(kTrsvThreads), args, 0, st);
    nk::note_launch();
    if (e != cudaSuccess) return e;
    e = cudaLaunchCooperativeKernel((const void *)k_trsv_bwd, dim3(gb), dim3(kTrsvThreads), args, 0, st);
    nk::note_launch();
    prof_end(slot, st, 2.0 * (double)n * (double)n);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Lower triangle of K = T T^T by tensor cores with S slices per 64-column
// chunk of T [Ns][M], then the Jacobian-row Gram s.s + t.t + (t.t)(s.s)
// written to both triangles.
// Lower triangle of C = scale X^T X + eps I for X [rows][ncols] (row stride
// ncols): 64 rows of X per tensor-core pass, each sliced by columns (one
// exponent per column and pass) and accumulated in FP64.
cudaError_t launch_gram_cols_tc(const double *X, int64_t rows, int64_t ncols, double scale, double eps, double *C,
                                int *err, void *ws, cudaStream_t st) {
    if (rows <= 0 || ncols <= 0) return cudaSuccess;
    TcWs w = carve_tc(ws, ncols);
    const int S = kMaxSlices;
    const int slot = prof_begin(NK_PROF_GRAM, st);
    cudaError_t e = cudaSuccess;
    for (int64_t r0 = 0; r0 < rows && e == cudaSuccess; r0 += kTileK) {
        const int kr = (int)(rows - r0 < kTileK ? rows - r0 : kTileK);
        (k_slice_cols<<<nblk(ncols, 32), 256, 0, st>>>(X, ncols, r0, kr, ncols, S, w.Asl, w.expA), nk::note_launch());
        e = launch_ozaki_gemm(w.Asl, w.expA, ncols, w.Asl, w.expA, ncols, S, C, ncols, r0 == 0 ? 0 : 2, true, err, st);
    }
    if (e == cudaSuccess) {
        const dim3 grid(nblk(ncols, 256), (unsigned)(ncols < 65535 ? ncols : 65535));
        (k_scale_shift_lower<<<grid, 256, 0, st>>>(C, ncols, scale, eps), nk::note_launch());
    }
    prof_end(slot, st, (double)rows * ncols * (double)(ncols + 1),
             (double)((rows + kTileK - 1) / kTileK) * ozaki_mma_flops(ncols, ncols, S, true));
    return e != cudaSuccess ? e : cudaGetLastError();
}

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
    // the lower triangle of the Jacobian-row Gram through s.s + t.t + (t.t)(s.s):
    // (N + M) flops per entry, the count of the FP64 path
    prof_end(slot, st, (double)Ns * (Ns + 1) * (double)(N + M),
             (double)((M + kTileK - 1) / kTileK) * ozaki_mma_flops(Ns, Ns, S, true));
    return cudaGetLastError();
}

}  // namespace nk
