// Tensor-core products with the spin configurations as one operand.
//
// The three dense contractions of the RBM path all multiply the +-1
// configuration matrix by a real matrix (NetKet 3, Sec. 3.2 model
// evaluation; App. B.1 Jacobian products):
//   theta = S W^T + b           (batched hidden activations, [Ns][M])
//   J v   = rowdot(T', S' V'^T)  (S' = [S, 1], V' = [[V_W, v_b], [v_a, 0]])
//   J^T g via P^T = S'^T (T'o g) (T' = [T, 1])
// +-1 and 1 are exact in BF16.  The real operand B is cut, row by row with one
// power-of-two exponent per row, into SB slices of 8-bit integers (as in
// k_tc.cu).  Every slice level t then needs one MMA chain,
//   D_t[m][n] = sum_k a_mk beta_t,nk,
// whose FP32 accumulation is exact: |D_t| <= K 255 < 2^24 for K <= 65792.
// The epilogue recombines sum_t D_t 2^{-8t} 2^{f_n} in integers and writes
// FP64.  With SB = 7 the products are exact up to the 2^-56 truncation of B
// (FP64-level: the batched theta rebuild, the force and the sample-space
// solve products); with SB = 4 up to 2^-32 (the NK_MIXED QGT products of CG).
//
// Kernel: 128 x 64 output tile per CTA, K in chunks of 64 through a TMA /
// mbarrier ring (3 stages; 2 for SB <= 4, so that two CTAs share an SM and
// one drains while the other multiplies).  Thread 0 produces, thread 32
// issues tcgen05.mma M=128 K=16 into SB TMEM accumulators of 64 columns,
// with the slices side by side as one B operand (N = 64 SB up to 256), then the
// four warps drain TMEM through the integer recombination.  Outputs: a
// staged, coalesced store (C =, -=, += R; a long K range may be split over
// blockIdx.z into partial outputs summed afterwards), or, for J v, the row
// products with t' = [t, 1] taken in the epilogue (one partial per row and
// 64-column tile), so that the Ns x (M+1) product never reaches HBM.
// Every wait is bounded by the global timer.

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "nk_common.cuh"
#include "nk_internal.h"
#include "tc_ptx.cuh"

namespace nk {

namespace {

constexpr int kBM = 128, kBN = 64, kBK = 64;
constexpr int kMaxSB = 7;
constexpr int kSgThreads = 128;
constexpr int kAB = kBM * kBK * 2;             // A tile, bytes
constexpr int kBB = kBN * kBK * 2;             // one B slice tile, bytes
constexpr int kSgOutLd = kBN + 1;

struct SgArgs {
    int64_t rows, cols;
    int kchunks, SB;
    int kc_split;         // K-chunks per split (blockIdx.z)
    int nstages, stage_bytes;
    uint32_t tmem_cols;
    const int *expB;      // [cols]
    double *C;            // modes 0-2: output (+ blockIdx.z * split_stride); mode 3: row partials
    int64_t ldc, split_stride;
    int mode;             // 0: C = R (+ bias), 1: C -= R, 2: C += R, 3: C[row][bx] = sum_col R t'
    const double *bias;   // [cols] or null
    const double *T;      // mode 3: T [rows][Mt]; t'_col = T[col] for col < Mt, 1 at col = Mt
    int Mt;
    int *err;
};

// Smem: nstages x (A tile + SB B-slice tiles), reused by the staged output
// tile after the MMAs.  With SB <= 4 two stages and 256 TMEM columns let two
// CTAs share an SM, so that one CTA's epilogue overlaps the other's MMAs.
__global__ void __launch_bounds__(kSgThreads, 2)
    k_sgemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, SgArgs a) {
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *ops = smem_raw + ((1024 - (base & 1023)) & 1023);
    const size_t ops_bytes = (size_t)a.nstages * a.stage_bytes > (size_t)kBM * kSgOutLd * 8
                                 ? (size_t)a.nstages * a.stage_bytes
                                 : (size_t)kBM * kSgOutLd * 8;
    uint64_t *full = reinterpret_cast<uint64_t *>(ops + ops_bytes);
    uint64_t *empty = full + 4;
    uint64_t *done = empty + 4;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t m0 = (int64_t)blockIdx.y * kBM, n0 = (int64_t)blockIdx.x * kBN;
    const int SB = a.SB, NS = a.nstages;
    const int kc0 = (int)blockIdx.z * a.kc_split;
    const int kc1 = kc0 + a.kc_split < a.kchunks ? kc0 + a.kc_split : a.kchunks;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (threadIdx.x == 0) {
        // TMA producer
        const uint32_t tx = (uint32_t)(kAB + SB * kBB);
        for (int kc = kc0; kc < kc1; ++kc) {
            const int i = kc - kc0, s = i % NS;
            if (i >= NS && !mbar_wait(&empty[s], (uint32_t)(((i / NS) - 1) & 1))) {
                *abort_flag = 1;
                atomicExch(a.err, 3);
                break;
            }
            unsigned char *sp = ops + (size_t)s * a.stage_bytes;
            mbar_expect_tx(&full[s], tx);
            tma_load_2d(sp, &mapA, &full[s], kc * kBK, (int)m0);
            for (int t = 0; t < SB; ++t) tma_load_3d(sp + kAB + t * kBB, &mapB, &full[s], kc * kBK, (int)n0, t);
        }
    } else if (threadIdx.x == 32) {
        // MMA issuer
        // the SB slice tiles of a stage lie back to back ([SB][64][64] BF16), so
        // slices 0 .. 3 form one operand of 64 min(SB, 4) rows for one MMA into
        // TMEM columns 0 .. 64 min(SB, 4) - 1, and slices 4 .. SB-1 a second one
        const int nlo = SB < 4 ? SB : 4, nhi = SB - nlo;
        const uint32_t idesc_lo = idesc_bf16(kBM, kBN * nlo), idesc_hi = idesc_bf16(kBM, kBN * (nhi > 0 ? nhi : 1));
        bool ok = true;
        for (int kc = kc0; kc < kc1; ++kc) {
            const int i = kc - kc0, s = i % NS;
            if (!mbar_wait(&full[s], (uint32_t)((i / NS) & 1))) {
                ok = false;
                break;
            }
            tc_fence_after();
            unsigned char *sp = ops + (size_t)s * a.stage_bytes;
            const uint64_t da = sw128_desc(sp), dlo = sw128_desc(sp + kAB), dhi = sw128_desc(sp + kAB + 4 * kBB);
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
                umma_bf16(tmem, da + (uint64_t)(kk * 2), dlo + (uint64_t)(kk * 2), idesc_lo, acc);
                if (nhi > 0)
                    umma_bf16(tmem + (uint32_t)(4 * kBN), da + (uint64_t)(kk * 2), dhi + (uint64_t)(kk * 2), idesc_hi,
                              acc);
            }
            umma_commit(&empty[s]);
        }
        if (!ok) {
            *abort_flag = 1;
            atomicExch(a.err, 4);
        }
        umma_commit(done);
    }
    __syncthreads();
    double *tile = reinterpret_cast<double *>(ops);
    const int rloc = warp * 32 + lane;
    const int64_t row = m0 + rloc;
    if (!*abort_flag) {
        int ok = 1;
        if (lane == 0) ok = mbar_wait(done, 0) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) {
            if (lane == 0) {
                atomicExch(a.err, 5);
                *abort_flag = 2;
            }
        } else {
            tc_fence_after();
            const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
            const bool row_ok = row < a.rows;
            const double *trow = (a.mode == 3 && row_ok) ? a.T + (size_t)row * a.Mt : nullptr;
            double racc = 0.0;
#pragma unroll 1
            for (int c8 = 0; c8 < kBN; c8 += 8) {
                // column exponents of this chunk (lane & 7) and, for the fused
                // row product, the chunk's t' values, loaded before the TMEM drain
                const int64_t fcol = n0 + c8 + (lane & 7);
                const int fj_lane = fcol < a.cols ? a.expB[fcol] : 0;
                double tv[8];
                if (a.mode == 3) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int64_t col = n0 + c8 + j;
                        tv[j] = trow == nullptr ? 0.0 : (col < a.Mt ? trow[col] : (col == a.Mt ? 1.0 : 0.0));
                    }
                }
                uint32_t r[kMaxSB][8];
#pragma unroll
                for (int t = 0; t < kMaxSB; ++t)
                    if (t < SB) tmem_ld8(lane_base + (uint32_t)(t * kBN + c8), r[t]);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    int d[kMaxSB];
#pragma unroll
                    for (int t = 0; t < kMaxSB; ++t) d[t] = t < SB ? __float2int_rn(__uint_as_float(r[t][j])) : 0;
                    // V 2^(f_n - 56) with V = sum_t D_t 2^(8 (7 - t))
                    const int fn = __shfl_sync(0xffffffffu, fj_lane, j);
                    const double v = window_to_double(sgemm_window10(d), fn - 46);
                    if (a.mode == 3)
                        racc = fma(v, tv[j], racc);
                    else
                        tile[rloc * kSgOutLd + c8 + j] = v;
                }
            }
            if (a.mode == 3 && row_ok) a.C[(size_t)row * a.ldc + blockIdx.x] = racc;
        }
    }
    __syncthreads();
    if (!*abort_flag && a.mode != 3) {
        double *C = a.C + (size_t)blockIdx.z * a.split_stride;
        const int cx = threadIdx.x & 63, ry = threadIdx.x >> 6;
        const int64_t col = n0 + cx;
        constexpr int kStep = kSgThreads / 64, kBatch = 8;
        if (col < a.cols) {
            const double bcol = (a.bias && a.mode == 0) ? a.bias[col] : 0.0;
            for (int rb = ry; rb < kBM; rb += kStep * kBatch) {
                double cv[kBatch];
                bool on[kBatch];
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    const int rl = rb + kStep * u;
                    on[u] = rl < kBM && m0 + rl < a.rows;
                    cv[u] = (on[u] && a.mode != 0) ? C[(size_t)(m0 + rl) * a.ldc + col] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < kBatch; ++u) {
                    if (!on[u]) continue;
                    const int rl = rb + kStep * u;
                    const double v = tile[rl * kSgOutLd + cx];
                    C[(size_t)(m0 + rl) * a.ldc + col] = a.mode == 0 ? v + bcol : (a.mode == 1 ? cv[u] - v : cv[u] + v);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

// ------------------------------ J v and J^T g: persistent, 3 FP16 slices ---
//
// The CG products of NK_MIXED as one persistent kernel per SM, on FP16
// slices: B (V' for J v, (T' o g')^T for J^T g) is cut into 3 slices of
// 11-bit digits on a 33-bit grid per operand row (FP16 holds every integer up
// to 2048 exactly), A is the +-1 operand in FP16, and each FP32 level sums
// K products of at most 2^11 in magnitude, exact while K 2^11 <= 2^24 (K <=
// 8192 per unit).
// Warp 0 streams A / B K-chunks through a 5-stage TMA ring (40 KB a stage),
// warp 1 issues the MMAs of a 128 x 64 tile (3 slices side by side, N = 192)
// into one of two TMEM accumulator sets, and 16 epilogue warps drain the
// other set meanwhile: warp (q, g) owns TMEM lane quarter q (tile rows 32q ..
// 32q + 31) and the 16 tile columns 16g .. 16g + 15.
//
// J v (mode 0) needs sum_j t'_j V_j 2^(f_j - 33) per row, V_j = D_0 2^22 +
// D_1 2^11 + D_2 from the exact FP32 levels.  It runs in FP32 on tanh(theta)
// stored as an FP32 pair t = th + tl (|tl| <= 2^-24 |th|, built once per
// solve): with u = th 2^(f_j - F) and ul = tl 2^(f_j - F) (F the largest
// column exponent of the tile, so that the scale is a power of two <= 1),
// the row sum is 2^(F - 11) sum_j (D_0 + D_1 2^-11 + D_2 2^-22)(u + ul).  The
// products D_0 u and D_1 u are split exactly by FMA (p + e), p is summed
// exactly by two-sum into FP32 pairs, and the smaller terms go to a plain
// FP32 sum: about 2^-44 of the summed magnitudes, below the 2^-33 of the
// slicing, with no FP64 work per entry.  The four column groups of a row meet
// as FP32 pairs in shared memory (a ring of 4 tiles, an mbarrier per quarter
// and slot), and warp (q, 0) writes the tile's row partial P[nt][row] in
// FP64.  J^T g (mode 1) recombines V exactly in int64 and writes FP64 split-K
// partials.  Units go round robin over the clusters.  Every wait is bounded;
// a time-out sets err and drains the copies and MMAs in flight before the
// TMEM is released.
constexpr int kJvEpiWarps = 16;
constexpr int kJvThreads = 64 + 32 * kJvEpiWarps;
constexpr int kJvStages = 5;
constexpr int kJvSB = 3;                            // FP16 slices of 11-bit digits
constexpr int kJvStageBytes = kAB + kJvSB * kBB;  // 40 KB
constexpr int kJvRing = 4;                          // row-partial slots
constexpr uint32_t kJvAccCols = kJvSB * kBN;        // 192 per accumulator set
constexpr uint32_t kJvTmemCols = 512;               // two sets, rounded up to a power of two
constexpr int kTcRowDot = 0, kTcStoreT = 1;         // epilogue modes of k_tc4

struct Tc4Args {
    int64_t rows, cols;
    int kchunks;          // K-chunks of the whole product
    int kc_split;         // K-chunks per unit (mode 1; kchunks in mode 0)
    int ks;               // K splits
    int n_nt, n_mg;       // column tiles; row-tile groups of C tiles
    int C;                // CTAs per cluster (1, 2, 4): B slices multicast across them
    int64_t groups;       // n_mg * n_nt * ks
    const int *expB;      // [n_nt * 64] (read up to the tile end; columns >= cols unused)
    const float4 *Thl;    // mode 0: t' as FP32 pairs, tile-major (launch_split_t)
    double *P;            // mode 0: [n_nt][rows]; mode 1: [ks][cols][ldp] (column-major tiles)
    int64_t ldp, split_stride;
    int *err;
    const int *skip;      // optional: nothing is done while *skip is set (a converged CG)
};

// s + e = a + b exactly (Knuth's two-sum, no ordering of |a|, |b| needed)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

constexpr size_t jv_smem_bytes() {
    return 1024 + (size_t)kJvStages * kJvStageBytes + (size_t)kJvRing * 4 * kBM * 8 +
           (size_t)(2 * kJvStages + 4 + kJvRing * 4) * 8 + 16;
}

// Unit li of cluster slot `cl` (of ncl): the cluster's row-tile group mg,
// column tile nt and K split z, this CTA's row tile mt = mg C + rank.
// Mode 0 walks the column tiles fastest (the A tiles of a group are reused),
// mode 1 the row-tile groups (the B range of (nt, z) is reused from L2).
struct Tc4Unit {
    int64_t mt;
    int nt, z;
};
template <int kMode>
__device__ __forceinline__ Tc4Unit tc4_unit(const Tc4Args &a, int64_t g, uint32_t rank) {
    Tc4Unit u;
    int64_t mg;
    if (kMode == kTcRowDot) {
        mg = g / a.n_nt;
        u.nt = (int)(g % a.n_nt);
        u.z = 0;
    } else {
        mg = g % a.n_mg;
        const int64_t r = g / a.n_mg;
        u.nt = (int)(r % a.n_nt);
        u.z = (int)(r / a.n_nt);
    }
    u.mt = mg * a.C + rank;
    return u;
}
template <int kMode>
__global__ void __launch_bounds__(kJvThreads, 1)
    k_tc4(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, Tc4Args a) {
    // every thread of every CTA reads the same word, written before the launch
    if (a.skip && *a.skip) return;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t base = smem_u32(smem_raw);
    unsigned char *ops = smem_raw + ((1024 - (base & 1023)) & 1023);
    float2 *red = reinterpret_cast<float2 *>(ops + (size_t)kJvStages * kJvStageBytes);  // [ring][4 groups][128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(red + (size_t)kJvRing * 4 * kBM);
    uint64_t *full = bars, *empty = bars + kJvStages;
    uint64_t *acc_full = bars + 2 * kJvStages, *acc_empty = acc_full + 2;
    uint64_t *red_full = acc_empty + 2;  // [ring][quarter]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(red_full + kJvRing * 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = a.C;
    const uint32_t rank = C > 1 ? cluster_rank() : 0u;
    const uint16_t mask = (uint16_t)((1u << C) - 1u);
    const int64_t cl = blockIdx.x / C, ncl = gridDim.x / C;
    const int64_t nunits = a.groups > cl ? (a.groups - 1 - cl) / ncl + 1 : 0;
    const int64_t n_mt = (a.rows + kBM - 1) / kBM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kJvStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], (uint32_t)C);  // one commit from every CTA of the cluster
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], kJvEpiWarps);
        }
        for (int i = 0; i < kJvRing * 4; ++i) mbar_init(&red_full[i], 4);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tmem_alloc(tslot, kJvTmemCols);
    tc_fence_before();
    if (C > 1)
        cluster_sync_all();  // the peers' barriers exist before any multicast reaches them
    else
        __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    auto fail = [&](int code) {
        *abort_flag = 1;
        atomicExch(a.err, code);
    };

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------- producer
        // own A tile; B slices rank * 3 / C .. (rank + 1) * 3 / C - 1 to every CTA
        const int t0 = (int)rank * kJvSB / C, t1 = ((int)rank + 1) * kJvSB / C;
        int64_t g = 0;  // K-chunks issued (all units)
        for (int64_t li = 0; li < nunits && !*abort_flag; ++li) {
            const Tc4Unit u = tc4_unit<kMode>(a, cl + li * ncl, rank);
            const int m0 = (int)(u.mt * kBM), n0 = u.nt * kBN;
            const int kc0 = u.z * a.kc_split;
            const int kc1 = kc0 + a.kc_split < a.kchunks ? kc0 + a.kc_split : a.kchunks;
            for (int kc = kc0; kc < kc1; ++kc, ++g) {
                const int s = (int)(g % kJvStages);
                if (g >= kJvStages &&
                    !mbar_wait_or_abort_sleep(&empty[s], (uint32_t)((g / kJvStages - 1) & 1), abort_flag)) {
                    fail(20);
                    break;
                }
                unsigned char *sp = ops + (size_t)s * kJvStageBytes;
                mbar_expect_tx(&full[s], (uint32_t)kJvStageBytes);
                tma_load_2d(sp, &mapA, &full[s], kc * kBK, m0);
                for (int t = t0; t < t1; ++t) {
                    if (C > 1)
                        tma_load_3d_mc(sp + kAB + t * kBB, &mapB, &full[s], kc * kBK, n0, t, mask);
                    else
                        tma_load_3d(sp + kAB + t * kBB, &mapB, &full[s], kc * kBK, n0, t);
                }
            }
        }
        if (*abort_flag) {
            // the copies in flight land before the CTA exits
            for (int64_t h = g - kJvStages > 0 ? g - kJvStages : 0; h < g; ++h)
                mbar_wait(&full[h % kJvStages], (uint32_t)((h / kJvStages) & 1));
        }
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------- MMA issuer
        const uint32_t idesc = idesc_f16(kBM, kBN * kJvSB);
        int64_t g = 0;
        int64_t committed = -1;  // last unit whose accumulator commit was issued
        for (int64_t li = 0; li < nunits && !*abort_flag; ++li) {
            const Tc4Unit u = tc4_unit<kMode>(a, cl + li * ncl, rank);
            const int kc0 = u.z * a.kc_split;
            const int kc1 = kc0 + a.kc_split < a.kchunks ? kc0 + a.kc_split : a.kchunks;
            const int b = (int)(li & 1);
            const uint32_t use = (uint32_t)(li >> 1);
            if (use > 0 && !mbar_wait_or_abort(&acc_empty[b], (use - 1) & 1, abort_flag)) {
                fail(21);
                break;
            }
            tc_fence_after();
            bool ok = true;
            for (int kc = kc0; kc < kc1; ++kc, ++g) {
                const int s = (int)(g % kJvStages);
                if (!mbar_wait_or_abort_sleep(&full[s], (uint32_t)((g / kJvStages) & 1), abort_flag)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                unsigned char *sp = ops + (size_t)s * kJvStageBytes;
                const uint64_t da = sw128_desc(sp), db = sw128_desc(sp + kAB);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk)
                    umma_bf16(tmem + (uint32_t)b * kJvAccCols, da + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2),
                              idesc, (kc > kc0 || kk > 0) ? 1u : 0u);
                // the stage is free once every CTA of the cluster has read it
                if (C > 1)
                    umma_commit_mc(&empty[s], mask);
                else
                    umma_commit(&empty[s]);
            }
            umma_commit(&acc_full[b]);
            committed = li;
            if (!ok) {
                fail(22);
                break;
            }
        }
        if (*abort_flag && committed >= 0) {
            // the MMAs in flight finish before the TMEM is released
            mbar_wait(&acc_full[committed & 1], (uint32_t)((committed >> 1) & 1));
        }
    } else if (warp >= 2) {
        // --------------------------------------------------------- epilogue
        const int q = warp & 3, grp = (warp - 2) >> 2, c0 = grp * 16;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        for (int64_t li = 0; li < nunits; ++li) {
            const Tc4Unit u = tc4_unit<kMode>(a, cl + li * ncl, rank);
            const int64_t m0 = u.mt * kBM;
            const int n0 = u.nt * kBN;
            const int64_t row = m0 + q * 32 + lane;
            const bool row_ok = row < a.rows;
            const int col0 = n0 + c0;
            // mode 0: t' of the warp's 16 columns, in flight while the MMAs
            // run (tile-major pairs: a warp's 32 rows of a column pair are 512
            // contiguous bytes, one 16-byte load per lane and column pair)
            float2 tv[16];
            if (kMode == kTcRowDot) {
                if (u.mt < n_mt) {
                    const float4 *src =
                        a.Thl + (((size_t)u.mt * a.n_nt + u.nt) * (kBN / 2) + (c0 >> 1)) * kBM + q * 32 + lane;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 v4 = __ldcs(src + (size_t)j * kBM);
                        tv[2 * j] = make_float2(v4.x, v4.y);
                        tv[2 * j + 1] = make_float2(v4.z, v4.w);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) tv[j] = make_float2(0.f, 0.f);
                }
            }
            // the warp's column exponents; mode 0 scales them against the
            // tile's largest one F (lanes cover its 64 columns): 2^(f_j - F)
            int fe[16];
            {
                const int4 *ep = reinterpret_cast<const int4 *>(a.expB + col0);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int4 e4 = __ldg(ep + j);
                    fe[4 * j] = e4.x;
                    fe[4 * j + 1] = e4.y;
                    fe[4 * j + 2] = e4.z;
                    fe[4 * j + 3] = e4.w;
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) fe[j] = col0 + j < a.cols ? fe[j] : -100000;
            }
            int F = 0;
            float cs[16];
            if (kMode == kTcRowDot) {
                const int ca = n0 + lane, cb = n0 + 32 + lane;
                const int ea = ca < a.cols ? __ldg(a.expB + ca) : -100000;
                const int eb = cb < a.cols ? __ldg(a.expB + cb) : -100000;
                F = __reduce_max_sync(0xffffffffu, ea > eb ? ea : eb);
                if (F == -100000) F = 0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int e = fe[j] - F + 127;
                    cs[j] = e >= 1 ? __int_as_float(e << 23) : 0.f;
                }
            }
            const int b = (int)(li & 1);
            const uint32_t use = (uint32_t)(li >> 1);
            int ok = 1;
            if (lane == 0) ok = mbar_wait_or_abort_sleep(&acc_full[b], use & 1, abort_flag) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) {
                if (lane == 0) fail(23);
                break;
            }
            tc_fence_after();
            if (kMode == kTcStoreT) {
                // P^T[z][col][row] = V 2^(f_col - 33), V = D_0 2^22 + D_1 2^11 + D_2 exact
                // (|D_t| < 2^24: K per unit <= 8192)
                double *dst = a.P + (size_t)u.z * a.split_stride + row;
#pragma unroll
                for (int c8 = 0; c8 < 16; c8 += 8) {
                    uint32_t r[kJvSB][8];
#pragma unroll
                    for (int t = 0; t < kJvSB; ++t)
                        tmem_ld8(tmem + (uint32_t)b * kJvAccCols + lane_base + (uint32_t)(t * kBN + c0 + c8), r[t]);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const long long V = ((long long)__float2int_rn(__uint_as_float(r[0][j])) << 22) +
                                            ((long long)__float2int_rn(__uint_as_float(r[1][j])) << 11) +
                                            (long long)__float2int_rn(__uint_as_float(r[2][j]));
                        const int col = col0 + c8 + j;
                        if (row_ok && col < a.cols) dst[(size_t)col * a.ldp] = exact_to_double(V, fe[c8 + j] - 33);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[b]);
                continue;
            }
            // mode 0.  A: sum of D_0 u (exact pairs); B: sum of D_1 u; sm: the smaller terms
            float ah = 0.f, al = 0.f, bh = 0.f, bl = 0.f, sm = 0.f;
#pragma unroll
            for (int c8 = 0; c8 < 16; c8 += 8) {
                uint32_t r[kJvSB][8];
#pragma unroll
                for (int t = 0; t < kJvSB; ++t)
                    tmem_ld8(tmem + (uint32_t)b * kJvAccCols + lane_base + (uint32_t)(t * kBN + c0 + c8), r[t]);
                tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const float d0 = __uint_as_float(r[0][j]), d1 = __uint_as_float(r[1][j]);
                    const float d2 = __uint_as_float(r[2][j]);
                    const float u0 = __fmul_rn(tv[c8 + j].x, cs[c8 + j]), ul = __fmul_rn(tv[c8 + j].y, cs[c8 + j]);
                    const float p0 = __fmul_rn(d0, u0), e0 = __fmaf_rn(d0, u0, -p0);
                    const float p1 = __fmul_rn(d1, u0), e1 = __fmaf_rn(d1, u0, -p1);
                    // 2^-24-level: e0 + D_0 ul; 2^-35: (e1 + D_1 ul) 2^-11; 2^-22: D_2 u 2^-22
                    float lo = __fmaf_rn(d0, ul, e0);
                    lo = __fmaf_rn(__fmaf_rn(d1, ul, e1), 4.8828125e-04f, lo);
                    lo = __fmaf_rn(d2, __fmul_rn(u0, 2.384185791015625e-07f), lo);
                    sm = __fadd_rn(sm, lo);
                    float s, e;
                    two_sum(ah, p0, s, e);
                    ah = s;
                    al = __fadd_rn(al, e);
                    two_sum(bh, p1, s, e);
                    bh = s;
                    bl = __fadd_rn(bl, e);
                }
            }
            // the accumulator set is drained: hand it back to the MMA warp
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
            // (H, L) = A + B 2^-11 + sm as one FP32 pair
            float H, L;
            two_sum(ah, __fmul_rn(bh, 4.8828125e-04f), H, L);
            L = __fadd_rn(L, __fadd_rn(al, __fmaf_rn(bl, 4.8828125e-04f, sm)));
            // the four column groups of each row meet in the ring slot of this unit
            const int slot = (int)(li % kJvRing);
            red[((size_t)slot * 4 + grp) * kBM + q * 32 + lane] = make_float2(H, L);
            __syncwarp();
            if (lane == 0) mbar_arrive(&red_full[slot * 4 + q]);
            if (grp == 0) {
                int rok = 1;
                if (lane == 0)
                    rok = mbar_wait_or_abort_sleep(&red_full[slot * 4 + q], (uint32_t)((li / kJvRing) & 1), abort_flag)
                              ? 1
                              : 0;
                rok = __shfl_sync(0xffffffffu, rok, 0);
                if (!rok) {
                    if (lane == 0) fail(24);
                    break;
                }
                const float2 *rs = red + (size_t)slot * 4 * kBM + q * 32 + lane;
                float sh = rs[0].x, sl = rs[0].y;
#pragma unroll
                for (int g2 = 1; g2 < 4; ++g2) {
                    float s, e;
                    two_sum(sh, rs[g2 * kBM].x, s, e);
                    sh = s;
                    sl = __fadd_rn(sl, __fadd_rn(e, rs[g2 * kBM].y));
                }
                // 2^(F - 11) (sh + sl) in FP64 (the power of two by its exponent bits)
                const int ebias = F - 11 + 1023;
                const double scale = __longlong_as_double(
                    ebias < 1 ? 0LL : (ebias > 2046 ? 0x7FF0000000000000LL : (long long)ebias << 52));
                if (row_ok) a.P[(size_t)u.nt * a.rows + row] = ((double)sh + (double)sl) * scale;
            }
        }
    }
    tc_fence_before();
    // no peer multicasts into this CTA's shared memory or arrives on its
    // barriers after the cluster barrier; then the TMEM goes back
    if (C > 1)
        cluster_sync_all();
    else
        __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kJvTmemCols);
    }
}

int sgemm_stages(int SB) { return SB <= 4 ? 2 : 3; }

size_t sgemm_smem_bytes(int SB) {
    const size_t st = (size_t)sgemm_stages(SB) * (kAB + SB * kBB);
    const size_t tile = (size_t)kBM * kSgOutLd * 8;
    return 1024 + (st > tile ? st : tile) + 9 * sizeof(uint64_t) + 16;
}

// ------------------------------------------------------- operand staging ---

// S [B][N] int8 -> BF16 [B][ld]; column N holds 1.0 when augment, the rest of
// the padding 0.
// +-1, 1 and 0 as 16-bit operands: BF16 (the k_sgemm products) or FP16 (the
// 3-slice products of k_tc4); all three values are exact in both.
template <typename H>
__device__ __forceinline__ H to16(float v);
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half to16<__half>(float v) {
    return __float2half_rn(v);
}

template <typename H>
__global__ void k_pm1_rows(const int8_t *__restrict__ s, int64_t B, int N, int augment, int64_t ld,
                           H *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * ld) return;
    const int64_t k = idx / ld;
    const int i = (int)(idx % ld);
    float v = 0.f;
    if (i < N)
        v = (float)s[(size_t)k * N + i];
    else if (augment && i == N)
        v = 1.f;
    out[idx] = to16<H>(v);
}

// S^T with a row of ones: out [N+1][ld] (row i, column k) = s_ki (i < N) or 1.
template <typename H>
__global__ void k_pm1_cols(const int8_t *__restrict__ s, int64_t Ns, int N, int64_t ld, H *__restrict__ out) {
    __shared__ int8_t tile[32][33];
    const int64_t k0 = (int64_t)blockIdx.x * 32;
    const int i0 = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t k = k0 + r;
        const int i = i0 + threadIdx.x;
        tile[r][threadIdx.x] = (k < Ns && i < N) ? s[(size_t)k * N + i] : (int8_t)0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int i = i0 + r;
        const int64_t k = k0 + threadIdx.x;
        if (i > N || k >= ld) continue;
        float v = 0.f;
        if (k < Ns) v = i < N ? (float)tile[threadIdx.x][r] : 1.f;
        out[(size_t)i * ld + k] = to16<H>(v);
    }
}

// Largest binary exponent of |x| (frexp convention, |x| < 2^e); -100000 for 0.
__device__ __forceinline__ int exp_of(double x) {
    int b;
    unsigned long long m;
    bool n;
    split_bits(x, b, m, n);
    return m ? b - 1022 : -100000;
}

// Slice one value with row exponent e into SB bytes (sign applied).
__device__ __forceinline__ void slice_value(double x, int e, int SB, __nv_bfloat16 *out, int64_t plane) {
    int b;
    unsigned long long m;
    bool neg;
    split_bits(x, b, m, neg);
    unsigned long long y = 0;
    if (m) {
        const int sh = b - 1075 + 8 * SB - e;
        y = sh >= 0 ? (m << sh) : (sh <= -64 ? 0ULL : m >> (-sh));
    }
    for (int t = 0; t < SB; ++t) {
        const int d = (int)((y >> (8 * (SB - 1 - t))) & 0xFFULL);
        out[(size_t)t * plane] = __int2bfloat16_rn(neg ? -d : d);
    }
}

// slice_value for two neighbouring values of one row, written as BF16 pairs
// (4-byte stores, so that a warp writes whole 128-byte lines per plane).
__device__ __forceinline__ void slice_pair(double x0, double x1, int e, int SB, __nv_bfloat162 *out,
                                           int64_t plane2) {
    unsigned long long y[2] = {0ULL, 0ULL};
    bool neg[2];
    const double x[2] = {x0, x1};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        int b;
        unsigned long long m;
        split_bits(x[h], b, m, neg[h]);
        if (m) {
            const int sh = b - 1075 + 8 * SB - e;
            y[h] = sh >= 0 ? (m << sh) : (sh <= -64 ? 0ULL : m >> (-sh));
        }
    }
    for (int t = 0; t < SB; ++t) {
        const int d0 = (int)((y[0] >> (8 * (SB - 1 - t))) & 0xFFULL), d1 = (int)((y[1] >> (8 * (SB - 1 - t))) & 0xFFULL);
        out[(size_t)t * plane2] = __halves2bfloat162(__int2bfloat16_rn(neg[0] ? -d0 : d0),
                                                     __int2bfloat16_rn(neg[1] ? -d1 : d1));
    }
}

// The 4-slice case of slice_pair (grid32 and bf16_digit_pair, tc_ptx.cuh).
__device__ __forceinline__ void slice_pair4(double x0, double x1, int e, uint32_t *out, int64_t plane2) {
    uint32_t s0, s1;
    const uint32_t y0 = grid32(x0, e, s0), y1 = grid32(x1, e, s1);
    const uint32_t sg = (s0 << 15) | (s1 << 31);
#pragma unroll
    for (int t = 0; t < 4; ++t) out[(size_t)t * plane2] = bf16_digit_pair(y0, y1, 3u - (uint32_t)t, sg);
}

// Rows of a row-major FP64 matrix into 3 FP16 slices of 11-bit digits (the
// 33-bit grid of the row's exponent): out [3][rows][ld], one block per row.
__global__ void k_slice_rows_h3(const double *__restrict__ X, int64_t ldx, int64_t rows, int64_t K, int64_t ld,
                                uint32_t *__restrict__ out, int *__restrict__ expo) {
    const int64_t r = blockIdx.x;
    if (r >= rows) return;
    int ex = -100000;
    for (int64_t k = threadIdx.x; k < K; k += blockDim.x) ex = max(ex, exp_of(X[(size_t)r * ldx + k]));
    __shared__ int red[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ex;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -100000;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const int e = red[0] == -100000 ? 0 : red[0];
    const int64_t plane2 = rows * ld / 2;  // in FP16 pairs (ld even)
    for (int64_t k = 2 * threadIdx.x; k < ld; k += 2 * blockDim.x) {
        const double x0 = k < K ? X[(size_t)r * ldx + k] : 0.0, x1 = k + 1 < K ? X[(size_t)r * ldx + k + 1] : 0.0;
        uint32_t s0, s1;
        const unsigned long long y0 = grid33(x0, e, s0), y1 = grid33(x1, e, s1);
        const uint32_t sg = (s0 << 15) | (s1 << 31);
        uint32_t *o = out + ((size_t)r * ld + k) / 2;
#pragma unroll
        for (int t = 0; t < 3; ++t) o[(size_t)t * plane2] = f16_digit_pair(y0, y1, 22 - 11 * t, sg);
    }
    if (threadIdx.x == 0) expo[r] = e;
}

// Rows of a row-major FP64 matrix (row r, column k: X[r * ldx + k] for k < K;
// with augment, column K holds aug[r] and the operand has K + 1 columns) ->
// SB slices [SB][rows][ld] with one exponent per row.  One block per row.
__global__ void k_slice_long_rows(const double *__restrict__ X, int64_t ldx, int64_t rows, int64_t K,
                                  const double *__restrict__ aug, int SB, int64_t ld,
                                  __nv_bfloat16 *__restrict__ out, int *__restrict__ expo) {
    const int64_t r = blockIdx.x;
    if (r >= rows) return;
    const int64_t Ke = aug ? K + 1 : K;
    auto val = [&](int64_t k) -> double { return k < K ? X[(size_t)r * ldx + k] : aug[r]; };
    int ex = -100000;
    for (int64_t k = threadIdx.x; k < Ke; k += blockDim.x) ex = max(ex, exp_of(val(k)));
    __shared__ int red[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ex;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -100000;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (threadIdx.x == 0) red[0] = v;
    }
    __syncthreads();
    const int e = red[0] == -100000 ? 0 : red[0];
    const int64_t plane = rows * ld;
    for (int64_t k = threadIdx.x; k < ld; k += blockDim.x) {
        const double x = k < Ke ? val(k) : 0.0;
        slice_value(x, e, SB, out + (size_t)r * ld + k, plane);
    }
    if (threadIdx.x == 0) expo[r] = e;
}

__global__ void k_fill_int(int64_t n, int v, int *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

// Exponent of every row j <= M of (T' o g)^T: max over samples k of
// |t'_kj g'_k|, t'_kM = 1, g'_k = scale (g_k - shift).  Blocks of 32 rows x
// 256 samples, combined with atomicMax (-100000 marks an all-zero row).
// g'_k = scale (g_k - shift) and its exponent (|g'_k| < 2^ge_k).
__global__ void k_scale_g(int64_t Ns, const double *__restrict__ g, double scale, const double *__restrict__ shift,
                          double *__restrict__ gp, int *__restrict__ ge) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ns) return;
    const double v = scale * (g[k] - (shift ? *shift : 0.0));
    gp[k] = v;
    ge[k] = exp_of(v);
}

// Column exponents of T' o g' (column j of (T' o g')^T): an upper bound
// max_k (exp(T'_kj) + exp(g'_k)) of the exact exponent, at most one above it,
// taken with integer operations only.
__global__ void k_tg_colexp(const double *__restrict__ T, const int *__restrict__ ge, int64_t Ns, int M,
                            int *__restrict__ expo) {
    const int j = blockIdx.x * 32 + threadIdx.x;
    const int64_t k0 = (int64_t)blockIdx.y * 256;
    int ex = -100000;
    if (j <= M) {
        const int64_t kend = k0 + 256 < Ns ? k0 + 256 : Ns;
#pragma unroll 4
        for (int64_t k = k0 + threadIdx.y; k < kend; k += blockDim.y) {  // loads of 4 rows in flight
            const int et = j < M ? exp_of(T[(size_t)k * M + j]) : 1, eg = ge[k];
            if (et != -100000 && eg != -100000) ex = max(ex, et + eg);
        }
    }
    __shared__ int red[8][32];
    red[threadIdx.y][threadIdx.x] = ex;
    __syncthreads();
    if (threadIdx.y == 0 && j <= M) {
        for (int y = 1; y < (int)blockDim.y; ++y) ex = max(ex, red[y][threadIdx.x]);
        if (ex != -100000) atomicMax(&expo[j], ex);
    }
}

// max over k of ge[k] (-100000 marks zero): one block.
__global__ void k_max_exp(int64_t n, const int *__restrict__ ge, int *__restrict__ out) {
    __shared__ int red[32];
    int m = -100000;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) m = max(m, ge[k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        int v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : -100000;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (threadIdx.x == 0) *out = v;
    }
}

// Column exponents of T' o g' from the bound max_k |t'_kj| max_k |g'_k|:
// expo[j] = colexpT[j] + gmax (an upper bound of the per-entry exponents).
__global__ void k_colexp_bound(int M, const int *__restrict__ colexpT, const int *__restrict__ gmax,
                               int *__restrict__ expo) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > M) return;
    const int a = colexpT[j], b = *gmax;
    expo[j] = (a == -100000 || b == -100000) ? -100000 : a + b;
}

// (T' o g')^T sliced: out [SB][M+1][ld], row j, column k, through tiles of
// 64 k x 64 j in shared memory (FP64, row pitch 65).  A warp reads rows of T
// as 512 contiguous bytes (one 16-byte load per lane), all eight of a
// thread's loads issued before their first use; it writes BF16 pairs, 128
// contiguous bytes per plane and row j (ld is even).
constexpr int kTgPitch = 65;
__global__ void __launch_bounds__(256) k_tg_slice(const double *__restrict__ T, const double *__restrict__ gp,
                                                  int64_t Ns, int M, int SB, int64_t ld, int vec,
                                                  const int *__restrict__ expo, __nv_bfloat16 *__restrict__ out) {
    __shared__ double tile[64 * kTgPitch];  // [k][j]
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * 64;
    const int j0 = blockIdx.y * 64;
    const int jl = 2 * lane, j = j0 + jl;
    double2 v[8];
    double gk[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t k = k0 + w + 8 * i;
        gk[i] = k < Ns ? gp[k] : 0.0;
        if (k < Ns && vec && j + 1 < M) {
            v[i] = __ldcs(reinterpret_cast<const double2 *>(T + (size_t)k * M + j));
        } else {
            v[i].x = (k < Ns && j < M) ? T[(size_t)k * M + j] : (j == M ? 1.0 : 0.0);
            v[i].y = (k < Ns && j + 1 < M) ? T[(size_t)k * M + j + 1] : (j + 1 == M ? 1.0 : 0.0);
        }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = w + 8 * i;
        tile[r * kTgPitch + jl] = v[i].x * gk[i];
        tile[r * kTgPitch + jl + 1] = v[i].y * gk[i];
    }
    __syncthreads();
    const int64_t plane2 = (int64_t)(M + 1) * ld / 2;
    const int64_t k = k0 + 2 * lane;
#pragma unroll 2
    for (int i = 0; i < 8; ++i) {
        const int jr = w + 8 * i, jj = j0 + jr;
        if (jj > M || k >= ld) continue;
        const int e = expo[jj] == -100000 ? 0 : expo[jj];
        const double x0 = k < Ns ? tile[(2 * lane) * kTgPitch + jr] : 0.0;
        const double x1 = k + 1 < Ns ? tile[(2 * lane + 1) * kTgPitch + jr] : 0.0;
        if (SB == 4)
            slice_pair4(x0, x1, e, reinterpret_cast<uint32_t *>(out + (size_t)jj * ld + k), plane2);
        else
            slice_pair(x0, x1, e, SB, reinterpret_cast<__nv_bfloat162 *>(out + (size_t)jj * ld + k), plane2);
    }
}

// g'' = 2^-G g' as FP32 pairs (gh = fl32(g''), gl = fl32(g'' - gh): g'' - gh
// is exact in FP64), G = *gmax (|g'_k| < 2^G for every k, so |g''| < 1);
// an all-zero g' (G = -100000) gives zero pairs.
__global__ void k_g_pairs(int64_t Ns, const double *__restrict__ gp, const int *__restrict__ gmax,
                          float2 *__restrict__ g2) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Ns) return;
    const int G = *gmax;
    float2 v = make_float2(0.f, 0.f);
    if (G != -100000) {
        const double x = ldexp(gp[k], -G);
        const float h = __double2float_rn(x);
        v = make_float2(h, __double2float_rn(x - (double)h));
    }
    g2[k] = v;
}

// (T' o g')^T as 3 FP16 slices of signed 11-bit digits on the 33-bit grid of
// the column exponent e_j = colexpT[j] + G, from FP32 pairs only (no FP64
// arithmetic): t' from the tile-major pairs of k_split_t, g'' = 2^-G g' from
// k_g_pairs.  Per entry, x = t' g'' 2^(11 - colexpT[j]) (|x| <= 2^11) is
// formed as a pair by mul_pairs and scaled exactly, then cut by
// h3_signed_digits: x 2^22 = d0 2^22 + d1 2^11 + d2 within 1.25 units, the
// recombination V 2^(e_j - 33) of the J^T g epilogue.  Columns whose
// |t'| stays below 2^-100 (or are all zero) get zero digits.
// out [3][M+1][ld] FP16, four samples per 8-byte store.  One block per 128 x
// 64 tile of t' (the tile order of k_split_t): warp w takes column pairs 4w
// .. 4w + 3, lane l samples 4l .. 4l + 3 of the tile.  With skip set (the CG
// has converged) the kernel does nothing.
__global__ void __launch_bounds__(256) k_tg_slice_hl(int64_t Ns, int M, int n_nt, int64_t ld,
                                                     const float4 *__restrict__ Thl, const float2 *__restrict__ g2,
                                                     const int *__restrict__ colexpT, const int *__restrict__ skip,
                                                     uint2 *__restrict__ out) {
    if (skip && *skip) return;
    const int nt = blockIdx.x;
    const int64_t mt = blockIdx.y;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t k0 = mt * kBM + 4 * lane;
    if (k0 >= ld) return;  // ld is a multiple of 8: a lane's four samples are all in or all out
    float gh[4], gl[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float2 v = k0 + i < Ns ? __ldg(g2 + k0 + i) : make_float2(0.f, 0.f);
        gh[i] = v.x;
        gl[i] = v.y;
    }
    const float4 *src = Thl + ((size_t)mt * n_nt + nt) * (kBN / 2) * kBM + 4 * lane;
    const int64_t plane = (int64_t)(M + 1) * ld / 4;  // uint2 per plane
#pragma unroll 2
    for (int c = 0; c < 4; ++c) {
        const int cp = 4 * w + c;
        const int j0 = nt * kBN + 2 * cp;
        if (j0 > M) break;
        float4 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = __ldcs(src + (size_t)cp * kBM + i);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + h;
            if (j > M) break;
            const int cT = __ldg(colexpT + j);
            float d[3][4];
            if (cT < -100) {
#pragma unroll
                for (int i = 0; i < 4; ++i) d[0][i] = d[1][i] = d[2][i] = 0.f;
            } else {
                // 2^(11 - cT) in two exact factors (11 - cT <= 111 here)
                const int a1 = 11 - cT > 64 ? 64 : 11 - cT, a2 = 11 - cT - a1;
                const float s1 = __int_as_float((127 + a1) << 23), s2 = __int_as_float((127 + a2) << 23);
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float ph, pl;
                    mul_pairs(h ? v[i].z : v[i].x, h ? v[i].w : v[i].y, gh[i], gl[i], ph, pl);
                    h3_signed_digits(__fmul_rn(__fmul_rn(ph, s1), s2), __fmul_rn(__fmul_rn(pl, s1), s2), d[0][i],
                                     d[1][i], d[2][i]);
                }
            }
            uint2 *dst = out + ((size_t)j * ld + k0) / 4;
#pragma unroll
            for (int t = 0; t < 3; ++t)
                dst[(size_t)t * plane] = make_uint2(f16_int_pair(d[t][0], d[t][1]), f16_int_pair(d[t][2], d[t][3]));
        }
    }
}

// t' = [tanh(theta), 1] as FP32 pairs th = fl32(t), tl = fl32(t - th) (t - th
// is exact in FP64: th + tl = t within 2^-48 |t|), in the tile order of
// k_tc4 (mode 0): one block per 128 x 64 tile (row tile mt, column tile nt), stored
// at ((mt n_nt + nt) 32 + column pair) 128 + row as float4 (th, tl) of the
// pair's two columns.  Rows >= Ns and columns > M hold 0, column M holds 1.
// The tile passes through shared memory in FP64 (row pitch 65).
constexpr int kSplitPitch = kBN + 1;
__global__ void __launch_bounds__(256) k_split_t(int64_t Ns, int M, int n_nt, const double *__restrict__ T,
                                                 float4 *__restrict__ out) {
    extern __shared__ double tile[];  // [128][65]
    const int nt = blockIdx.x;
    const int64_t mt = blockIdx.y;
    const int64_t m0 = mt * kBM;
    const int n0 = nt * kBN;
    for (int e = threadIdx.x; e < kBM * kBN; e += blockDim.x) {
        const int r = e / kBN, c = e % kBN;
        const int64_t row = m0 + r;
        const int col = n0 + c;
        double v = 0.0;
        if (row < Ns) v = col < M ? __ldcs(T + (size_t)row * M + col) : (col == M ? 1.0 : 0.0);
        tile[r * kSplitPitch + c] = v;
    }
    __syncthreads();
    float4 *dst = out + ((size_t)mt * n_nt + nt) * (kBN / 2) * kBM;
    for (int e = threadIdx.x; e < kBM * (kBN / 2); e += blockDim.x) {
        const int cp = e / kBM, r = e % kBM;
        const double t0 = tile[r * kSplitPitch + 2 * cp], t1 = tile[r * kSplitPitch + 2 * cp + 1];
        const float h0 = __double2float_rn(t0), h1 = __double2float_rn(t1);
        dst[e] = make_float4(h0, __double2float_rn(t0 - (double)h0), h1, __double2float_rn(t1 - (double)h1));
    }
}

// w[r] = sum_t P[t][r] (tile-major partials of k_tc4 mode 0), in tile order.
__global__ void k_rowsum_tiles(int64_t rows, int ntc, const double *__restrict__ P, double *__restrict__ w) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double acc = 0.0;
    for (int t = 0; t < ntc; ++t) acc += P[(size_t)t * rows + r];
    w[r] = acc;
}

// w[row] = sum over the ntc column tiles of P[row][t], in tile order.
__global__ void k_rowsum_partials(int64_t rows, int ntc, const double *__restrict__ P, double *__restrict__ w) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= rows) return;
    double acc = 0.0;
    for (int t = 0; t < ntc; ++t) acc += P[(size_t)r * ntc + t];
    w[r] = acc;
}

// P^T as [ks][M+1][N+1] (column j, row i: k_tc4 mode 1) -> J^T g in the
// parameter layout, the ks partials summed in order.
__global__ void k_scatter_vjp_t(int N, int M, int ks, const double *__restrict__ PT, double *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(N + 1) * (M + 1);
    if (idx >= tot) return;
    const int j = (int)(idx / (N + 1)), i = (int)(idx % (N + 1));
    double v = PT[idx];
    for (int z = 1; z < ks; ++z) v += PT[(size_t)z * tot + idx];
    if (i == N && j == M) return;
    if (j == M)
        out[i] = v;
    else if (i == N)
        out[N + j] = v;
    else
        out[N + M + (size_t)j * N + i] = v;
}

// P^T [N+1][M+1] (row i, column j) -> J^T g in the parameter layout; PT
// holds ks K-split partial products [ks][(N+1)][(M+1)], summed in order.
__global__ void k_scatter_vjp(int N, int M, int ks, const double *__restrict__ PT, double *__restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(N + 1) * (M + 1);
    if (idx >= tot) return;
    const int i = (int)(idx / (M + 1)), j = (int)(idx % (M + 1));
    double v = PT[idx];
    for (int z = 1; z < ks; ++z) v += PT[(size_t)z * tot + idx];
    if (i == N && j == M) return;
    if (j == M)
        out[i] = v;
    else if (i == N)
        out[N + j] = v;
    else
        out[N + M + (size_t)j * N + i] = v;
}

// V' [(M+1)][(N+1)] from the parameter-shaped vector v: row j < M is
// [V_W[j][0..N-1], v_b[j]], row M is [v_a, 0].
__global__ void k_build_vaug(int N, int M, const double *__restrict__ v, double *__restrict__ Vp) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)(M + 1) * (N + 1);
    if (idx >= tot) return;
    const int j = (int)(idx / (N + 1)), i = (int)(idx % (N + 1));
    double x;
    if (j < M)
        x = i < N ? v[N + M + (size_t)j * N + i] : v[N + j];
    else
        x = i < N ? v[i] : 0.0;
    Vp[idx] = x;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }
inline int64_t pad8(int64_t x) { return (x + 7) / 8 * 8; }

bool make_rows_map(CUtensorMap *map, const __nv_bfloat16 *p, int64_t rows, int64_t K, int64_t ld, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool make_sliced_map(CUtensorMap *map, const __nv_bfloat16 *p, int64_t rows, int64_t K, int64_t ld, int SB,
                     int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)SB};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)rows * ld * 2};
    cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(p), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C (mode) A B^T + bias: A BF16 [rows][ldA] (K used), B slices [SB][cols][ldB].
// ksplit > 1 (mode 0 only): split z of the K range writes C + z split_stride.
// mode 3: C [rows][ldc >= col tiles] receives, per 64-column tile, the row
// products sum_col R[row][col] t'_col with t' = [T[row][0 .. Mt-1], 1, 0 ...].
cudaError_t sgemm(const __nv_bfloat16 *A, int64_t rows, int64_t ldA, const __nv_bfloat16 *Bsl, const int *expB,
                  int64_t cols, int64_t ldB, int64_t K, int SB, double *C, int64_t ldc, int mode,
                  const double *bias, int *err, cudaStream_t st, const double *T = nullptr, int Mt = 0,
                  int ksplit = 1, int64_t split_stride = 0) {
    if (rows <= 0 || cols <= 0 || K <= 0) return cudaSuccess;
    if (SB < 1 || SB > kMaxSB || rows > (1LL << 31) - kBM || cols > (1LL << 31) - kBN) return cudaErrorInvalidValue;
    if (ksplit < 1 || (ksplit > 1 && mode != 0) || (mode == 3 && T == nullptr)) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_rows_map(&ma, A, rows, K, ldA, kBM) || !make_sliced_map(&mb, Bsl, cols, K, ldB, SB, kBN))
        return cudaErrorInvalidValue;
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_sgemm);
    if (e != cudaSuccess) return e;
    const int kchunks = (int)((K + kBK - 1) / kBK);
    const int kc_split = (kchunks + ksplit - 1) / ksplit;
    uint32_t tcols = 32;
    while (tcols < (uint32_t)(SB * kBN)) tcols <<= 1;
    SgArgs a{rows, cols, kchunks, SB, kc_split, sgemm_stages(SB), kAB + SB * kBB, tcols, expB, C, ldc,
             split_stride, mode, bias, T, Mt, err};
    dim3 grid(nblk(cols, kBN), nblk(rows, kBM), (unsigned)((kchunks + kc_split - 1) / kc_split));
    (k_sgemm<<<grid, kSgThreads, sgemm_smem_bytes(SB), st>>>(ma, mb, a), nk::note_launch());
    return cudaGetLastError();
}

// One launch of k_tc4: as many clusters of a.C CTAs as fit at once (one CTA
// per SM), each walking its units round robin.
template <int kMode>
cudaError_t launch_tc4(const CUtensorMap &ma, const CUtensorMap &mb, const Tc4Args &a, cudaStream_t st) {
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_tc4<kMode>);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(kJvThreads);
    cfg.dynamicSmemBytes = jv_smem_bytes();
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int64_t ncl = sms / a.C;
    if (a.C > 1) {
        int fit = 0;
        cfg.gridDim = dim3((unsigned)(ncl * a.C));
        e = cudaOccupancyMaxActiveClusters(&fit, (const void *)k_tc4<kMode>, &cfg);
        if (e != cudaSuccess) return e;
        if (fit < 1) return cudaErrorInvalidConfiguration;  // the caller falls back to single CTAs
        if (fit < ncl) ncl = fit;
    }
    if (ncl > a.groups) ncl = a.groups;
    cfg.gridDim = dim3((unsigned)(ncl * a.C));
    e = cudaLaunchKernelEx(&cfg, k_tc4<kMode>, ma, mb, a);
    nk::note_launch();
    return e != cudaSuccess ? e : cudaGetLastError();
}

// CTAs per cluster of the J v product (B slices multicast across row tiles).
constexpr int kJvCluster = 2;

// The largest K whose FP32 levels stay exact with 11-bit digits (K 2047 < 2^24).
constexpr int kH3MaxK = 8192;

// J v partials P [n_nt][rows] = per 64-column tile, sum_col (A B^T)[row][col]
// t'_col by k_tc4 mode 0 (A FP16 +-1, B 3 FP16 slices; K <= 8192).
cudaError_t jvp4(const void *A, int64_t rows, int64_t ldA, const void *Bsl, const int *expB, int64_t cols,
                 int64_t ldB, int64_t K, const void *Thl, int Mt, double *P, int *err, cudaStream_t st,
                 const int *skip) {
    if (rows <= 0 || cols <= 0 || K <= 0) return cudaSuccess;
    if (K > kH3MaxK || rows > (1LL << 31) - kBM || cols > (1LL << 31) - kBN || Thl == nullptr)
        return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(Thl) & 15) != 0 || Mt + 1 != cols) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_rows_map(&ma, static_cast<const __nv_bfloat16 *>(A), rows, K, ldA, kBM) ||
        !make_sliced_map(&mb, static_cast<const __nv_bfloat16 *>(Bsl), cols, K, ldB, kJvSB, kBN))
        return cudaErrorInvalidValue;
    const int n_nt = (int)((cols + kBN - 1) / kBN);
    const int64_t n_mt = (rows + kBM - 1) / kBM;
    const int kchunks = (int)((K + kBK - 1) / kBK);
    for (int C = n_mt >= 2 * kJvCluster ? kJvCluster : 1;; C = 1) {
        const int n_mg = (int)((n_mt + C - 1) / C);
        Tc4Args a{rows, cols, kchunks, kchunks, 1, n_nt, n_mg, C, (int64_t)n_mg * n_nt, expB,
                  reinterpret_cast<const float4 *>(Thl), P, 0, 0, err, skip};
        const cudaError_t e = launch_tc4<kTcRowDot>(ma, mb, a, st);
        if (e == cudaErrorInvalidConfiguration && C > 1) continue;  // no cluster fits: single CTAs
        return e;
    }
}

// P^T [ks][cols][ldp] (column-major split-K partial products) = A B^T by
// k_tc4 mode 1 (A FP16 +-1, B 3 FP16 slices), with ks such that a unit is at
// most 128 K-chunks (K <= 8192: exact FP32 levels) and the last round of
// units is nearly full.
cudaError_t vjp4(const void *A, int64_t rows, int64_t ldA, const void *Bsl, const int *expB, int64_t cols,
                 int64_t ldB, int64_t K, double *P, int64_t ldp, int64_t split_stride, int max_ks, int *ks_out,
                 int *err, cudaStream_t st, const int *skip) {
    if (rows <= 0 || cols <= 0 || K <= 0) return cudaSuccess;
    if (rows > (1LL << 31) - kBM || cols > (1LL << 31) - kBN || ldp < rows) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_rows_map(&ma, static_cast<const __nv_bfloat16 *>(A), rows, K, ldA, kBM) ||
        !make_sliced_map(&mb, static_cast<const __nv_bfloat16 *>(Bsl), cols, K, ldB, kJvSB, kBN))
        return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int n_nt = (int)((cols + kBN - 1) / kBN);
    const int n_mt = (int)((rows + kBM - 1) / kBM);
    const int kchunks = (int)((K + kBK - 1) / kBK);
    const int ks_min = (kchunks + kH3MaxK / kBK - 1) / (kH3MaxK / kBK);
    if (ks_min > max_ks) return cudaErrorInvalidValue;
    // All row tiles of a unit in one cluster when there are 2 to 8 of them
    // (N + 1 <= 1024): each tile of digits is then read from L2 once and
    // multicast to every row tile (on the 24 x 24 workload, 5 row tiles:
    // 100.5 against 102.4 ms of products a step).  Single CTAs otherwise, or
    // where no cluster of that size fits.
    for (int C = n_mt >= 2 && n_mt <= 8 ? n_mt : 1;; C = 1) {
        const int n_mg = (n_mt + C - 1) / C, slots = sms / C;
        int ks = ks_min;
        double best = -1.0;
        for (int k = ks_min; k <= max_ks; ++k) {
            const int64_t units = (int64_t)n_mg * n_nt * k, rounds = (units + slots - 1) / slots;
            const double score = (double)units / (double)(rounds * slots) - 0.01 * (k - ks_min);
            if (score > best + 1e-12) best = score, ks = k;
        }
        const int kc_split = (kchunks + ks - 1) / ks;
        ks = (kchunks + kc_split - 1) / kc_split;
        *ks_out = ks;
        Tc4Args a{rows, cols, kchunks, kc_split, ks, n_nt, n_mg, C, (int64_t)n_mg * n_nt * ks, expB, nullptr, P,
                  ldp, split_stride, err, skip};
        e = launch_tc4<kTcStoreT>(ma, mb, a, st);
        if (e == cudaErrorInvalidConfiguration && C > 1) continue;
        return e;
    }
}

double sgemm_flops(int64_t rows, int64_t cols, int64_t K, int SB) {
    return 2.0 * (double)((rows + kBM - 1) / kBM * kBM) * (double)((cols + kBN - 1) / kBN * kBN) *
           (double)((K + kBK - 1) / kBK * kBK) * SB;
}

}  // namespace

// ============================================================ launchers ====

size_t tc_theta_ws_bytes(int N, int M, int64_t B) {
    const int64_t ld = pad8(N);
    return ((size_t)B * ld * 2 + 255) / 256 * 256 + ((size_t)kMaxSB * M * ld * 2 + 255) / 256 * 256 +
           ((size_t)M * 4 + 255) / 256 * 256 + 256;
}

// theta [B][M] = S W^T + b with W sliced 7 ways: exact up to 2^-56 of max|W_j|.
cudaError_t launch_theta_tc(int N, int M, const double *b, const double *W, const int8_t *s, int64_t B,
                            double *theta, int *err, void *ws, cudaStream_t st, int64_t ldtheta) {
    if (B <= 0) return cudaSuccess;
    const int64_t ld = pad8(N);
    char *p = static_cast<char *>(ws);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    auto *As = reinterpret_cast<__nv_bfloat16 *>(take((size_t)B * ld * 2));
    auto *Ws = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kMaxSB * M * ld * 2));
    auto *ew = reinterpret_cast<int *>(take((size_t)M * 4));
    (k_pm1_rows<<<nblk(B * ld, 256), 256, 0, st>>>(s, B, N, 0, ld, As), nk::note_launch());
    (k_slice_long_rows<<<M, 128, 0, st>>>(W, N, M, N, nullptr, kMaxSB, ld, Ws, ew), nk::note_launch());
    const int slot = prof_begin(NK_PROF_JVP_VJP, st);
    cudaError_t e = sgemm(As, B, ld, Ws, ew, M, ld, N, kMaxSB, theta, ldtheta > 0 ? ldtheta : M, 0, b, err, st);
    prof_end(slot, st, 2.0 * (double)B * N * (double)M, sgemm_flops(B, M, N, kMaxSB));
    return e != cudaSuccess ? e : cudaGetLastError();
}

size_t tc_jvp_ws_bytes(int N, int M, int64_t Ns) {
    const int64_t ld = pad8(N + 1), ntc = (M + 1 + kBN - 1) / kBN;
    return ((size_t)Ns * ld * 2 + 255) / 256 * 256 + ((size_t)kMaxSB * (M + 1) * ld * 2 + 255) / 256 * 256 +
           ((size_t)(M + 1) * (N + 1) * 8 + 255) / 256 * 256 + ((size_t)(M + 1) * 4 + 255) / 256 * 256 +
           ((size_t)Ns * ntc * 8 + 255) / 256 * 256 + tc_split_t_bytes(M, Ns) + 256;
}

size_t tc_split_t_bytes(int M, int64_t Ns) {
    return (size_t)((Ns + kBM - 1) / kBM) * kBM * (size_t)((M + 1 + kBN - 1) / kBN) * kBN * sizeof(float2);
}

cudaError_t launch_split_t(int M, int64_t Ns, const double *T, void *Thl, cudaStream_t st) {
    if (Ns <= 0) return cudaSuccess;
    const int n_nt = (M + 1 + kBN - 1) / kBN;
    const int64_t n_mt = (Ns + kBM - 1) / kBM;
    if (n_mt > 65535) return cudaErrorInvalidValue;
    const size_t smem = (size_t)kBM * kSplitPitch * sizeof(double);
    cudaError_t e = nk::allow_max_dynamic_smem((const void *)k_split_t);
    if (e != cudaSuccess) return e;
    (k_split_t<<<dim3(n_nt, (unsigned)n_mt), 256, smem, st>>>(Ns, M, n_nt, T, static_cast<float4 *>(Thl)),
     nk::note_launch());
    return cudaGetLastError();
}

size_t tc_jvp_operand_bytes(int N, int64_t Ns) { return (size_t)Ns * pad8(N + 1) * 2; }
size_t tc_vjp_operand_bytes(int N, int64_t Ns) { return (size_t)(N + 1) * pad8(Ns) * 2; }

cudaError_t launch_jacobian_operands(int N, int64_t Ns, const int8_t *s, void *opA, void *opT, cudaStream_t st) {
    if (Ns <= 0) return cudaSuccess;
    const int64_t lda = pad8(N + 1), ldt = pad8(Ns);
    (k_pm1_rows<<<nblk(Ns * lda, 256), 256, 0, st>>>(s, Ns, N, 1, lda, static_cast<__half *>(opA)),
     nk::note_launch());
    (k_pm1_cols<<<dim3(nblk(ldt, 32), nblk(N + 1, 32)), dim3(32, 8), 0, st>>>(s, Ns, N, ldt, static_cast<__half *>(opT)),
     nk::note_launch());
    return cudaGetLastError();
}

// out = J v with V' cut into SB slices: w = rowdot(T', S' V'^T), the row
// products taken in the S-GEMM epilogue per 64-column tile and summed after.
cudaError_t launch_jvp_tc(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *v,
                          double *out, int SB, int *err, void *ws, cudaStream_t st, const void *opA,
                          const void *Thl, const int *skip) {
    const int64_t ld = pad8(N + 1);
    char *p = static_cast<char *>(ws);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    auto *As = reinterpret_cast<__nv_bfloat16 *>(take((size_t)Ns * ld * 2));
    auto *Vs = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kMaxSB * (M + 1) * ld * 2));
    auto *Vp = reinterpret_cast<double *>(take((size_t)(M + 1) * (N + 1) * 8));
    auto *ev = reinterpret_cast<int *>(take((size_t)(M + 1) * 4));
    const int ntc = (M + 1 + kBN - 1) / kBN;
    auto *P = reinterpret_cast<double *>(take((size_t)Ns * ntc * 8));
    const int64_t tot = (int64_t)(M + 1) * (N + 1);
    // 4 slices' accuracy (the CG products) through the persistent kernel on 3
    // FP16 slices of 11-bit digits (33 bits), where K = N + 1 allows it
    const bool persistent = SB == 4 && N + 1 <= kH3MaxK;
    if (persistent && opA)
        As = static_cast<__nv_bfloat16 *>(const_cast<void *>(opA));  // FP16 bits
    else if (persistent)
        (k_pm1_rows<<<nblk(Ns * ld, 256), 256, 0, st>>>(s, Ns, N, 1, ld, reinterpret_cast<__half *>(As)),
         nk::note_launch());
    else
        (k_pm1_rows<<<nblk(Ns * ld, 256), 256, 0, st>>>(s, Ns, N, 1, ld, As), nk::note_launch());
    (k_build_vaug<<<nblk(tot, 256), 256, 0, st>>>(N, M, v, Vp), nk::note_launch());
    if (persistent)
        (k_slice_rows_h3<<<M + 1, 128, 0, st>>>(Vp, N + 1, M + 1, N + 1, ld, reinterpret_cast<uint32_t *>(Vs), ev),
         nk::note_launch());
    else
        (k_slice_long_rows<<<M + 1, 128, 0, st>>>(Vp, N + 1, M + 1, N + 1, nullptr, SB, ld, Vs, ev),
         nk::note_launch());
    if (persistent && Thl == nullptr) {
        void *own = take(tc_split_t_bytes(M, Ns));
        cudaError_t es = launch_split_t(M, Ns, T, own, st);
        if (es != cudaSuccess) return es;
        Thl = own;
    }
    const int slot = prof_begin(NK_PROF_JVP_VJP, st);
    cudaError_t e = persistent ? jvp4(As, Ns, ld, Vs, ev, M + 1, ld, N + 1, Thl, M, P, err, st, skip)
                               : sgemm(As, Ns, ld, Vs, ev, M + 1, ld, N + 1, SB, P, ntc, 3, nullptr, err, st, T, M);
    prof_end(slot, st, 2.0 * (double)Ns * (N + 1) * (double)(M + 1),
             sgemm_flops(Ns, M + 1, N + 1, persistent ? kJvSB : SB));
    if (e != cudaSuccess) return e;
    if (persistent)
        (k_rowsum_tiles<<<nblk(Ns, 256), 256, 0, st>>>(Ns, ntc, P, out), nk::note_launch());
    else
        (k_rowsum_partials<<<nblk(Ns, 256), 256, 0, st>>>(Ns, ntc, P, out), nk::note_launch());
    return cudaGetLastError();
}

constexpr int kMaxKSplit = 16;

// K-split count for a grid of `tiles` output tiles over `slots` resident
// CTAs: the share of the last wave's slots that hold work, less 1 % per extra
// split (its partial output is written and summed), best over 1 .. 8 splits
// of at least 4 K-chunks each.
static int pick_ksplit(int64_t tiles, int64_t kchunks, int64_t slots) {
    int best = 1;
    double best_score = -1.0;
    for (int ks = 1; ks <= kMaxKSplit; ++ks) {
        if (ks > 1 && kchunks / ks < 4) break;
        const int64_t ctas = tiles * ks, waves = (ctas + slots - 1) / slots;
        const double score = (double)ctas / (double)(waves * slots) - 0.01 * (ks - 1);
        if (score > best_score + 1e-12) best_score = score, best = ks;
    }
    return best;
}

size_t tc_vjp_ws_bytes(int N, int M, int64_t Ns) {
    const int64_t ld = pad8(Ns);
    return ((size_t)(N + 1) * ld * 2 + 255) / 256 * 256 + ((size_t)kMaxSB * (M + 1) * ld * 2 + 255) / 256 * 256 +
           ((size_t)(M + 2) * 4 + 255) / 256 * 256 +
           ((size_t)kMaxKSplit * (N + 1) * (M + 1) * 8 + 255) / 256 * 256 + ((size_t)Ns * 8 + 255) / 256 * 256 +
           ((size_t)Ns * 4 + 255) / 256 * 256 + 256 +
           // the 3-slice path: g'' pairs, and the column exponents and t'
           // pairs of T when the caller does not pass them
           ((size_t)Ns * 8 + 255) / 256 * 256 + ((size_t)(M + 1) * 4 + 255) / 256 * 256 +
           (tc_colexp_ws_bytes(M, Ns) + 255) / 256 * 256 + (tc_split_t_bytes(M, Ns) + 255) / 256 * 256;
}

// out = J^T g' with g' = scale (g - shift), (T' o g')^T cut into SB slices.
size_t tc_colexp_ws_bytes(int M, int64_t Ns) { return ((size_t)Ns * 4 + 255) / 256 * 256 + (size_t)(M + 1) * 4; }

// colexpT[j] = exponent of max_k |t'_kj| (t'_kM = 1), once per T.
cudaError_t launch_colexp_t(int M, int64_t Ns, const double *T, int *colexpT, void *ws, cudaStream_t st) {
    int *zero = static_cast<int *>(ws);
    (k_fill_int<<<nblk(Ns, 256), 256, 0, st>>>(Ns, 0, zero), nk::note_launch());
    (k_fill_int<<<nblk(M + 1, 256), 256, 0, st>>>(M + 1, -100000, colexpT), nk::note_launch());
    (k_tg_colexp<<<dim3(nblk(M + 1, 32), nblk(Ns, 256)), dim3(32, 8), 0, st>>>(T, zero, Ns, M, colexpT),
     nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_vjp_tc(int N, int M, int64_t Ns, const int8_t *s, const double *T, const double *g,
                          double scale, const double *shift, double *out, int SB, int *err, void *ws,
                          cudaStream_t st, const int *colexpT, const void *opT, const void *Thl,
                          const int *skip) {
    const int64_t ld = pad8(Ns);
    char *p = static_cast<char *>(ws);
    auto take = [&](size_t bytes) {
        char *q = p;
        p += (bytes + 255) / 256 * 256;
        return q;
    };
    auto *St = reinterpret_cast<__nv_bfloat16 *>(take((size_t)(N + 1) * ld * 2));
    auto *Gs = reinterpret_cast<__nv_bfloat16 *>(take((size_t)kMaxSB * (M + 1) * ld * 2));
    auto *eg = reinterpret_cast<int *>(take((size_t)(M + 2) * 4));
    auto *PT = reinterpret_cast<double *>(take((size_t)kMaxKSplit * (N + 1) * (M + 1) * 8));
    auto *gp = reinterpret_cast<double *>(take((size_t)Ns * 8));
    auto *ge = reinterpret_cast<int *>(take((size_t)Ns * 4));
    dim3 tb(32, 8);
    const int64_t kchunks = (Ns + kBK - 1) / kBK;
    // 4 slices' accuracy (the CG products) through the persistent kernel on 3
    // FP16 slices of 11-bit digits (33 bits), in units of at most 8192 samples
    const bool h3 = SB == 4 && (kchunks + kH3MaxK / kBK - 1) / (kH3MaxK / kBK) <= kMaxKSplit;
    if (h3 && opT)
        St = static_cast<__nv_bfloat16 *>(const_cast<void *>(opT));  // FP16 bits
    else if (h3)
        (k_pm1_cols<<<dim3(nblk(ld, 32), nblk(N + 1, 32)), tb, 0, st>>>(s, Ns, N, ld, reinterpret_cast<__half *>(St)),
         nk::note_launch());
    else
        (k_pm1_cols<<<dim3(nblk(ld, 32), nblk(N + 1, 32)), tb, 0, st>>>(s, Ns, N, ld, St), nk::note_launch());
    (k_scale_g<<<nblk(Ns, 256), 256, 0, st>>>(Ns, g, scale, shift, gp, ge), nk::note_launch());
    if (h3) {
        // 3 FP16 slices from FP32 pairs: the column exponents of T and its
        // tile-major pairs (given once per solve by the CG, else built here),
        // the bound e_j = colexpT[j] + max_k exp(g'_k), g'' = 2^-G g' as pairs
        const int *cT = colexpT;
        if (cT == nullptr) {
            int *own = reinterpret_cast<int *>(take((size_t)(M + 1) * 4));
            cudaError_t ec = launch_colexp_t(M, Ns, T, own, take(tc_colexp_ws_bytes(M, Ns)), st);
            if (ec != cudaSuccess) return ec;
            cT = own;
        }
        if (Thl == nullptr) {
            void *own = take(tc_split_t_bytes(M, Ns));
            cudaError_t es = launch_split_t(M, Ns, T, own, st);
            if (es != cudaSuccess) return es;
            Thl = own;
        }
        auto *g2 = reinterpret_cast<float2 *>(take((size_t)Ns * 8));
        (k_max_exp<<<1, 1024, 0, st>>>(Ns, ge, eg + M + 1), nk::note_launch());
        (k_colexp_bound<<<nblk(M + 1, 256), 256, 0, st>>>(M, cT, eg + M + 1, eg), nk::note_launch());
        (k_g_pairs<<<nblk(Ns, 256), 256, 0, st>>>(Ns, gp, eg + M + 1, g2), nk::note_launch());
        const int n_nt = (M + 1 + kBN - 1) / kBN;
        const int64_t n_mt = (Ns + kBM - 1) / kBM;
        if (n_mt > 65535) return cudaErrorInvalidValue;
        (k_tg_slice_hl<<<dim3(n_nt, (unsigned)n_mt), 256, 0, st>>>(Ns, M, n_nt, ld, static_cast<const float4 *>(Thl),
                                                                   g2, cT, skip, reinterpret_cast<uint2 *>(Gs)),
         nk::note_launch());
    } else {
        (k_fill_int<<<nblk(M + 1, 256), 256, 0, st>>>(M + 1, -100000, eg), nk::note_launch());
        (k_tg_colexp<<<dim3(nblk(M + 1, 32), nblk(Ns, 256)), dim3(32, 8), 0, st>>>(T, ge, Ns, M, eg),
         nk::note_launch());
        const int vec = (M % 2 == 0) && ((reinterpret_cast<uintptr_t>(T) & 15) == 0);
        (k_tg_slice<<<dim3(nblk(ld, 64), nblk(M + 1, 64)), 256, 0, st>>>(T, gp, Ns, M, SB, ld, vec, eg, Gs),
         nk::note_launch());
    }
    // split the long K = Ns range so that the last wave of CTAs is nearly
    // full (every split keeps >= 4 chunks; each split's FP32 levels stay exact)
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = nk::allow_max_dynamic_smem((const void *)k_sgemm);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sgemm, kSgThreads, sgemm_smem_bytes(SB));
    if (e != cudaSuccess) return e;
    const int64_t tiles = (int64_t)nblk(M + 1, kBN) * nblk(N + 1, kBM);
    const int64_t tot = (int64_t)(N + 1) * (M + 1);
    if (h3) {
        // the persistent kernel, P^T column-major
        int ks4 = 1;
        const int slot = prof_begin(NK_PROF_JVP_VJP, st);
        e = vjp4(St, N + 1, ld, Gs, eg, M + 1, ld, Ns, PT, N + 1, tot, kMaxKSplit, &ks4, err, st, skip);
        prof_end(slot, st, 2.0 * (double)Ns * (N + 1) * (double)(M + 1), sgemm_flops(N + 1, M + 1, Ns, kJvSB));
        if (e != cudaSuccess) return e;
        (k_scatter_vjp_t<<<nblk(tot, 256), 256, 0, st>>>(N, M, ks4, PT, out), nk::note_launch());
        return cudaGetLastError();
    }
    int ks = pick_ksplit(tiles, kchunks, (int64_t)sms * (per_sm > 0 ? per_sm : 1));
    const int kc_split = (int)((kchunks + ks - 1) / ks);
    ks = (int)((kchunks + kc_split - 1) / kc_split);  // splits the kernel launches
    const int slot = prof_begin(NK_PROF_JVP_VJP, st);
    e = sgemm(St, N + 1, ld, Gs, eg, M + 1, ld, Ns, SB, PT, M + 1, 0, nullptr, err, st, nullptr, 0, ks, tot);
    prof_end(slot, st, 2.0 * (double)Ns * (N + 1) * (double)(M + 1), sgemm_flops(N + 1, M + 1, Ns, SB));
    if (e != cudaSuccess) return e;
    (k_scatter_vjp<<<nblk(tot, 256), 256, 0, st>>>(N, M, ks, PT, out), nk::note_launch());
    return cudaGetLastError();
}

}  // namespace nk
