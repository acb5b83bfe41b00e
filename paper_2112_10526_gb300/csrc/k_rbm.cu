// RBM kernels: flip-ratio tables, ln psi, chain initialisation, Metropolis
// sweeps and local energies.
//
// Model (NetKet 3, Sec. 3.2, Table tab:nk.models, RBM):
//   ln psi(s) = sum_i a_i s_i + sum_j ln cosh theta_j,  theta = b + W s.
//
// Flip-ratio identity used by the sweep and local-energy kernels.  With
// t_j = tanh theta_j and s_i = +-1, cosh(theta - d) = cosh theta cosh d
// (1 - tanh theta tanh d) gives, for flipping site i (d_j = 2 W_ji s_i):
//   ln psi(s^(i)) - ln psi(s) = -2 a_i s_i + K_i + sum_j ln(1 - s_i t_j tau_ji)
// with tau_ji = tanh(2 W_ji), K_i = sum_j ln cosh(2 W_ji); and for swapping an
// antiparallel pair (i, k) (d_j = 2 s_i (W_ji - W_jk)):
//   ln psi(s^(ik)) - ln psi(s) = -2 s_i (a_i - a_k) + K_e + sum_j ln(1 - s_i t_j tau_ej)
// with tau_ej = tanh(2 (W_ji - W_jk)), K_e = sum_j ln cosh(2 (W_ji - W_jk)).
// The sum of logs is taken as the log of one renormalised product, so a
// ratio costs one FMA and one multiply per hidden unit.  After an accepted
// move t_j becomes tanh(theta_j - d_j) = (t_j - s_i tau_j) / (1 - s_i t_j tau_j).

#include <cuda_runtime.h>

#include "nk_common.cuh"
#include "nk_internal.h"

namespace nk {

namespace {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- tables ---

__global__ void k_transpose_W(int N, int M, const double *__restrict__ W, double *__restrict__ Wt) {
    __shared__ double tile[32][33];
    int j0 = blockIdx.y * 32, i0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int j = j0 + r, i = i0 + threadIdx.x;
        if (j < M && i < N) tile[r][threadIdx.x] = W[(size_t)j * N + i];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        int i = i0 + r, j = j0 + threadIdx.x;
        if (i < N && j < M) Wt[(size_t)i * M + j] = tile[threadIdx.x][r];
    }
}

// One block per site (or edge): tau row, its transpose and K by a fixed-order
// block reduction.
template <typename R>
__global__ void k_tau_rows(int N, int M, int nrows, const double *__restrict__ Wt,
                           const int32_t *__restrict__ edges, R *__restrict__ tau,
                           R *__restrict__ tauT, R *__restrict__ K) {
    int r = blockIdx.x;
    if (r >= nrows) return;
    const double *w0, *w1 = nullptr;
    if (edges) {
        const int i = edges[2 * r], k = edges[2 * r + 1];
        if ((unsigned)i >= (unsigned)N || (unsigned)k >= (unsigned)N) return;  // never used
        w0 = Wt + (size_t)i * M;
        w1 = Wt + (size_t)k * M;
    } else {
        w0 = Wt + (size_t)r * M;
    }
    double part = 0.0;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        double d = w1 ? (w0[j] - w1[j]) : w0[j];
        double v = tanh(2.0 * d);
        tau[(size_t)r * M + j] = (R)v;
        tauT[(size_t)j * nrows + r] = (R)v;
        part += lncosh(2.0 * d);
    }
    __shared__ double red[32];
    part = warp_sum(part);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        int nw = blockDim.x >> 5;
        double v = threadIdx.x < nw ? red[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) K[r] = (R)v;
    }
}

// ------------------------------------------------------------------ ln psi ---

// One warp per configuration; theta rebuilt in FP64 from the transposed W.
__global__ void k_logpsi(int N, int M, const double *__restrict__ a, const double *__restrict__ b,
                         const double *__restrict__ Wt, const int8_t *__restrict__ s, int64_t B,
                         double *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char sm[];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (k >= B) return;
    int8_t *sv = reinterpret_cast<int8_t *>(sm) + (size_t)warp * ((N + 15) & ~15);
    for (int i = lane; i < N; i += 32) sv[i] = s[(size_t)k * N + i];
    __syncwarp();
    double part = 0.0;
    for (int i = lane; i < N; i += 32) part += a[i] * (double)sv[i];
    for (int j = lane; j < M; j += 32) {
        double th = b[j];
        for (int i = 0; i < N; ++i) th = fma(Wt[(size_t)i * M + j], (double)sv[i], th);
        part += lncosh(th);
    }
    part = warp_sum(part);
    if (lane == 0) out[k] = part;
}

// ln psi from a precomputed theta [B][M]: one warp per configuration.
__global__ void k_logpsi_theta(int N, int M, const double *__restrict__ a, const double *__restrict__ theta,
                               const int8_t *__restrict__ s, int64_t B, double *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (k >= B) return;
    double part = 0.0;
    for (int i = lane; i < N; i += 32) part += a[i] * (double)s[(size_t)k * N + i];
    for (int j = lane; j < M; j += 32) part += lncosh(theta[(size_t)k * M + j]);
    part = warp_sum(part);
    if (lane == 0) out[k] = part;
}

__global__ void k_tanh_inplace(int64_t n, double *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = tanh(x[i]);
}

// ------------------------------------------------------------- chain init ---

__global__ void k_chain_init(int N, int C, int rule, unsigned long long seed, unsigned stream_id,
                             int8_t *__restrict__ s) {
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    int8_t *sc = s + (size_t)c * N;
    if (rule == NK_RULE_LOCAL) {
        for (int blk = 0; blk * 256 < N; ++blk) {
            Philox4 y = philox4x64_10((unsigned long long)blk, (unsigned long long)c, stream_id, 1ULL,
                                      seed, 0ULL);
            for (int bit = 0; bit < 256 && blk * 256 + bit < N; ++bit)
                sc[blk * 256 + bit] = ((y.v[bit >> 6] >> (bit & 63)) & 1ULL) ? 1 : -1;
        }
    } else {
        for (int i = 0; i < N; ++i) sc[i] = i < N / 2 ? 1 : -1;
        for (int i = N - 1; i >= 1; --i) {
            Philox4 y = philox4x64_10((unsigned long long)i, (unsigned long long)c, stream_id, 1ULL,
                                      seed, 0ULL);
            int j = pick_index(y.v[0], i + 1);
            int8_t tmp = sc[i];
            sc[i] = sc[j];
            sc[j] = tmp;
        }
    }
}

// ------------------------------------------------------ ratio products ---

// prod over j = j0, j0 + step, ... < M of (1 - si t_j tau[j * tstride]) as
// mantissa x 2^exp.  Four independent running products (each renormalised
// every RenormEvery factors) keep several loads and multiplies in flight.
template <typename R>
__device__ __forceinline__ Prod<R> strided_product(const R *__restrict__ t, const R *__restrict__ tau, size_t tstride,
                                                   R si, int j0, int step, int M) {
    R m0 = R(1), m1 = R(1), m2 = R(1), m3 = R(1);
    int e = 0, cnt = 0;
    int j = j0;
    for (; j + 3 * step < M; j += 4 * step) {
        m0 *= R(1) - si * t[j] * tau[(size_t)j * tstride];
        m1 *= R(1) - si * t[j + step] * tau[(size_t)(j + step) * tstride];
        m2 *= R(1) - si * t[j + 2 * step] * tau[(size_t)(j + 2 * step) * tstride];
        m3 *= R(1) - si * t[j + 3 * step] * tau[(size_t)(j + 3 * step) * tstride];
        if (++cnt == RenormEvery<R>::value) {
            Prod<R> q0{m0, 0}, q1{m1, 0}, q2{m2, 0}, q3{m3, 0};
            renorm(q0);
            renorm(q1);
            renorm(q2);
            renorm(q3);
            m0 = q0.m;
            m1 = q1.m;
            m2 = q2.m;
            m3 = q3.m;
            e += q0.e + q1.e + q2.e + q3.e;
            cnt = 0;
        }
    }
    for (; j < M; j += step) m0 *= R(1) - si * t[j] * tau[(size_t)j * tstride];
    Prod<R> p{m0, e};
    renorm(p);
    p.m *= m1;
    renorm(p);
    p.m *= m2;
    renorm(p);
    p.m *= m3;
    renorm(p);
    return p;
}

// Lanes over hidden units, four consecutive units per lane (16-byte loads of
// t and tau): prod over this lane's units of (1 - si t_j tau_j).  Needs
// M % 4 == 0 and 16-byte aligned rows.  kSharedTau: the tau row is in shared
// memory (plain loads instead of the read-only global path); the arithmetic
// is the same either way.
template <bool kSharedTau>
__device__ __forceinline__ float4 load_tau4(const float *tau) {
    if (kSharedTau) return *reinterpret_cast<const float4 *>(tau);
    return __ldg(reinterpret_cast<const float4 *>(tau));
}

// frexp of a positive running product: m = f 2^k, f in [0.5, 1), from the
// exponent bits (zero and subnormal m are left as they are, k = 0; the
// products here are renormalised every 8 factors in (0, 2)).
__device__ __forceinline__ float renorm_bits(float m, int &e) {
    const int b = __float_as_int(m);
    const int be = (b >> 23) & 0xFF;
    e += be ? be - 126 : 0;
    return be ? __int_as_float((b & 0x807FFFFF) | 0x3F000000) : m;
}

// A lane's tau row in groups g of four 16-byte loads (units j0 + 512 g + 128
// u, u < 4), for g = 0 .. full - 1: f(uv, g) runs on each group in order,
// while a ring of four keeps the loads of the next three groups in flight
// (large M reads the row from L2, one round trip per group otherwise).
// Returns full.
template <class F>
__device__ __forceinline__ int tau_ring4(const float *__restrict__ tau, int j0, int full, F &&f) {
    float4 r0[4], r1[4], r2[4], r3[4];
    auto load = [&](float4 (&r)[4], int g) {
#pragma unroll
        for (int u = 0; u < 4; ++u) r[u] = __ldg(reinterpret_cast<const float4 *>(tau + j0 + g * 512 + u * 128));
    };
    if (0 < full) load(r0, 0);
    if (1 < full) load(r1, 1);
    if (2 < full) load(r2, 2);
    int g = 0;
    for (; g + 3 < full; g += 4) {
        load(r3, g + 3);
        f(r0, g);
        if (g + 4 < full) load(r0, g + 4);
        f(r1, g + 1);
        if (g + 5 < full) load(r1, g + 5);
        f(r2, g + 2);
        if (g + 6 < full) load(r2, g + 6);
        f(r3, g + 3);
    }
    // up to three groups left, already in r0 / r1 / r2
    if (g < full) f(r0, g++);
    if (g < full) f(r1, g++);
    if (g < full) f(r2, g++);
    return g;
}

// groups of four units (j + 384 < M) of the lane starting at unit j
__device__ __forceinline__ int lane_groups(int M, int j) { return M - j - 3 * 128 > 0 ? (M - j - 3 * 128 + 511) / 512 : 0; }

// kPos: s_i = +1 (factors 1 - t tau), else s_i = -1 (1 + t tau), the sign
// in the FMA operand; the running products are renormalised by their
// exponent bits.
template <bool kSharedTau, bool kRing, bool kPos>
__device__ __forceinline__ Prod<float> lane_product4_signed(const float *__restrict__ t, const float *__restrict__ tau,
                                                            int lane, int M) {
    float m0 = 1.f, m1 = 1.f;
    int e = 0;
    int j = 4 * lane;
    // Large M: the ring of tau_ring4 (the products and renormalisations run
    // in the order of the plain loop below, so the result is the same).
    if (kRing && !kSharedTau && M >= 6 * 512) {
        const int j0 = j;
        j += 512 * tau_ring4(tau, j0, lane_groups(M, j0), [&](const float4 (&uv)[4], int g) {
            float4 tv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) tv[u] = *reinterpret_cast<const float4 *>(t + j0 + g * 512 + u * 128);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                m0 *= fmaf(kPos ? -tv[u].x : tv[u].x, uv[u].x, 1.f) * fmaf(kPos ? -tv[u].y : tv[u].y, uv[u].y, 1.f);
                m1 *= fmaf(kPos ? -tv[u].z : tv[u].z, uv[u].z, 1.f) * fmaf(kPos ? -tv[u].w : tv[u].w, uv[u].w, 1.f);
            }
            m0 = renorm_bits(m0, e);
            m1 = renorm_bits(m1, e);
        });
    }
    // groups of four 16-byte loads in flight (large M reads the tau row from L2),
    // renormalised after each group as before
    for (; j + 3 * 128 < M; j += 4 * 128) {
        float4 uv[4], tv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) uv[u] = load_tau4<kSharedTau>(tau + j + u * 128);
#pragma unroll
        for (int u = 0; u < 4; ++u) tv[u] = *reinterpret_cast<const float4 *>(t + j + u * 128);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            m0 *= fmaf(kPos ? -tv[u].x : tv[u].x, uv[u].x, 1.f) * fmaf(kPos ? -tv[u].y : tv[u].y, uv[u].y, 1.f);
            m1 *= fmaf(kPos ? -tv[u].z : tv[u].z, uv[u].z, 1.f) * fmaf(kPos ? -tv[u].w : tv[u].w, uv[u].w, 1.f);
        }
        m0 = renorm_bits(m0, e);
        m1 = renorm_bits(m1, e);
    }
    for (; j < M; j += 128) {
        const float4 tv = *reinterpret_cast<const float4 *>(t + j);
        const float4 uv = load_tau4<kSharedTau>(tau + j);
        m0 *= fmaf(kPos ? -tv.x : tv.x, uv.x, 1.f) * fmaf(kPos ? -tv.y : tv.y, uv.y, 1.f);
        m1 *= fmaf(kPos ? -tv.z : tv.z, uv.z, 1.f) * fmaf(kPos ? -tv.w : tv.w, uv.w, 1.f);
    }
    Prod<float> p{m0, e};
    renorm(p);
    p.m *= m1;
    renorm(p);
    return p;
}

template <bool kSharedTau = false, bool kRing = false>
__device__ __forceinline__ Prod<float> lane_product4(const float *__restrict__ t, const float *__restrict__ tau,
                                                     float si, int lane, int M) {
    return si > 0.f ? lane_product4_signed<kSharedTau, kRing, true>(t, tau, lane, M)
                    : lane_product4_signed<kSharedTau, kRing, false>(t, tau, lane, M);
}

template <bool kRing>
__device__ __forceinline__ Prod<double> unit_lanes_product(const double *t, const double *tau, double si, int lane,
                                                           int M, bool vec4) {
    return strided_product<double>(t, tau, 1, si, lane, 32, M);
}
template <bool kRing>
__device__ __forceinline__ Prod<float> unit_lanes_product(const float *t, const float *tau, float si, int lane, int M,
                                                          bool vec4) {
    return vec4 ? lane_product4<false, kRing>(t, tau, si, lane, M)
                : strided_product<float>(t, tau, 1, si, lane, 32, M);
}

// lane_product4 on a tau row already held in registers: uv[u] is the chunk j
// = 4 lane + 128 u (zero past M).  The groups, renormalisations and tail are
// those of lane_product4, in the same order, so the result is identical; only
// the loads are gone (the caller issues all of them at once, one L2 round
// trip per row instead of one per group of four).
template <int kC>
__device__ __forceinline__ Prod<float> lane_product4_regs(const float *__restrict__ t, const float4 (&uv)[kC],
                                                          float si, int lane, int M) {
    float m0 = 1.f, m1 = 1.f;
    int e = 0;
    int j = 4 * lane, G = 0;
#pragma unroll
    for (int g = 0; g < kC / 4; ++g) {
        if (j + 3 * 128 < M) {
            float4 tv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) tv[u] = *reinterpret_cast<const float4 *>(t + j + u * 128);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 w = uv[4 * g + u];
                m0 *= fmaf(-si * tv[u].x, w.x, 1.f) * fmaf(-si * tv[u].y, w.y, 1.f);
                m1 *= fmaf(-si * tv[u].z, w.z, 1.f) * fmaf(-si * tv[u].w, w.w, 1.f);
            }
            m0 = renorm_bits(m0, e);
            m1 = renorm_bits(m1, e);
            j += 4 * 128;
            ++G;
        }
    }
#pragma unroll
    for (int u = 0; u < kC; ++u) {
        if (u >= 4 * G && 4 * lane + 128 * u < M) {
            const float4 tv = *reinterpret_cast<const float4 *>(t + 4 * lane + 128 * u);
            const float4 w = uv[u];
            m0 *= fmaf(-si * tv.x, w.x, 1.f) * fmaf(-si * tv.y, w.y, 1.f);
            m1 *= fmaf(-si * tv.z, w.z, 1.f) * fmaf(-si * tv.w, w.w, 1.f);
        }
    }
    Prod<float> p{m0, e};
    renorm(p);
    p.m *= m1;
    renorm(p);
    return p;
}

// ------------------------------------------------------------------ sweep ---

// Edge e of the list joins two sites of [0, N) holding different spins, after
// the spins of sites i and k are flipped (i = k = -1: as they are).
__device__ __forceinline__ bool antiparallel(const int32_t *__restrict__ edges, int e, int N, const int8_t *sv,
                                             int i, int k) {
    const int a = edges[2 * e], b = edges[2 * e + 1];
    if ((unsigned)a >= (unsigned)N || (unsigned)b >= (unsigned)N) return false;
    const int sa = (a == i || a == k) ? -sv[a] : sv[a], sb = (b == i || b == k) ? -sv[b] : sv[b];
    return sa != sb;
}

// MetropolisHamiltonian proposal of a Heisenberg-type Hamiltonian (Sec. 3.4):
// the connected configurations are the swaps across the n(s) antiparallel
// edges; the proposal is the r-th of them in edge order, r = floor(hi n(s) /
// 2^32), and n(s') is counted on the swapped state.  Warp-uniform results;
// e_sel = -1 when n(s) = 0.
__device__ __forceinline__ void hamiltonian_pick(const int32_t *__restrict__ edges, int E, int N, const int8_t *sv,
                                                 unsigned hi, int lane, int &e_sel, int &ns, int &nsp) {
    ns = 0;
    nsp = 0;
    e_sel = -1;
    for (int e0 = 0; e0 < E; e0 += 32) {
        const int e = e0 + lane;
        ns += __popc(__ballot_sync(kFull, e < E && antiparallel(edges, e, N, sv, -1, -1)));
    }
    if (ns == 0) return;
    int r = (int)(((unsigned long long)hi * (unsigned long long)ns) >> 32);  // r < ns
    for (int e0 = 0; e0 < E; e0 += 32) {
        const int e = e0 + lane;
        const bool f = e < E && antiparallel(edges, e, N, sv, -1, -1);
        const unsigned m = __ballot_sync(kFull, f);
        const int cnt = __popc(m);
        if (r < cnt) {  // warp-uniform
            const bool hit = f && __popc(m & ((1u << lane) - 1u)) == r;
            e_sel = e0 + __ffs(__ballot_sync(kFull, hit)) - 1;
            break;
        }
        r -= cnt;
    }
    if (e_sel < 0) {
        ns = 0;
        return;
    }
    const int i = edges[2 * e_sel], k = edges[2 * e_sel + 1];
    for (int e0 = 0; e0 < E; e0 += 32) {
        const int e = e0 + lane;
        nsp += __popc(__ballot_sync(kFull, e < E && antiparallel(edges, e, N, sv, i, k)));
    }
}

template <typename R>
struct SweepK {
    Tables<R> t;
    SweepArgs a;
    int warp_bytes, t_bytes;
    bool vec4;  // FP32 with M % 4 == 0: 16-byte loads in the ratio products
};

// One warp per chain.  Hidden units are spread over the lanes (j = lane,
// lane + 32, ...); t = tanh theta and the spins live in shared memory.  The
// 32 lanes evaluate the Philox blocks of 32 consecutive proposals at once and
// broadcast them one per proposal.  kHam: the Hamiltonian rule, whose edge
// depends on the state (a separate instantiation keeps the registers of the
// local and exchange rules as they are).
// kRing: the FP32 form with the pipelined tau loads (M >= 3072), given the
// registers of 3 blocks of 4 warps per SM (what shared memory allows there);
// otherwise the registers of 7 blocks, for the small-M occupancy.
template <typename R, bool kHam, bool kRing>
__global__ void __launch_bounds__(128, kRing ? 3 : 7) k_sweep(SweepK<R> P) {
    extern __shared__ __align__(16) unsigned char sm[];
    const Tables<R> &T = P.t;
    const SweepArgs &A = P.a;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= A.C) return;
    const int N = T.N, M = T.M;
    R *t = reinterpret_cast<R *>(sm + (size_t)warp * P.warp_bytes);
    int8_t *sv = reinterpret_cast<int8_t *>(sm + (size_t)warp * P.warp_bytes + P.t_bytes);
    for (int i = lane; i < N; i += 32) sv[i] = A.s[(size_t)c * N + i];
    __syncwarp();
    unsigned long long acc = 0;
    const int n_sweeps = A.n_discard + A.n_samples;
    constexpr bool kF32 = sizeof(R) == 4;
    using Acc = R;  // precision of the accept arithmetic
    for (int w = 0; w < n_sweeps; ++w) {
        // From-scratch FP64 theta = b + W s (rebuilt here, or given by the
        // tensor-core product), t = tanh theta, ln psi.
        double lp = 0.0;
        for (int j = lane; j < M; j += 32) {
            double th;
            if (A.theta_in) {
                th = A.theta_in[(size_t)c * (A.theta_ld > 0 ? A.theta_ld : M) + j];
            } else {
                th = T.b[j];
                for (int i = 0; i < N; ++i) th = fma(T.Wt[(size_t)i * M + j], (double)sv[i], th);
            }
            if (kF32) {
                // FP32 path: t and the ln cosh terms in FP32 lanes (the FP64
                // pipe of this part runs at 1/64 of the FP32 rate)
                const float thf = (float)th;
                t[j] = (R)tanhf(thf);
                lp += (double)lncosh(thf);
            } else {
                t[j] = (R)tanh(th);
                lp += lncosh(th);
            }
        }
        for (int i = lane; i < N; i += 32) lp += T.a[i] * (double)sv[i];
        lp = warp_sum(lp);
        __syncwarp();
        const unsigned long long qbase = (unsigned long long)(A.sweep0 + w) * (unsigned long long)N;
        // Lane l prepares proposal q0 + l of each batch of 32: its Philox
        // block, ln u, the site / edge, K and the visible-bias difference, so
        // that a proposal only broadcasts them.
        // The FP32 path takes the accept decision in FP32 (ln u and the
        // ratio), the FP64 path in FP64.
        int b_i = 0, b_k = -1, b_row = 0, b_ok = 1;
        unsigned b_hi = 0;
        R b_K = R(0);
        Acc b_aa = Acc(0), b_lu = Acc(0);
        for (int q = 0; q < N; ++q) {
            if ((q & 31) == 0) {
                Philox4 y = philox4x64_10(qbase + (unsigned long long)(q + lane), (unsigned long long)c,
                                          (unsigned long long)A.stream_id, 0ULL, A.seed, 0ULL);
                if (kF32)
                    b_lu = (Acc)logf((float)uniform53(y.v[1]));
                else
                    b_lu = (Acc)log(uniform53(y.v[1]));
                if (A.rule == NK_RULE_LOCAL) {
                    b_i = pick_index(y.v[0], N);
                    b_k = -1;
                    b_row = b_i;
                    b_K = T.K_site[b_i];
                    b_aa = (Acc)T.a[b_i];
                } else if (kHam) {
                    b_hi = (unsigned)(y.v[0] >> 32);  // the edge depends on the state
                } else {
                    const int e = pick_index(y.v[0], T.E);
                    const int i0 = A.edges[2 * e], k0 = A.edges[2 * e + 1];
                    // an edge outside [0, N) is never a move (bounds guard)
                    b_ok = (unsigned)i0 < (unsigned)N && (unsigned)k0 < (unsigned)N;
                    b_i = b_ok ? i0 : 0;
                    b_k = b_ok ? k0 : 0;
                    b_row = e;
                    b_K = T.K_edge[e];
                    b_aa = b_ok ? (Acc)(T.a[b_i] - T.a[b_k]) : Acc(0);
                }
            }
            const int src = q & 31;
            int i = __shfl_sync(kFull, b_i, src), k = __shfl_sync(kFull, b_k, src);
            int row = __shfl_sync(kFull, b_row, src);
            R K = __shfl_sync(kFull, b_K, src);
            Acc aa = __shfl_sync(kFull, b_aa, src);
            const Acc lu = __shfl_sync(kFull, b_lu, src);
            const size_t slot = ((size_t)c * A.dec_stride + A.dec_offset + w) * N + q;
            const R *tau;
            Acc corr = Acc(0);  // ln g(s|s') - ln g(s'|s)
            if (A.rule == NK_RULE_LOCAL) {
                tau = T.tau_site + (size_t)row * M;
            } else if (kHam) {
                int e, ns, nsp;
                hamiltonian_pick(A.edges, T.E, N, sv, __shfl_sync(kFull, b_hi, src), lane, e, ns, nsp);
                if (e < 0) {
                    if (lane == 0 && A.decisions) A.decisions[slot] = 2;
                    continue;
                }
                i = A.edges[2 * e];
                k = A.edges[2 * e + 1];
                row = e;
                K = T.K_edge[e];
                aa = (Acc)(T.a[i] - T.a[k]);
                if (kF32)
                    corr = (Acc)(logf((float)ns) - logf((float)nsp));
                else
                    corr = (Acc)(log((double)ns) - log((double)nsp));
                tau = T.tau_edge + (size_t)row * M;
            } else {
                if (!__shfl_sync(kFull, b_ok, src) || sv[i] == sv[k]) {
                    if (lane == 0 && A.decisions) A.decisions[slot] = 2;
                    continue;
                }
                tau = T.tau_edge + (size_t)row * M;
            }
            const Acc d0 = Acc(-2) * aa * (Acc)sv[i];
            const R si = (R)sv[i];
            Prod<R> pr = unit_lanes_product<kRing>(t, tau, si, lane, M, P.vec4);
            pr = warp_prod_normalised(pr);
            const Acc delta = d0 + (Acc)(K + prod_log(pr));
            const bool accept = lu < Acc(2) * delta + corr;
            if (lane == 0 && A.decisions) A.decisions[slot] = accept ? 1 : 0;
            if (accept) {
                if (kF32 && P.vec4) {
                    // FP32 path: 16-byte accesses, fast division (t is rebuilt
                    // exactly from theta after every sweep)
                    float *tf = reinterpret_cast<float *>(t);
                    const float *uf = reinterpret_cast<const float *>(tau);
                    const float sf = (float)si;
                    auto upd = [&](float4 tv, const float4 &uv, int j) {
                        const float v0 = sf * uv.x, v1 = sf * uv.y, v2 = sf * uv.z, v3 = sf * uv.w;
                        tv.x = __fdividef(tv.x - v0, fmaf(-tv.x, v0, 1.f));
                        tv.y = __fdividef(tv.y - v1, fmaf(-tv.y, v1, 1.f));
                        tv.z = __fdividef(tv.z - v2, fmaf(-tv.z, v2, 1.f));
                        tv.w = __fdividef(tv.w - v3, fmaf(-tv.w, v3, 1.f));
                        *reinterpret_cast<float4 *>(tf + j) = tv;
                    };
                    // the row again in groups of four 16-byte loads (one round
                    // trip per group where it has left L1)
                    int j = 4 * lane;
                    for (; j + 3 * 128 < M; j += 4 * 128) {
                        float4 uv[4], tv[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) uv[u] = __ldg(reinterpret_cast<const float4 *>(uf + j + u * 128));
#pragma unroll
                        for (int u = 0; u < 4; ++u) tv[u] = *reinterpret_cast<const float4 *>(tf + j + u * 128);
#pragma unroll
                        for (int u = 0; u < 4; ++u) upd(tv[u], uv[u], j + u * 128);
                    }
                    for (; j < M; j += 128)
                        upd(*reinterpret_cast<const float4 *>(tf + j), __ldg(reinterpret_cast<const float4 *>(uf + j)), j);
                } else {
                    for (int j = lane; j < M; j += 32) {
                        const R tj = t[j], tv = si * tau[j];
                        t[j] = (tj - tv) / (R(1) - tj * tv);
                    }
                }
                __syncwarp();
                if (lane == 0) {
                    sv[i] = (int8_t)-sv[i];
                    if (k >= 0) sv[k] = (int8_t)-sv[k];
                }
                lp += (double)delta;
                ++acc;
            }
            __syncwarp();
        }
        if (w >= A.n_discard) {
            const size_t row = (size_t)c * A.out_stride + A.out_offset + (w - A.n_discard);
            for (int i = lane; i < N; i += 32) A.samples[row * N + i] = sv[i];
            if (lane == 0 && A.logpsi) A.logpsi[row] = lp;
        }
        __syncwarp();
    }
    for (int i = lane; i < N; i += 32) A.s[(size_t)c * N + i] = sv[i];
    if (lane == 0 && A.n_accepted) A.n_accepted[c] += acc;
}

// FP32 sweeps of the local and exchange rules with the flip-ratio row of a
// proposal held in registers: every lane issues the loads of all its kC
// chunks of the row at once, so a proposal waits for one L2 round trip
// (k_sweep<float, false> waits for one per group of four chunks: nine at M =
// 4608).  The accepted move's update of t reuses the registers.  The
// arithmetic and the order of every product are those of
// k_sweep<float, false>, so the decisions are identical.  Needs M % 4 == 0 and
// M <= 128 kC.
template <int kC>
__global__ void __launch_bounds__(128) k_sweep_rows(SweepK<float> P) {
    extern __shared__ __align__(16) unsigned char sm[];
    const Tables<float> &T = P.t;
    const SweepArgs &A = P.a;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int c = blockIdx.x * (blockDim.x >> 5) + warp;
    if (c >= A.C) return;
    const int N = T.N, M = T.M;
    unsigned char *base = sm + (size_t)warp * P.warp_bytes;
    float *t = reinterpret_cast<float *>(base);
    int8_t *sv = reinterpret_cast<int8_t *>(base + P.t_bytes);
    const bool local = A.rule == NK_RULE_LOCAL;
    const float *tab = local ? T.tau_site : T.tau_edge;
    for (int i = lane; i < N; i += 32) sv[i] = A.s[(size_t)c * N + i];
    __syncwarp();
    unsigned long long acc = 0;
    const int n_sweeps = A.n_discard + A.n_samples;
    for (int w = 0; w < n_sweeps; ++w) {
        double lp = 0.0;
        for (int j = lane; j < M; j += 32) {
            double th;
            if (A.theta_in) {
                th = A.theta_in[(size_t)c * (A.theta_ld > 0 ? A.theta_ld : M) + j];
            } else {
                th = T.b[j];
                for (int i = 0; i < N; ++i) th = fma(T.Wt[(size_t)i * M + j], (double)sv[i], th);
            }
            const float thf = (float)th;
            t[j] = tanhf(thf);
            lp += (double)lncosh(thf);
        }
        for (int i = lane; i < N; i += 32) lp += T.a[i] * (double)sv[i];
        lp = warp_sum(lp);
        __syncwarp();
        const unsigned long long qbase = (unsigned long long)(A.sweep0 + w) * (unsigned long long)N;
        int b_i = 0, b_k = -1, b_row = 0, b_ok = 1;
        float b_K = 0.f, b_aa = 0.f, b_lu = 0.f;
        for (int q = 0; q < N; ++q) {
            const int src = q & 31;
            if (src == 0) {
                Philox4 y = philox4x64_10(qbase + (unsigned long long)(q + lane), (unsigned long long)c,
                                          (unsigned long long)A.stream_id, 0ULL, A.seed, 0ULL);
                b_lu = logf((float)uniform53(y.v[1]));
                if (local) {
                    b_i = pick_index(y.v[0], N);
                    b_k = -1;
                    b_row = b_i;
                    b_K = T.K_site[b_i];
                    b_aa = (float)T.a[b_i];
                } else {
                    const int e = pick_index(y.v[0], T.E);
                    const int i0 = A.edges[2 * e], k0 = A.edges[2 * e + 1];
                    // an edge outside [0, N) is never a move (bounds guard)
                    b_ok = (unsigned)i0 < (unsigned)N && (unsigned)k0 < (unsigned)N;
                    b_i = b_ok ? i0 : 0;
                    b_k = b_ok ? k0 : 0;
                    b_row = e;
                    b_K = T.K_edge[e];
                    b_aa = b_ok ? (float)(T.a[b_i] - T.a[b_k]) : 0.f;
                }
            }
            const int i = __shfl_sync(kFull, b_i, src), k = __shfl_sync(kFull, b_k, src);
            const int row = __shfl_sync(kFull, b_row, src);
            const float K = __shfl_sync(kFull, b_K, src), aa = __shfl_sync(kFull, b_aa, src);
            const float lu = __shfl_sync(kFull, b_lu, src);
            const int ok = __shfl_sync(kFull, b_ok, src);
            const size_t slot = ((size_t)c * A.dec_stride + A.dec_offset + w) * N + q;
            if (!local && (!ok || sv[i] == sv[k])) {
                if (lane == 0 && A.decisions) A.decisions[slot] = 2;
                continue;
            }
            const float d0 = -2.f * aa * (float)sv[i];
            const float si = (float)sv[i];
            float4 uv[kC];
            const float *row_p = tab + (size_t)row * M;
#pragma unroll
            for (int u = 0; u < kC; ++u) {
                const int j = 4 * lane + 128 * u;
                uv[u] = j < M ? __ldg(reinterpret_cast<const float4 *>(row_p + j)) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            Prod<float> pr = lane_product4_regs<kC>(t, uv, si, lane, M);
            pr = warp_prod_normalised(pr);
            const float delta = d0 + (K + prod_log(pr));
            const bool accept = lu < 2.f * delta;
            if (lane == 0 && A.decisions) A.decisions[slot] = accept ? 1 : 0;
            if (accept) {
#pragma unroll
                for (int u = 0; u < kC; ++u) {
                    const int j = 4 * lane + 128 * u;
                    if (j >= M) continue;
                    float4 tv = *reinterpret_cast<const float4 *>(t + j);
                    const float v0 = si * uv[u].x, v1 = si * uv[u].y, v2 = si * uv[u].z, v3 = si * uv[u].w;
                    tv.x = __fdividef(tv.x - v0, fmaf(-tv.x, v0, 1.f));
                    tv.y = __fdividef(tv.y - v1, fmaf(-tv.y, v1, 1.f));
                    tv.z = __fdividef(tv.z - v2, fmaf(-tv.z, v2, 1.f));
                    tv.w = __fdividef(tv.w - v3, fmaf(-tv.w, v3, 1.f));
                    *reinterpret_cast<float4 *>(t + j) = tv;
                }
                __syncwarp();
                if (lane == 0) {
                    sv[i] = (int8_t)-sv[i];
                    if (k >= 0) sv[k] = (int8_t)-sv[k];
                }
                lp += (double)delta;
                ++acc;
            }
            __syncwarp();
        }
        if (w >= A.n_discard) {
            const size_t row = (size_t)c * A.out_stride + A.out_offset + (w - A.n_discard);
            for (int i = lane; i < N; i += 32) A.samples[row * N + i] = sv[i];
            if (lane == 0 && A.logpsi) A.logpsi[row] = lp;
        }
        __syncwarp();
    }
    for (int i = lane; i < N; i += 32) A.s[(size_t)c * N + i] = sv[i];
    if (lane == 0 && A.n_accepted) A.n_accepted[c] += acc;
}

// ----------------------------------------------------------- local energy ---

template <typename R>
struct ElocK {
    Tables<R> t;
    ElocArgs a;
    int warp_bytes, t_bytes, s_bytes;
    int units;  // 1: lanes over hidden units (large M), 0: lanes over connections
};

// Hidden-unit count from which the local energy spreads the units over the
// lanes (one warp reduction per connection) instead of the connections.
constexpr int kUnitsMappingM = 1024;

// One warp per sample.  theta and t are rebuilt from s; the connected
// configurations are spread over the lanes (sites for the Ising field term,
// antiparallel edges for the Heisenberg exchange term), each lane running
// over all hidden units with the unit-major tables.
template <typename R>
__global__ void __launch_bounds__(128) k_eloc(ElocK<R> P) {
    extern __shared__ __align__(16) unsigned char sm[];
    const Tables<R> &T = P.t;
    const ElocArgs &A = P.a;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (k >= A.Ns) return;
    const int N = T.N, M = T.M, E = T.E;
    unsigned char *base = sm + (size_t)warp * P.warp_bytes;
    R *t = reinterpret_cast<R *>(base);
    int8_t *sv = reinterpret_cast<int8_t *>(base + P.t_bytes);
    int *list = reinterpret_cast<int *>(base + P.t_bytes + P.s_bytes);
    for (int i = lane; i < N; i += 32) sv[i] = A.s[(size_t)k * N + i];
    __syncwarp();
    for (int j = lane; j < M; j += 32) {
        double th;
        if (A.theta_in) {
            th = A.theta_in[(size_t)k * M + j];
        } else {
            th = T.b[j];
            for (int i = 0; i < N; ++i) th = fma(T.Wt[(size_t)i * M + j], (double)sv[i], th);
        }
        const double tj = tanh(th);
        t[j] = (R)tj;
        if (A.t_out) A.t_out[(size_t)k * M + j] = tj;
    }
    // edges [0, E1) couple with J, the next-nearest ones [E1, E) with J2
    const int E1 = E - A.E2;
    double diag = 0.0;
    for (int e = lane; e < E; e += 32) {
        const int i = T.edges[2 * e], kk = T.edges[2 * e + 1];
        if ((unsigned)i < (unsigned)N && (unsigned)kk < (unsigned)N)
            diag += (e < E1 ? A.J : A.J2) * (double)sv[i] * (double)sv[kk];
    }
    __syncwarp();
    double off = 0.0;
    if (A.kind == NK_TFIM && P.units) {
        // large M: lanes over hidden units, one warp reduction per site
        for (int i = 0; i < N; ++i) {
            const R si = (R)sv[i];
            Prod<R> pr = strided_product<R>(t, T.tau_site + (size_t)i * M, 1, si, lane, 32, M);
            pr = warp_prod(pr);
            const double delta = -2.0 * T.a[i] * (double)si + (double)(T.K_site[i] + prod_log(pr));
            if (lane == 0) off += -A.h * exp(delta);
        }
    } else if (A.kind == NK_TFIM) {
        // small M: lanes over sites, each over all hidden units
        for (int i = lane; i < N; i += 32) {
            const R si = (R)sv[i];
            Prod<R> pr = strided_product<R>(t, T.tau_siteT + i, (size_t)N, si, 0, 1, M);
            const double delta = -2.0 * T.a[i] * (double)si + (double)(T.K_site[i] + prod_log(pr));
            off += -A.h * exp(delta);
        }
    } else {
        // compact the antiparallel edges
        int n = 0;
        for (int e0 = 0; e0 < E; e0 += 32) {
            const int e = e0 + lane;
            bool f = false;
            if (e < E) {
                const int i = T.edges[2 * e], kk = T.edges[2 * e + 1];
                f = (unsigned)i < (unsigned)N && (unsigned)kk < (unsigned)N && sv[i] != sv[kk];
            }
            const unsigned mask = __ballot_sync(kFull, f);
            if (f) list[n + __popc(mask & ((1u << lane) - 1u))] = e;
            n += __popc(mask);
        }
        __syncwarp();
        // off-diagonal elements; the Marshall sign flips only the edges that
        // join the two sublattices (the nearest-neighbour class)
        const double hoff = A.marshall ? -2.0 * A.J : 2.0 * A.J, hoff2 = 2.0 * A.J2;
        if (P.units) {
            for (int idx = 0; idx < n; ++idx) {
                const int e = list[idx];
                const int i = T.edges[2 * e], kk = T.edges[2 * e + 1];
                const R si = (R)sv[i];
                Prod<R> pr = strided_product<R>(t, T.tau_edge + (size_t)e * M, 1, si, lane, 32, M);
                pr = warp_prod(pr);
                const double delta =
                    -2.0 * (double)si * (T.a[i] - T.a[kk]) + (double)(T.K_edge[e] + prod_log(pr));
                if (lane == 0) off += (e < E1 ? hoff : hoff2) * exp(delta);
            }
        } else {
            for (int idx = lane; idx < n; idx += 32) {
                const int e = list[idx];
                const int i = T.edges[2 * e], kk = T.edges[2 * e + 1];
                const R si = (R)sv[i];
                Prod<R> pr = strided_product<R>(t, T.tau_edgeT + e, (size_t)E, si, 0, 1, M);
                const double delta =
                    -2.0 * (double)si * (T.a[i] - T.a[kk]) + (double)(T.K_edge[e] + prod_log(pr));
                off += (e < E1 ? hoff : hoff2) * exp(delta);
            }
        }
    }
    const double tot = warp_sum(diag + off);
    if (lane == 0) A.eloc[k] = tot;
}

// ------------------------------------------- sample-batched local energy ---
// Large M (NK_MIXED, theta given): one CTA of eloc_warps(kU) warps holds
// tanh(theta) of kEG samples in shared memory; every warp takes connections
// (sites, or edges) in turn, loads each tau row once (16-byte loads, lanes
// over units) and applies it to all kEG samples, so the tau traffic per ratio
// term drops kEG-fold.  One warp reduction per (connection, sample).
constexpr int kEG = 8;
// Warps per CTA.  At M >= 4096 the t of kEG samples (147 KB at M = 4608)
// leaves room for one CTA per SM, and the kernel waits on shared-memory and
// fixed latencies: 32 warps instead of 16 took the 24 x 24 local energies
// from 62.1 to 52.1 ms a step.
__host__ __device__ constexpr int eloc_warps(int kU) { return kU == 4 ? 32 : 16; }

struct ElocBK {
    Tables<float> t;
    ElocArgs a;
    int t_ld, s_ld;
};

// kU tau loads in flight per lane: 4 where M is large enough that the
// shared-memory t of kEG samples allows one CTA per SM anyway (M >= 4096),
// else 1 (the extra registers of 4 would halve the resident CTAs).
template <int kU>
__global__ void __launch_bounds__(eloc_warps(kU) * 32) k_eloc_batched(ElocBK P) {
    constexpr int kEW = eloc_warps(kU);
    extern __shared__ __align__(16) unsigned char sm[];
    const Tables<float> &T = P.t;
    const ElocArgs &A = P.a;
    const int N = T.N, M = T.M, E = T.E, E1 = E - A.E2;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t k0 = (int64_t)blockIdx.x * kEG;
    const int G = (int)(A.Ns - k0 < kEG ? A.Ns - k0 : kEG);
    float *t = reinterpret_cast<float *>(sm);                                    // [kEG][t_ld]
    int8_t *sv = reinterpret_cast<int8_t *>(sm + (size_t)kEG * P.t_ld * 4);      // [kEG][s_ld]
    double *part = reinterpret_cast<double *>(sm + (size_t)kEG * P.t_ld * 4 + (size_t)kEG * P.s_ld);  // [kEW][kEG]
    double *diag = part + kEW * kEG;                                              // [kEG]
    float *offw = reinterpret_cast<float *>(diag + kEG);                          // [kEW][kEG]
    for (int x = threadIdx.x; x < kEG * N; x += blockDim.x) {
        const int g = x / N, i = x % N;
        sv[g * P.s_ld + i] = g < G ? A.s[(size_t)(k0 + g) * N + i] : (int8_t)1;
    }
    for (int x = threadIdx.x; x < kEG * M; x += blockDim.x) {
        const int g = x / M, j = x % M;
        float tv = 0.f;
        if (g < G) {
            const double tj = tanh(A.theta_in[(size_t)(k0 + g) * M + j]);
            tv = (float)tj;
            if (A.t_out) A.t_out[(size_t)(k0 + g) * M + j] = tj;
        }
        t[g * P.t_ld + j] = tv;
    }
    __syncthreads();
    // diagonal part: warp g sums J_e s_i s_k over the edges of sample g
    if (warp < G) {
        double d = 0.0;
        const int8_t *s = sv + warp * P.s_ld;
        for (int e = lane; e < E; e += 32) {
            const int i = T.edges[2 * e], kk = T.edges[2 * e + 1];
            if ((unsigned)i < (unsigned)N && (unsigned)kk < (unsigned)N)
                d += (e < E1 ? A.J : A.J2) * (double)s[i] * (double)s[kk];
        }
        d = warp_sum(d);
        if (lane == 0) diag[warp] = d;
    }
    // FP32 path: ratios, exponentials and the per-warp partial sums in FP32
    // lanes (each warp adds about nconn / kEW terms); the diagonal part and
    // the final sum stay in FP64.
    if (lane < kEG) offw[warp * kEG + lane] = 0.f;
    __syncwarp();
    const bool tfim = A.kind == NK_TFIM;
    const int nconn = tfim ? N : E;
    const float hoff = (float)(A.marshall ? -2.0 * A.J : 2.0 * A.J), hoff2 = (float)(2.0 * A.J2),
                hfield = (float)(-A.h);
    for (int c = warp; c < nconn; c += kEW) {
        int i, kk = -1;
        const float *tau;
        float K, aa;
        if (tfim) {
            i = c;
            tau = T.tau_site + (size_t)c * M;
            K = T.K_site[c];
            aa = (float)T.a[i];
        } else {
            i = T.edges[2 * c];
            kk = T.edges[2 * c + 1];
            if ((unsigned)i >= (unsigned)N || (unsigned)kk >= (unsigned)N) continue;
            tau = T.tau_edge + (size_t)c * M;
            K = T.K_edge[c];
            aa = (float)(T.a[i] - T.a[kk]);
        }
        unsigned active = 0;
#pragma unroll
        for (int g = 0; g < kEG; ++g)
            if (g < G && (tfim || sv[g * P.s_ld + i] != sv[g * P.s_ld + kk])) active |= 1u << g;
        if (!active) continue;
        // The active samples of this connection as slots 0 .. cnt - 1 (in
        // increasing sample order, so every product is formed as before):
        // the loops below stop at cnt, so inactive samples cost nothing.
        const int cnt = __popc(active);
        float m[kEG];
        int ex[kEG];
        float sg[kEG];
        const float *tg[kEG];
        int gs[kEG];
        unsigned rest = active;
#pragma unroll
        for (int q = 0; q < kEG; ++q) {
            const int g = rest ? __ffs(rest) - 1 : 0;
            rest &= rest - 1u;
            gs[q] = g;
            m[q] = 1.f;
            ex[q] = 0;
            sg[q] = (float)sv[g * P.s_ld + i];
            tg[q] = t + (size_t)g * P.t_ld;
        }
        // This lane's units j = 4 lane + 128 it, it = j >> 7: the tau loads
        // of kU iterations are issued together (the row comes from L2), and
        // the products are renormalised after every odd iteration.
        for (int j0 = 4 * lane; j0 < M; j0 += kU * 128) {
            float4 uv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                uv[u] = j0 + u * 128 < M ? __ldg(reinterpret_cast<const float4 *>(tau + j0 + u * 128))
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int j = j0 + u * 128;
                if (j >= M) break;
#pragma unroll
                for (int q = 0; q < kEG; ++q) {
                    if (q >= cnt) break;
                    const float4 tv = *reinterpret_cast<const float4 *>(tg[q] + j);
                    const float ns = -sg[q];
                    m[q] *= fmaf(ns * tv.x, uv[u].x, 1.f) * fmaf(ns * tv.y, uv[u].y, 1.f) *
                            fmaf(ns * tv.z, uv[u].z, 1.f) * fmaf(ns * tv.w, uv[u].w, 1.f);
                }
                if ((j >> 7) & 1) {
#pragma unroll
                    for (int q = 0; q < kEG; ++q) {
                        if (q >= cnt) break;
                        m[q] = renorm_bits(m[q], ex[q]);
                    }
                }
            }
        }
#pragma unroll
        for (int q = 0; q < kEG; ++q) {
            if (q >= cnt) break;
            Prod<float> p{m[q], ex[q]};
            renorm(p);
            p = warp_prod_normalised(p);
            const float delta = -2.f * aa * sg[q] + (K + prod_log(p));
            if (lane == 0) {
                float &o = offw[warp * kEG + gs[q]];
                o = fmaf(tfim ? hfield : (c < E1 ? hoff : hoff2), expf(delta), o);
            }
        }
    }
    __syncwarp();
    if (lane == 0) {
#pragma unroll
        for (int g = 0; g < kEG; ++g) part[warp * kEG + g] = (double)offw[warp * kEG + g];
    }
    __syncthreads();
    if (threadIdx.x < G) {
        double tot = diag[threadIdx.x];
        for (int w = 0; w < kEW; ++w) tot += part[w * kEG + threadIdx.x];
        A.eloc[k0 + threadIdx.x] = tot;
    }
}

// --------------------------------------------------------- batched theta ---

// T[k][j] = tanh(b_j + sum_i W_ji s_ki): 64 x 64 output tile per block,
// 256 threads with 4 x 4 outputs each, FP64 FMA.
__global__ void __launch_bounds__(256) k_theta_tanh(int N, int M, const double *__restrict__ b,
                                                    const double *__restrict__ W,
                                                    const int8_t *__restrict__ s, int64_t B,
                                                    double *__restrict__ T) {
    __shared__ double Sa[16][64 + 1];
    __shared__ double Wb[16][64 + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t k0 = (int64_t)blockIdx.y * 64;
    const int j0 = blockIdx.x * 64;
    double acc[4][4] = {};
    for (int i0 = 0; i0 < N; i0 += 16) {
        for (int e = threadIdx.x; e < 16 * 64; e += 256) {
            const int ii = e & 15, rr = e >> 4;
            const int64_t kk = k0 + rr;
            const int jj = j0 + rr, ic = i0 + ii;
            Sa[ii][rr] = (kk < B && ic < N) ? (double)s[(size_t)kk * N + ic] : 0.0;
            Wb[ii][rr] = (jj < M && ic < N) ? W[(size_t)jj * N + ic] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int ii = 0; ii < 16; ++ii) {
            double av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                av[u] = Sa[ii][ty * 4 + u];
                bv[u] = Wb[ii][tx * 4 + u];
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
        const int64_t kk = k0 + ty * 4 + u;
        if (kk >= B) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int jj = j0 + tx * 4 + v;
            if (jj < M) T[(size_t)kk * M + jj] = tanh(acc[u][v] + b[jj]);
        }
    }
}

template <typename R>
static int align16(int x) {
    return (x + 15) & ~15;
}

}  // namespace

// ------------------------------------------------------------- launchers ---

template <typename R>
cudaError_t launch_tables(const Tables<R> &t, bool need_site, bool need_edge, cudaStream_t st) {
    dim3 tb(32, 8), tg((t.N + 31) / 32, (t.M + 31) / 32);
    (k_transpose_W<<<tg, tb, 0, st>>>(t.N, t.M, t.W, t.Wt), nk::note_launch());
    if (need_site)
        (k_tau_rows<R><<<t.N, 256, 0, st>>>(t.N, t.M, t.N, t.Wt, nullptr, t.tau_site, t.tau_siteT,
                                           t.K_site), nk::note_launch());
    if (need_edge && t.E > 0)
        (k_tau_rows<R><<<t.E, 256, 0, st>>>(t.N, t.M, t.E, t.Wt, t.edges, t.tau_edge, t.tau_edgeT,
                                           t.K_edge), nk::note_launch());
    return cudaGetLastError();
}

template cudaError_t launch_tables<double>(const Tables<double> &, bool, bool, cudaStream_t);
template cudaError_t launch_tables<float>(const Tables<float> &, bool, bool, cudaStream_t);

cudaError_t launch_logpsi(int N, int M, const double *a, const double *b, const double *Wt,
                          const int8_t *s, int64_t B, double *out, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const int wpb = 4;
    size_t smem = (size_t)wpb * ((N + 15) & ~15);
    unsigned grid = (unsigned)((B + wpb - 1) / wpb);
    (k_logpsi<<<grid, 32 * wpb, smem, st>>>(N, M, a, b, Wt, s, B, out), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_logpsi_theta(int N, int M, const double *a, const double *theta, const int8_t *s, int64_t B,
                                double *out, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    (k_logpsi_theta<<<(unsigned)((B + 7) / 8), 256, 0, st>>>(N, M, a, theta, s, B, out), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_tanh_inplace(int64_t n, double *x, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    (k_tanh_inplace<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, x), nk::note_launch());
    return cudaGetLastError();
}

cudaError_t launch_chain_init(int N, int C, int rule, uint64_t seed, uint32_t stream_id,
                              int8_t *s, cudaStream_t st) {
    if (C <= 0) return cudaSuccess;
    (k_chain_init<<<(C + 127) / 128, 128, 0, st>>>(N, C, rule, seed, stream_id, s), nk::note_launch());
    return cudaGetLastError();
}

// The register-row sweep for kC chunks of 128 floats per lane.
template <int kC>
cudaError_t launch_sweep_rows_kc(const SweepK<float> &P, cudaStream_t st) {
    int wpb = 4;
    while (wpb > 1 && (size_t)wpb * P.warp_bytes > 200 * 1024) wpb >>= 1;
    const size_t smem = (size_t)wpb * P.warp_bytes;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t err = nk::allow_max_dynamic_smem((const void *)k_sweep_rows<kC>);
    if (err != cudaSuccess) return err;
    const unsigned grid = (unsigned)((P.a.C + wpb - 1) / wpb);
    const int slot = prof_begin(NK_PROF_SWEEP, st);
    (k_sweep_rows<kC><<<grid, 32 * wpb, smem, st>>>(P), nk::note_launch());
    prof_end(slot, st, (double)P.a.C * (P.a.n_discard + P.a.n_samples) * P.t.N * (double)P.t.M);
    return cudaGetLastError();
}

// FP32 local and exchange rules with M % 4 == 0 and M <= 512: the
// register-row kernel (4 chunks a lane, 72 registers, the occupancy of
// k_sweep).  Measured on GB300: 0.62 against 0.71 ms a step at M = 200; at
// M = 1600 (16 chunks, 161 registers) and M = 4608 (36 chunks, 254
// registers) the larger register footprint made it slower than k_sweep
// (10.9 against 8.4 ms, 140 against 125 ms), so those sizes keep k_sweep.
cudaError_t launch_sweep_rows(const SweepK<float> &P, cudaStream_t st) { return launch_sweep_rows_kc<4>(P, st); }

template <typename R>
cudaError_t launch_sweep(const Tables<R> &t, const SweepArgs &a, cudaStream_t st) {
    if (a.C <= 0 || a.n_discard + a.n_samples <= 0) return cudaSuccess;
    SweepK<R> P;
    P.t = t;
    P.a = a;
    if (P.a.out_stride <= 0) {
        P.a.out_stride = a.n_samples;
        P.a.out_offset = 0;
    }
    if (P.a.dec_stride <= 0) {
        P.a.dec_stride = a.n_discard + a.n_samples;
        P.a.dec_offset = 0;
    }
    P.t_bytes = align16<R>(t.M * (int)sizeof(R));
    P.warp_bytes = P.t_bytes + align16<R>(t.N);
    P.vec4 = sizeof(R) == 4 && (t.M % 4) == 0;
    // FP32 local and exchange rules: the prefetching kernel, when two more
    // rows per warp fit in shared memory
    if constexpr (sizeof(R) == 4) {
        if (P.vec4 && a.rule != NK_RULE_HAMILTONIAN && t.M <= 4 * 128) return launch_sweep_rows(P, st);
    }
    int wpb = 4;
    while (wpb > 1 && (size_t)wpb * P.warp_bytes > 200 * 1024) wpb >>= 1;
    size_t smem = (size_t)wpb * P.warp_bytes;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const bool ham = a.rule == NK_RULE_HAMILTONIAN;
    const bool ring = sizeof(R) == 4 && P.vec4 && t.M >= 6 * 512;
    const void *fn = ham ? (ring ? (const void *)k_sweep<R, true, true> : (const void *)k_sweep<R, true, false>)
                         : (ring ? (const void *)k_sweep<R, false, true> : (const void *)k_sweep<R, false, false>);
    cudaError_t err = nk::allow_max_dynamic_smem(fn);
    if (err != cudaSuccess) return err;
    unsigned grid = (unsigned)((a.C + wpb - 1) / wpb);
    const int slot = prof_begin(NK_PROF_SWEEP, st);
    if (ham && ring)
        (k_sweep<R, true, true><<<grid, 32 * wpb, smem, st>>>(P), nk::note_launch());
    else if (ham)
        (k_sweep<R, true, false><<<grid, 32 * wpb, smem, st>>>(P), nk::note_launch());
    else if (ring)
        (k_sweep<R, false, true><<<grid, 32 * wpb, smem, st>>>(P), nk::note_launch());
    else
        (k_sweep<R, false, false><<<grid, 32 * wpb, smem, st>>>(P), nk::note_launch());
    prof_end(slot, st, (double)a.C * (a.n_discard + a.n_samples) * t.N * (double)t.M);
    return cudaGetLastError();
}

template cudaError_t launch_sweep<double>(const Tables<double> &, const SweepArgs &, cudaStream_t);
template cudaError_t launch_sweep<float>(const Tables<float> &, const SweepArgs &, cudaStream_t);

size_t eloc_batched_smem(int N, int M, int warps) {
    const size_t t_ld = (size_t)(M + 3) / 4 * 4, s_ld = (size_t)(N + 15) / 16 * 16;
    return (size_t)kEG * t_ld * 4 + (size_t)kEG * s_ld + (size_t)(warps * kEG + kEG) * 8 + (size_t)warps * kEG * 4;
}

template <typename R>
cudaError_t launch_eloc_batched(const Tables<R> &, const ElocArgs &, cudaStream_t) {
    return cudaErrorNotSupported;
}

template <>
cudaError_t launch_eloc_batched<float>(const Tables<float> &t, const ElocArgs &a, cudaStream_t st) {
    ElocBK P;
    P.t = t;
    P.a = a;
    P.t_ld = (t.M + 3) / 4 * 4;
    P.s_ld = (t.N + 15) / 16 * 16;
    const bool wide = t.M >= 4096;
    const int warps = wide ? eloc_warps(4) : eloc_warps(1);
    const size_t smem = eloc_batched_smem(t.N, t.M, warps);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const void *fn = wide ? (const void *)k_eloc_batched<4> : (const void *)k_eloc_batched<1>;
    cudaError_t err = nk::allow_max_dynamic_smem(fn);
    if (err != cudaSuccess) return err;
    const unsigned grid = (unsigned)((a.Ns + kEG - 1) / kEG);
    const int slot = prof_begin(NK_PROF_ELOC, st);
    if (wide)
        (k_eloc_batched<4><<<grid, warps * 32, smem, st>>>(P), nk::note_launch());
    else
        (k_eloc_batched<1><<<grid, warps * 32, smem, st>>>(P), nk::note_launch());
    const double conn = a.kind == NK_TFIM ? (double)t.N : 0.5 * (double)t.E;
    prof_end(slot, st, (double)a.Ns * conn * (double)t.M);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_eloc(const Tables<R> &t, const ElocArgs &a, cudaStream_t st) {
    if (a.Ns <= 0) return cudaSuccess;
    if (sizeof(R) == 4 && a.theta_in && t.M >= kUnitsMappingM && (t.M % 4) == 0 &&
        eloc_batched_smem(t.N, t.M, t.M >= 4096 ? eloc_warps(4) : eloc_warps(1)) <= 227 * 1024)
        return launch_eloc_batched<R>(t, a, st);
    ElocK<R> P;
    P.t = t;
    P.a = a;
    P.units = t.M >= kUnitsMappingM ? 1 : 0;
    P.t_bytes = align16<R>(t.M * (int)sizeof(R));
    P.s_bytes = align16<R>(t.N);
    P.warp_bytes = P.t_bytes + P.s_bytes + align16<R>(4 * (a.kind == NK_HEIS ? t.E : 0));
    int wpb = 4;
    while (wpb > 1 && (size_t)wpb * P.warp_bytes > 200 * 1024) wpb >>= 1;
    size_t smem = (size_t)wpb * P.warp_bytes;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t err = nk::allow_max_dynamic_smem((const void *)k_eloc<R>);
    if (err != cudaSuccess) return err;
    unsigned grid = (unsigned)((a.Ns + wpb - 1) / wpb);
    const int slot = prof_begin(NK_PROF_ELOC, st);
    (k_eloc<R><<<grid, 32 * wpb, smem, st>>>(P), nk::note_launch());
    // nominal connections per sample: N sites (Ising field) or E / 2 edges
    // (antiparallel on average at S_z = 0)
    const double conn = a.kind == NK_TFIM ? (double)t.N : 0.5 * (double)t.E;
    prof_end(slot, st, (double)a.Ns * conn * (double)t.M);
    return cudaGetLastError();
}

template cudaError_t launch_eloc<double>(const Tables<double> &, const ElocArgs &, cudaStream_t);
template cudaError_t launch_eloc<float>(const Tables<float> &, const ElocArgs &, cudaStream_t);

cudaError_t launch_theta_tanh(int N, int M, const double *b, const double *W, const int8_t *s,
                              int64_t B, double *T, cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    dim3 grid((M + 63) / 64, (unsigned)((B + 63) / 64));
    (k_theta_tanh<<<grid, 256, 0, st>>>(N, M, b, W, s, B, T), nk::note_launch());
    return cudaGetLastError();
}

}  // namespace nk
