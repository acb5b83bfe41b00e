// Internal: PTX wrappers for tcgen05 / TMA / mbarrier, exact integer-to-FP64
// assembly, and host-side tensor-map encoding, shared by the tensor-core
// translation units.  Everything is in an anonymous namespace (one copy per
// translation unit).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

namespace nk {
namespace {

constexpr unsigned long long kWaitNs = 2000000000ULL;  // 2 s bound on every wait
constexpr int kSliceK = 64;  // K extent of one slice row (128 bytes of BF16)

// ------------------------------------------------------------ PTX helpers ---

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false after kWaitNs.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < (1LL << 40); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255 && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand written by a TMA load with
// 128-byte swizzle (8-row groups of 1024 bytes), sm_100 descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(const void *p) {
    const uint64_t addr = smem_u32(p);
    uint64_t d = (addr & 0x3FFFFULL) >> 4;    // start address
    d |= (uint64_t)(16 >> 4) << 16;           // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 D.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with FP16 A and B (format field 0).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld2(uint32_t taddr, uint32_t (&r)[2]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up as soon as *abort is set (by another role
// of the same CTA); false on time-out or abort.
__device__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, const volatile int *abort) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < (1LL << 40); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 255) {
            if (*abort) return false;
            if (global_ns() - t0 > kWaitNs) return false;
        }
    }
    return false;
}

// A poll of the mbarrier phase that may suspend the thread for up to ns
// nanoseconds; it resumes as soon as the phase completes.
__device__ __forceinline__ bool mbar_try_wait_hint(uint64_t *bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// mbar_wait_or_abort whose polls may sleep up to 1 us each: a waiting warp
// (an epilogue waiting for its accumulators, a producer or MMA thread
// waiting for a stage) then gives its issue slots to the warps that have
// work.  The same bounds: false after kWaitNs or once *abort is set
// (checked every 16 polls).
__device__ bool mbar_wait_or_abort_sleep(uint64_t *bar, uint32_t parity, const volatile int *abort) {
    const unsigned long long t0 = global_ns();
    for (long long it = 0; it < (1LL << 40); ++it) {
        if (mbar_try_wait_hint(bar, parity, 1000U)) return true;
        if ((it & 15) == 15) {
            if (*abort) return false;
            if (global_ns() - t0 > kWaitNs) return false;
        }
    }
    return false;
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }


// ------------------------------------------------------------- clusters ---
// A CTA's rank in its cluster, and a cluster-wide barrier (every thread of
// every CTA of the cluster arrives; release / acquire orders shared memory;
// the warp is reconverged first, as the aligned form requires).
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// A 3-D tensor tile written to the same shared-memory offset in every CTA of
// cta_mask, each of whose mbarrier at the offset of bar receives the bytes.
__device__ __forceinline__ void tma_load_3d_mc(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1,
                                               int c2, uint16_t cta_mask) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster "
        "[%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar)), "h"(cta_mask)
        : "memory");
}

// Completion of this CTA's MMAs issued so far, as one arrival on the mbarrier
// at the offset of bar in every CTA of cta_mask.
__device__ __forceinline__ void umma_commit_mc(uint64_t *bar, uint16_t cta_mask) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(cta_mask)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void split_bits(double x, int &biased, unsigned long long &mant, bool &neg) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    neg = (b >> 63) != 0;
    biased = (int)((b >> 52) & 0x7FF);
    mant = b & 0xFFFFFFFFFFFFFULL;
    if (biased != 0) mant |= 1ULL << 52;
    else biased = 1;  // subnormal: value = mant 2^(1 - 1075)
}

__host__ __device__ __forceinline__ int clz64_any(unsigned long long x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// The tensor-core epilogues turn the exact FP32 levels D of a sliced product
// into one signed 64-bit window of the fixed-point value V = sum D 2^(8 k),
// then round the window to FP64.  The window drops only the lowest bits of V
// (8 or 10), fewer than the slicing itself leaves undetermined, so the result
// is the FP64 value of V within one rounding plus 2^(bits dropped) units of
// V's last place.  Power-of-two multiply-adds build it in a few 64-bit
// integer instructions.

// floor(V / 2^8) for the Ozaki levels V = sum_{g=2..8} D_g 2^(8 (8 - g)),
// d[g - 2] = D_g.  With |D_g| <= (g - 1) 64 255^2 (K = 64, 8-bit slices) the
// window is below 2^62.01 in magnitude.
__host__ __device__ __forceinline__ long long ozaki_window8(const int (&d)[7]) {
    long long w = (long long)(d[5] + (d[6] >> 8));  // D_7 + floor(D_8 / 2^8)
    w += (long long)d[4] * 256;
    w += (long long)d[3] * 65536;
    w += (long long)d[2] * 16777216;
    w += (long long)d[1] * 4294967296LL;
    w += (long long)d[0] * 1099511627776LL;
    return w;
}

// floor(V / 2^10) for the S-GEMM levels V = sum_{t=1..7} D_t 2^(8 (7 - t)),
// d[t - 1] = D_t (0 beyond the slices in use).  With |D_t| < 2^24 (K <= 65792,
// a +-1 operand against 8-bit slices) the window is below 2^62.01.
__host__ __device__ __forceinline__ long long sgemm_window10(const int (&d)[7]) {
    long long w = ((long long)d[5] * 256 + d[6]) >> 10;  // floor((D_6 2^8 + D_7) / 2^10)
    w += (long long)d[4] * 64;
    w += (long long)d[3] * 16384;
    w += (long long)d[2] * 4194304;
    w += (long long)d[1] * 1073741824LL;
    w += (long long)d[0] * 274877906944LL;
    return w;
}

// x 2^sc for |x| < 2^63 as FP64, rounded to nearest with ties away from zero,
// from integer operations: normalise |x| to a leading one at bit 63, round at
// bit 10, and add the 53-bit result (implicit bit included) to (exponent - 1)
// 2^52, so that a rounding carry lifts the exponent.  Results below 2^-1022
// in magnitude become a signed zero, at or above 2^1024 an infinity.
__host__ __device__ __forceinline__ double window_to_double(long long x, int sc) {
    const unsigned long long sgn = (unsigned long long)x & 0x8000000000000000ULL;
    const unsigned long long m = sgn ? 0ULL - (unsigned long long)x : (unsigned long long)x;
    const int z = clz64_any(m);                             // 1 .. 64
    const unsigned long long n = m << (z & 63);             // leading one at bit 63 (m != 0)
    const unsigned long long r = ((n >> 10) + 1ULL) >> 1;   // in [2^52, 2^53]
    const int eb = 1086 - z + sc;                           // biased exponent of the leading one
    const int ef = eb + (int)(r >> 53);                     // ... after the rounding carry
    unsigned long long bits = sgn | (((unsigned long long)(eb - 1) << 52) + r);  // mod 2^64
    bits = ef > 2046 ? (sgn | 0x7FF0000000000000ULL) : bits;
    bits = (m == 0ULL || ef < 1) ? sgn : bits;
    double v;
#ifdef __CUDA_ARCH__
    v = __longlong_as_double((long long)bits);
#else
    __builtin_memcpy(&v, &bits, 8);
#endif
    return v;
}

// The four FP32 levels of a 4-slice product (exact integers, |D_t| < 2^22)
// as the signed 64-bit V = D_0 2^24 + D_1 2^16 + D_2 2^8 + D_3.  One FP32 add
// of 1.5 2^23 turns a level into the bit pattern 0x4B400000 + D_t (ulp 1 in
// [2^23, 2^24)); the pairs D_0 2^8 + D_1 and D_2 2^8 + D_3 follow in 32-bit
// arithmetic modulo 2^32 (exact: both below 2^31 in magnitude), and V in one
// 64-bit multiply-add.
__host__ __device__ __forceinline__ unsigned int biased_level_bits(float d) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(__fadd_rn(d, 12582912.0f));
#else
    const float x = d + 12582912.0f;
    unsigned int u;
    __builtin_memcpy(&u, &x, 4);
    return u;
#endif
}

__host__ __device__ __forceinline__ long long levels4_to_i64(float d0, float d1, float d2, float d3) {
    const unsigned int bias = 257u * 0x4B400000u;  // mod 2^32
    const int hi = (int)(biased_level_bits(d0) * 256u + biased_level_bits(d1) - bias);
    const int lo = (int)(biased_level_bits(d2) * 256u + biased_level_bits(d3) - bias);
    return (long long)hi * 65536 + lo;
}

// V 2^sc as FP64 for |V| < 2^53, where the value needs no rounding: the
// leading one of |V| moves to bit 52 and (exponent - 1) 2^52 is added, as in
// window_to_double.  A signed zero for V = 0 or a result below 2^-1022, an
// infinity from 2^1024 on.
__host__ __device__ __forceinline__ double exact_to_double(long long V, int sc) {
    const unsigned long long sgn = (unsigned long long)V & 0x8000000000000000ULL;
    const unsigned long long m = sgn ? 0ULL - (unsigned long long)V : (unsigned long long)V;
    const int z = clz64_any(m);                              // 11 .. 64
    const unsigned long long n = m << ((z - 11) & 63);       // leading one at bit 52 (m != 0)
    const int eb = 1086 - z + sc;                            // biased exponent
    unsigned long long bits = sgn | (((unsigned long long)(eb - 1) << 52) + n);  // mod 2^64
    bits = eb > 2046 ? (sgn | 0x7FF0000000000000ULL) : bits;
    bits = (m == 0ULL || eb < 1) ? sgn : bits;
    double v;
#ifdef __CUDA_ARCH__
    v = __longlong_as_double((long long)bits);
#else
    __builtin_memcpy(&v, &bits, 8);
#endif
    return v;
}

// 4-slice digits with 32-bit integer operations.  grid32: y = trunc(|x|
// 2^(32 - e)) for |x| < 2^e is the top 32 bits of the mantissa (implicit one
// included) shifted right by 1022 + e - (biased exponent); the 21 dropped
// mantissa bits cannot carry into the truncated value.  Subnormal x give 0.
// bf16_digit_pair: byte `byte` of y0 and of y1 as the low and high BF16 of a
// pair, exactly (a byte d becomes the float 2^23 + d by its bit pattern,
// minus 2^23, whose upper 16 bits are the BF16 of d), signs OR-ed in.
__host__ __device__ __forceinline__ uint32_t byte_perm_any(uint32_t x, uint32_t y, uint32_t s) {
#ifdef __CUDA_ARCH__
    return __byte_perm(x, y, s);
#else
    const unsigned long long v = ((unsigned long long)y << 32) | x;
    uint32_t r = 0;
    for (int i = 0; i < 4; ++i) r |= (uint32_t)((v >> (8 * ((s >> (4 * i)) & 7))) & 0xFFu) << (8 * i);
    return r;
#endif
}

__host__ __device__ __forceinline__ uint32_t grid32(double x, int e, uint32_t &sgn) {
    unsigned long long b;
#ifdef __CUDA_ARCH__
    b = (unsigned long long)__double_as_longlong(x);
#else
    __builtin_memcpy(&b, &x, 8);
#endif
    const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
    sgn = hi >> 31;
    const int be = (int)((hi >> 20) & 0x7FFu);
    const uint32_t top = (((hi & 0xFFFFFu) | 0x100000u) << 11) | (lo >> 21);
    const int rs = 1022 + e - be;  // >= 0 for |x| < 2^e
    return (be == 0 || rs >= 32) ? 0u : (rs <= 0 ? top : top >> rs);
}

__host__ __device__ __forceinline__ uint32_t bf16_digit_pair(uint32_t y0, uint32_t y1, uint32_t byte,
                                                             uint32_t sgnmask) {
    const uint32_t sel = 0x7540u | byte;  // bytes: y.b[byte], 0, 0, 0x4B
    const uint32_t u0 = byte_perm_any(y0, 0x4B000000u, sel), u1 = byte_perm_any(y1, 0x4B000000u, sel);
    float f0, f1;
#ifdef __CUDA_ARCH__
    f0 = __fsub_rn(__uint_as_float(u0), 8388608.0f);
    f1 = __fsub_rn(__uint_as_float(u1), 8388608.0f);
    return __byte_perm(__float_as_uint(f0), __float_as_uint(f1), 0x7632u) | sgnmask;
#else
    __builtin_memcpy(&f0, &u0, 4);
    __builtin_memcpy(&f1, &u1, 4);
    f0 -= 8388608.0f;
    f1 -= 8388608.0f;
    uint32_t v0, v1;
    __builtin_memcpy(&v0, &f0, 4);
    __builtin_memcpy(&v1, &f1, 4);
    return byte_perm_any(v0, v1, 0x7632u) | sgnmask;
#endif
}

// 3-slice FP16 digits (11 bits each, exact in FP16 up to 2047).  grid33: y =
// trunc(|x| 2^(33 - e)) for |x| < 2^e, the mantissa (implicit one included)
// shifted right by 1042 + e - (biased exponent) >= 20; subnormal x give 0.
// f16_digit_pair: the 11-bit digit at bit `shift` of y0 and of y1 as the low
// and high FP16 of a pair (the float 2^23 + d from its bit pattern, minus
// 2^23, converted exactly), signs OR-ed in.
__host__ __device__ __forceinline__ unsigned long long grid33(double x, int e, uint32_t &sgn) {
    unsigned long long b;
#ifdef __CUDA_ARCH__
    b = (unsigned long long)__double_as_longlong(x);
#else
    __builtin_memcpy(&b, &x, 8);
#endif
    sgn = (uint32_t)(b >> 63);
    const int be = (int)((b >> 52) & 0x7FFu);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFULL) | (1ULL << 52);
    const int rs = 1042 + e - be;  // >= 20 for |x| < 2^e
    return (be == 0 || rs >= 64) ? 0ULL : (rs <= 0 ? m : m >> rs);
}

// The FP16 bit pattern of an integer 0 <= d < 2048 (exact), for the host.
__host__ __device__ __forceinline__ uint32_t f16_of_digit_bits(uint32_t d) {
    if (d == 0) return 0u;
    const int E = 63 - clz64_any((unsigned long long)d);  // floor(log2 d)
    return ((uint32_t)(E + 15) << 10) | ((d << (10 - E)) & 0x3FFu);
}

__host__ __device__ __forceinline__ uint32_t f16_digit_pair(unsigned long long y0, unsigned long long y1, int shift,
                                                            uint32_t sgnmask) {
    const uint32_t d0 = (uint32_t)(y0 >> shift) & 0x7FFu, d1 = (uint32_t)(y1 >> shift) & 0x7FFu;
#ifdef __CUDA_ARCH__
    const float f0 = __fsub_rn(__uint_as_float(0x4B000000u | d0), 8388608.0f);
    const float f1 = __fsub_rn(__uint_as_float(0x4B000000u | d1), 8388608.0f);
    const __half2 h = __floats2half2_rn(f0, f1);
    return *reinterpret_cast<const uint32_t *>(&h) | sgnmask;
#else
    return (f16_of_digit_bits(d0) | (f16_of_digit_bits(d1) << 16)) | sgnmask;
#endif
}

// The product t g of two FP32 pairs (t = th + tl, g = gh + gl, |tl| <=
// 2^-24 |th|, |gl| <= 2^-24 |gh|) as an unevaluated FP32 pair (ph, pl):
// ph = fl(th gh), whose rounding error th gh - ph the FMA gives exactly, and
// pl = fl(th gl + fl(tl gh + (th gh - ph))).  tl gl is dropped; |t g - ph -
// pl| stays below about 2^-44 |t g|.
__host__ __device__ __forceinline__ void mul_pairs(float th, float tl, float gh, float gl, float &ph, float &pl) {
#ifdef __CUDA_ARCH__
    ph = __fmul_rn(th, gh);
    pl = __fmaf_rn(th, gl, __fmaf_rn(tl, gh, __fmaf_rn(th, gh, -ph)));
#else
    ph = th * gh;
    pl = fmaf(th, gl, fmaf(tl, gh, fmaf(th, gh, -ph)));
#endif
}

// Three signed 11-bit digits of x = xh + xl (|xh| <= 2^11, |xl| <= 2^-22
// |xh|, FP32), rounded to nearest:
//     d0 = rint(xh),  s1 = fl(2^11 (xh - d0) + 2^11 xl),  d1 = rint(s1),
//     d2 = rint(2^11 (s1 - d1)).
// xh - d0 and s1 - d1 are exact (an FP32 value minus its nearest integer),
// and the scalings by 2^11 are exact, so the only roundings are the sum s1
// (at most 2^-14, |s1| <= 1024.5) and the last digit: |x - (d0 + 2^-11 d1 +
// 2^-22 d2)| <= 2^-23 + 2^-25.  |d0| <= 2048, |d1| <= 1025, |d2| <= 1024:
// integers that FP16 holds exactly.
__host__ __device__ __forceinline__ void h3_signed_digits(float xh, float xl, float &d0, float &d1, float &d2) {
#ifdef __CUDA_ARCH__
    d0 = rintf(xh);
    const float s1 = __fmaf_rn(__fsub_rn(xh, d0), 2048.0f, __fmul_rn(xl, 2048.0f));
    d1 = rintf(s1);
    d2 = rintf(__fmul_rn(__fsub_rn(s1, d1), 2048.0f));
#else
    d0 = rintf(xh);
    const float s1 = fmaf(xh - d0, 2048.0f, xl * 2048.0f);
    d1 = rintf(s1);
    d2 = rintf((s1 - d1) * 2048.0f);
#endif
}

// Two integer-valued floats |a|, |b| <= 2048 as the low and high FP16 of a
// pair (exact).
__host__ __device__ __forceinline__ uint32_t f16_int_pair(float a, float b) {
#ifdef __CUDA_ARCH__
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
#else
    auto one = [](float v) -> uint32_t {
        uint32_t bits;
        __builtin_memcpy(&bits, &v, 4);
        const uint32_t sg = (bits >> 16) & 0x8000u;  // -0 keeps its sign, as on the device
        const uint32_t d = (uint32_t)(v < 0.0f ? -v : v);
        return sg | (d == 2048u ? 0x6800u : f16_of_digit_bits(d));
    };
    return one(a) | (one(b) << 16);
#endif
}

// ------------------------------------------------------ host: tensor maps ---

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 3-D map over slices [S][rows][64] BF16 (consecutive slices stride_rows rows
// apart) with a box of one slice x box_rows rows.
bool make_slice_map(CUtensorMap *map, const __nv_bfloat16 *slices, int64_t rows, int S, int box_rows,
                    int64_t stride_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)kSliceK, (cuuint64_t)rows, (cuuint64_t)S};
    cuuint64_t strides[2] = {(cuuint64_t)kSliceK * 2, (cuuint64_t)stride_rows * kSliceK * 2};
    cuuint32_t box[3] = {(cuuint32_t)kSliceK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16 *>(slices), dims, strides,
                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}


}  // namespace
}  // namespace nk
