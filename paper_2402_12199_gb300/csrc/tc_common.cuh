// tcgen05 helpers shared by the tensor-core network kernels: swizzled BF16
// tile addressing, shared-memory and instruction descriptors, MMA issue and
// commit, bounded mbarrier waits, bulk async copies, tensor-memory loads and
// stores, fences.  All inline PTX for sm_103a.
#pragma once

#include <cstdint>

#include <cuda_bf16.h>

#include "nn_common.cuh"

namespace rb {
namespace tc {

constexpr int kM = 128;          // pairs per tile (MMA M, TMEM lanes)
constexpr int kW = 128;          // hidden width handled by this kernel
constexpr int kK1 = 64;          // layer-1 K (10 features padded)
constexpr int kNX = 16;          // reverse output columns (10 padded)

// Byte offset of element (row r, col c) in a K-major, 128-byte-swizzled BF16
// tile of `rows` rows: 64-column atoms stacked along K, 8-row groups of
// 1024 B inside an atom, the 16-byte chunk index XOR-ed with (row % 8).
__host__ __device__ constexpr uint32_t sw128_offset(int rows, int r, int c) {
    return (uint32_t)((c >> 6) * rows * 128 + r * 128 + ((((c & 63) >> 3) ^ (r & 7)) << 4) +
                      ((c & 7) << 1));
}

// ---------------------------------------------------------------- PTX helpers
__device__ inline uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (stride byte offset), descriptor version 1, base offset 0.
__device__ inline uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;                  // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset
    d |= (uint64_t)1 << 46;                  // descriptor version
    d |= (uint64_t)2 << 61;                  // 128-byte swizzle
    return d;
}

// Descriptor of the tile `off` bytes (a multiple of 16) after the one that
// `d` describes, same layout: the start address field (bits 0..13, in 16-byte
// units) takes the offset.  Shared-memory addresses stay below 2^18 bytes, so
// the field never carries into the next one; with `off` a compile-time
// constant this is a single add.
__device__ inline uint64_t sdesc_at(uint64_t d, uint32_t off) { return d + (uint64_t)(off >> 4); }

// Instruction descriptor, kind::f16: BF16 A and B, FP32 D, K-major A and B.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ inline void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ inline void mma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ inline void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ inline void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ inline void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ inline void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Bounded wait on an mbarrier phase: gives up (returns false) after about
// `limit_cycles` SM clock cycles.
__device__ inline bool mbar_wait(uint32_t bar, uint32_t parity, long long limit_cycles) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > limit_cycles) return false;
    }
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ inline void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Split form: issue a 32-column load, then wait; the wait names the
// destination registers so no use can be scheduled before it.
__device__ inline void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
}
__device__ inline void tmem_wait32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                   "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                   "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                   "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ inline float tanh_approx(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ inline float sigm(float z) { return fmaf(0.5f, tanh_approx(0.5f * z), 0.5f); }

__device__ inline uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}
__device__ inline uint32_t pack_bf16(float2 a) { return pack_bf16(a.x, a.y); }

// Two BF16 values (low half first) widened to FP32: a BF16 is the upper
// 16 bits of the FP32 with the same value.
__device__ inline float2 widen_bf16x2(uint32_t u) {
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}

// SiLU and its derivative for two pre-activations z = acc + b, given half
// the bias hb = b / 2, in packed FP32x2 arithmetic.  With h = z / 2 and
// t = tanh(h) the logistic function is s = (1 + t) / 2, so
//   silu(z)  = z s = h + h t,
//   silu'(z) = s (1 + z (1 - s)) = s + s u,  u = h (1 - t) = h - h t:
// five packed FMAs and two tanh per pair of elements.
__device__ inline void silu2(float2 acc, float2 hb, float2& y, float2& dy) {
    const float2 half2 = make_float2(0.5f, 0.5f);
    const float2 h = __ffma2_rn(acc, half2, hb);
    const float2 t = make_float2(tanh_approx(h.x), tanh_approx(h.y));
    const float2 u = __ffma2_rn(h, make_float2(-t.x, -t.y), h);
    const float2 s = __ffma2_rn(t, half2, half2);
    y = __ffma2_rn(h, t, h);
    dy = __ffma2_rn(s, u, s);
}

// Store 32 columns (c0..c0+31 of row r) given as 16 packed BF16 pairs into
// a swizzled tile of `rows` rows.
__device__ inline void store_row32p(unsigned char* tile, int rows, int r, int c0,
                                    const uint32_t (&p)[16]) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
        *reinterpret_cast<uint4*>(tile + sw128_offset(rows, r, c0 + 8 * q)) =
            make_uint4(p[4 * q], p[4 * q + 1], p[4 * q + 2], p[4 * q + 3]);
}

// Store 32 FP32 values (columns c0..c0+31 of row r) as BF16 into a swizzled
// tile of `rows` rows.
__device__ inline void store_row32(unsigned char* tile, int rows, int r, int c0,
                                   const float (&v)[32]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint4 w;
        w.x = pack_bf16(v[8 * q + 0], v[8 * q + 1]);
        w.y = pack_bf16(v[8 * q + 2], v[8 * q + 3]);
        w.z = pack_bf16(v[8 * q + 4], v[8 * q + 5]);
        w.w = pack_bf16(v[8 * q + 6], v[8 * q + 7]);
        *reinterpret_cast<uint4*>(tile + sw128_offset(rows, r, c0 + 8 * q)) = w;
    }
}


// Bulk async copy global -> shared (16-byte aligned, size a multiple of 16),
// completing `bytes` of transaction count on the mbarrier.
__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ inline void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of this thread's lane, stored without
// waiting: the values are taken from the registers at issue; tmem_wait_st
// orders every store issued so far before later TMEM accesses.
__device__ inline void tmem_st16_issue(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
}
__device__ inline void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive 32-bit TMEM columns of this thread's lane (stored, then
// waited for).
__device__ inline void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
        "r"(r[15])
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_ld16u(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Split form of tmem_ld16u (see tmem_ld32_issue / tmem_wait32).
__device__ inline void tmem_ld16_issue(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ inline void tmem_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                   "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15])
                 :
                 : "memory");
}
__device__ inline float2 unpack_bf16(uint32_t u) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(h);
}

constexpr long long kWaitCycles = 2000000000LL;  // ~1 s at 2 GHz

// Issue the MMAs of one layer GEMM (K in steps of 16) and commit to `bar`.
// A: [128 x K] tile, B: [N x K] tile, both swizzled K-major, ROWS_B rows.
// With K and ROWS_B compile-time the loop unrolls into the MMAs alone, with
// constant descriptor offsets: a single thread issues them, so per-MMA
// address arithmetic would otherwise delay the tensor pipe.
template <int K, int ROWS_B>
__device__ inline void issue_gemm_k(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                    uint32_t bar) {
    fence_after();
#pragma unroll
    for (int k = 0; k < K / 16; ++k)
        mma_bf16(tmem_d, sdesc_at(da, (k >> 2) * (kM * 128) + (k & 3) * 32),
                 sdesc_at(db, (k >> 2) * (ROWS_B * 128) + (k & 3) * 32), idesc, k > 0 ? 1u : 0u);
    mma_commit(bar);
}

// Runtime shape: the network kernels' shapes take the unrolled form, others
// (the single-tile GEMM check) the loop.
__device__ inline void issue_gemm(uint32_t tmem_d, uint32_t a_base, uint32_t b_base, int K,
                                  int rows_b, uint32_t idesc, uint32_t bar) {
    const uint64_t da = sdesc(a_base), db = sdesc(b_base);
    if (K == 128 && rows_b == 128) return issue_gemm_k<128, 128>(tmem_d, da, db, idesc, bar);
    if (K == 16 && rows_b == 128) return issue_gemm_k<16, 128>(tmem_d, da, db, idesc, bar);
    if (K == 64 && rows_b == 128) return issue_gemm_k<64, 128>(tmem_d, da, db, idesc, bar);
    if (K == 128 && rows_b == 16) return issue_gemm_k<128, 16>(tmem_d, da, db, idesc, bar);
    if (K == 256 && rows_b == 256) return issue_gemm_k<256, 256>(tmem_d, da, db, idesc, bar);
    if (K == 16 && rows_b == 256) return issue_gemm_k<16, 256>(tmem_d, da, db, idesc, bar);
    if (K == 256 && rows_b == 16) return issue_gemm_k<256, 16>(tmem_d, da, db, idesc, bar);
    fence_after();
    for (int k = 0; k < K / 16; ++k) {
        const uint32_t koff_a = (uint32_t)(k >> 2) * (kM * 128) + (uint32_t)(k & 3) * 32;
        const uint32_t koff_b = (uint32_t)(k >> 2) * (uint32_t)(rows_b * 128) + (uint32_t)(k & 3) * 32;
        mma_bf16(tmem_d, sdesc(a_base + koff_a), sdesc(b_base + koff_b), idesc, k > 0 ? 1u : 0u);
    }
    mma_commit(bar);
}

}  // namespace tc

// nn_tc2p.cu (width 128, two tile pipelines per CTA; same weight image)
template <bool SYSTEM>
rb_status launch_tc2p(const rb_mlp* m, cudaStream_t stream, int grid, const PairSrc& src,
                      const PairDst& dst, unsigned* status);
// nn_tc256.cu (width 256, streamed weights)
bool nn_tc256_supported(const rb_mlp* m);
rb_status nn_tc256_prepare(rb_mlp* m);
template <bool SYSTEM>
rb_status launch_tc256(const rb_mlp* m, cudaStream_t stream, int grid, const PairSrc& src,
                       const PairDst& dst, unsigned* status);

}  // namespace rb
