// FP32-accurate GEMM on the tensor cores for the force-matching training
// (the forward, reverse and weight-gradient products of the training pass,
// Methods: training of the pair network by force matching).
//
//   C = alpha A B + beta C,  A(m, k) = A[m sam + k sak],  B(k, n) = B[k sbk + n sbn],
//   C row-major with leading dimension ldc.
//
// Every operand x is split into two TF32 parts, x_hi = tf32(x) (round to
// nearest) and x_lo = x - x_hi (exact in FP32), and the product is formed as
// A_hi B_hi + A_hi B_lo + A_lo B_hi with tcgen05.mma kind::tf32, accumulated in
// FP32 in tensor memory.  TF32 keeps FP32's exponent range, so no scaling is
// needed; what is dropped (A_lo B_lo, the truncation of the lo parts to TF32)
// is about 2^-21 of each product, the accuracy class of an FP32 dot product.
//
// CTA tile: 128 rows of A (the TMEM lanes) x BN columns of B, 256 threads; K
// in chunks of 64 (two 128-byte swizzle atoms of FP32): each chunk is read
// from global memory along the operand's unit stride into registers while
// the previous chunk's MMAs run, split, and stored K-major with the 128-byte
// swizzle into one of two shared-memory stages.  One thread issues the 24
// MMAs of a chunk (three products x two atoms x four K steps of 8) and
// commits them to the stage's mbarrier, which the threads wait on (bounded)
// before they overwrite that stage.  The epilogue splits the tile's columns
// between the two warps that share each TMEM lane quarter.
// Split K (gridDim.z > 1): CTA z sums its K range into a partial tile at
// C + z csplit; k_splitk_sum adds the partials in a fixed order.
#include <algorithm>
#include <cstdint>

#include "tc_common.cuh"

namespace rb {
namespace gemm {

using namespace tc;

constexpr int kTM = 128, kTK = 64, kThreads = 256;

// status word for callers that pass none
__device__ unsigned g_status;

// Byte offset of element (r, k) of a [ROWS x 64] FP32 tile, K-major,
// 128-byte swizzle: two atoms of 32 columns (ROWS x 128 bytes each), one
// 128-byte row per r, 8-row groups of 1024 bytes, the 16-byte chunk index
// XOR-ed with (r % 8).
template <int ROWS>
__device__ __forceinline__ uint32_t off32(int r, int k) {
    return (uint32_t)((k >> 5) * (ROWS * 128) + r * 128 + ((((k >> 2) ^ r) & 7) << 4) + ((k & 3) << 2));
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(hi) : "f"(x));
    lo = __float_as_uint(x - __uint_as_float(hi));
}

// Instruction descriptor, kind::tf32: TF32 A and B, FP32 D, K-major A and B.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

template <int BN>
struct Shape {
    static constexpr uint32_t kA = kTM * kTK * 4;  // one part of the A chunk (32 KB)
    static constexpr uint32_t kB = BN * kTK * 4;   // one part of the B chunk
    static constexpr uint32_t kStage = 2 * kA + 2 * kB;
    static constexpr uint32_t kBar = 2 * kStage;   // two mbarriers, then the TMEM slot
    static constexpr uint32_t kSmem = kBar + 32 + 1024;  // + alignment slack
    static constexpr uint32_t kCols = BN < 32 ? 32 : BN;  // TMEM columns (power of two)
    static constexpr int kPerA = kTM * kTK / kThreads;     // 32 elements per thread
    static constexpr int kPerB = BN * kTK / kThreads;
};

template <int BN>
__global__ void __launch_bounds__(kThreads)
    k_gemm_tf32x3(int M, int N, int K, const float* __restrict__ A, int64_t sam, int64_t sak,
                  const float* __restrict__ B, int64_t sbk, int64_t sbn, float* __restrict__ C,
                  int64_t ldc, float alpha, float beta, int kchunk, int64_t csplit,
                  unsigned* status) {
    using S = Shape<BN>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int nch = ke > kb ? (ke - kb + kTK - 1) / kTK : 0;
    const uint32_t bar0 = smem_u32(sm + S::kBar), bar1 = bar0 + 8;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + S::kBar + 16);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(S::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_slot;

    // coalesced along the operand's unit stride
    const bool a_kfast = sak == 1 || sam != 1;
    const bool b_kfast = sbk == 1 || sbn != 1;
    float ra[S::kPerA], rb[S::kPerB];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < S::kPerA; ++i) {
            const int e = i * kThreads + tid;
            const int r = a_kfast ? e / kTK : e % kTM, kk = a_kfast ? e % kTK : e / kTM;
            const int gm = m0 + r, gk = k0 + kk;
            ra[i] = (gm < M && gk < ke) ? __ldg(A + gm * sam + gk * sak) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < S::kPerB; ++i) {
            const int e = i * kThreads + tid;
            const int n = b_kfast ? e / kTK : e % BN, kk = b_kfast ? e % kTK : e / BN;
            const int gn = n0 + n, gk = k0 + kk;
            rb[i] = (gn < N && gk < ke) ? __ldg(B + gk * sbk + gn * sbn) : 0.f;
        }
    };
    auto store = [&](unsigned char* st) {
#pragma unroll
        for (int i = 0; i < S::kPerA; ++i) {
            const int e = i * kThreads + tid;
            const int r = a_kfast ? e / kTK : e % kTM, kk = a_kfast ? e % kTK : e / kTM;
            uint32_t hi, lo;
            split_tf32(ra[i], hi, lo);
            const uint32_t o = off32<kTM>(r, kk);
            *reinterpret_cast<uint32_t*>(st + o) = hi;
            *reinterpret_cast<uint32_t*>(st + S::kA + o) = lo;
        }
#pragma unroll
        for (int i = 0; i < S::kPerB; ++i) {
            const int e = i * kThreads + tid;
            const int n = b_kfast ? e / kTK : e % BN, kk = b_kfast ? e % kTK : e / BN;
            uint32_t hi, lo;
            split_tf32(rb[i], hi, lo);
            const uint32_t o = off32<BN>(n, kk);
            *reinterpret_cast<uint32_t*>(st + 2 * S::kA + o) = hi;
            *reinterpret_cast<uint32_t*>(st + 2 * S::kA + S::kB + o) = lo;
        }
    };

    constexpr uint32_t idesc = idesc_tf32(kTM, BN);
    bool ok = true;      // the same in every thread
    int issued = 0;      // chunks whose MMAs were committed
    if (nch > 0) load(kb);
    for (int c = 0; c < nch && ok; ++c) {
        const int s = c & 1;
        unsigned char* st = sm + s * S::kStage;
        if (c >= 2) {  // the MMAs of chunk c - 2 read this stage
            const bool got = mbar_wait(s ? bar1 : bar0, ((c - 2) >> 1) & 1, kWaitCycles);
            if (__syncthreads_or(!got)) {
                ok = false;
                break;
            }
        }
        store(st);
        fence_proxy_async();
        fence_before();
        __syncthreads();
        if (tid == 0) {
            fence_after();
            const uint32_t a = smem_u32(st);
            const uint64_t dah = sdesc(a), dal = sdesc(a + S::kA);
            const uint64_t dbh = sdesc(a + 2 * S::kA), dbl = sdesc(a + 2 * S::kA + S::kB);
#pragma unroll
            for (int k = 0; k < kTK / 8; ++k) {  // atom k / 4, K step k % 4 of 8
                const uint32_t oa = (k >> 2) * (kTM * 128) + (k & 3) * 32;
                const uint32_t ob = (k >> 2) * (BN * 128) + (k & 3) * 32;
                const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
                mma_tf32(tmem, sdesc_at(dah, oa), sdesc_at(dbh, ob), idesc, acc);
                mma_tf32(tmem, sdesc_at(dah, oa), sdesc_at(dbl, ob), idesc, 1u);
                mma_tf32(tmem, sdesc_at(dal, oa), sdesc_at(dbh, ob), idesc, 1u);
            }
            mma_commit(s ? bar1 : bar0);
        }
        issued = c + 1;
        if (c + 1 < nch) load(kb + (c + 1) * kTK);  // in flight while the MMAs run
    }
    // the last commit covers every MMA issued before it
    bool done = issued == 0;
    if (issued > 0) {
        const int c = issued - 1;
        done = !__syncthreads_or(!mbar_wait((c & 1) ? bar1 : bar0, (c >> 1) & 1, kWaitCycles));
    }
    fence_after();
    // warps w and w + 4 read TMEM lanes 32 (w % 4) .. +31: column halves
    // (BN = 16: the first four warps take all of them)
    constexpr int kHalf = BN >= 32 ? BN / 2 : BN;
    const int half = warp >> 2;
    if (ok && done && half * kHalf < BN) {
        const int r = m0 + (warp & 3) * 32 + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + half * kHalf;
        const bool split = gridDim.z > 1;
        float* Cz = C + blockIdx.z * csplit;
#pragma unroll
        for (int c0 = 0; c0 < kHalf; c0 += 16) {
            float v[16];
            if (nch > 0)
                tmem_ld16(lane_addr + c0, v);
            else
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
            if (r < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + half * kHalf + c0 + j;
                    if (n >= N) break;
                    float* cp = Cz + (int64_t)r * ldc + n;
                    *cp = split ? v[j] : (beta == 0.f ? alpha * v[j] : fmaf(beta, *cp, alpha * v[j]));
                }
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(S::kCols));
    }
    if (!(ok && done) && tid == 0) atomicOr(status ? status : &g_status, ST_TC_TIMEOUT);
}

template <int BN>
static rb_status launch(cudaStream_t st, dim3 grid, int M, int N, int K, const float* A, int64_t sam,
                        int64_t sak, const float* B, int64_t sbk, int64_t sbn, float* C,
                        int64_t ldc, float alpha, float beta, int kchunk, int64_t csplit,
                        unsigned* status) {
    static bool attr = false;
    if (!attr) {
        RB_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Shape<BN>::kSmem));
        attr = true;
    }
    k_gemm_tf32x3<BN><<<grid, kThreads, Shape<BN>::kSmem, st>>>(
        M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, alpha, beta, kchunk, csplit, status);
    RB_CUDA(cudaGetLastError());
    return RB_OK;
}

}  // namespace gemm

// C = beta C + alpha (sum over the S partial tiles, in order; eight partials
// are loaded before they are added, the additions keep the order).
__global__ void k_splitk_sum(int M, int N, int S, const float* __restrict__ P, float* __restrict__ C,
                             int64_t ldc, float alpha, float beta) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t mn = (int64_t)M * N;
    if (t >= mn) return;
    const int m = (int)(t / N), n = (int)(t % N);
    float sum = 0.f;
    int z = 0;
    for (; z + 8 <= S; z += 8) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcs(P + (int64_t)(z + u) * mn + t);
#pragma unroll
        for (int u = 0; u < 8; ++u) sum += v[u];
    }
    for (; z < S; ++z) sum += __ldcs(P + (int64_t)z * mn + t);
    float* c = C + m * ldc + n;
    *c = beta == 0.f ? alpha * sum : fmaf(beta, *c, alpha * sum);
}

static int device_sms() {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

rb_status sgemm(cudaStream_t st, int M, int N, int K, const float* A, int64_t sam, int64_t sak,
                const float* B, int64_t sbk, int64_t sbn, float* C, int64_t ldc, float alpha,
                float beta, unsigned* status, float* ws, size_t ws_floats) {
    if (M <= 0 || N <= 0) return RB_OK;
    // column tile: the narrowest that covers N up to 32, else 32 or 64 so that
    // a batch-long M still gives about one CTA per SM
    const int BN = N <= 16 ? 16 : (N <= 32 || N <= 128 ? 32 : 64);
    const int gm = (M + gemm::kTM - 1) / gemm::kTM, gn = (N + BN - 1) / BN;
    int S = 1;
    if (ws && K >= 512) {  // a long reduction on a small output: split K to fill the GPU
        const int want = (2 * device_sms() + gm * gn - 1) / (gm * gn);
        const size_t fit = ws_floats / ((size_t)M * N);
        S = std::max(1, std::min({want, K / 128, kSplitMax, (int)std::min<size_t>(fit, 1 << 20)}));
    }
    const int kchunk = S == 1 ? std::max(K, 1)
                              : (((K + S - 1) / S) + gemm::kTK - 1) / gemm::kTK * gemm::kTK;
    S = S == 1 ? 1 : (K + kchunk - 1) / kchunk;
    float* out = S == 1 ? C : ws;
    const int64_t ld = S == 1 ? ldc : N;
    const float a = S == 1 ? alpha : 1.f, b = S == 1 ? beta : 0.f;
    const dim3 grid(gn, gm, S);
    const int64_t cs = S == 1 ? 0 : (int64_t)M * N;
    switch (BN) {
        case 16: RB_TRY(gemm::launch<16>(st, grid, M, N, K, A, sam, sak, B, sbk, sbn, out, ld, a, b, kchunk, cs, status)); break;
        case 32: RB_TRY(gemm::launch<32>(st, grid, M, N, K, A, sam, sak, B, sbk, sbn, out, ld, a, b, kchunk, cs, status)); break;
        default: RB_TRY(gemm::launch<64>(st, grid, M, N, K, A, sam, sak, B, sbk, sbn, out, ld, a, b, kchunk, cs, status)); break;
    }
    if (S > 1) {
        const int64_t mn = (int64_t)M * N;
        k_splitk_sum<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>(M, N, S, ws, C, ldc, alpha, beta);
        RB_CUDA(cudaGetLastError());
    }
    return RB_OK;
}

rb_status gemm_status_take(cudaStream_t st, bool* timed_out) {
    unsigned v = 0;
    RB_CUDA(cudaMemcpyFromSymbolAsync(&v, gemm::g_status, sizeof(unsigned), 0,
                                      cudaMemcpyDeviceToHost, st));
    RB_CUDA(cudaStreamSynchronize(st));
    if (v) {
        const unsigned zero = 0;
        RB_CUDA(cudaMemcpyToSymbolAsync(gemm::g_status, &zero, sizeof(unsigned), 0,
                                        cudaMemcpyHostToDevice, st));
        RB_CUDA(cudaStreamSynchronize(st));
    }
    *timed_out = v != 0;
    return RB_OK;
}

}  // namespace rb

using namespace rb;

extern "C" rb_status rb_gemm_f32(int64_t M, int64_t N, int64_t K, const float* A, int64_t sam,
                                 int64_t sak, const float* B, int64_t sbk, int64_t sbn, float* C,
                                 int64_t ldc, float alpha, float beta, float* ws, int64_t ws_floats,
                                 void* stream) {
    if (M < 0 || N < 0 || K < 0 || M > (1 << 30) || N > (1 << 30) || K > (1 << 30))
        return fail(RB_EINVAL, "M, N, K in [0, 2^30]");
    if ((M > 0 && N > 0) && (!C || (K > 0 && (!A || !B)) || ldc < N))
        return fail(RB_EINVAL, "null operand or ldc < N");
    if (ws_floats < 0 || (ws_floats > 0 && !ws)) return fail(RB_EINVAL, "ws_floats > 0 needs ws");
    cudaStream_t st = (cudaStream_t)stream;
    RB_TRY(sgemm(st, (int)M, (int)N, (int)K, A, sam, sak, B, sbk, sbn, C, ldc, alpha, beta, nullptr,
                 ws, (size_t)ws_floats));
    bool bad = false;
    RB_TRY(gemm_status_take(st, &bad));
    if (bad) return fail(RB_EFAULT, "tensor-core GEMM timed out waiting for an MMA");
    return RB_OK;
}
