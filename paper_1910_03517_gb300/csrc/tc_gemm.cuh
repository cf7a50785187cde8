// BF16 GEMM on the 5th-generation tensor cores (tcgen05, accumulators in
// tensor memory), operands staged in shared memory by TMA.
//
//   D[M x N] (FP32, in TMEM) = A[M x K] * B[N x K]^T,  A and B K-major BF16
//
// One CTA computes one 128 x BN tile with 4 warps:
//   warp 0, one lane: TMA producer (kStages-deep ring of A/B stages);
//   warp 1, one lane: MMA issuer (tcgen05.mma.cta_group::1.kind::f16, K 16 per
//                     instruction, 4 per 64-wide stage), tcgen05.commit frees
//                     the stage and finally signals the accumulator;
//   warps 0-3: epilogue, each reading its 32 TMEM lanes (rows) with
//              tcgen05.ld.32x32b and calling the fused epilogue functor.
// Shared-memory tiles use the 128-byte swizzle that TMA writes and the MMA
// descriptors describe (8-row groups 1024 bytes apart).
//
// Every wait is bounded: after kSpinLimit polls the waiting thread records an
// error code in *err and gives up; the CTA still frees its tensor memory.
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_bf16.h>

namespace rt {
namespace tc {

constexpr int kBM = 128;
constexpr int kBK = 64;                 // 64 BF16 = 128 bytes = one swizzle row
constexpr int kStages = 4;
constexpr uint32_t kSpinLimit = 1u << 24;

enum : int { kErrTimeoutFull = 1, kErrTimeoutEmpty = 2, kErrTimeoutAcc = 3 };

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(a), "r"(parity) : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar)) : "memory");
}

// Shared-memory matrix descriptor (sm_100 UMMA): start address >> 4 in
// bits [0,14), leading-byte offset >> 4 in [16,30) (unused for K-major
// swizzled tiles), stride-byte offset >> 4 in [32,46) (1024 B between 8-row
// groups), version 1 in [46,48), layout type in [61,64) (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits [4,6) = 1),
// A and B BF16 (bits [7,10) and [10,13) = 1), both K-major, N >> 3 in
// [17,23), M >> 4 in [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_after_sync()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_before_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared memory of one CTA (dynamic, 1024-byte aligned base).
template <int BN>
struct Smem {
    static constexpr int kABytes = kBM * kBK * 2;
    static constexpr int kBBytes = BN * kBK * 2;
    static constexpr int kStageBytes = kABytes + kBBytes;
    static constexpr int kBytes = kStages * kStageBytes + 1024 /*align*/ + 256 /*barriers*/;
};

// The GEMM mainloop + epilogue over the K range [k0, k0 + K) (a split of a
// longer contraction when k0 > 0).  Epi is called per thread with
// (row, col0, 32 FP32 values of columns col0..col0+31).
template <int BN, class Epi>
__device__ __forceinline__ void gemm_tile(const CUtensorMap *tmA, const CUtensorMap *tmB, int k0, int K,
                                          const Epi &epi, int *err)
{
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 256, "BN");
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *tiles = base;
    uint64_t *full = reinterpret_cast<uint64_t *>(base + kStages * Smem<BN>::kStageBytes);
    uint64_t *empty = full + kStages;
    uint64_t *accb = empty + kStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(accb + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int nk = K / kBK;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;   // power of two >= 32 columns of TMEM

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tslot;

    __shared__ int s_fail;
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();

    if (warp == 0 && lane == 0) {
        // producer
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (kb >= kStages && !mbar_wait(&empty[s], ((kb / kStages) & 1) ^ 1)) {
                atomicExch(err, kErrTimeoutEmpty);
                s_fail = 1;
                break;
            }
            uint8_t *a = tiles + s * Smem<BN>::kStageBytes;
            uint8_t *b = a + Smem<BN>::kABytes;
            mbar_expect_tx(&full[s], Smem<BN>::kStageBytes);
            tma_load_2d(a, tmA, &full[s], k0 + kb * kBK, m0);
            tma_load_2d(b, tmB, &full[s], k0 + kb * kBK, n0);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        constexpr uint32_t idesc = idesc_bf16_f32(kBM, BN);
        bool ok = true;
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kStages;
            if (!mbar_wait(&full[s], (kb / kStages) & 1)) {
                atomicExch(err, kErrTimeoutFull);
                s_fail = 1;
                ok = false;
                break;
            }
            fence_after_sync();
            const uint32_t a = smem_u32(tiles + s * Smem<BN>::kStageBytes);
            const uint32_t b = a + Smem<BN>::kABytes;
            const uint64_t ad = smem_desc_sw128(a), bd = smem_desc_sw128(b);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)   // +32 bytes per K=16 step inside the swizzle row
                mma_bf16(tmem, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (kb | k) != 0);
            mma_commit(&empty[s]);
        }
        mma_commit(accb);   // arrives when every issued MMA has completed
        (void)ok;
    }
    __syncwarp();
    // epilogue: all four warps
    const bool acc_ok = mbar_wait(accb, 0);
    if (!acc_ok && lane == 0) atomicExch(err, kErrTimeoutAcc);
    fence_after_sync();
    if (acc_ok && !s_fail) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (int c = 0; c < BN; c += 32) {
            float v[32];
            tmem_ld32(tmem + lane_base + (uint32_t)c, v);
            epi(row, n0 + c, v);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

}  // namespace tc
}  // namespace rt
