// dvc_gemm.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) of
// sm_103a, for the value network's dense layers:
//     C[m, n] = act(sum_k A[m, k] * B[n, k] + bias[n])      (A, B K-major BF16)
// One CTA computes a 128 x BN tile with FP32 accumulators in tensor memory.
// Operand tiles of 64 K-elements are staged in shared memory in the 128-byte
// swizzled K-major layout (8-row atoms of 1024 bytes, 16-byte chunks XOR-ed
// with the row index) by cp.async, double-buffered; one thread issues the
// tcgen05.mma instructions (K = 16 each) and commits them to an mbarrier;
// four warps read the accumulators back with tcgen05.ld for the epilogue.
// Every wait on an mbarrier is bounded: on time-out the kernel records an
// error, waits (bounded) for its own MMAs, frees its tensor memory and exits.
#pragma once
#include <stdint.h>

namespace dvc {

constexpr int kGemmBM = 128;
constexpr int kGemmBK = 64;
constexpr uint32_t kWaitLimit = 1u << 22;

enum : int { kActNone = 0, kActGelu = 1 };

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (sm_100 family): start address >> 4 in bits
// 0-13, leading-dimension byte offset >> 4 in 16-29 (unused for swizzled
// K-major tiles: 1), stride-dimension byte offset >> 4 in 32-45 (1024 bytes
// between 8-row atoms), descriptor version 1 in bits 46-47, swizzle mode in
// bits 61-63 (2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor for kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// Bounded wait; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 lanes x 16 columns of 32-bit accumulators (lane = row of the tile).
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* g, uint32_t bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(saddr), "l"(g), "r"(bytes) : "memory");
}

// Byte offset of 16-byte chunk j (0..7) of row r in a 128-byte-swizzled tile.
__device__ __forceinline__ uint32_t sw128(uint32_t r, uint32_t j) {
    return (r >> 3) * 1024u + (r & 7u) * 128u + ((j ^ (r & 7u)) << 4);
}

// Stage rows [0, rows) x 64 K-elements starting at column k0 of a row-major
// K-major matrix (ld elements per row) into a swizzled tile; rows at or
// beyond `valid` are zero-filled.
__device__ __forceinline__ void stage_tile(uint32_t sbase, const __nv_bfloat16* g, int ld, int k0, int rows,
                                           int valid, int tid, int nthr) {
    for (int c = tid; c < rows * 8; c += nthr) {
        const int r = c >> 3, j = c & 7;
        const bool ok = r < valid;
        const __nv_bfloat16* src = g + (size_t)(ok ? r : 0) * ld + k0 + j * 8;
        cp_async16(sbase + sw128((uint32_t)r, (uint32_t)j), src, ok ? 16u : 0u);
    }
}

__device__ __forceinline__ float gelu_erf(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

struct GemmArgs {
    const __nv_bfloat16* A;  // M x K
    const __nv_bfloat16* B;  // N x K
    const float* bias;       // N (may be null)
    __nv_bfloat16* C;        // M x N, act(acc + bias) (may be null)
    float* Cf;               // M x N, acc + bias before the activation, FP32 (may be null)
    int M, N, K;             // K % 64 == 0, N % BN == 0
    int act;
    int32_t* flags;
};

// BN in {16, 32, 64, 128, 256}.  128 threads, dynamic smem = 2 stages x
// (16 KB + BN x 128 B) + 1024 alignment slack.
template <int BN>
__global__ void __launch_bounds__(128) gemm_bf16_tc_kernel(GemmArgs a) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ uint64_t s_bar[2];
    __shared__ uint64_t s_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    constexpr uint32_t kATile = kGemmBM * kGemmBK * 2;  // 16 KB
    constexpr uint32_t kBTile = BN * kGemmBK * 2;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kGemmBM, n0 = blockIdx.y * BN;
    const uint32_t base = (smem_u32(gsm) + 1023u) & ~1023u;
    const uint32_t sA[2] = {base, base + kATile + kBTile};
    const uint32_t sB[2] = {base + kATile, base + 2 * kATile + kBTile};
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_init(&s_done, 1);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc_alloc(&s_tmem, kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = idesc_bf16_f32(kGemmBM, BN);
    const int nk = a.K / kGemmBK;
    const int mvalid = min(kGemmBM, a.M - m0);
    uint32_t issued[2] = {0, 0};  // MMA batches committed per stage (phase tracking)
    // prologue: stage 0
    stage_tile(sA[0], a.A + (size_t)m0 * a.K, a.K, 0, kGemmBM, mvalid, tid, 128);
    stage_tile(sB[0], a.B + (size_t)n0 * a.K, a.K, 0, BN, BN, tid, 128);
    asm volatile("cp.async.commit_group;" ::: "memory");
    for (int kc = 0; kc < nk; ++kc) {
        const int st = kc & 1;
        // prefetch the next chunk into the other stage once its previous MMAs are done
        if (kc + 1 < nk) {
            const int nx = st ^ 1;
            if (issued[nx]) {
                if (!mbar_wait(&s_bar[nx], (issued[nx] - 1) & 1)) {
                    if (tid == 0) s_fail = 1;
                }
            }
            stage_tile(sA[nx], a.A + (size_t)m0 * a.K, a.K, (kc + 1) * kGemmBK, kGemmBM, mvalid, tid, 128);
            stage_tile(sB[nx], a.B + (size_t)n0 * a.K, a.K, (kc + 1) * kGemmBK, BN, BN, tid, 128);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (s_fail) break;
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kGemmBK / 16; ++kk) {
                const uint64_t ad = smem_desc_sw128(sA[st] + kk * 32);
                const uint64_t bd = smem_desc_sw128(sB[st] + kk * 32);
                tc_mma(tmem, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&s_bar[st]);
        }
        issued[st]++;
    }
    // all MMAs done -> accumulators readable
    if (tid == 0) tc_commit(&s_done);
    __syncthreads();
    const bool ok = mbar_wait(&s_done, 0) && !s_fail;
    tc_fence_after();
    if (!ok) {
        if (tid == 0 && a.flags) atomicCAS(a.flags, 0, -4);  // DVC_E_TIMEOUT
    } else {
        const int row = m0 + warp * 32 + lane;
        const bool live = row < a.M;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            tc_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (live) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int n = n0 + c0 + i;
                    float x = v[i] + (a.bias ? a.bias[n] : 0.0f);
                    if (a.Cf) a.Cf[(size_t)row * a.N + n] = x;
                    if (a.act == kActGelu) x = gelu_erf(x);
                    v[i] = x;
                }
                if (a.C) {
                    __nv_bfloat16* dst = a.C + (size_t)row * a.N + n0 + c0;
#pragma unroll
                    for (int i = 0; i < 16; i += 2) {
                        __nv_bfloat162 p;
                        p.x = __float2bfloat16_rn(v[i]);
                        p.y = __float2bfloat16_rn(v[i + 1]);
                        *reinterpret_cast<__nv_bfloat162*>(dst + i) = p;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, kCols);
    }
}

__host__ __device__ inline uint32_t gemm_smem_bytes(int BN) { return 2u * (16384u + (uint32_t)BN * 128u) + 1024u; }

}  // namespace dvc
