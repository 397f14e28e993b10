// dvc_gemm.cuh -- BF16 GEMM on the 5th-generation tensor cores (tcgen05) of
// sm_103a, for the value network's dense layers:
//     C[m, n] = act(sum_k A[m, k] * B[n, k] + bias[n])      (A, B K-major BF16)
// A persistent, warp-specialised kernel: one CTA per SM walks its 128 x BN
// output tiles (N tile fastest, so CTAs working at the same time share A
// tiles in L2).  Warp 0 streams 64-wide K slices of A and B by TMA
// (cp.async.bulk.tensor, 128-byte swizzle) into a ring of S stages guarded by
// full/empty mbarriers; warp 1 issues tcgen05.mma (K = 16 each, FP32
// accumulators in tensor memory) as slices land and frees each stage by
// tcgen05.commit; the accumulators are double-buffered in tensor memory, so
// warps 4-19 drain tile i (tcgen05.ld, bias, activation, 16-byte stores)
// while the tensor cores compute tile i + 1.  Every wait on an mbarrier is
// bounded: on time-out the kernel records an error, waits (bounded) for its
// own copies and MMAs, frees its tensor memory and exits.
#pragma once
#include <cuda.h>  // CUtensorMap (the type only; maps are encoded through the runtime's driver entry point)
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

// The same for a K-major tile without swizzle: core matrices of 8 rows x 16
// bytes; lbo = bytes between the two 8-element halves of a 16-wide K slice,
// sbo = bytes between 8-row groups; swizzle mode 0.
__device__ __forceinline__ uint64_t smem_desc_noswz(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;
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

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait: false once limit_ns of global time have passed (checked every
// 64 polls) or after kWaitLimit polls, whichever comes first.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try_wait(bar, phase)) return true;
        if ((i & 63u) == 63u && global_ns() - t0 > limit_ns) return false;
    }
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

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// Contiguous copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned) from global to shared memory, completing `bytes` of the barrier's
// transaction count.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// 2-D TMA load of box (x = K offset, y = row offset) into shared memory,
// completing `bytes` of the barrier's transaction count.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// GELU in its tanh form (Hendrycks and Gimpel, "Gaussian Error Linear Units",
// 2016): 0.5 x (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3))), with the hardware
// tanh (tanh.approx.f32).
__device__ __forceinline__ float tanh_hw(float u) {
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    return t;
}
__device__ __forceinline__ float gelu(float x) {
    return 0.5f * x * (1.0f + tanh_hw(0.79788456080286536f * (x + 0.044715f * x * x * x)));
}

struct GemmArgs {
    const __nv_bfloat16* A;  // M x K
    const __nv_bfloat16* B;  // N x K
    const float* bias;       // N (may be null)
    __nv_bfloat16* C;        // M x N, act(acc + bias) (may be null)
    float* Cf;               // M x N, acc + bias before the activation, FP32 (may be null)
    int M, N, K;             // K % 64 == 0, N % BN == 0
    int act;
    int32_t* flags;
    uint64_t wait_ns;  // limit of every mbarrier wait (global time)
    int starve;        // test hook: the producer issues no copy, so every consumer wait runs out
    // Optional 4-output head folded into the epilogue (N = 512, BN = 256):
    // head_out[row][part][o] = sum over the part's columns c of
    // act(acc + bias)[row][c] * head_w[o][c], one part per (N tile, column
    // group), 8 parts per row, summed in a fixed order by the consumer.
    const __nv_bfloat16* head_w;  // 4 (or more) x N BF16, row-major; null: no head
    float* head_out;              // M x 8 x 4 FP32
    int wide;   // C and Cf 32-byte aligned: 256-bit stores (half the store instructions)
    int bias4;  // bias 16-byte aligned: read four floats per load
    // K-blocked layout (M % 128 == 0): a matrix of R rows and W columns is
    // stored as R/128 x W/16 blocks of 4 KB in that order, block (i, j) holding
    // rows 128i.. and columns 16j.. as two halves of 8 columns, each 128 rows x
    // 16 bytes.  A 64-wide K slice of a row tile is then 16 KB in one piece (one
    // bulk copy, read by the MMA without swizzle), and an epilogue warp's 32
    // rows x 8 columns are 512 contiguous bytes (one coalesced store).
    int a_blocked;  // A in the K-blocked layout
    int c_blocked;  // C written in the K-blocked layout
};

// Element (r, c) of a K-blocked matrix with W columns.
__host__ __device__ inline size_t kblocked_index(int r, int c, int W) {
    return (((size_t)(r >> 7) * (size_t)(W >> 4) + (size_t)(c >> 4)) * 2 + (size_t)((c >> 3) & 1)) * 1024 +
           (size_t)(r & 127) * 8 + (size_t)(c & 7);
}

// 32 bytes to global memory in one instruction (p 32-byte aligned).
__device__ __forceinline__ void st_global_v8(void* p, const uint32_t* w) {
    asm volatile("st.global.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]), "r"(w[1]),
                 "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

constexpr int kHeadParts = 8;

// Stage geometry for a BN-column tile: A 128 x 64 and B BN x 64 BF16 per
// stage, as many stages as fit in 192 KB (at most 6); two accumulator
// buffers of max(BN, 32) tensor-memory columns.
template <int BN>
struct GemmCfg {
    static constexpr uint32_t kA = (uint32_t)kGemmBM * kGemmBK * 2;  // 16 KB
    static constexpr uint32_t kB = (uint32_t)BN * kGemmBK * 2;
    static constexpr uint32_t kStage = kA + kB;
    static constexpr int kStages = (int)((192u * 1024u) / kStage) > 6 ? 6 : (int)((192u * 1024u) / kStage);
    static constexpr uint32_t kSmem = (uint32_t)kStages * kStage + 1024u;  // + alignment slack
    static constexpr uint32_t kAccCols = BN < 32 ? 32u : (uint32_t)BN;
    static constexpr uint32_t kCols = 2u * kAccCols;  // a power of two, >= 64
};

constexpr int kGemmEpiWarps = 16;                       // four per tensor-memory lane quarter
constexpr int kGemmThreads = 32 * (4 + kGemmEpiWarps);  // warp 0 TMA, warp 1 MMA, warps 2-3 idle, then epilogue

// BN in {16, 32, 64, 128, 256}.  tA: A as a (K, M) tensor, box (64, 128);
// tB: B as (K, N), box (64, BN); both 128-byte swizzled.  Grid: at most one
// CTA per SM; CTA c takes tiles c, c + gridDim.x, ...
template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    gemm_bf16_tc_kernel(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, GemmArgs a) {
    using Cfg = GemmCfg<BN>;
    constexpr int S = Cfg::kStages;
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ uint64_t s_full[S], s_empty[S], s_accf[2], s_acce[2], s_done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail, s_issued, s_consumed;
    __shared__ float4 s_head[512];  // head weights per column (outputs 0..3), when a.head_w is set
    volatile int* fail = &s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntn = a.N / BN;
    const int tiles = ((a.M + kGemmBM - 1) / kGemmBM) * ntn;
    const int nk = a.K / kGemmBK;
    const uint32_t base = (smem_u32(gsm) + 1023u) & ~1023u;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&s_full[s], 1);
            mbar_init(&s_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&s_accf[b], 1);
            mbar_init(&s_acce[b], kGemmEpiWarps);  // one arrival per epilogue warp
        }
        mbar_init(&s_done, 1);
        s_fail = 0;
        s_issued = 0;
        s_consumed = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (a.head_w)
        for (int c = tid; c < a.N && c < 512; c += blockDim.x)
            s_head[c] = make_float4(__bfloat162float(a.head_w[c]), __bfloat162float(a.head_w[a.N + c]),
                                    __bfloat162float(a.head_w[2 * a.N + c]), __bfloat162float(a.head_w[3 * a.N + c]));
    if (warp == 0) tc_alloc(&s_tmem, Cfg::kCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    if (warp == 0) {
        if (lane == 0) {
            // producer: K slices of every tile of this CTA, up to S in flight
            int it = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x) {
                const int m0 = (t / ntn) * kGemmBM, n0 = (t % ntn) * BN;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % S, r = it / S;
                    if (a.starve || (it >= S && !mbar_wait(&s_empty[s], (uint32_t)(r - 1) & 1u, a.wait_ns)) ||
                        *fail) {
                        *fail = 1;
                        stop = true;
                        break;
                    }
                    const uint32_t sa = base + (uint32_t)s * Cfg::kStage;
                    mbar_expect_tx(&s_full[s], Cfg::kStage);
                    if (a.a_blocked)  // the four 4 KB blocks of K slice kc of row tile m0 / 128
                        bulk_load(sa, a.A + kblocked_index(m0, kc * kGemmBK, a.K), Cfg::kA, &s_full[s]);
                    else
                        tma_load_2d(sa, &tA, kc * kGemmBK, m0, &s_full[s]);
                    tma_load_2d(sa + Cfg::kA, &tB, kc * kGemmBK, n0, &s_full[s]);
                }
            }
            s_issued = it;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile j accumulates into buffer j & 1 once the
            // epilogue has drained that buffer's previous tile
            const uint32_t idesc = idesc_bf16_f32(kGemmBM, BN);
            int it = 0, j = 0;
            bool stop = false;
            for (int t = blockIdx.x; t < tiles && !stop; t += gridDim.x, ++j) {
                const int b = j & 1, u = j >> 1;
                if (u > 0 && !mbar_wait(&s_acce[b], (uint32_t)(u - 1) & 1u, a.wait_ns)) {
                    *fail = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)b * Cfg::kAccCols;
                for (int kc = 0; kc < nk; ++kc, ++it) {
                    const int s = it % S, r = it / S;
                    if (!mbar_wait(&s_full[s], (uint32_t)r & 1u, a.wait_ns) || *fail) {
                        *fail = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + (uint32_t)s * Cfg::kStage;
#pragma unroll
                    for (int kk = 0; kk < kGemmBK / 16; ++kk) {
                        const uint64_t ad = a.a_blocked ? smem_desc_noswz(sa + (uint32_t)kk * 4096u, 2048u, 128u)
                                                        : smem_desc_sw128(sa + (uint32_t)kk * 32u);
                        const uint64_t bd = smem_desc_sw128(sa + Cfg::kA + (uint32_t)kk * 32u);
                        tc_mma(acc, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                    }
                    tc_commit(&s_empty[s]);
                }
                if (!stop) tc_commit(&s_accf[b]);
            }
            s_consumed = it;
            tc_commit(&s_done);  // arrives when every MMA issued above has completed
        }
    } else if (warp >= 4) {
        // epilogue: warp w reads tensor-memory lanes 32 (w mod 4) .. +31 (one
        // output row per thread) and one of up to four column groups
        constexpr int kGroups = BN / 16 < kGemmEpiWarps / 4 ? BN / 16 : kGemmEpiWarps / 4;
        constexpr int cw = BN / kGroups;
        const int quarter = warp & 3, group = (warp - 4) >> 2;
        const int cbeg = group < kGroups ? group * cw : BN;
        int j = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++j) {
            const int b = j & 1, u = j >> 1;
            const bool got = mbar_wait(&s_accf[b], (uint32_t)u & 1u, a.wait_ns);
            if (!__all_sync(0xFFFFFFFFu, got) || *fail) {
                if (lane == 0) *fail = 1;
                break;
            }
            tc_fence_after();
            const int m0 = (t / ntn) * kGemmBM, n0 = (t % ntn) * BN;
            const int row = m0 + quarter * 32 + lane;
            const bool live = row < a.M;
            const uint32_t acc = tmem + (uint32_t)b * Cfg::kAccCols + ((uint32_t)(quarter * 32) << 16);
            float4 head = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 1
            for (int c0 = cbeg; c0 < cbeg + cw && c0 < BN; c0 += 16) {  // cw is a multiple of 16
                float v[16];
                tc_ld16(acc + (uint32_t)c0, v);
                if (live) {
                    const int nb = n0 + c0;
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += (a.bias && !a.bias4) ? __ldg(a.bias + nb + i) : 0.0f;
                    if (a.bias4) {  // the 16 biases as four 16-byte loads (nb is a multiple of 16)
                        const float4* b4 = reinterpret_cast<const float4*>(a.bias + nb);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 x = __ldg(b4 + j);
                            v[4 * j] += x.x;
                            v[4 * j + 1] += x.y;
                            v[4 * j + 2] += x.z;
                            v[4 * j + 3] += x.w;
                        }
                    }
                    if (a.Cf) {
                        float* cf = a.Cf + (size_t)row * a.N + nb;
                        if (a.wide) {
                            st_global_v8(cf, reinterpret_cast<const uint32_t*>(v));
                            st_global_v8(cf + 8, reinterpret_cast<const uint32_t*>(v + 8));
                        } else {
                            float4* f = reinterpret_cast<float4*>(cf);
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                f[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                        }
                    }
                    if (a.act == kActGelu) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = gelu(v[i]);
                    }
                    if (a.head_out) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float4 hw = s_head[nb + i];
                            head.x += v[i] * hw.x;
                            head.y += v[i] * hw.y;
                            head.z += v[i] * hw.z;
                            head.w += v[i] * hw.w;
                        }
                    }
                    if (a.C) {
                        uint32_t w[8];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            __nv_bfloat162 p = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                            w[i] = *reinterpret_cast<uint32_t*>(&p);
                        }
                        if (a.c_blocked) {
                            __nv_bfloat16* blk = a.C + kblocked_index(m0, nb, a.N) + (size_t)(quarter * 32 + lane) * 8;
                            *reinterpret_cast<uint4*>(blk) = make_uint4(w[0], w[1], w[2], w[3]);
                            *reinterpret_cast<uint4*>(blk + 1024) = make_uint4(w[4], w[5], w[6], w[7]);
                        } else if (a.wide) {
                            st_global_v8(a.C + (size_t)row * a.N + nb, w);
                        } else {
                            uint4* dst = reinterpret_cast<uint4*>(a.C + (size_t)row * a.N + nb);
                            dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
                            dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
                        }
                    }
                }
            }
            if (a.head_out && live && group < kGroups)
                reinterpret_cast<float4*>(a.head_out)[(size_t)row * kHeadParts + (t % ntn) * kGroups + group] = head;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s_acce[b]);
        }
    }
    __syncthreads();
    // every MMA has completed before tensor memory is freed; on failure the
    // copies still in flight land first
    const bool ok = __syncthreads_and(mbar_wait(&s_done, 0, a.wait_ns) && !*fail) != 0;
    if (!ok && tid == 0) {
        for (int it = s_consumed; it < s_issued; ++it) mbar_wait(&s_full[it % S], (uint32_t)(it / S) & 1u, a.wait_ns);
        if (a.flags) atomicCAS(a.flags, 0, -4);  // DVC_E_TIMEOUT
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, Cfg::kCols);
    }
}

}  // namespace dvc
