// dvc_value.cu -- the value network: a learned leaf evaluator that can stand in
// for random playouts (the workload's extension of the method; the paper's
// own leaf evaluation is the playout of Sec. II-B).
//
// Features (640): per tile, owner seat relative to the mover, face-down/up
// and drawn-this-turn; per opponent slot, the values it may hold given the
// face-up numbered neighbours and the tiles the mover cannot see.  Network
// 640 -> 512 -> 512 -> 512 (GELU) -> 4 logits over relative seats, softmax
// over the seats in play.  BF16 weights and activations, FP32 accumulation in
// tensor memory (tcgen05), FP32 master weights and AdamW moments.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "dvc_device.cuh"
#include "dvc_gemm.cuh"
#include "dvc_internal.h"

using namespace dvc;
using namespace dvc_host;

namespace {

constexpr int VF = 640, VH = 512, VO = 16;
// floats per row of the logit buffers: VO logits (training) or kHeadParts x 4
// partial logits (inference with the output layer folded into layer 3)
constexpr int kLogitFloats = kHeadParts * 4 > VO ? kHeadParts * 4 : VO;
constexpr size_t OFF_W1 = 0, OFF_B1 = OFF_W1 + (size_t)VH * VF, OFF_W2 = OFF_B1 + VH, OFF_B2 = OFF_W2 + (size_t)VH * VH,
                 OFF_W3 = OFF_B2 + VH, OFF_B3 = OFF_W3 + (size_t)VH * VH, OFF_W4 = OFF_B3 + VH,
                 OFF_B4 = OFF_W4 + 4 * VH, NPARAM = OFF_B4 + 4;

}  // namespace

struct dvc_value_net {
    float *master, *m, *v, *grad;
    __nv_bfloat16 *W1, *W2, *W3, *W4;  // W4: 16 x 512, rows 4.. zero
    __nv_bfloat16 *W2T, *W3T, *W4T;    // W4T: 512 x 64, columns 4.. zero
    float* b4p;                        // 16
    int cap;                           // workspace rows (multiple of 128)
    __nv_bfloat16 *X, *H1, *H2, *H3, *XT, *H1T, *H2T, *H3T, *dZ, *dZT, *dZ4, *dZ4T;
    float *Z1, *Z2, *Z3, *L, *dH, *dZ4f, *tmp, *part, *loss;
    long long step;
};

namespace {

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ uint32_t unknown_mask(const G& g) { return g.tmask & ~g.hand(g.cur) & ~g.rev; }

// One thread per state: the row's 640 feature bits are built in registers at
// fixed positions (every loop below is unrolled), parked in the thread's own
// shared-memory row, and then each warp writes its 32 consecutive rows -- one
// contiguous stretch of X -- with coalesced 16-byte stores: a byte of feature
// bits becomes 8 BF16 values through a 256-entry table (4 FP32 values per
// nibble for Xf).  Rows n .. npad-1 are written as zeros.  Blocks of 256.
constexpr int kFeatWords = VF / 32;         // 20
constexpr int kFeatPitch = kFeatWords + 1;  // 21: the 32 rows of a warp start in 32 different banks

// OR a field of `width` bits into the bit vector f at position pos (both
// known at compile time once the caller's loops are unrolled).
__device__ __forceinline__ void or_bits(uint32_t* f, int pos, uint32_t field, int width) {
    const int w = pos >> 5, sh = pos & 31;
    f[w] |= field << sh;
    if (sh + width > 32) f[w + 1] |= field >> (32 - sh);
}

__global__ void __launch_bounds__(256) features_kernel(const dvc_state* states, int n, int npad, __nv_bfloat16* X,
                                                       float* Xf, int blocked) {
    __shared__ uint32_t s_rows[256 * kFeatPitch];
    __shared__ uint4 s_lut[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int b = tid; b < 256; b += blockDim.x) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            w[j] = (((b >> (2 * j)) & 1) ? 0x3F80u : 0u) | (((b >> (2 * j + 1)) & 1) ? 0x3F800000u : 0u);
        s_lut[b] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    uint32_t f[kFeatWords];
#pragma unroll
    for (int k = 0; k < kFeatWords; ++k) f[k] = 0u;
    const int row = blockIdx.x * blockDim.x + tid;
    if (row < n) {
        const G g = load_state(states[row]);
        uint32_t q1 = g.cur + 1u, q2 = g.cur + 2u, q3 = g.cur + 3u;
        q1 = q1 >= g.np ? q1 - g.np : q1;
        q2 = q2 >= g.np ? q2 - g.np : q2;
        q3 = q3 >= g.np ? q3 - g.np : q3;
        const uint32_t M1 = g.hand(q1), M2 = g.np > 2u ? g.hand(q2) : 0u, M3 = g.np > 3u ? g.hand(q3) : 0u;
        const uint32_t held = g.h0 | g.h1 | g.h2 | g.h3;
        // tiles: bit 7t + (owner seat relative to the mover), 7t + 4 + face-up,
        // 7t + 6 if drawn this turn; tiles in the pool have none
#pragma unroll
        for (int t = 0; t < 26; ++t) {
            const uint32_t r = ((M1 >> t) & 1u) | (((M2 >> t) & 1u) << 1) | (((M3 >> t) & 1u) * 3u);
            const uint32_t grp = (1u << r) | (16u << ((g.rev >> t) & 1u)) | ((uint32_t)t == g.drawn ? 64u : 0u);
            or_bits(f, 7 * t, ((held >> t) & 1u) ? grp : 0u, 7);
        }
        const uint32_t U = unknown_mask(g);
        const uint32_t jok = (U & kJokerMask) ? 1u << 12 : 0u;
        // opponent k (seat cur + k), slot s: 13 bits at 182 + ((k - 1) * 11 + s) * 13;
        // a face-up tile sets its value (a joker 12); a face-down slot sets every
        // value the mover cannot see strictly between its face-up numbered
        // neighbours, plus bit 12 if a joker is unseen.  Slots are walked left
        // to right: numbered tiles ascend by id, each joker stands where its
        // gap puts it, and a joker's right-hand threshold is the next numbered
        // tile of the row (or 24).
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            const uint32_t hq = k == 1 ? M1 : (k == 2 ? M2 : M3);
            const uint32_t len = (uint32_t)k < g.np ? (uint32_t)__popc(hq) : 0u;
            const uint32_t num = hq & kNumMask, R = num & g.rev;
            const uint32_t jp0 = (hq >> 24) & 1u ? joker_pos(g, hq, 0u) : 0xFFu;
            const uint32_t jp1 = (hq >> 25) & 1u ? joker_pos(g, hq, 1u) : 0xFFu;
            uint32_t rem = num;
#pragma unroll
            for (int sl = 0; sl < 11; ++sl) {
                if ((uint32_t)sl < len) {
                    const bool j0 = (uint32_t)sl == jp0, j1 = (uint32_t)sl == jp1;
                    const uint32_t low = rem ? (uint32_t)__ffs(rem) - 1u : 24u;
                    const uint32_t t = j0 ? 24u : (j1 ? 25u : low);
                    const uint32_t thr = low;  // a numbered slot's own tile, or the tile right of a joker
                    if (!j0 && !j1) rem &= rem - 1u;
                    uint32_t field;
                    if ((g.rev >> t) & 1u) {
                        field = 1u << (t < 24u ? t >> 1 : 12u);
                    } else {
                        const uint32_t below_thr = thr >= 32u ? 0xFFFFFFFFu : (1u << thr) - 1u;
                        const uint32_t left = R & below_thr, right = R & ~below_thr;
                        const int lo = left ? 31 - __clz(left) : -1;
                        const int hi = right ? __ffs(right) - 1 : 24;
                        const uint32_t above = lo < 0 ? 0x00FFFFFFu : (0x00FFFFFFu & ~((2u << lo) - 1u));
                        const uint32_t below = (1u << hi) - 1u;
                        const uint32_t m = U & above & below;
                        uint32_t x = (m | (m >> 1)) & 0x00555555u;
                        x = (x | (x >> 1)) & 0x00333333u;
                        x = (x | (x >> 2)) & 0x000F0F0Fu;
                        x = ((x | (x >> 4)) & 0x000000FFu) | ((x >> 8) & 0x00000F00u);
                        field = x | jok;
                    }
                    or_bits(f, 182 + ((k - 1) * 11 + sl) * 13, field, 13);
                }
            }
        }
    }
    if (blocked) {
        // K-blocked X (npad a multiple of 128): each thread writes its own row,
        // 16 bytes per 8 features; the warp's 32 rows are contiguous in a block
        __syncthreads();  // the table
        if (X && row < npad) {
            __nv_bfloat16* xr = X + kblocked_index(row, 0, VF);
#pragma unroll
            for (int b = 0; b < VF / 8; ++b)
                *reinterpret_cast<uint4*>(xr + (size_t)(b >> 1) * 2048 + (size_t)(b & 1) * 1024) =
                    s_lut[(f[b >> 2] >> (8 * (b & 3))) & 0xFFu];
        }
        return;
    }
    uint32_t* mine = s_rows + tid * kFeatPitch;
#pragma unroll
    for (int k = 0; k < kFeatWords; ++k) mine[k] = f[k];
    __syncthreads();
    const int row0 = blockIdx.x * blockDim.x + warp * 32;
    const int nrows = min(32, npad - row0);
    const uint32_t* wrows = s_rows + warp * 32 * kFeatPitch;
    if (X && nrows > 0) {
        uint4* dst = reinterpret_cast<uint4*>(X + (size_t)row0 * VF);
        for (int c = lane; c < nrows * (VF / 8); c += 32) {
            const int r = c / (VF / 8), k = c - r * (VF / 8);
            dst[c] = s_lut[(wrows[r * kFeatPitch + (k >> 2)] >> (8 * (k & 3))) & 0xFFu];
        }
    }
    if (Xf && nrows > 0) {
        float4* dst = reinterpret_cast<float4*>(Xf + (size_t)row0 * VF);
        for (int c = lane; c < nrows * (VF / 4); c += 32) {
            const int r = c / (VF / 4), k = c - r * (VF / 4);
            const uint32_t nib = (wrows[r * kFeatPitch + (k >> 3)] >> (4 * (k & 7))) & 0xFu;
            dst[c] = make_float4((float)(nib & 1u), (float)((nib >> 1) & 1u), (float)((nib >> 2) & 1u),
                                 (float)((nib >> 3) & 1u));
        }
    }
}

// Softmax over relative seats 0..P-1, written per absolute seat, of logits
// given as 8 partial sums per row (the output layer folded into layer 3):
// z[r] = b4[r] + parts[0][r] + ... + parts[7][r].
__global__ void softmax_head_kernel(const float* parts, const float* b4, const dvc_state* states, int n, float* out) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const dvc_state& s = states[row];
    const int P = (s.nplayers >= 2 && s.nplayers <= 4) ? s.nplayers : 2;
    const int cur = s.cur < P ? s.cur : 0;
    const float4* pp = reinterpret_cast<const float4*>(parts) + (size_t)row * kHeadParts;
    float4 z = make_float4(b4[0], b4[1], b4[2], b4[3]);
#pragma unroll
    for (int p = 0; p < kHeadParts; ++p) {
        const float4 q = pp[p];
        z.x += q.x;
        z.y += q.y;
        z.z += q.z;
        z.w += q.w;
    }
    const float zz[4] = {z.x, z.y, z.z, z.w};
    float mx = zz[0];
    for (int r = 1; r < P; ++r) mx = fmaxf(mx, zz[r]);
    float e[4], sum = 0.0f;
    for (int r = 0; r < P; ++r) {
        e[r] = expf(zz[r] - mx);
        sum += e[r];
    }
    float* o = out + (size_t)row * 4;
    o[0] = o[1] = o[2] = o[3] = 0.0f;
    for (int r = 0; r < P; ++r) o[(cur + r) % P] = e[r] / sum;
}

// Cross-entropy against soft labels (absolute seats) and dL/dlogits / n.
// Rows >= n get zero gradient.  dZ4 (npad x 64, BF16, K-padded), dZ4T (16 x
// npad, BF16), dZ4f (npad x 16, FP32); per-row loss into rowloss.
__global__ void loss_grad_kernel(const float* L, const dvc_state* states, const float* labels, int n, int npad,
                                 __nv_bfloat16* dZ4, __nv_bfloat16* dZ4T, float* dZ4f, float* rowloss) {
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= npad) return;
    float d[VO];
    for (int r = 0; r < VO; ++r) d[r] = 0.0f;
    float loss = 0.0f;
    if (row < n) {
        const dvc_state& s = states[row];
        const int P = (s.nplayers >= 2 && s.nplayers <= 4) ? s.nplayers : 2;
        const int cur = s.cur < P ? s.cur : 0;
        const float* z = L + (size_t)row * VO;
        float mx = z[0];
        for (int r = 1; r < P; ++r) mx = fmaxf(mx, z[r]);
        float sum = 0.0f;
        for (int r = 0; r < P; ++r) sum += expf(z[r] - mx);
        const float lse = mx + logf(sum);
        for (int r = 0; r < P; ++r) {
            const float y = labels[(size_t)row * 4 + (cur + r) % P];
            const float p = expf(z[r] - lse);
            if (y > 0.0f) loss -= y * (z[r] - lse);
            d[r] = (p - y) / (float)n;
        }
    }
    rowloss[row] = loss;
    for (int r = 0; r < 64; ++r) dZ4[(size_t)row * 64 + r] = __float2bfloat16_rn(r < VO ? d[r] : 0.0f);
    for (int r = 0; r < VO; ++r) {
        dZ4T[(size_t)r * npad + row] = __float2bfloat16_rn(d[r]);
        dZ4f[(size_t)row * VO + r] = d[r];
    }
}

// out[c][r] = in[r][c] for an R x C BF16 matrix (R, C multiples of 32).
__global__ void transpose_bf16_kernel(const __nv_bfloat16* in, __nv_bfloat16* out, int R, int C) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) tile[i][threadIdx.x] = in[(size_t)(r0 + i) * C + c0 + threadIdx.x];
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y)
        out[(size_t)(c0 + i) * R + r0 + threadIdx.x] = tile[threadIdx.x][i];
}

// Derivative of the tanh-form GELU (dvc_gemm.cuh): with u = k (z + a z^3),
// t = tanh(u): 0.5 (1 + t) + 0.5 z (1 - t^2) k (1 + 3 a z^2).
__device__ __forceinline__ float gelu_grad(float z) {
    const float k = 0.79788456080286536f, a = 0.044715f;
    const float t = tanh_hw(k * (z + a * z * z * z));
    return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * k * (1.0f + 3.0f * a * z * z);
}

// dZ = dH * GELU'(Z): FP32 in place in dH, BF16 copy in dZ.
__global__ void gelu_back_kernel(float* dH, const float* Z, __nv_bfloat16* dZ, size_t count) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float v = dH[i] * gelu_grad(Z[i]);
        dH[i] = v;
        dZ[i] = __float2bfloat16_rn(v);
    }
}

// Column sums of an R x C FP32 matrix in a fixed order: partial sums over
// row blocks of 256, then one thread per column adds the blocks in order.
__global__ void colsum_partial_kernel(const float* A, int R, int C, float* part) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int rb = blockIdx.y;
    if (c >= C) return;
    float acc = 0.0f;
    const int r1 = min(R, (rb + 1) * 256);
    for (int r = rb * 256; r < r1; ++r) acc += A[(size_t)r * C + c];
    part[(size_t)rb * C + c] = acc;
}

__global__ void colsum_final_kernel(const float* part, int nb, int C, float* out, int cols_out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols_out) return;
    float acc = 0.0f;
    for (int b = 0; b < nb; ++b) acc += part[(size_t)b * C + c];
    out[c] = acc;
}

__global__ void mean_kernel(const float* x, int n, float* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    float acc = 0.0f;
    for (int i = 0; i < n; ++i) acc += x[i];
    *out = acc / (float)n;
}

__global__ void copy_rows_kernel(const float* src, float* dst, size_t count) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// AdamW on the FP32 master copy; weight decay on weight matrices only.
__global__ void adamw_kernel(float* w, float* m, float* v, const float* g, size_t count, float lr, float b1, float b2,
                             float eps, float wd, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const bool is_bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) ||
                             (i >= OFF_B3 && i < OFF_W4) || i >= OFF_B4;
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float upd = (mi / c1) / (sqrtf(vi / c2) + eps);
        if (!is_bias) upd += wd * w[i];
        w[i] -= lr * upd;
    }
}

// BF16 working copies (and transposes) of the master weights.
__global__ void refresh_kernel(const float* w, __nv_bfloat16* W1, __nv_bfloat16* W2, __nv_bfloat16* W3,
                               __nv_bfloat16* W4, __nv_bfloat16* W2T, __nv_bfloat16* W3T, __nv_bfloat16* W4T,
                               float* b4p) {
    const size_t total = (size_t)VH * VF + 2 * (size_t)VH * VH + (size_t)VO * VH;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        if (i < (size_t)VH * VF) {
            W1[i] = __float2bfloat16_rn(w[OFF_W1 + i]);
            continue;
        }
        size_t j = i - (size_t)VH * VF;
        if (j < (size_t)VH * VH) {
            const __nv_bfloat16 b = __float2bfloat16_rn(w[OFF_W2 + j]);
            W2[j] = b;
            W2T[(j % VH) * VH + j / VH] = b;
            continue;
        }
        j -= (size_t)VH * VH;
        if (j < (size_t)VH * VH) {
            const __nv_bfloat16 b = __float2bfloat16_rn(w[OFF_W3 + j]);
            W3[j] = b;
            W3T[(j % VH) * VH + j / VH] = b;
            continue;
        }
        j -= (size_t)VH * VH;  // W4 padded: 16 x 512
        const size_t r = j / VH, c = j % VH;
        const __nv_bfloat16 b = __float2bfloat16_rn(r < 4 ? w[OFF_W4 + r * VH + c] : 0.0f);
        W4[j] = b;
    }
    // W4T: 512 x 64 (K-padded), b4 padded
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < (size_t)VH * 64; i += (size_t)gridDim.x * blockDim.x) {
        const size_t k = i / 64, r = i % 64;
        W4T[i] = __float2bfloat16_rn(r < 4 ? w[OFF_W4 + r * VH + k] : 0.0f);
    }
    if (blockIdx.x == 0 && threadIdx.x < VO) b4p[threadIdx.x] = threadIdx.x < 4 ? w[OFF_B4 + threadIdx.x] : 0.0f;
}

// Glorot-uniform weights from Philox (key = seed, counter = index), zero biases.
__global__ void init_params_kernel(float* w, uint64_t seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NPARAM; i += (size_t)gridDim.x * blockDim.x) {
        float fan_in = 0.0f, fan_out = 0.0f;
        bool bias = true;
        if (i < OFF_B1) { fan_in = VF; fan_out = VH; bias = false; }
        else if (i >= OFF_W2 && i < OFF_B2) { fan_in = VH; fan_out = VH; bias = false; }
        else if (i >= OFF_W3 && i < OFF_B3) { fan_in = VH; fan_out = VH; bias = false; }
        else if (i >= OFF_W4 && i < OFF_B4) { fan_in = VH; fan_out = 4; bias = false; }
        if (bias) {
            w[i] = 0.0f;
            continue;
        }
        uint32_t a = (uint32_t)i, b = (uint32_t)(i >> 32), c = 7u, d = 0u;
        philox10(a, b, c, d, (uint32_t)seed, (uint32_t)(seed >> 32));
        const float u = ((float)(a >> 8) + 0.5f) * (1.0f / 16777216.0f);  // (0, 1)
        const float lim = sqrtf(6.0f / (fan_in + fan_out));
        w[i] = (2.0f * u - 1.0f) * lim;
    }
}

// ------------------------------------------------------------------ host helpers

template <int BN>
cudaError_t gemm_attributes() {
    return cudaFuncSetAttribute(gemm_bf16_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)GemmCfg<BN>::kSmem);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point, so the
// library needs no link against the driver library.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    }();
    return fn;
}

// A row-major rows x K BF16 matrix as the 2-D tensor (K, rows) read in boxes
// of 64 x box_rows with the 128-byte swizzle; rows past the end read as zero.
bool encode_kmajor(CUtensorMap* m, const __nv_bfloat16* p, int rows, int K, int box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2u};
    const cuuint32_t box[2] = {(cuuint32_t)kGemmBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t st) {
    // inside a stream capture the attributes were set beforehand (dvc_value_prepare)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cs);
    if (e == cudaSuccess && cs == cudaStreamCaptureStatusNone) e = gemm_attributes<BN>();
    if (e != cudaSuccess) return e;
    CUtensorMap tA, tB;
    if (!encode_kmajor(&tA, a.A, a.M, a.K, kGemmBM) || !encode_kmajor(&tB, a.B, a.N, a.K, BN))
        return cudaErrorInvalidValue;
    const long long tiles = (long long)((a.M + kGemmBM - 1) / kGemmBM) * (a.N / BN);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::min<long long>(tiles, std::max(sms, 1));
    gemm_bf16_tc_kernel<BN><<<grid, kGemmThreads, GemmCfg<BN>::kSmem, st>>>(tA, tB, a);
    return cudaGetLastError();
}

constexpr uint64_t kGemmWaitNs = 2000000000ull;  // 2 s: far beyond any wait of a working GEMM

// a_blocked / c_blocked: A read / C written in the K-blocked layout (M a
// multiple of 128; the inference path's activations).
cudaError_t gemm(const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, __nv_bfloat16* C, float* Cf, int M,
                 int N, int K, int act, int32_t* flags, cudaStream_t st, bool a_blocked = false,
                 bool c_blocked = false) {
    const int wide = ((uintptr_t)C % 32 == 0 && (uintptr_t)Cf % 32 == 0) ? 1 : 0;  // null counts as aligned
    GemmArgs a{A, B, bias, C, Cf, M, N, K, act, flags, kGemmWaitNs, 0, nullptr, nullptr, wide,
               bias && (uintptr_t)bias % 16 == 0, a_blocked ? 1 : 0, c_blocked ? 1 : 0};
    if (N % 256 == 0) return launch_gemm<256>(a, st);
    if (N % 128 == 0) return launch_gemm<128>(a, st);
    if (N % 64 == 0) return launch_gemm<64>(a, st);
    if (N % 32 == 0) return launch_gemm<32>(a, st);
    return launch_gemm<16>(a, st);
}

// Layer 3 with the 512 -> 4 output layer folded into its epilogue: no H3
// written; 8 partial logit vectors per row into `parts` (rows x 8 x 4).
cudaError_t gemm_head(const __nv_bfloat16* A, const __nv_bfloat16* B, const float* bias, float* Cf, int M,
                      const __nv_bfloat16* W4, float* parts, int32_t* flags, cudaStream_t st, bool a_blocked) {
    GemmArgs a{A,     B,  bias, nullptr, Cf, M, VH, VH, kActGelu, flags, kGemmWaitNs, 0, W4, parts,
               (uintptr_t)Cf % 32 == 0, bias && (uintptr_t)bias % 16 == 0, a_blocked ? 1 : 0, 0};
    return launch_gemm<256>(a, st);  // N = 512: two 256-column tiles x four column groups = kHeadParts
}

int net_alloc(dvc_ctx* c) {
    if (c->vnet) return DVC_OK;
    dvc_value_net* v = new dvc_value_net();
    std::memset(v, 0, sizeof(*v));
    bool ok = cudaMalloc(&v->master, NPARAM * 4) == cudaSuccess && cudaMalloc(&v->m, NPARAM * 4) == cudaSuccess &&
              cudaMalloc(&v->v, NPARAM * 4) == cudaSuccess && cudaMalloc(&v->grad, NPARAM * 4) == cudaSuccess &&
              cudaMalloc(&v->W1, (size_t)VH * VF * 2) == cudaSuccess &&
              cudaMalloc(&v->W2, (size_t)VH * VH * 2) == cudaSuccess &&
              cudaMalloc(&v->W3, (size_t)VH * VH * 2) == cudaSuccess &&
              cudaMalloc(&v->W4, (size_t)VO * VH * 2) == cudaSuccess &&
              cudaMalloc(&v->W2T, (size_t)VH * VH * 2) == cudaSuccess &&
              cudaMalloc(&v->W3T, (size_t)VH * VH * 2) == cudaSuccess &&
              cudaMalloc(&v->W4T, (size_t)VH * 64 * 2) == cudaSuccess && cudaMalloc(&v->b4p, VO * 4) == cudaSuccess;
    if (!ok || cudaMemset(v->m, 0, NPARAM * 4) != cudaSuccess || cudaMemset(v->v, 0, NPARAM * 4) != cudaSuccess ||
        cudaMemset(v->grad, 0, NPARAM * 4) != cudaSuccess) {
        cudaGetLastError();
        c->vnet = v;
        return fail(c, DVC_E_OOM, "value network: parameter allocation");
    }
    c->vnet = v;
    return DVC_OK;
}

void free_work(dvc_value_net* v) {
    void* ptrs[] = {v->X,  v->H1,  v->H2, v->H3,   v->XT,   v->H1T, v->H2T, v->H3T, v->dZ,  v->dZT, v->dZ4,
                    v->dZ4T, v->Z1, v->Z2, v->Z3, v->L, v->dH, v->dZ4f, v->tmp, v->part, v->loss};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    v->X = v->H1 = v->H2 = v->H3 = v->XT = v->H1T = v->H2T = v->H3T = v->dZ = v->dZT = v->dZ4 = v->dZ4T = nullptr;
    v->Z1 = v->Z2 = v->Z3 = v->L = v->dH = v->dZ4f = v->tmp = v->part = v->loss = nullptr;
    v->cap = 0;
}

int ensure_work(dvc_ctx* c, int npad) {
    dvc_value_net* v = c->vnet;
    if (npad <= v->cap) return DVC_OK;
    free_work(v);
    const size_t r = (size_t)npad;
    auto al = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    const bool ok = al((void**)&v->X, r * VF * 2) && al((void**)&v->H1, r * VH * 2) && al((void**)&v->H2, r * VH * 2) &&
                    al((void**)&v->H3, r * VH * 2) && al((void**)&v->XT, r * VF * 2) && al((void**)&v->H1T, r * VH * 2) &&
                    al((void**)&v->H2T, r * VH * 2) && al((void**)&v->H3T, r * VH * 2) &&
                    al((void**)&v->dZ, r * VH * 2) && al((void**)&v->dZT, r * VH * 2) && al((void**)&v->dZ4, r * 64 * 2) &&
                    al((void**)&v->dZ4T, r * VO * 2) && al((void**)&v->Z1, r * VH * 4) && al((void**)&v->Z2, r * VH * 4) &&
                    al((void**)&v->Z3, r * VH * 4) && al((void**)&v->L, r * kLogitFloats * 4) && al((void**)&v->dH, r * VH * 4) &&
                    al((void**)&v->dZ4f, r * VO * 4) && al((void**)&v->tmp, (size_t)VO * VH * 4) &&
                    al((void**)&v->part, ((r + 255) / 256) * (size_t)VF * 4) && al((void**)&v->loss, (r + 1) * 4);
    if (!ok) {
        cudaGetLastError();
        free_work(v);
        return fail(c, DVC_E_OOM, "value network: workspace of " + std::to_string(npad) + " rows");
    }
    v->cap = npad;
    return DVC_OK;
}

int refresh(dvc_ctx* c, cudaStream_t st) {
    dvc_value_net* v = c->vnet;
    refresh_kernel<<<256, 256, 0, st>>>(v->master, v->W1, v->W2, v->W3, v->W4, v->W2T, v->W3T, v->W4T, v->b4p);
    return check_launch(c, "refresh_kernel");
}

int need_net(dvc_ctx* c) {
    if (!c->vnet || !c->vnet->master) return fail(c, DVC_E_INVALID, "value network not initialised (dvc_value_init)");
    return DVC_OK;
}

// Forward pass for n rows (npad = n rounded up to 128).  With train = true,
// keeps pre-activations and transposed activations for the backward pass.
// Features and the four layers of npad rows (n live) into the given
// activation buffers; Z1..Z3 (pre-activation FP32, training) may be null.
// With head = true (inference) the output layer is folded into layer 3's
// epilogue: L receives 8 partial logit vectors per row (softmax_head_kernel
// sums them) and H3 is not written; with head = false (training) layer 4 is
// a GEMM of its own and L holds the logits (16 columns per row).
int forward_into(dvc_ctx* c, const dvc_state* states, int n, int npad, __nv_bfloat16* X, __nv_bfloat16* H1,
                 __nv_bfloat16* H2, __nv_bfloat16* H3, float* L, float* Z1, float* Z2, float* Z3, bool head,
                 cudaStream_t st) {
    dvc_value_net* v = c->vnet;
    int32_t* fl = c->d_flags;
    // inference (head folded in): X, H1 and H2 in the K-blocked layout; training keeps them row-major
    const bool kb = head;
    features_kernel<<<(npad + 255) / 256, 256, 0, st>>>(states, n, npad, X, nullptr, kb ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = gemm(X, v->W1, v->master + OFF_B1, H1, Z1, npad, VH, VF, kActGelu, fl, st, kb, kb);
    if (e == cudaSuccess) e = gemm(H1, v->W2, v->master + OFF_B2, H2, Z2, npad, VH, VH, kActGelu, fl, st, kb, kb);
    if (head) {
        if (e == cudaSuccess) e = gemm_head(H2, v->W3, v->master + OFF_B3, Z3, npad, v->W4, L, fl, st, kb);
    } else {
        if (e == cudaSuccess) e = gemm(H2, v->W3, v->master + OFF_B3, H3, Z3, npad, VH, VH, kActGelu, fl, st);
        if (e == cudaSuccess) e = gemm(H3, v->W4, v->b4p, nullptr, L, npad, VO, VH, kActNone, fl, st);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "value forward");
    return DVC_OK;
}

int forward(dvc_ctx* c, const dvc_state* states, int n, int npad, bool train, cudaStream_t st) {
    dvc_value_net* v = c->vnet;
    return forward_into(c, states, n, npad, v->X, v->H1, v->H2, v->H3, v->L, train ? v->Z1 : nullptr,
                        train ? v->Z2 : nullptr, train ? v->Z3 : nullptr, !train, st);
}

int transpose(dvc_ctx* c, const __nv_bfloat16* in, __nv_bfloat16* out, int R, int C, cudaStream_t st) {
    transpose_bf16_kernel<<<dim3(C / 32, R / 32), dim3(32, 8), 0, st>>>(in, out, R, C);
    return check_launch(c, "transpose_bf16_kernel");
}

int colsum(dvc_ctx* c, const float* A, int R, int C, float* out, int cols_out, cudaStream_t st) {
    dvc_value_net* v = c->vnet;
    const int nb = (R + 255) / 256;
    colsum_partial_kernel<<<dim3((C + 127) / 128, nb), 128, 0, st>>>(A, R, C, v->part);
    colsum_final_kernel<<<(cols_out + 127) / 128, 128, 0, st>>>(v->part, nb, C, out, cols_out);
    return check_launch(c, "colsum");
}

int check_states_args(dvc_ctx* c, const void* d_states, int n) {
    if (n < 0) return fail(c, DVC_E_INVALID, "value network: n < 0");
    if (n > (1 << 24)) return fail(c, DVC_E_UNSUPPORTED, "value network: more than 2^24 rows");
    if (n > 0 && !is_device_ptr(d_states, c->device)) return fail(c, DVC_E_INVALID, "value network: states must be device memory");
    return DVC_OK;
}

}  // namespace

extern "C" {

int dvc_value_init(dvc_ctx* c, uint64_t seed, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (int rc = set_device(c)) return rc;
    if (int rc = net_alloc(c)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    dvc_value_net* v = c->vnet;
    init_params_kernel<<<512, 256, 0, st>>>(v->master, seed);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(v->m, 0, NPARAM * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(v->v, 0, NPARAM * 4, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dvc_value_init");
    v->step = 0;
    return refresh(c, st);
}

int dvc_value_params(dvc_ctx* c, float* d_params, int direction, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (!is_device_ptr(d_params, c->device) || (direction != 0 && direction != 1))
        return fail(c, DVC_E_INVALID, "dvc_value_params: device pointer and direction 0 (out) or 1 (in)");
    if (int rc = set_device(c)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (direction == 1 && !c->vnet) {
        if (int rc = net_alloc(c)) return rc;
    }
    if (int rc = need_net(c)) return rc;
    dvc_value_net* v = c->vnet;
    const cudaError_t e = direction == 0 ? cudaMemcpyAsync(d_params, v->master, NPARAM * 4, cudaMemcpyDeviceToDevice, st)
                                         : cudaMemcpyAsync(v->master, d_params, NPARAM * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "dvc_value_params");
    return direction == 1 ? refresh(c, st) : DVC_OK;
}

int dvc_value_features(dvc_ctx* c, const dvc_state* d_states, int n, float* d_out, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (int rc = check_states_args(c, d_states, n)) return rc;
    if (n == 0) return DVC_OK;
    if (!is_device_ptr(d_out, c->device)) return fail(c, DVC_E_INVALID, "dvc_value_features: d_out must be device memory");
    if (int rc = set_device(c)) return rc;
    features_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(d_states, n, n, nullptr, d_out, 0);
    return check_launch(c, "features_kernel");
}

int dvc_value_eval(dvc_ctx* c, const dvc_state* d_leaves, int n, float* d_winprob, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (int rc = check_states_args(c, d_leaves, n)) return rc;
    if (n == 0) return DVC_OK;
    if (!is_device_ptr(d_winprob, c->device)) return fail(c, DVC_E_INVALID, "dvc_value_eval: d_winprob must be device memory");
    if (int rc = set_device(c)) return rc;
    if (int rc = need_net(c)) return rc;
    const int npad = (n + 127) / 128 * 128;
    if (int rc = ensure_work(c, npad)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if (int rc = forward(c, d_leaves, n, npad, false, st)) return rc;
    softmax_head_kernel<<<(n + 127) / 128, 128, 0, st>>>(c->vnet->L, c->vnet->b4p, d_leaves, n, d_winprob);
    return check_launch(c, "softmax_head_kernel");
}

int dvc_value_train_step(dvc_ctx* c, const dvc_state* d_states, const float* d_labels, int n, float lr, float* d_loss,
                         void* stream) {
    if (!c) return DVC_E_INVALID;
    if (int rc = check_states_args(c, d_states, n)) return rc;
    if (n == 0) return DVC_OK;
    if (!is_device_ptr(d_labels, c->device) || (d_loss && !is_device_ptr(d_loss, c->device)) || !(lr >= 0.0f))
        return fail(c, DVC_E_INVALID, "dvc_value_train_step: device labels/loss, lr >= 0");
    if (int rc = set_device(c)) return rc;
    if (int rc = need_net(c)) return rc;
    const int npad = (n + 127) / 128 * 128;
    if (int rc = ensure_work(c, npad)) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    dvc_value_net* v = c->vnet;
    int32_t* fl = c->d_flags;
    if (int rc = forward(c, d_states, n, npad, true, st)) return rc;
    loss_grad_kernel<<<(npad + 127) / 128, 128, 0, st>>>(v->L, d_states, d_labels, n, npad, v->dZ4, v->dZ4T, v->dZ4f,
                                                          v->loss);
    if (int rc = check_launch(c, "loss_grad_kernel")) return rc;
    if (d_loss) mean_kernel<<<1, 32, 0, st>>>(v->loss, n, d_loss);
    int rc = transpose(c, v->X, v->XT, npad, VF, st);
    if (!rc) rc = transpose(c, v->H1, v->H1T, npad, VH, st);
    if (!rc) rc = transpose(c, v->H2, v->H2T, npad, VH, st);
    if (!rc) rc = transpose(c, v->H3, v->H3T, npad, VH, st);
    if (rc) return rc;
    float* g = v->grad;
    cudaError_t e;
    // layer 4
    e = gemm(v->dZ4T, v->H3T, nullptr, nullptr, v->tmp, VO, VH, npad, kActNone, fl, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "value backward 4");
    copy_rows_kernel<<<16, 256, 0, st>>>(v->tmp, g + OFF_W4, (size_t)4 * VH);
    if ((rc = colsum(c, v->dZ4f, npad, VO, g + OFF_B4, 4, st))) return rc;
    e = gemm(v->dZ4, v->W4T, nullptr, nullptr, v->dH, npad, VH, 64, kActNone, fl, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "value backward dH3");
    // layers 3, 2, 1
    const float* Zs[3] = {v->Z3, v->Z2, v->Z1};
    const __nv_bfloat16* Hin_T[3] = {v->H2T, v->H1T, v->XT};
    const __nv_bfloat16* WT[3] = {v->W3T, v->W2T, nullptr};
    const size_t offW[3] = {OFF_W3, OFF_W2, OFF_W1}, offB[3] = {OFF_B3, OFF_B2, OFF_B1};
    const int kin[3] = {VH, VH, VF};
    for (int l = 0; l < 3; ++l) {
        const size_t cnt = (size_t)npad * VH;
        gelu_back_kernel<<<1024, 256, 0, st>>>(v->dH, Zs[l], v->dZ, cnt);
        if ((rc = check_launch(c, "gelu_back_kernel"))) return rc;
        if ((rc = colsum(c, v->dH, npad, VH, g + offB[l], VH, st))) return rc;
        if ((rc = transpose(c, v->dZ, v->dZT, npad, VH, st))) return rc;
        e = gemm(v->dZT, Hin_T[l], nullptr, nullptr, g + offW[l], VH, kin[l], npad, kActNone, fl, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "value backward dW");
        if (WT[l]) {
            e = gemm(v->dZ, WT[l], nullptr, nullptr, v->dH, npad, VH, VH, kActNone, fl, st);
            if (e != cudaSuccess) return cuda_fail(c, e, "value backward dH");
        }
    }
    // AdamW
    v->step += 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f, wd = 1e-4f;
    const float c1 = 1.0f - powf(b1, (float)v->step), c2 = 1.0f - powf(b2, (float)v->step);
    adamw_kernel<<<1024, 256, 0, st>>>(v->master, v->m, v->v, g, NPARAM, lr, b1, b2, eps, wd, c1, c2);
    if ((rc = check_launch(c, "adamw_kernel"))) return rc;
    return refresh(c, st);
}

int dvc_value_grads(dvc_ctx* c, float* d_out, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (!is_device_ptr(d_out, c->device)) return fail(c, DVC_E_INVALID, "dvc_value_grads: d_out must be device memory");
    if (int rc = need_net(c)) return rc;
    if (int rc = set_device(c)) return rc;
    const cudaError_t e =
        cudaMemcpyAsync(d_out, c->vnet->grad, NPARAM * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return e == cudaSuccess ? DVC_OK : cuda_fail(c, e, "dvc_value_grads");
}

// File: "DVCV" magic, u32 version 1, u64 parameter count, i64 Adam step,
// then master weights, first and second moments (FP32 each).
int dvc_value_save(dvc_ctx* c, const char* path) {
    if (!c || !path) return DVC_E_INVALID;
    if (int rc = need_net(c)) return rc;
    if (int rc = set_device(c)) return rc;
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(c, DVC_E_CUDA, "dvc_value_save: sync");
    dvc_value_net* v = c->vnet;
    std::vector<float> buf(3 * NPARAM);
    if (cudaMemcpy(buf.data(), v->master, NPARAM * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + NPARAM, v->m, NPARAM * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(buf.data() + 2 * NPARAM, v->v, NPARAM * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(c, DVC_E_CUDA, "dvc_value_save: copy");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(c, DVC_E_INVALID, std::string("dvc_value_save: cannot open ") + path);
    const char magic[4] = {'D', 'V', 'C', 'V'};
    const uint32_t ver = 1;
    const uint64_t np = NPARAM;
    const int64_t step = v->step;
    bool ok = std::fwrite(magic, 1, 4, f) == 4 && std::fwrite(&ver, 4, 1, f) == 1 && std::fwrite(&np, 8, 1, f) == 1 &&
              std::fwrite(&step, 8, 1, f) == 1 && std::fwrite(buf.data(), 4, buf.size(), f) == buf.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? DVC_OK : fail(c, DVC_E_INVALID, "dvc_value_save: write failed");
}

int dvc_value_load(dvc_ctx* c, const char* path) {
    if (!c || !path) return DVC_E_INVALID;
    if (int rc = set_device(c)) return rc;
    if (int rc = net_alloc(c)) return rc;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, DVC_E_INVALID, std::string("dvc_value_load: cannot open ") + path);
    char magic[4];
    uint32_t ver = 0;
    uint64_t np = 0;
    int64_t step = 0;
    std::vector<float> buf(3 * NPARAM);
    bool ok = std::fread(magic, 1, 4, f) == 4 && std::memcmp(magic, "DVCV", 4) == 0 && std::fread(&ver, 4, 1, f) == 1 &&
              ver == 1 && std::fread(&np, 8, 1, f) == 1 && np == NPARAM && std::fread(&step, 8, 1, f) == 1 &&
              std::fread(buf.data(), 4, buf.size(), f) == buf.size();
    std::fclose(f);
    if (!ok) return fail(c, DVC_E_INVALID, "dvc_value_load: not a version-1 value-network file");
    dvc_value_net* v = c->vnet;
    if (cudaMemcpy(v->master, buf.data(), NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(v->m, buf.data() + NPARAM, NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(v->v, buf.data() + 2 * NPARAM, NPARAM * 4, cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(c, DVC_E_CUDA, "dvc_value_load: copy");
    v->step = step;
    if (int rc = refresh(c, nullptr)) return rc;
    return cudaDeviceSynchronize() == cudaSuccess ? DVC_OK : fail(c, DVC_E_CUDA, "dvc_value_load: sync");
}

int dvc_gemm_timeout_probe(dvc_ctx* c, const void* d_A, const void* d_B, float* d_Cf, int M, int N, int K,
                           int wait_ms, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (M < 1 || N < 16 || N % 16 || K < 64 || K % 64 || wait_ms < 1 || wait_ms > 1000)
        return fail(c, DVC_E_INVALID, "dvc_gemm_timeout_probe: M >= 1, N % 16 == 0, K % 64 == 0, wait 1..1000 ms");
    if (!is_device_ptr(d_A, c->device) || !is_device_ptr(d_B, c->device) || !is_device_ptr(d_Cf, c->device))
        return fail(c, DVC_E_INVALID, "dvc_gemm_timeout_probe: device pointers");
    if (int rc = set_device(c)) return rc;
    GemmArgs a{(const __nv_bfloat16*)d_A, (const __nv_bfloat16*)d_B, nullptr, nullptr, d_Cf, M, N, K, kActNone,
               c->d_flags, (uint64_t)wait_ms * 1000000ull, 1, nullptr, nullptr, 0};
    cudaError_t e;
    if (N % 256 == 0) e = launch_gemm<256>(a, (cudaStream_t)stream);
    else if (N % 128 == 0) e = launch_gemm<128>(a, (cudaStream_t)stream);
    else if (N % 64 == 0) e = launch_gemm<64>(a, (cudaStream_t)stream);
    else if (N % 32 == 0) e = launch_gemm<32>(a, (cudaStream_t)stream);
    else e = launch_gemm<16>(a, (cudaStream_t)stream);
    return e == cudaSuccess ? DVC_OK : cuda_fail(c, e, "dvc_gemm_timeout_probe");
}

int dvc_gemm_bf16(dvc_ctx* c, const void* d_A, const void* d_B, const float* d_bias, void* d_C, float* d_Cf, int M,
                  int N, int K, int act, void* stream) {
    if (!c) return DVC_E_INVALID;
    if (M < 1 || N < 16 || N % 16 || K < 64 || K % 64 || (act != kActNone && act != kActGelu))
        return fail(c, DVC_E_INVALID, "dvc_gemm_bf16: M >= 1, N % 16 == 0, K % 64 == 0, act 0 or 1");
    if (!is_device_ptr(d_A, c->device) || !is_device_ptr(d_B, c->device) || (d_bias && !is_device_ptr(d_bias, c->device)) ||
        (d_C && !is_device_ptr(d_C, c->device)) || (d_Cf && !is_device_ptr(d_Cf, c->device)) || (!d_C && !d_Cf))
        return fail(c, DVC_E_INVALID, "dvc_gemm_bf16: device pointers, at least one output");
    if ((uintptr_t)d_C % 16 || (uintptr_t)d_Cf % 16 || (uintptr_t)d_A % 16 || (uintptr_t)d_B % 16)
        return fail(c, DVC_E_INVALID, "dvc_gemm_bf16: A, B, C and Cf must be 16-byte aligned");
    if (int rc = set_device(c)) return rc;
    const cudaError_t e = gemm((const __nv_bfloat16*)d_A, (const __nv_bfloat16*)d_B, d_bias, (__nv_bfloat16*)d_C, d_Cf,
                               M, N, K, act, c->d_flags, (cudaStream_t)stream);
    return e == cudaSuccess ? DVC_OK : cuda_fail(c, e, "dvc_gemm_bf16");
}

}  // extern "C"

int dvc_value_forward_probs(dvc_ctx* c, const dvc_state* d_leaves, int n, float* d_probs, cudaStream_t st) {
    if (int rc = need_net(c)) return rc;
    const int npad = (n + 127) / 128 * 128;
    if (int rc = ensure_work(c, npad)) return rc;
    if (int rc = forward(c, d_leaves, n, npad, false, st)) return rc;
    softmax_head_kernel<<<(n + 127) / 128, 128, 0, st>>>(c->vnet->L, c->vnet->b4p, d_leaves, n, d_probs);
    return check_launch(c, "softmax_head_kernel");
}

int dvc_value_rows_alloc(dvc_ctx* c, dvc_value_rows* r, int rows) {
    dvc_value_rows_free(r);
    const size_t n = (size_t)rows;
    const bool ok = cudaMalloc(&r->X, n * VF * 2) == cudaSuccess && cudaMalloc(&r->H1, n * VH * 2) == cudaSuccess &&
                    cudaMalloc(&r->H2, n * VH * 2) == cudaSuccess && cudaMalloc(&r->H3, n * VH * 2) == cudaSuccess &&
                    cudaMalloc(&r->L, n * kLogitFloats * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        dvc_value_rows_free(r);
        return fail(c, DVC_E_OOM, "value network: activation rows");
    }
    r->rows = rows;
    return DVC_OK;
}

void dvc_value_rows_free(dvc_value_rows* r) {
    void* ptrs[] = {r->X, r->H1, r->H2, r->H3, r->L};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    *r = dvc_value_rows{};
}

int dvc_value_prepare(dvc_ctx* c) {
    if (int rc = need_net(c)) return rc;
    cudaError_t e = gemm_attributes<256>();
    if (e == cudaSuccess) e = gemm_attributes<128>();
    if (e == cudaSuccess) e = gemm_attributes<64>();
    if (e == cudaSuccess) e = gemm_attributes<32>();
    if (e == cudaSuccess) e = gemm_attributes<16>();
    return e == cudaSuccess ? DVC_OK : cuda_fail(c, e, "value network attributes");
}

int dvc_value_forward_rows(dvc_ctx* c, const dvc_state* d_leaves, int n, dvc_value_rows* r, int row0, float* d_probs,
                           cudaStream_t st) {
    if (n <= 0) return DVC_OK;
    const int npad = (n + 127) / 128 * 128;
    if (row0 < 0 || row0 + npad > r->rows) return fail(c, DVC_E_INVALID, "value network: activation rows");
    const size_t o = (size_t)row0;
    float* L = r->L + o * kLogitFloats;
    if (int rc = forward_into(c, d_leaves, n, npad, (__nv_bfloat16*)r->X + o * VF, (__nv_bfloat16*)r->H1 + o * VH,
                              (__nv_bfloat16*)r->H2 + o * VH, (__nv_bfloat16*)r->H3 + o * VH, L, nullptr, nullptr,
                              nullptr, true, st))
        return rc;
    softmax_head_kernel<<<(n + 127) / 128, 128, 0, st>>>(L, c->vnet->b4p, d_leaves, n, d_probs);
    return check_launch(c, "softmax_head_kernel");
}

void dvc_value_free(dvc_ctx* c) {
    if (!c || !c->vnet) return;
    dvc_value_net* v = c->vnet;
    free_work(v);
    void* ptrs[] = {v->master, v->m, v->v, v->grad, v->W1, v->W2, v->W3, v->W4, v->W2T, v->W3T, v->W4T, v->b4p};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete v;
    c->vnet = nullptr;
}
