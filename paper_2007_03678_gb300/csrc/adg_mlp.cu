// adg_mlp.cu -- the triage network of the screening pipeline: a three-layer
// perceptron nin -> 256 -> 256 -> 1 with ReLU, BF16 weights and FP32
// accumulation on the tensor cores (two engines: tcgen05 MMAs with tensor
// memory accumulators, and warp-level mma m16n8k16), trained on the GPU by
// these kernels (forward, backward, Adam).  The paper has no learned part; the network predicts a ligand's
// final best docking energy from its descriptors and the first generations
// of its best-energy trace, so that ligands predicted hopeless can skip the
// full search.
//
// Numerics (what is stored in BF16, what stays FP32):
//   x_hat = (x - mu) / sigma                 FP32, stored BF16 (operand)
//   h1 = relu(W1 x_hat + b1)                 FP32 accumulate, stored BF16 (operand)
//   h2 = relu(W2 h1 + b2)                    FP32
//   y  = w3 . h2 + b3                        FP32 (w3 BF16)
//   dh2 = dy w3 [h2 > 0]                     FP32 (bias gradient), BF16 as operand
//   dh1 = (dh2 W2) [h1 > 0]                  FP32 (bias gradient), BF16 as operand
//   dW2 = dh2^T h1, dW1 = dh1^T x_hat        FP32 accumulate over the batch
// Master weights and Adam moments are FP32; the BF16 copies are rewritten
// after every update (round to nearest even).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "adg_internal.h"

namespace {

using bf16 = __nv_bfloat16;
constexpr int H = ADG_MLP_HIDDEN;   // 256
constexpr int KIN = ADG_MLP_NIN_MAX;  // 32: input width padded for the k = 16 steps
constexpr int TR = 32;              // rows per tile of the activation kernel
constexpr int LW2 = H + 8;          // shared-memory row strides (bf16 elements)
constexpr int LW1 = KIN + 8;
constexpr int LX = KIN + 8;
constexpr int LH = H + 8;
constexpr int LF = H + 4;           // float rows
constexpr size_t kActSmem = sizeof(bf16) * ((size_t)H * LW2 + (size_t)H * LW1 + TR * LX + 2 * TR * LH) +
                            sizeof(float) * ((size_t)TR * LF + TR);

struct Norm {
    float mu[KIN], sigma[KIN];
    float mu_y, sigma_y;
};

struct Offs {
    int w1, b1, w2, b2, w3, b3, n;
};

Offs offsets(int nin)
{
    Offs o;
    o.w1 = 0;
    o.b1 = H * nin;
    o.w2 = o.b1 + H;
    o.b2 = o.w2 + H * H;
    o.w3 = o.b2 + H;
    o.b3 = o.w3 + H;
    o.n = o.b3 + 1;
    return o;
}

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// acc (16x8, FP32) += A (16x16) * B (16x8), operands BF16 in shared memory.
// AK: A(m,k) = a[m*lda + k], else a[k*lda + m].
// BK: B(k,n) = b[n*ldb + k], else b[k*ldb + n].
// Fragment layout of mma.m16n8k16 (g = lane/4, t = lane%4): A regs hold
// (g,2t..2t+1), (g+8,2t..), (g,2t+8..), (g+8,2t+8..); B regs (2t..2t+1, g),
// (2t+8..2t+9, g); C holds (g,2t), (g,2t+1), (g+8,2t), (g+8,2t+1).
template <bool AK, bool BK>
__device__ __forceinline__ void mma16816(float (&c)[4], const bf16* a, int lda, const bf16* b, int ldb, int lane)
{
    const int g = lane >> 2, t = lane & 3;
    uint32_t a0, a1, a2, a3, b0, b1;
    if (AK) {
        a0 = *reinterpret_cast<const uint32_t*>(a + g * lda + 2 * t);
        a1 = *reinterpret_cast<const uint32_t*>(a + (g + 8) * lda + 2 * t);
        a2 = *reinterpret_cast<const uint32_t*>(a + g * lda + 2 * t + 8);
        a3 = *reinterpret_cast<const uint32_t*>(a + (g + 8) * lda + 2 * t + 8);
    } else {
        a0 = pack2(a[(2 * t) * lda + g], a[(2 * t + 1) * lda + g]);
        a1 = pack2(a[(2 * t) * lda + g + 8], a[(2 * t + 1) * lda + g + 8]);
        a2 = pack2(a[(2 * t + 8) * lda + g], a[(2 * t + 9) * lda + g]);
        a3 = pack2(a[(2 * t + 8) * lda + g + 8], a[(2 * t + 9) * lda + g + 8]);
    }
    if (BK) {
        b0 = *reinterpret_cast<const uint32_t*>(b + g * ldb + 2 * t);
        b1 = *reinterpret_cast<const uint32_t*>(b + g * ldb + 2 * t + 8);
    } else {
        b0 = pack2(b[(2 * t) * ldb + g], b[(2 * t + 1) * ldb + g]);
        b1 = pack2(b[(2 * t + 8) * ldb + g], b[(2 * t + 9) * ldb + g]);
    }
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float wsum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct ActArgs {
    const float* theta;  // FP32 master parameters (biases read from here)
    const bf16* w1;      // [H][KIN]
    const bf16* w2;      // [H][H]
    const bf16* w3;      // [H]
    Offs o;
    int nin;
    Norm nm;
    const float* x;      // [*][nin]
    const float* t;      // [*] raw targets (training)
    const int* idx;      // rows of x / t to use, or NULL (identity)
    int B;
    float* y;            // forward: denormalised predictions [B]
    // training
    bf16* xh;            // [Bpad][KIN]
    bf16* h1;            // [Bpad][H]
    bf16* dh2;           // [Bpad][H]
    bf16* dh1;           // [Bpad][H]
    float* part;         // per tile: b1 [H], b2 [H], w3 [H], b3, sum of squared residuals (kPart floats)
    float inv_B;
};

constexpr int kPart = 3 * H + 2;  // partial sums per tile

// Forward (and, TRAIN, the backward pass down to the activations) of 32-row
// tiles; persistent CTAs keep W1 and W2 in shared memory across tiles.  The
// bias / w3 gradients and the loss leave as per-tile partial sums, reduced
// in tile order by k_mlp_wgrad, so training is bit-reproducible.
template <bool TRAIN>
__global__ void __launch_bounds__(256, 1) k_mlp_act(ActArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    bf16* W2s = reinterpret_cast<bf16*>(smem);
    bf16* W1s = W2s + H * LW2;
    bf16* Xs = W1s + H * LW1;
    bf16* H1s = Xs + TR * LX;
    bf16* D2s = H1s + TR * LH;
    float* H2s = reinterpret_cast<float*>(D2s + TR * LH);
    float* dys = H2s + TR * LF;
    __shared__ float wloss[8];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    for (int i = tid; i < H * H / 8; i += 256) {
        const int r = i >> 5, c8 = i & 31;
        *reinterpret_cast<uint4*>(W2s + r * LW2 + c8 * 8) = *reinterpret_cast<const uint4*>(A.w2 + r * H + c8 * 8);
    }
    for (int i = tid; i < H * KIN / 8; i += 256) {
        const int r = i >> 2, c8 = i & 3;
        *reinterpret_cast<uint4*>(W1s + r * LW1 + c8 * 8) = *reinterpret_cast<const uint4*>(A.w1 + r * KIN + c8 * 8);
    }
    const float* b1 = A.theta + A.o.b1;
    const float* b2 = A.theta + A.o.b2;
    const float b3 = A.theta[A.o.b3];
    __syncthreads();
    const int ntiles = (A.B + TR - 1) / TR;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int r0 = tile * TR;
        // 1. normalised inputs
        for (int i = tid; i < TR * KIN; i += 256) {
            const int r = i / KIN, k = i % KIN, row = r0 + r;
            float v = 0.f;
            if (row < A.B && k < A.nin) {
                const int src = A.idx ? A.idx[row] : row;
                v = (A.x[(long)src * A.nin + k] - A.nm.mu[k]) / A.nm.sigma[k];
            }
            const bf16 hv = __float2bfloat16_rn(v);
            Xs[r * LX + k] = hv;
            if (TRAIN) A.xh[(long)row * KIN + k] = hv;
        }
        __syncthreads();
        // 2. h1 = relu(x_hat W1^T + b1); warp w owns columns [32w, 32w+32)
        {
            float acc[2][4][4] = {};
#pragma unroll
            for (int ks = 0; ks < KIN; ks += 16)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        mma16816<true, true>(acc[mt][nt], Xs + mt * 16 * LX + ks, LX,
                                             W1s + (warp * 32 + nt * 8) * LW1 + ks, LW1, lane);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = mt * 16 + g + (q >> 1) * 8, j = warp * 32 + nt * 8 + 2 * t4 + (q & 1);
                        const bf16 hv = __float2bfloat16_rn(fmaxf(acc[mt][nt][q] + b1[j], 0.f));
                        H1s[r * LH + j] = hv;
                        if (TRAIN) A.h1[(long)(r0 + r) * H + j] = hv;
                    }
        }
        __syncthreads();
        // 3. h2 = relu(h1 W2^T + b2), FP32 in shared memory
        {
            float acc[2][4][4] = {};
#pragma unroll 4
            for (int ks = 0; ks < H; ks += 16)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        mma16816<true, true>(acc[mt][nt], H1s + mt * 16 * LH + ks, LH,
                                             W2s + (warp * 32 + nt * 8) * LW2 + ks, LW2, lane);
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int r = mt * 16 + g + (q >> 1) * 8, j = warp * 32 + nt * 8 + 2 * t4 + (q & 1);
                        H2s[r * LF + j] = fmaxf(acc[mt][nt][q] + b2[j], 0.f);
                    }
        }
        __syncthreads();
        // 4. y = w3 . h2 + b3; warp w owns rows 4w..4w+3
        float lsum = 0.f;
        for (int q = 0; q < 4; ++q) {
            const int r = warp * 4 + q, row = r0 + r;
            float s = 0.f;
            for (int j = lane; j < H; j += 32) s += H2s[r * LF + j] * __bfloat162float(A.w3[j]);
            const float y = wsum(s) + b3;
            if (!TRAIN) {
                if (lane == 0 && row < A.B) A.y[row] = y * A.nm.sigma_y + A.nm.mu_y;
            } else {
                float res = 0.f;
                if (row < A.B) {
                    const int src = A.idx ? A.idx[row] : row;
                    res = y - (A.t[src] - A.nm.mu_y) / A.nm.sigma_y;
                }
                if (lane == 0) dys[r] = 2.f * res * A.inv_B;
                lsum += res * res;
            }
        }
        if (!TRAIN) {
            __syncthreads();
            continue;
        }
        float* part = A.part + (long)tile * kPart;
        if (lane == 0) wloss[warp] = lsum;
        __syncthreads();
        if (tid == 0) {
            float l = 0.f;
            for (int w = 0; w < 8; ++w) l += wloss[w];
            part[3 * H + 1] = l;
        }
        // 5. per column j: dW3, dh2 = dy w3 [h2 > 0], db2
        {
            const int j = tid;
            const float w3j = __bfloat162float(A.w3[j]);
            float gw3 = 0.f, gb2 = 0.f, gb3 = 0.f;
            for (int r = 0; r < TR; ++r) {
                const float h = H2s[r * LF + j], d = dys[r];
                gw3 += d * h;
                gb3 += d;
                const float dh = h > 0.f ? d * w3j : 0.f;
                gb2 += dh;
                const bf16 db = __float2bfloat16_rn(dh);
                D2s[r * LH + j] = db;
                A.dh2[(long)(r0 + r) * H + j] = db;
            }
            part[2 * H + j] = gw3;
            part[H + j] = gb2;
            if (j == 0) part[3 * H] = gb3;
        }
        __syncthreads();
        // 6. dh1 = (dh2 W2) [h1 > 0], db1; warp w owns columns [32w, 32w+32)
        {
            float acc[2][4][4] = {};
#pragma unroll 4
            for (int ks = 0; ks < H; ks += 16)
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int nt = 0; nt < 4; ++nt)
                        mma16816<true, false>(acc[mt][nt], D2s + mt * 16 * LH + ks, LH,
                                              W2s + ks * LW2 + warp * 32 + nt * 8, LW2, lane);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int i = warp * 32 + nt * 8 + 2 * t4 + c;
                    float colsum = 0.f;
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const int r = mt * 16 + g + hh * 8;
                            const float v = __bfloat162float(H1s[r * LH + i]) > 0.f ? acc[mt][nt][hh * 2 + c] : 0.f;
                            colsum += v;
                            A.dh1[(long)(r0 + r) * H + i] = __float2bfloat16_rn(v);
                        }
                    // sum over the 8 row groups g (lanes t4, t4+4, ..., t4+28)
                    colsum += __shfl_xor_sync(0xffffffffu, colsum, 4);
                    colsum += __shfl_xor_sync(0xffffffffu, colsum, 8);
                    colsum += __shfl_xor_sync(0xffffffffu, colsum, 16);
                    if (g == 0) part[i] = colsum;
                }
        }
        __syncthreads();
    }
}

struct WgradArgs {
    const bf16* dh2;  // [Bpad][H]
    const bf16* h1;   // [Bpad][H]
    const bf16* dh1;  // [Bpad][H]
    const bf16* xh;   // [Bpad][KIN]
    int Bpad, nin;
    Offs o;
    float* grad;
    const float* part;  // [Bpad / 32][kPart] from k_mlp_act
    float* loss;        // += sum of squared residuals * loss_scale
    float loss_scale;
};

// Weight gradients summed over the batch (rows r):
//   dW2[j][i] = sum_r dh2[r][j] h1[r][i]   (16 CTAs, 64x64 tiles)
//   dW1[j][k] = sum_r dh1[r][j] xh[r][k]   (4 CTAs, 64x32 tiles)
// Each output element is produced by one CTA (plain stores, no atomics).
// CTA 20 sums the per-tile partials (biases, w3, loss) in tile order.
__global__ void __launch_bounds__(256) k_mlp_wgrad(WgradArgs A)
{
    if (blockIdx.x == 20) {
        const int ntiles = A.Bpad / 32;
        for (int c = threadIdx.x; c < kPart; c += blockDim.x) {
            float sum = 0.f;
            for (int t = 0; t < ntiles; ++t) sum += A.part[(long)t * kPart + c];
            if (c < H) A.grad[A.o.b1 + c] = sum;
            else if (c < 2 * H) A.grad[A.o.b2 + c - H] = sum;
            else if (c < 3 * H) A.grad[A.o.w3 + c - 2 * H] = sum;
            else if (c == 3 * H) A.grad[A.o.b3] = sum;
            else *A.loss += sum * A.loss_scale;
        }
        return;
    }
    constexpr int RC = 32;                 // rows per chunk
    constexpr int LA = 64 + 8, LB = 64 + 8;
    __shared__ __align__(16) bf16 As[RC * LA];
    __shared__ __align__(16) bf16 Bs[RC * LB];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const bool w1part = blockIdx.x >= 16;
    const int jt = w1part ? (int)blockIdx.x - 16 : (int)blockIdx.x / 4;
    const int it = w1part ? 0 : (int)blockIdx.x % 4;
    const int ncols = w1part ? KIN : 64;   // output columns of this tile
    const bf16* Asrc = w1part ? A.dh1 : A.dh2;
    const bf16* Bsrc = w1part ? A.xh : A.h1;
    const int ldb_src = w1part ? KIN : H;
    const int mtile = warp & 3, nhalf = warp >> 2;
    const int nnt = ncols / 16;            // n-tiles (of 8) per warp: 4 for 64 columns, 2 for 32
    float acc[4][4] = {};
    for (int rc = 0; rc < A.Bpad; rc += RC) {
        for (int i = tid; i < RC * 8; i += 256) {  // A chunk: 32 rows x 64 columns j
            const int r = i >> 3, c8 = i & 7;
            *reinterpret_cast<uint4*>(As + r * LA + c8 * 8) =
                *reinterpret_cast<const uint4*>(Asrc + (long)(rc + r) * H + jt * 64 + c8 * 8);
        }
        for (int i = tid; i < RC * (ncols / 8); i += 256) {  // B chunk: 32 rows x ncols columns
            const int r = i / (ncols / 8), c8 = i % (ncols / 8);
            *reinterpret_cast<uint4*>(Bs + r * LB + c8 * 8) =
                *reinterpret_cast<const uint4*>(Bsrc + (long)(rc + r) * ldb_src + it * 64 + c8 * 8);
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < RC; ks += 16)
            for (int nt = 0; nt < nnt; ++nt)
                mma16816<false, false>(acc[nt], As + ks * LA + mtile * 16, LA,
                                       Bs + ks * LB + nhalf * (ncols / 2) + nt * 8, LB, lane);
        __syncthreads();
    }
    for (int nt = 0; nt < nnt; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = jt * 64 + mtile * 16 + g + (q >> 1) * 8;
            const int c = it * 64 + nhalf * (ncols / 2) + nt * 8 + 2 * t4 + (q & 1);
            if (w1part) {
                if (c < A.nin) A.grad[A.o.w1 + j * A.nin + c] = acc[nt][q];
            } else {
                A.grad[A.o.w2 + j * H + c] = acc[nt][q];
            }
        }
}

// Adam on the FP32 master parameters (update != 0), then the BF16 copies.
__global__ void k_mlp_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, Offs o, int nin, int update, float lr, float c1, float c2,
                           bf16* __restrict__ w1, bf16* __restrict__ w2, bf16* __restrict__ w3)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= o.n) return;
    float th = theta[p];
    if (update) {
        const float gr = grad[p];
        const float mm = 0.9f * m[p] + 0.1f * gr;
        const float vv = 0.999f * v[p] + 0.001f * gr * gr;
        m[p] = mm;
        v[p] = vv;
        th -= lr * (mm * c1) / (sqrtf(vv * c2) + 1e-8f);
        theta[p] = th;
    }
    if (p < o.b1) w1[(p / nin) * KIN + p % nin] = __float2bfloat16_rn(th);
    else if (p >= o.w2 && p < o.b2) w2[p - o.w2] = __float2bfloat16_rn(th);
    else if (p >= o.w3 && p < o.b3) w3[p - o.w3] = __float2bfloat16_rn(th);
}


// ------------------------------------------------------------------ tcgen05 forward
// Inference on the 5th-generation tensor cores: persistent CTAs (16 warps, one
// per SM) run 128-row tiles, W1 and W2 staged once per CTA.  x_hat, W1, h1 and W2 sit in shared memory in the canonical K-major
// no-swizzle layout (8-row x 16-byte core matrices: element (r, k) of an
// R x K operand at ((r/8)(K/8) + k/8) * 128 + (r%8) * 16 + (k%8) * 2 bytes);
// one thread issues tcgen05.mma (M = 128, N = 256, K = 16 per instruction,
// BF16 in, FP32 accumulators in tensor memory): x_hat W1^T into TMEM columns
// 0-255, then h1 W2^T into columns 256-511.  Four threads own a row (its TMEM
// lane), one per quarter of the columns (four warps per lane quarter keep the
// epilogue's tensor-memory and shared-memory latencies covered); they read
// their accumulators back with tcgen05.ld and finish the row (bias, ReLU,
// BF16 h1; then bias, ReLU and the w3 dot product, the quarters summed
// through shared memory).
constexpr int TC_ROWS = 128;
constexpr size_t kTcW2 = (size_t)H * H * 2;
constexpr size_t kTcW1 = (size_t)H * KIN * 2;
constexpr size_t kTcX = (size_t)TC_ROWS * KIN * 2;
constexpr size_t kTcH1 = (size_t)TC_ROWS * H * 2;
constexpr size_t kTcSmem = kTcW2 + kTcW1 + kTcX + kTcH1 + 3 * H * sizeof(float) + 32;
constexpr long long kTcWaitNs = 1000000000ll;   // default bound of a wait on an MMA completion barrier (1 s)
constexpr long long kTcDrainNs = 1000000000ll;  // bound of the final wait for every issued MMA (1 s)

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;      // leading byte offset: next core matrix along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;      // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;                            // descriptor version of this architecture
    return d;                                          // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the given phase parity of an mbarrier, for at most wait_ns
// nanoseconds; wait_ns <= 0 tests the barrier once without waiting.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity, long long wait_ns)
{
    if (wait_ns <= 0) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        return done != 0;
    }
    const long long t0 = global_ns();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > wait_ns) return false;
    }
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// relu(a + b[0]) and relu(c + b[1]) rounded to BF16 and packed (first value in
// the low half): one two-wide add and one conversion that applies the ReLU
// to the rounded values (the same result as rounding the ReLU's output).
__device__ __forceinline__ uint32_t bias_relu_bf16x2(float a, float c, const float* b)
{
    const float2 h = __fadd2_rn(make_float2(a, c), *reinterpret_cast<const float2*>(b));
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(h.y), "f"(h.x));
    return r;
}

constexpr int TC_THREADS = 512;  // 16 warps: warps w, w + 4, w + 8, w + 12 share TMEM lanes 32 (w % 4).., a column quarter each

// status: bit 0 set when a wait on an MMA completion barrier gave up after
// wait_ns (the tile's rows are then written as NaN), bit 1 when the final
// wait for every issued MMA gave up.
__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_fwd_tc(ActArgs A, int* status, long long wait_ns)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* W2s = smem;
    unsigned char* W1s = W2s + kTcW2;
    unsigned char* Xs = W1s + kTcW1;
    unsigned char* H1s = Xs + kTcX;
    float* b1s = reinterpret_cast<float*>(H1s + kTcH1);
    float* b2s = b1s + H;
    float* w3s = b2s + H;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(w3s + H);  // [0]: layer-1 MMAs, [1]: layer-2 MMAs, [2]: drain
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);
    __shared__ float part[3][TC_ROWS];  // the other column quarters' shares of each row's output
    const int tid = threadIdx.x, warp = tid >> 5;
    const int r = (warp & 3) * 32 + (tid & 31);  // this thread's row = its TMEM lane
    const int half = warp >> 2;                  // column quarter: columns [64 half, 64 half + 64)
    const uint32_t s_base = smem_u32(smem), s_mbar1 = smem_u32(mbar), s_mbar2 = smem_u32(mbar + 1),
                   s_mbar3 = smem_u32(mbar + 2);
    if (warp == 0) {  // 512 TMEM columns: layer 1 in 0-255, layer 2 in 256-511
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_mbar1) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_mbar2) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s_mbar3) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < H * H / 8; i += TC_THREADS) {
        const int n = i >> 5, k8 = i & 31;
        *reinterpret_cast<uint4*>(W2s + (((n >> 3) * (H / 8) + k8) << 7) + ((n & 7) << 4)) =
            *reinterpret_cast<const uint4*>(A.w2 + n * H + k8 * 8);
    }
    for (int i = tid; i < H * KIN / 8; i += TC_THREADS) {
        const int n = i >> 2, k8 = i & 3;
        *reinterpret_cast<uint4*>(W1s + (((n >> 3) * (KIN / 8) + k8) << 7) + ((n & 7) << 4)) =
            *reinterpret_cast<const uint4*>(A.w1 + n * KIN + k8 * 8);
    }
    for (int j = tid; j < H; j += TC_THREADS) {
        b1s[j] = A.theta[A.o.b1 + j];
        b2s[j] = A.theta[A.o.b2 + j];
        w3s[j] = __bfloat162float(A.w3[j]);
    }
    // kind::f16 instruction descriptor: FP32 accumulate, BF16 A and B, both K-major, N = 256, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(TC_ROWS >> 4) << 24);
    // x_hat of one tile (BF16, canonical layout, K = 32); each column quarter writes one of the four 8-column chunks
    auto stage_x = [&](int tile) {
        const int row = tile * TC_ROWS + r;
#pragma unroll
        for (int k8 = half; k8 < half + 1; ++k8) {
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k8 * 8 + 2 * q;
                float v0 = 0.f, v1 = 0.f;
                if (row < A.B) {
                    const int src = A.idx ? A.idx[row] : row;
                    if (k < A.nin) v0 = (A.x[(long)src * A.nin + k] - A.nm.mu[k]) / A.nm.sigma[k];
                    if (k + 1 < A.nin) v1 = (A.x[(long)src * A.nin + k + 1] - A.nm.mu[k + 1]) / A.nm.sigma[k + 1];
                }
                pk[q] = pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
            }
            *reinterpret_cast<uint4*>(Xs + (((r >> 3) * (KIN / 8) + k8) << 7) + ((r & 7) << 4)) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // smem writes visible to the tensor cores
    };
    auto issue_layer1 = [&](uint32_t tbase) {
        for (int s = 0; s < KIN / 16; ++s)
            tc_mma(tbase, tc_smem_desc(s_base + (uint32_t)(kTcW2 + kTcW1) + s * 256, 128, (KIN / 8) * 128),
                   tc_smem_desc(s_base + (uint32_t)kTcW2 + s * 256, 128, (KIN / 8) * 128), idesc, s > 0);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_mbar1)
                     : "memory");
    };
    bool ok = true;
    uint32_t ph1 = 0, ph2 = 0;  // parity of the next completion of each barrier
    const int ntiles = (A.B + TC_ROWS - 1) / TC_ROWS;
    int tile = blockIdx.x;
    if (tile < ntiles) stage_x(tile);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // TMEM address, barriers, weights and the first x_hat are ready
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = *tslot;
    const uint32_t trow = tbase + ((uint32_t)((warp & 3) * 32) << 16);
    if (tid == 0 && tile < ntiles) issue_layer1(tbase);
    // persistent CTAs, W1 and W2 resident; the next tile's x_hat and layer-1 MMAs
    // overlap this tile's layer-2 MMAs and epilogue
    for (; tile < ntiles; tile += gridDim.x) {
        const int row = tile * TC_ROWS + r;
        ok = tc_wait(s_mbar1, ph1, wait_ns) && ok;
        ph1 ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int c = half * 2; c < half * 2 + 2; ++c) {  // h1 = relu(x_hat W1^T + b1) -> BF16, row-major K = 256
            float v[32];
            tc_ld32(trow + c * 32, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = c * 32 + q * 8 + 2 * e;
                    pk[e] = bias_relu_bf16x2(v[q * 8 + 2 * e], v[q * 8 + 2 * e + 1], b1s + j);
                }
                *reinterpret_cast<uint4*>(H1s + (((r >> 3) * (H / 8) + c * 4 + q) << 7) + ((r & 7) << 4)) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            for (int s = 0; s < H / 16; ++s)
                tc_mma(tbase + H,
                       tc_smem_desc(s_base + (uint32_t)(kTcW2 + kTcW1 + kTcX) + s * 256, 128, (H / 8) * 128),
                       tc_smem_desc(s_base + s * 256, 128, (H / 8) * 128), idesc, s > 0);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_mbar2)
                         : "memory");
        }
        // the next tile: x_hat (its buffer is free: layer 1 of this tile is done) and, once every thread has
        // written it, its layer-1 MMAs into columns 0-255 (their accumulators were read above)
        const int next = tile + gridDim.x;
        if (next < ntiles) stage_x(next);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && next < ntiles) issue_layer1(tbase);
        ok = tc_wait(s_mbar2, ph2, wait_ns) && ok;
        ph2 ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float2 acc2 = make_float2(0.f, 0.f);
        for (int c = half * 2; c < half * 2 + 2; ++c) {  // w3 . relu(h1 W2^T + b2) over this quarter's columns
            float v[32];
            tc_ld32(trow + H + c * 32, v);
#pragma unroll
            for (int e = 0; e < 32; e += 2) {  // two columns at a time (even and odd partial sums)
                const float2 h = __fadd2_rn(make_float2(v[e], v[e + 1]),
                                            *reinterpret_cast<const float2*>(b2s + c * 32 + e));
                acc2 = __ffma2_rn(make_float2(fmaxf(h.x, 0.f), fmaxf(h.y, 0.f)),
                                  *reinterpret_cast<const float2*>(w3s + c * 32 + e), acc2);
            }
        }
        const float acc = acc2.x + acc2.y;
        if (half > 0) part[half - 1][r] = acc;
        // h1 and columns 256-511 are rewritten for the next tile only after every thread is done with them;
        // a wait that gave up in any thread of the CTA marks the tile's rows (any row may have read
        // an accumulator too early)
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        const bool all_ok = __syncthreads_and(ok) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (half == 0 && row < A.B)
            A.y[row] = all_ok ? (acc + part[0][r] + part[1][r] + part[2][r] + A.theta[A.o.b3]) * A.nm.sigma_y + A.nm.mu_y
                              : __int_as_float(0x7fc00000);
    }
    if (!ok) atomicOr(status, 1);
    // every MMA this CTA issued has completed before its tensor memory is released: one more commit
    // tracks all of them, waited for under the normal bound whatever wait_ns was
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s_mbar3)
                     : "memory");
    if (!tc_wait(s_mbar3, 0u, kTcDrainNs) && tid == 0) atomicOr(status, 2);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tbase) : "memory");
}

// ------------------------------------------------------------------ tcgen05 training
// The training contractions on the 5th-generation tensor cores, in three
// kernels over 128-row tiles, with the numerics of the warp-level engine
// (x_hat, h1, dh2 and dh1 stored BF16 as operands, FP32 accumulation):
//   k_mlp_train_fwd_tc   x_hat W1^T, h1 W2^T (tensor memory), then per row the
//                        output, residual and dh2 = dy w3 [h2 > 0]; per-tile
//                        column sums of dh2 (b2), dy h2 (w3), dy (b3), res^2
//   k_mlp_train_bwd_tc   dh1 = (dh2 W2) [h1 > 0] with W2^T staged; per-tile
//                        column sums of dh1 (b1)
//   k_mlp_wgrad_tc       dW2 = dh2^T h1 and dW1 = dh1^T x_hat, the batch as the
//                        K dimension in chunks of 64 rows (transposed into the
//                        canonical K-major layout while staging); one CTA sums
//                        the per-tile partials in tile order.
// Every sum has a fixed order, so training stays bit-reproducible.  Waits on
// the MMA barriers are bounded as in the forward kernel (status bit 0 when
// one gives up; the tile's values are then zero), and every CTA waits for
// all its MMAs before freeing tensor memory (bit 1 if that wait gives up).
struct TrainArgs {
    const float* theta;
    const bf16* w1;      // [H][KIN]
    const bf16* w2;      // [H][H]
    const bf16* w3;      // [H]
    Offs o;
    int nin;
    Norm nm;
    const float* x;      // [*][nin]
    const float* t;      // [*] raw targets
    const int* idx;      // rows of x / t, or NULL
    int B, Bpad;         // rows, rows padded to whole 128-row tiles
    float inv_B;
    bf16* xh;            // [Bpad][KIN]
    bf16* h1;            // [Bpad][H]
    bf16* dh2;           // [Bpad][H]
    bf16* dh1;           // [Bpad][H]
    float* part;         // [Bpad / 128][kPart]
    float* grad;
    float* loss;         // += sum of squared residuals * loss_scale
    float loss_scale;
};

// Sum over the warp's 32 lanes of each of 32 per-lane values: afterwards lane
// l holds the sum of v[l] (fixed order: a butterfly that halves the list each
// round, the upper half going to the lanes with the round's bit set).
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32], int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const float send = up ? v[i] : v[i + s];
            const float keep = up ? v[i + s] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return v[0];
}

// Element (r, k) of an R x K BF16 operand in the canonical K-major layout
// without swizzle (8-row x 16-byte core matrices), as a byte offset.
__device__ __forceinline__ uint32_t kmajor_off(int r, int k, int K)
{
    return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void tc_sync()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Every MMA the CTA issued is complete (a last commit by the issuing thread,
// waited for under the normal bound) before the tensor memory is freed.
__device__ __forceinline__ void tc_drain_dealloc(uint32_t mbar_drain, uint32_t tbase, uint32_t ncols, int* status,
                                                 int warp, int tid)
{
    tc_sync();
    if (tid == 0) tc_commit(mbar_drain);
    if (!tc_wait(mbar_drain, 0u, kTcDrainNs) && tid == 0) atomicOr(status, 2);
    tc_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(ncols) : "memory");
}

constexpr size_t kTfSmem = kTcW2 + kTcW1 + kTcX + kTcH1 + (3 * H + 2 * TC_ROWS) * sizeof(float) + 64;
static_assert(kTcX == 8 * H * sizeof(float), "the column sums of a tile fill the x_hat operand buffer exactly");

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_train_fwd_tc(TrainArgs A, int* status, long long wait_ns)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* W2s = smem;
    unsigned char* W1s = W2s + kTcW2;
    unsigned char* Xs = W1s + kTcW1;
    unsigned char* H1s = Xs + kTcX;
    float* b1s = reinterpret_cast<float*>(H1s + kTcH1);
    float* b2s = b1s + H;
    float* w3s = b2s + H;
    float* dys = w3s + H;           // [128] dy of each row
    float* rqs = dys + TC_ROWS;     // [128] squared residual of each row
    // per 32-row block the column sums of dh2 and of dy h2, [4][H] each, in the
    // x_hat buffer (free from the end of layer 1 until the next tile is staged)
    float* colb = reinterpret_cast<float*>(Xs);
    float* colw = colb + 4 * H;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(rqs + TC_ROWS);  // layer 1, layer 2, drain
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 3);
    __shared__ float part[3][TC_ROWS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = (warp & 3) * 32 + lane, quarter = warp >> 2, rb = warp & 3;
    const uint32_t s_base = smem_u32(smem), s_m1 = smem_u32(mbar), s_m2 = smem_u32(mbar + 1),
                   s_m3 = smem_u32(mbar + 2);
    if (warp == 0) tc_alloc(tslot, 512);
    if (tid == 0) {
        mbar_init(s_m1);
        mbar_init(s_m2);
        mbar_init(s_m3);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < H * H / 8; i += TC_THREADS) {
        const int n = i >> 5, k8 = i & 31;
        *reinterpret_cast<uint4*>(W2s + (((n >> 3) * (H / 8) + k8) << 7) + ((n & 7) << 4)) =
            *reinterpret_cast<const uint4*>(A.w2 + n * H + k8 * 8);
    }
    for (int i = tid; i < H * KIN / 8; i += TC_THREADS) {
        const int n = i >> 2, k8 = i & 3;
        *reinterpret_cast<uint4*>(W1s + (((n >> 3) * (KIN / 8) + k8) << 7) + ((n & 7) << 4)) =
            *reinterpret_cast<const uint4*>(A.w1 + n * KIN + k8 * 8);
    }
    for (int j = tid; j < H; j += TC_THREADS) {
        b1s[j] = A.theta[A.o.b1 + j];
        b2s[j] = A.theta[A.o.b2 + j];
        w3s[j] = __bfloat162float(A.w3[j]);
    }
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(TC_ROWS >> 4) << 24);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    const uint32_t tbase = *tslot;
    const uint32_t trow = tbase + ((uint32_t)(rb * 32) << 16);
    const float b3 = A.theta[A.o.b3];
    bool ok = true;
    uint32_t ph1 = 0, ph2 = 0;
    const int ntiles = A.Bpad / TC_ROWS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row = tile * TC_ROWS + r;
        // x_hat (BF16): canonical operand in shared memory and row-major copy for the weight gradient
        {
            const int k8 = quarter;
            uint32_t pk[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = k8 * 8 + 2 * q;
                float v0 = 0.f, v1 = 0.f;
                if (row < A.B) {
                    const int src = A.idx ? A.idx[row] : row;
                    if (k < A.nin) v0 = (A.x[(long)src * A.nin + k] - A.nm.mu[k]) / A.nm.sigma[k];
                    if (k + 1 < A.nin) v1 = (A.x[(long)src * A.nin + k + 1] - A.nm.mu[k + 1]) / A.nm.sigma[k + 1];
                }
                pk[q] = pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
            }
            const uint4 u = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            *reinterpret_cast<uint4*>(Xs + kmajor_off(r, k8 * 8, KIN)) = u;
            *reinterpret_cast<uint4*>(A.xh + (long)row * KIN + k8 * 8) = u;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
        if (tid == 0) {
            for (int s = 0; s < KIN / 16; ++s)
                tc_mma(tbase, tc_smem_desc(s_base + (uint32_t)(kTcW2 + kTcW1) + s * 256, 128, (KIN / 8) * 128),
                       tc_smem_desc(s_base + (uint32_t)kTcW2 + s * 256, 128, (KIN / 8) * 128), idesc, s > 0);
            tc_commit(s_m1);
        }
        ok = tc_wait(s_m1, ph1, wait_ns) && ok;
        ph1 ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // h1 = relu(x_hat W1^T + b1) -> BF16: operand of layer 2 and row-major copy
        for (int c = quarter * 2; c < quarter * 2 + 2; ++c) {
            float v[32];
            tc_ld32(trow + c * 32, v);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = c * 32 + q * 8 + 2 * e;
                    pk[e] = bias_relu_bf16x2(v[q * 8 + 2 * e], v[q * 8 + 2 * e + 1], b1s + j);
                }
                const uint4 u = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                *reinterpret_cast<uint4*>(H1s + kmajor_off(r, c * 32 + q * 8, H)) = u;
                *reinterpret_cast<uint4*>(A.h1 + (long)row * H + c * 32 + q * 8) = u;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
        if (tid == 0) {
            for (int s = 0; s < H / 16; ++s)
                tc_mma(tbase + H,
                       tc_smem_desc(s_base + (uint32_t)(kTcW2 + kTcW1 + kTcX) + s * 256, 128, (H / 8) * 128),
                       tc_smem_desc(s_base + s * 256, 128, (H / 8) * 128), idesc, s > 0);
            tc_commit(s_m2);
        }
        ok = tc_wait(s_m2, ph2, wait_ns) && ok;
        ph2 ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // output y = w3 . relu(h1 W2^T + b2) + b3 (column quarters summed through shared memory)
        float acc = 0.f;
        for (int c = quarter * 2; c < quarter * 2 + 2; ++c) {
            float v[32];
            tc_ld32(trow + H + c * 32, v);
#pragma unroll
            for (int e = 0; e < 32; ++e) acc += fmaxf(v[e] + b2s[c * 32 + e], 0.f) * w3s[c * 32 + e];
        }
        if (quarter > 0) part[quarter - 1][r] = acc;
        // a wait that gave up anywhere in the CTA voids the tile (its rows add nothing)
        const bool all_ok = __syncthreads_and(ok) != 0;
        if (quarter == 0) {
            float res = 0.f;
            if (row < A.B && all_ok) {
                const int src = A.idx ? A.idx[row] : row;
                const float y = acc + part[0][r] + part[1][r] + part[2][r] + b3;
                res = y - (A.t[src] - A.nm.mu_y) / A.nm.sigma_y;
            }
            dys[r] = 2.f * res * A.inv_B;
            rqs[r] = res * res;
        }
        __syncthreads();
        // dh2 = dy w3 [h2 > 0] (BF16, row-major), and per 32-row block the column
        // sums of dh2 (b2 gradient) and of dy h2 (w3 gradient)
        const float dy = dys[r];
        for (int c = quarter * 2; c < quarter * 2 + 2; ++c) {
            float v[32], gb[32], gw[32];
            tc_ld32(trow + H + c * 32, v);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int j = c * 32 + e;
                const float h = fmaxf(v[e] + b2s[j], 0.f);
                gb[e] = h > 0.f ? dy * w3s[j] : 0.f;
                gw[e] = dy * h;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    pk[e] = pack2(__float2bfloat16_rn(gb[q * 8 + 2 * e]), __float2bfloat16_rn(gb[q * 8 + 2 * e + 1]));
                *reinterpret_cast<uint4*>(A.dh2 + (long)row * H + c * 32 + q * 8) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            colb[rb * H + c * 32 + lane] = warp_transpose_sum(gb, lane);
            colw[rb * H + c * 32 + lane] = warp_transpose_sum(gw, lane);
        }
        __syncthreads();
        // this tile's partial sums, row blocks in order
        float* pt = A.part + (long)tile * kPart;
        for (int j = tid; j < H; j += TC_THREADS) {
            pt[H + j] = ((colb[j] + colb[H + j]) + colb[2 * H + j]) + colb[3 * H + j];
            pt[2 * H + j] = ((colw[j] + colw[H + j]) + colw[2 * H + j]) + colw[3 * H + j];
        }
        if (tid == 0) {
            float sd = 0.f, sq = 0.f;
            for (int q = 0; q < TC_ROWS; ++q) {
                sd += dys[q];
                sq += rqs[q];
            }
            pt[3 * H] = sd;
            pt[3 * H + 1] = sq;
        }
        // the next tile rewrites dys, rqs, colb, colw and the tensor memory only after every thread is done
        tc_sync();
    }
    if (!ok) atomicOr(status, 1);
    tc_drain_dealloc(s_m3, tbase, 512, status, warp, tid);
}

// dh1 = (dh2 W2) [h1 > 0] over 128-row tiles: W2^T staged once (operand B
// with N = output column i, K = j), the tile's dh2 as operand A; per 32-row
// block the column sums of dh1 (b1 gradient) into the tile's partials.
constexpr size_t kTbSmem = kTcW2 + kTcH1 + 4 * H * sizeof(float) + 64;

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_train_bwd_tc(TrainArgs A, int* status, long long wait_ns)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* W2t = smem;             // [i][j] canonical K-major (K = j)
    unsigned char* D2s = W2t + kTcW2;      // [r][j] canonical K-major
    float* colb = reinterpret_cast<float*>(D2s + kTcH1);  // [4][H]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(colb + 4 * H);  // MMA, drain
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int r = (warp & 3) * 32 + lane, quarter = warp >> 2, rb = warp & 3;
    const uint32_t s_base = smem_u32(smem), s_m1 = smem_u32(mbar), s_m3 = smem_u32(mbar + 1);
    if (warp == 0) tc_alloc(tslot, 256);
    if (tid == 0) {
        mbar_init(s_m1);
        mbar_init(s_m3);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // W2^T: element (i, j) = W2[j][i]; each thread gathers 8 consecutive j of one i
    for (int q = tid; q < H * H / 8; q += TC_THREADS) {
        const int i = q % H, j8 = q / H;
        uint32_t pk[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) pk[e] = pack2(A.w2[(j8 * 8 + 2 * e) * H + i], A.w2[(j8 * 8 + 2 * e + 1) * H + i]);
        *reinterpret_cast<uint4*>(W2t + kmajor_off(i, j8 * 8, H)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) |
                           ((uint32_t)(TC_ROWS >> 4) << 24);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_sync();
    const uint32_t tbase = *tslot;
    const uint32_t trow = tbase + ((uint32_t)(rb * 32) << 16);
    bool ok = true;
    uint32_t ph1 = 0;
    const int ntiles = A.Bpad / TC_ROWS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row = tile * TC_ROWS + r;
        for (int k8 = quarter * 8; k8 < quarter * 8 + 8; ++k8)  // this thread's row, a quarter of the 32 chunks
            *reinterpret_cast<uint4*>(D2s + kmajor_off(r, k8 * 8, H)) =
                *reinterpret_cast<const uint4*>(A.dh2 + (long)row * H + k8 * 8);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
        if (tid == 0) {
            for (int s = 0; s < H / 16; ++s)
                tc_mma(tbase, tc_smem_desc(s_base + (uint32_t)kTcW2 + s * 256, 128, (H / 8) * 128),
                       tc_smem_desc(s_base + s * 256, 128, (H / 8) * 128), idesc, s > 0);
            tc_commit(s_m1);
        }
        ok = tc_wait(s_m1, ph1, wait_ns) && ok;
        ph1 ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const bool all_ok = __syncthreads_and(ok) != 0;
        for (int c = quarter * 2; c < quarter * 2 + 2; ++c) {
            float v[32];
            tc_ld32(trow + c * 32, v);
            const uint4* hp = reinterpret_cast<const uint4*>(A.h1 + (long)row * H + c * 32);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 hu = hp[q];
                const uint32_t hw[4] = {hu.x, hu.y, hu.z, hu.w};
                uint32_t pk[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float h0 = __bfloat162float(__ushort_as_bfloat16((unsigned short)(hw[e] & 0xffffu)));
                    const float h1v = __bfloat162float(__ushort_as_bfloat16((unsigned short)(hw[e] >> 16)));
                    float& a0 = v[q * 8 + 2 * e];
                    float& a1 = v[q * 8 + 2 * e + 1];
                    a0 = (all_ok && h0 > 0.f) ? a0 : 0.f;
                    a1 = (all_ok && h1v > 0.f) ? a1 : 0.f;
                    pk[e] = pack2(__float2bfloat16_rn(a0), __float2bfloat16_rn(a1));
                }
                *reinterpret_cast<uint4*>(A.dh1 + (long)row * H + c * 32 + q * 8) =
                    make_uint4(pk[0], pk[1], pk[2], pk[3]);
            }
            colb[rb * H + c * 32 + lane] = warp_transpose_sum(v, lane);
        }
        __syncthreads();
        float* pt = A.part + (long)tile * kPart;
        for (int j = tid; j < H; j += TC_THREADS)
            pt[j] = ((colb[j] + colb[H + j]) + colb[2 * H + j]) + colb[3 * H + j];
        tc_sync();
    }
    if (!ok) atomicOr(status, 1);
    tc_drain_dealloc(s_m3, tbase, 256, status, warp, tid);
}

// Weight gradients on the tensor cores: dW2 = dh2^T h1 (N = 256) and dW1 =
// dh1^T x_hat (N = 32), each in two 128-row halves (j), with the batch as
// the K dimension.  The batch's 64-row chunks are split over `nsplit` CTAs
// per half (CTA mt * nsplit + sp: half mt & 1 of dW2 for mt < 2, of dW1
// otherwise; split sp); each CTA accumulates its chunks in tensor memory and
// writes its partial block (to the gradient itself when nsplit == 1, else to
// scratch, summed in split order by k_mlp_wgrad_reduce).  Chunks are staged
// by 8 x 8 blocks: eight 16-byte row loads, transposed in registers, stored
// as eight 16-byte rows of the canonical K-major layout.  The last CTA sums
// the per-tile partials (biases, w3, loss) in tile order.  128 threads:
// thread r reads tensor-memory lane r.
constexpr int WG_CHUNK = 64;
constexpr size_t kWgSmem = (size_t)TC_ROWS * WG_CHUNK * 2 + (size_t)H * WG_CHUNK * 2 + 64;
constexpr size_t kWgBlock = (size_t)H * H + (size_t)H * KIN;  // floats of one split's partial dW2 and dW1

// 8 x 8 BF16 block transpose: rows in[k] (8 elements each) -> out[e] = column e.
__device__ __forceinline__ void transpose8x8(const uint4 (&in)[8], uint4 (&out)[8])
{
    uint32_t w[8][4];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        w[k][0] = in[k].x; w[k][1] = in[k].y; w[k][2] = in[k].z; w[k][3] = in[k].w;
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const uint32_t sel = (e & 1) ? 0x7632u : 0x5410u;  // high or low halves of two words
        const int c = e >> 1;
        out[e] = make_uint4(__byte_perm(w[0][c], w[1][c], sel), __byte_perm(w[2][c], w[3][c], sel),
                            __byte_perm(w[4][c], w[5][c], sel), __byte_perm(w[6][c], w[7][c], sel));
    }
}

__global__ void __launch_bounds__(128, 1) k_mlp_wgrad_tc(TrainArgs A, float* scratch, int nsplit, int* status,
                                                         long long wait_ns)
{
    const int tid = threadIdx.x, warp = tid >> 5;
    if ((int)blockIdx.x == 4 * nsplit) {
        const int ntiles = A.Bpad / TC_ROWS;
        for (int c = tid; c < kPart; c += blockDim.x) {
            float sum = 0.f;
            for (int t = 0; t < ntiles; ++t) sum += A.part[(long)t * kPart + c];
            if (c < H) A.grad[A.o.b1 + c] = sum;
            else if (c < 2 * H) A.grad[A.o.b2 + c - H] = sum;
            else if (c < 3 * H) A.grad[A.o.w3 + c - 2 * H] = sum;
            else if (c == 3 * H) A.grad[A.o.b3] = sum;
            else *A.loss += sum * A.loss_scale;
        }
        return;
    }
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* As = smem;                                   // [128 j][64 rows]
    unsigned char* Bs = As + (size_t)TC_ROWS * WG_CHUNK * 2;     // [N][64 rows]
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Bs + (size_t)H * WG_CHUNK * 2);  // MMA, drain
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int mt = (int)blockIdx.x / nsplit, sp = (int)blockIdx.x % nsplit;
    const bool w1part = mt >= 2;
    const int j0 = (mt & 1) * TC_ROWS;
    const int N = w1part ? KIN : H;
    const bf16* Asrc = w1part ? A.dh1 : A.dh2;  // [rows][H]
    const bf16* Bsrc = w1part ? A.xh : A.h1;    // [rows][N]
    const uint32_t ncols = w1part ? 32u : 256u;
    const int nchunks = A.Bpad / WG_CHUNK;
    const int c0 = (int)((long)sp * nchunks / nsplit), c1 = (int)((long)(sp + 1) * nchunks / nsplit);
    const uint32_t s_base = smem_u32(smem), s_m1 = smem_u32(mbar), s_m3 = smem_u32(mbar + 1);
    if (warp == 0) tc_alloc(tslot, ncols);
    if (tid == 0) {
        mbar_init(s_m1);
        mbar_init(s_m3);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
                           ((uint32_t)(TC_ROWS >> 4) << 24);
    tc_sync();
    const uint32_t tbase = *tslot;
    bool ok = true;
    uint32_t ph1 = 0;
    for (int ch = c0; ch < c1; ++ch) {
        const long rc = (long)ch * WG_CHUNK;
        // A: element (m, k) = Asrc[rc + k][j0 + m]: 16 x 8 blocks of 8 x 8, one per thread
        {
            const int m8 = tid & 15, k8 = tid >> 4;
            uint4 in[8], out[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                in[k] = *reinterpret_cast<const uint4*>(Asrc + (rc + k8 * 8 + k) * H + j0 + m8 * 8);
            transpose8x8(in, out);
#pragma unroll
            for (int e = 0; e < 8; ++e) *reinterpret_cast<uint4*>(As + kmajor_off(m8 * 8 + e, k8 * 8, WG_CHUNK)) = out[e];
        }
        // B: element (n, k) = Bsrc[rc + k][n]: (N / 8) x 8 blocks
        for (int q = tid; q < (N / 8) * (WG_CHUNK / 8); q += 128) {
            const int n8 = q % (N / 8), k8 = q / (N / 8);
            uint4 in[8], out[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                in[k] = *reinterpret_cast<const uint4*>(Bsrc + (rc + k8 * 8 + k) * N + n8 * 8);
            transpose8x8(in, out);
#pragma unroll
            for (int e = 0; e < 8; ++e) *reinterpret_cast<uint4*>(Bs + kmajor_off(n8 * 8 + e, k8 * 8, WG_CHUNK)) = out[e];
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc_sync();
        if (tid == 0) {
            for (int s = 0; s < WG_CHUNK / 16; ++s)
                tc_mma(tbase, tc_smem_desc(s_base + s * 256, 128, (WG_CHUNK / 8) * 128),
                       tc_smem_desc(s_base + (uint32_t)(TC_ROWS * WG_CHUNK * 2) + s * 256, 128, (WG_CHUNK / 8) * 128),
                       idesc, (ch > c0 || s > 0) ? 1 : 0);
            tc_commit(s_m1);
        }
        ok = tc_wait(s_m1, ph1, wait_ns) && ok;  // the chunk's operands are rewritten only after its MMAs
        ph1 ^= 1u;
        tc_sync();
    }
    const bool all_ok = __syncthreads_and(ok) != 0;
    const bool any = c1 > c0;  // a split with no chunk contributes zeros
    // thread r holds row j0 + r of the block in tensor-memory lane r
    const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);
    const int j = j0 + tid;
    float* dst = nsplit == 1 ? nullptr : scratch + (size_t)sp * kWgBlock;
    for (int c = 0; c < N / 32; ++c) {
        float v[32];
        if (any) tc_ld32(trow + c * 32, v);
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const int col = c * 32 + e;
            const float g = (all_ok && any) ? v[e] : 0.f;
            if (dst) {
                if (w1part) dst[(size_t)H * H + j * KIN + col] = g;
                else dst[j * H + col] = g;
            } else if (w1part) {
                if (col < A.nin) A.grad[A.o.w1 + j * A.nin + col] = g;
            } else {
                A.grad[A.o.w2 + j * H + col] = g;
            }
        }
    }
    if (!ok) atomicOr(status, 1);
    tc_drain_dealloc(s_m3, tbase, ncols, status, warp, tid);
}

// The split partials of dW2 and dW1 summed in split order into the gradient.
__global__ void k_mlp_wgrad_reduce(const float* __restrict__ scratch, int nsplit, Offs o, int nin, float* grad)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int)kWgBlock) return;
    float sum = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) sum += scratch[(size_t)sp * kWgBlock + p];
    if (p < H * H) {
        grad[o.w2 + p] = sum;
    } else {
        const int q = p - H * H, j = q / KIN, col = q % KIN;
        if (col < nin) grad[o.w1 + j * nin + col] = sum;
    }
}

uint64_t splitmix64(uint64_t& s)
{
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct adg_mlp {
    int device = 0;
    int nin = 0;
    Offs o{};
    float* theta = nullptr;  // FP32 master parameters [n]
    float* m = nullptr;      // Adam moments [n]
    float* v = nullptr;
    float* grad = nullptr;   // [n]
    float* loss = nullptr;   // device scratch [1]
    bf16* w1 = nullptr;      // [H][KIN], zero beyond nin
    bf16* w2 = nullptr;      // [H][H]
    bf16* w3 = nullptr;      // [H]
    Norm nm{};
    long step = 0;
    void* act = nullptr;     // training activations
    size_t act_bytes = 0;
    int* idx = nullptr;      // fit(): permutation of the training rows
    size_t idx_n = 0;
    float* eloss = nullptr;  // fit(): loss per epoch
    size_t eloss_n = 0;
    int engine = ADG_MLP_TCGEN05;  // forward pass engine
    int* status = nullptr;   // device: bit 0 set when a bounded wait of the tcgen05 forward expired
    long long wait_ns = kTcWaitNs;  // bound of each wait of the tcgen05 forward on its MMAs
};

namespace {

int mlp_fail(adg_ctx* ctx, cudaError_t e)
{
    (void)ctx;
    return e == cudaErrorMemoryAllocation ? ADG_ENOMEM : ADG_ECUDA;
}

#define MCK(call)                                      \
    do {                                               \
        cudaError_t _e = (call);                       \
        if (_e != cudaSuccess) return mlp_fail(ctx, _e); \
    } while (0)

cudaError_t sync_bf16(cudaStream_t st, adg_mlp* M)
{
    k_mlp_adam<<<(M->o.n + 255) / 256, 256, 0, st>>>(M->theta, M->m, M->v, M->grad, M->o, M->nin, 0, 0.f, 0.f, 0.f,
                                                     M->w1, M->w2, M->w3);
    return cudaGetLastError();
}

ActArgs act_args(const adg_mlp* M, const float* x, int B)
{
    ActArgs a{};
    a.theta = M->theta;
    a.w1 = M->w1;
    a.w2 = M->w2;
    a.w3 = M->w3;
    a.o = M->o;
    a.nin = M->nin;
    a.nm = M->nm;
    a.x = x;
    a.B = B;
    return a;
}

unsigned act_blocks(int B, int device)
{
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
    const int ntiles = (B + TR - 1) / TR;
    return (unsigned)std::max(1, std::min(ntiles, nsm));
}

// The same gradient on the tcgen05 engine: forward with dh2, dh1, weight
// gradients (three launches over 128-row tiles; see k_mlp_train_fwd_tc).
int backprop_tc(adg_ctx* ctx, adg_mlp* M, cudaStream_t st, const float* x, const float* t, const int* idx, int B,
                float* loss, float loss_scale)
{
    const int Bpad = (B + TC_ROWS - 1) / TC_ROWS * TC_ROWS;
    const int ntiles = Bpad / TC_ROWS;
    const size_t act_b = sizeof(bf16) * (size_t)Bpad * (KIN + 3 * H);
    // the weight gradient's K (batch) split: about one CTA per SM over the four row halves
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, M->device);
    const int nsplit = std::max(1, std::min(Bpad / WG_CHUNK, nsm / 4));
    const size_t part_b = sizeof(float) * (size_t)ntiles * kPart;
    const size_t need = act_b + part_b + (nsplit > 1 ? sizeof(float) * (size_t)nsplit * kWgBlock : 0);
    if (need > M->act_bytes) {
        MCK(cudaStreamSynchronize(st));
        if (M->act) cudaFree(M->act);
        M->act = nullptr;
        M->act_bytes = 0;
        MCK(cudaMalloc(&M->act, need));
        M->act_bytes = need;
    }
    float* scratch = (float*)((char*)M->act + act_b + part_b);
    TrainArgs a{};
    a.theta = M->theta;
    a.w1 = M->w1;
    a.w2 = M->w2;
    a.w3 = M->w3;
    a.o = M->o;
    a.nin = M->nin;
    a.nm = M->nm;
    a.x = x;
    a.t = t;
    a.idx = idx;
    a.B = B;
    a.Bpad = Bpad;
    a.inv_B = 1.f / (float)B;
    a.xh = (bf16*)M->act;
    a.h1 = a.xh + (size_t)Bpad * KIN;
    a.dh2 = a.h1 + (size_t)Bpad * H;
    a.dh1 = a.dh2 + (size_t)Bpad * H;
    a.part = (float*)((char*)M->act + act_b);
    a.grad = M->grad;
    a.loss = loss;
    a.loss_scale = loss_scale;
    const unsigned grid = (unsigned)std::min(ntiles, nsm);
    MCK(cudaFuncSetAttribute(k_mlp_train_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTfSmem));
    MCK(cudaFuncSetAttribute(k_mlp_train_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTbSmem));
    MCK(cudaFuncSetAttribute(k_mlp_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem));
    k_mlp_train_fwd_tc<<<grid, TC_THREADS, kTfSmem, st>>>(a, M->status, M->wait_ns);
    MCK(cudaGetLastError());
    k_mlp_train_bwd_tc<<<grid, TC_THREADS, kTbSmem, st>>>(a, M->status, M->wait_ns);
    MCK(cudaGetLastError());
    k_mlp_wgrad_tc<<<4 * nsplit + 1, 128, kWgSmem, st>>>(a, scratch, nsplit, M->status, M->wait_ns);
    MCK(cudaGetLastError());
    if (nsplit > 1) {
        k_mlp_wgrad_reduce<<<(unsigned)((kWgBlock + 255) / 256), 256, 0, st>>>(scratch, nsplit, M->o, M->nin, M->grad);
        MCK(cudaGetLastError());
    }
    ctx->stats.kernel_launches += nsplit > 1 ? 4 : 3;
    return ADG_OK;
}

// Gradient of the batch loss into M->grad (and the loss, scaled, into *loss).
int backprop(adg_ctx* ctx, adg_mlp* M, cudaStream_t st, const float* x, const float* t, const int* idx, int B,
             float* loss, float loss_scale)
{
    if (M->engine == ADG_MLP_TCGEN05) return backprop_tc(ctx, M, st, x, t, idx, B, loss, loss_scale);
    const int Bpad = (B + TR - 1) / TR * TR;
    const size_t act_b = sizeof(bf16) * (size_t)Bpad * (KIN + 3 * H);
    const size_t need = act_b + sizeof(float) * (size_t)(Bpad / TR) * kPart;
    if (need > M->act_bytes) {
        MCK(cudaStreamSynchronize(st));
        if (M->act) cudaFree(M->act);
        M->act = nullptr;
        M->act_bytes = 0;
        MCK(cudaMalloc(&M->act, need));
        M->act_bytes = need;
    }
    bf16* xh = (bf16*)M->act;
    bf16* h1 = xh + (size_t)Bpad * KIN;
    bf16* dh2 = h1 + (size_t)Bpad * H;
    bf16* dh1 = dh2 + (size_t)Bpad * H;
    float* part = (float*)((char*)M->act + act_b);
    ActArgs a = act_args(M, x, B);
    a.t = t;
    a.idx = idx;
    a.xh = xh;
    a.h1 = h1;
    a.dh2 = dh2;
    a.dh1 = dh1;
    a.part = part;
    a.inv_B = 1.f / (float)B;
    MCK(cudaFuncSetAttribute(k_mlp_act<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kActSmem));
    k_mlp_act<true><<<act_blocks(B, M->device), 256, kActSmem, st>>>(a);
    MCK(cudaGetLastError());
    WgradArgs w{};
    w.dh2 = dh2;
    w.h1 = h1;
    w.dh1 = dh1;
    w.xh = xh;
    w.Bpad = Bpad;
    w.nin = M->nin;
    w.o = M->o;
    w.grad = M->grad;
    w.part = part;
    w.loss = loss;
    w.loss_scale = loss_scale;
    k_mlp_wgrad<<<21, 256, 0, st>>>(w);
    MCK(cudaGetLastError());
    ctx->stats.kernel_launches += 2;
    return ADG_OK;
}

int adam_step(adg_ctx* ctx, adg_mlp* M, cudaStream_t st, float lr)
{
    M->step += 1;
    const float c1 = (float)(1.0 / (1.0 - pow(0.9, (double)M->step)));
    const float c2 = (float)(1.0 / (1.0 - pow(0.999, (double)M->step)));
    k_mlp_adam<<<(M->o.n + 255) / 256, 256, 0, st>>>(M->theta, M->m, M->v, M->grad, M->o, M->nin, 1, lr, c1, c2,
                                                     M->w1, M->w2, M->w3);
    MCK(cudaGetLastError());
    ctx->stats.kernel_launches += 1;
    return ADG_OK;
}

}  // namespace

extern "C" {

int adg_mlp_nparams(int nin)
{
    if (nin < 1 || nin > ADG_MLP_NIN_MAX) return ADG_EINVAL;
    return offsets(nin).n;
}

int adg_mlp_create(adg_ctx* ctx, int nin, uint64_t seed, adg_mlp** out)
{
    if (!ctx || !out || nin < 1 || nin > ADG_MLP_NIN_MAX) return ADG_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ADG_ECUDA;
    adg_mlp* M = new (std::nothrow) adg_mlp();
    if (!M) return ADG_ENOMEM;
    M->device = ctx->device;
    M->nin = nin;
    M->o = offsets(nin);
    const size_t n = (size_t)M->o.n;
    for (int k = 0; k < KIN; ++k) {
        M->nm.mu[k] = 0.f;
        M->nm.sigma[k] = 1.f;
    }
    M->nm.mu_y = 0.f;
    M->nm.sigma_y = 1.f;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMalloc(&M->theta, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&M->m, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&M->v, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&M->grad, sizeof(float) * n);
    if (e == cudaSuccess) e = cudaMalloc(&M->loss, sizeof(float) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&M->w1, sizeof(bf16) * H * KIN);
    if (e == cudaSuccess) e = cudaMalloc(&M->w2, sizeof(bf16) * H * H);
    if (e == cudaSuccess) e = cudaMalloc(&M->w3, sizeof(bf16) * H);
    if (e == cudaSuccess) e = cudaMalloc(&M->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(M->status, 0, sizeof(int), ctx->stream);
    // He-uniform initial weights (bound sqrt(6 / fan_in)), zero biases
    std::vector<float> th(n, 0.f);
    uint64_t s = seed;
    auto uni = [&](float bound) { return bound * (2.f * (float)((splitmix64(s) >> 40) * (1.0 / 16777216.0)) - 1.f); };
    for (int i = 0; i < H * nin; ++i) th[M->o.w1 + i] = uni(sqrtf(6.f / nin));
    for (int i = 0; i < H * H; ++i) th[M->o.w2 + i] = uni(sqrtf(6.f / H));
    for (int i = 0; i < H; ++i) th[M->o.w3 + i] = uni(sqrtf(6.f / H));
    cudaStream_t st = ctx->stream;
    if (e == cudaSuccess) e = cudaMemcpyAsync(M->theta, th.data(), sizeof(float) * n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->m, 0, sizeof(float) * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->v, 0, sizeof(float) * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->w1, 0, sizeof(bf16) * H * KIN, st);
    if (e == cudaSuccess) e = sync_bf16(st, M);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        adg_mlp_destroy(M);
        return e == cudaErrorMemoryAllocation ? ADG_ENOMEM : ADG_ECUDA;
    }
    ctx->stats.h2d_bytes += (int64_t)(sizeof(float) * n);
    *out = M;
    return ADG_OK;
}

int adg_mlp_destroy(adg_mlp* M)
{
    if (!M) return ADG_EINVAL;
    cudaSetDevice(M->device);
    cudaFree(M->theta);
    cudaFree(M->m);
    cudaFree(M->v);
    cudaFree(M->grad);
    cudaFree(M->loss);
    cudaFree(M->w1);
    cudaFree(M->w2);
    cudaFree(M->w3);
    cudaFree(M->act);
    cudaFree(M->idx);
    cudaFree(M->eloss);
    cudaFree(M->status);
    delete M;
    return ADG_OK;
}

int adg_mlp_get_params(adg_ctx* ctx, const adg_mlp* M, float* out)
{
    if (!ctx || !M || !out) return ADG_EINVAL;
    MCK(cudaSetDevice(M->device));
    MCK(cudaMemcpyAsync(out, M->theta, sizeof(float) * M->o.n, cudaMemcpyDeviceToHost, ctx->stream));
    MCK(cudaStreamSynchronize(ctx->stream));
    ctx->stats.d2h_bytes += (int64_t)(sizeof(float) * M->o.n);
    return ADG_OK;
}

int adg_mlp_set_params(adg_ctx* ctx, adg_mlp* M, const float* in)
{
    if (!ctx || !M || !in) return ADG_EINVAL;
    MCK(cudaSetDevice(M->device));
    cudaStream_t st = ctx->stream;
    MCK(cudaMemcpyAsync(M->theta, in, sizeof(float) * M->o.n, cudaMemcpyHostToDevice, st));
    MCK(cudaMemsetAsync(M->m, 0, sizeof(float) * M->o.n, st));
    MCK(cudaMemsetAsync(M->v, 0, sizeof(float) * M->o.n, st));
    MCK(sync_bf16(st, M));
    MCK(cudaStreamSynchronize(st));
    M->step = 0;
    ctx->stats.h2d_bytes += (int64_t)(sizeof(float) * M->o.n);
    ctx->stats.kernel_launches += 1;
    return ADG_OK;
}

int adg_mlp_set_norm(adg_mlp* M, const float* mu, const float* sigma, float mu_y, float sigma_y)
{
    if (!M || !mu || !sigma || !(sigma_y > 0.f)) return ADG_EINVAL;
    for (int k = 0; k < M->nin; ++k)
        if (!(sigma[k] > 0.f)) return ADG_EINVAL;
    for (int k = 0; k < KIN; ++k) {
        M->nm.mu[k] = k < M->nin ? mu[k] : 0.f;
        M->nm.sigma[k] = k < M->nin ? sigma[k] : 1.f;
    }
    M->nm.mu_y = mu_y;
    M->nm.sigma_y = sigma_y;
    return ADG_OK;
}

int adg_mlp_forward(adg_ctx* ctx, const adg_mlp* M, const float* x, int B, float* y)
{
    if (!ctx || !M || B < 0 || (B > 0 && (!x || !y))) return ADG_EINVAL;
    if (B == 0) return ADG_OK;
    MCK(cudaSetDevice(M->device));
    ActArgs a = act_args(M, x, B);
    a.y = y;
    if (M->engine == ADG_MLP_TCGEN05) {
        MCK(cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
        int nsm = 148;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, M->device);
        const int ntiles = (B + TC_ROWS - 1) / TC_ROWS;
        k_mlp_fwd_tc<<<(unsigned)std::min(ntiles, nsm), TC_THREADS, kTcSmem, ctx->stream>>>(a, M->status,
                                                                                            M->wait_ns);
    } else {
        MCK(cudaFuncSetAttribute(k_mlp_act<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kActSmem));
        k_mlp_act<false><<<act_blocks(B, M->device), 256, kActSmem, ctx->stream>>>(a);
    }
    MCK(cudaGetLastError());
    ctx->stats.kernel_launches += 1;
    return ADG_OK;
}

int adg_mlp_set_engine(adg_mlp* M, int engine)
{
    if (!M || (engine != ADG_MLP_MMA_SYNC && engine != ADG_MLP_TCGEN05)) return ADG_EINVAL;
    M->engine = engine;
    return ADG_OK;
}

int adg_mlp_set_wait_ns(adg_mlp* M, long long ns)
{
    if (!M || ns < 0) return ADG_EINVAL;
    M->wait_ns = ns;
    return ADG_OK;
}

int adg_mlp_check(adg_ctx* ctx, adg_mlp* M)
{
    if (!ctx || !M) return ADG_EINVAL;
    MCK(cudaSetDevice(M->device));
    int h = 0;
    MCK(cudaMemcpyAsync(&h, M->status, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    MCK(cudaMemsetAsync(M->status, 0, sizeof(int), ctx->stream));
    MCK(cudaStreamSynchronize(ctx->stream));
    return h ? ADG_ETIMEOUT : ADG_OK;
}

int adg_mlp_grad(adg_ctx* ctx, adg_mlp* M, const float* x, const float* t, const int* idx, int B, float* grad,
                 float* loss)
{
    if (!ctx || !M || !x || !t || !grad || B <= 0) return ADG_EINVAL;
    MCK(cudaSetDevice(M->device));
    cudaStream_t st = ctx->stream;
    MCK(cudaMemsetAsync(M->loss, 0, sizeof(float), st));
    const int rc = backprop(ctx, M, st, x, t, idx, B, M->loss, 1.f / (float)B);
    if (rc != ADG_OK) return rc;
    MCK(cudaMemcpyAsync(grad, M->grad, sizeof(float) * M->o.n, cudaMemcpyDeviceToDevice, st));
    if (loss) MCK(cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    return ADG_OK;
}

int adg_mlp_train_step(adg_ctx* ctx, adg_mlp* M, const float* x, const float* t, const int* idx, int B, float lr,
                       float* loss)
{
    if (!ctx || !M || !x || !t || B <= 0 || !(lr >= 0.f)) return ADG_EINVAL;
    MCK(cudaSetDevice(M->device));
    cudaStream_t st = ctx->stream;
    MCK(cudaMemsetAsync(M->loss, 0, sizeof(float), st));
    int rc = backprop(ctx, M, st, x, t, idx, B, M->loss, 1.f / (float)B);
    if (rc != ADG_OK) return rc;
    rc = adam_step(ctx, M, st, lr);
    if (rc != ADG_OK) return rc;
    if (loss) MCK(cudaMemcpyAsync(loss, M->loss, sizeof(float), cudaMemcpyDeviceToDevice, st));
    return ADG_OK;
}

int adg_mlp_fit(adg_ctx* ctx, adg_mlp* M, const float* x, const float* t, int n, int batch, int epochs, float lr,
                uint64_t seed, float* epoch_loss)
{
    if (!ctx || !M || !x || !t || n <= 0 || batch <= 0 || epochs < 0 || !(lr >= 0.f)) return ADG_EINVAL;
    MCK(cudaSetDevice(M->device));
    cudaStream_t st = ctx->stream;
    if ((size_t)n > M->idx_n) {
        MCK(cudaStreamSynchronize(st));
        cudaFree(M->idx);
        M->idx = nullptr;
        M->idx_n = 0;
        MCK(cudaMalloc(&M->idx, sizeof(int) * n));
        M->idx_n = (size_t)n;
    }
    if ((size_t)epochs > M->eloss_n) {
        MCK(cudaStreamSynchronize(st));
        cudaFree(M->eloss);
        M->eloss = nullptr;
        M->eloss_n = 0;
        MCK(cudaMalloc(&M->eloss, sizeof(float) * std::max(epochs, 1)));
        M->eloss_n = (size_t)epochs;
    }
    if (epochs == 0) return ADG_OK;
    MCK(cudaMemsetAsync(M->eloss, 0, sizeof(float) * epochs, st));
    // one permutation per epoch (Fisher-Yates on a splitmix64 stream), uploaded
    // before the epoch's steps; the host buffer is pinned so the copy is async
    int* perm = nullptr;
    MCK(cudaMallocHost(&perm, sizeof(int) * (size_t)n * 2));
    uint64_t s = seed;
    int rc = ADG_OK;
    for (int ep = 0; ep < epochs && rc == ADG_OK; ++ep) {
        int* hp = perm + (size_t)(ep & 1) * n;
        if (ep >= 2) {
            // the copy that used this half two epochs ago has finished once the stream passed it
            if (cudaStreamSynchronize(st) != cudaSuccess) {
                rc = ADG_ECUDA;
                break;
            }
        }
        for (int i = 0; i < n; ++i) hp[i] = i;
        for (int i = n - 1; i > 0; --i) {
            const int j = (int)(splitmix64(s) % (uint64_t)(i + 1));
            std::swap(hp[i], hp[j]);
        }
        if (cudaMemcpyAsync(M->idx, hp, sizeof(int) * n, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = ADG_ECUDA;
            break;
        }
        ctx->stats.h2d_bytes += (int64_t)(sizeof(int) * n);
        for (int b0 = 0; b0 < n && rc == ADG_OK; b0 += batch) {
            const int B = std::min(batch, n - b0);
            rc = backprop(ctx, M, st, x, t, M->idx + b0, B, M->eloss + ep, 1.f / (float)n);
            if (rc == ADG_OK) rc = adam_step(ctx, M, st, lr);
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (rc == ADG_OK && e != cudaSuccess) rc = ADG_ECUDA;
    if (rc == ADG_OK && epoch_loss) {
        e = cudaMemcpy(epoch_loss, M->eloss, sizeof(float) * epochs, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) rc = ADG_ECUDA;
    }
    cudaFreeHost(perm);
    return rc;
}

}  // extern "C"
