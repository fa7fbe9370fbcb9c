// Constitutive surrogate network: 16 -> 128 -> 128 -> 128 -> 16, SiLU after the hidden
// layers.  Layer l maps a row x to z = x W_l^T + b_l (W_l is out x in, row-major).
//
// Tensor cores: mma.sync.m16n8k16 with BF16 operands and FP32 accumulation.  A warp owns
// 16 rows of the batch; its A fragments come from row-major activations (K contiguous),
// its B fragments from row-major weights W[n][k] (K contiguous), which is the "col"
// operand layout of the instruction.  Training keeps FP32 master weights (Adam) and BF16
// copies of W and W^T for the GEMMs.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace tl {

constexpr int kIn = 16, kHid = 128, kOut = 16;
// packed parameters: W0 (128x16), b0, W1 (128x128), b1, W2 (128x128), b2, W3 (16x128), b3
constexpr int kOffW0 = 0, kOffB0 = kOffW0 + kHid * kIn, kOffW1 = kOffB0 + kHid, kOffB1 = kOffW1 + kHid * kHid,
              kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid, kOffW3 = kOffB2 + kHid,
              kOffB3 = kOffW3 + kOut * kHid, kNumParams = kOffB3 + kOut;
constexpr int kNumWeights = kHid * kIn + 2 * kHid * kHid + kOut * kHid;  // bf16 weights (no biases)

// Derivative of SiLU for the backward pass (FP32, through the hardware tanh:
// sigma(z) = (1 + tanh(z / 2)) / 2, SiLU'(z) = sigma (1 + z (1 - sigma))).
__device__ __forceinline__ float tanh_fast(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = fmaf(0.5f, tanh_fast(0.5f * z), 0.5f);
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void mma_bf16_16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// The activations of a hidden layer as the next layer reads them: SiLU of the two pre-activations
// (lo, hi) in packed bf16 arithmetic, SiLU(z) = h + h tanh(h) with h = z / 2: one conversion, one
// multiply, one tanh and one fused multiply-add (single rounding) for two values.  Training and
// both inference paths use this same function.
__device__ __forceinline__ uint32_t silu_bf16x2(float lo, float hi) {
    uint32_t x, h, t, y;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(x) : "f"(hi), "f"(lo));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(h) : "r"(x), "r"(0x3F003F00u));  // (0.5, 0.5)
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(y) : "r"(h), "r"(t), "r"(h));
    return y;
}

// ------------------------------------------------------------------ generic GEMM (training)
// C[M x N] = A[M x K] * B[N x K]^T (+ bias), A and B bf16 row-major (K contiguous).
// M a multiple of 16, N of 8, K of 16.  One warp computes a 16 x 32 tile.
// EPI 0: C (f32) only; 1: also Zout = C (f32) and Aout = bf16(SiLU(C)); 2: Aout = bf16(C).
template <int EPI>
__global__ void k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B, const float *bias,
                            float *C, __nv_bfloat16 *Aout) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int tiles_n = (N + 31) / 32;
    const int tm = warp / tiles_n, tn = warp % tiles_n;
    if (tm * 16 >= M) return;
    const int r0 = tm * 16, n0 = tn * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[j][q] = 0.0f;
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        const __nv_bfloat16 *ar0 = A + (size_t)(r0 + g) * K + k0 + 2 * t;
        const __nv_bfloat16 *ar1 = A + (size_t)(r0 + g + 8) * K + k0 + 2 * t;
        a[0] = *reinterpret_cast<const uint32_t *>(ar0);
        a[1] = *reinterpret_cast<const uint32_t *>(ar1);
        a[2] = *reinterpret_cast<const uint32_t *>(ar0 + 8);
        a[3] = *reinterpret_cast<const uint32_t *>(ar1 + 8);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int nn = n0 + 8 * j;
            if (nn >= N) break;
            const __nv_bfloat16 *br = B + (size_t)(nn + g) * K + k0 + 2 * t;
            uint32_t b[2] = {*reinterpret_cast<const uint32_t *>(br), *reinterpret_cast<const uint32_t *>(br + 8)};
            mma_bf16_16816(acc[j], a, b);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++) {
        const int nn = n0 + 8 * j;
        if (nn >= N) break;
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int row = r0 + g + 8 * h;
            const int col = nn + 2 * t;
            float v0 = acc[j][2 * h], v1 = acc[j][2 * h + 1];
            if (bias) {
                v0 += bias[col];
                v1 += bias[col + 1];
            }
            C[(size_t)row * N + col] = v0;
            C[(size_t)row * N + col + 1] = v1;
            if (EPI == 1) {
                *reinterpret_cast<uint32_t *>(Aout + (size_t)row * N + col) = silu_bf16x2(v0, v1);
            } else if (EPI == 2) {
                *reinterpret_cast<uint32_t *>(Aout + (size_t)row * N + col) = pack_bf16(v0, v1);
            }
        }
    }
}

// out[c * rows + r] = in[r * cols + c] (bf16)
__global__ void k_transpose_bf16(int rows, int cols, const __nv_bfloat16 *in, __nv_bfloat16 *out) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int r = by + y, c = bx + threadIdx.x;
        if (r < rows && c < cols) tile[y][threadIdx.x] = in[(size_t)r * cols + c];
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int c = bx + y, r = by + threadIdx.x;
        if (r < rows && c < cols) out[(size_t)c * rows + r] = tile[threadIdx.x][y];
    }
}

__global__ void k_f32_to_bf16(int64_t n, const float *in, __nv_bfloat16 *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = __float2bfloat16_rn(in[i]);
}

// normalised rows: out = (x - mean) / std (row length 16), as f32 and bf16
__global__ void k_normalize(int64_t rows, const float *x, const float *mean, const float *stdv, float *outf,
                            __nv_bfloat16 *outb) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * 16) return;
    const int c = (int)(i & 15);
    const float v = (x[i] - mean[c]) / stdv[c];
    if (outf) outf[i] = v;
    if (outb) outb[i] = __float2bfloat16_rn(v);
}

// dL/dout of the mean squared error (sum over B x 16 elements / (B * 16)); loss partials per block
__global__ void k_mse_grad(int64_t n, const float *out, const float *y, float *dout, __nv_bfloat16 *dout_b,
                           float *loss_acc) {
    __shared__ float red[32];
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    float e2 = 0.0f;
    if (i < n) {
        const float e = out[i] - y[i];
        const float d = 2.0f * e / (float)n;
        dout[i] = d;
        dout_b[i] = __float2bfloat16_rn(d);
        e2 = e * e;
    }
    for (int o = 16; o > 0; o >>= 1) e2 += __shfl_xor_sync(0xffffffffu, e2, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e2;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w];
        atomicAdd(loss_acc, s / (float)n);
    }
}

// dZ = dA * SiLU'(Z) (f32 in, bf16 out)
__global__ void k_silu_back(int64_t n, const float *dA, const float *Z, __nv_bfloat16 *dZ) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dZ[i] = __float2bfloat16_rn(dA[i] * silu_grad_f(Z[i]));
}
__global__ void k_silu_back_f32(int64_t n, const float *dA, const float *Z, float *dZ) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dZ[i] = dA[i] * silu_grad_f(Z[i]);
}

// db[c] = sum over rows of dZ[r][c]
__global__ void k_colsum(int rows, int cols, const float *dZ, float *db) {
    const int c = blockIdx.x;
    float s = 0.0f;
    for (int r = threadIdx.x; r < rows; r += blockDim.x) s += dZ[(size_t)r * cols + c];
    __shared__ float red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        db[c] = t;
    }
}

// Adam (bias-corrected) on the FP32 master parameters
__global__ void k_adam(int n, float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ dataset statistics
// per-column sum, sum of squares, min and max of rows x 16 values (FP64 sums)
__global__ void k_col_stats(int64_t rows, const float *x, double *sum, double *sum2, float *mn, float *mx) {
    const int c = blockIdx.y;
    double s = 0.0, s2 = 0.0;
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[r * 16 + c];
        s += v;
        s2 += (double)v * v;
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sum[c], s);
        atomicAdd(&sum2[c], s2);
        // float min / max through the ordered-int trick (works for any sign)
        int ilo = __float_as_int(lo), ihi = __float_as_int(hi);
        if (ilo < 0) ilo = 0x80000000 - ilo;
        if (ihi < 0) ihi = 0x80000000 - ihi;
        atomicMin(reinterpret_cast<int *>(&mn[c]), ilo);
        atomicMax(reinterpret_cast<int *>(&mx[c]), ihi);
    }
}

// ------------------------------------------------------------------ block-level forward (inference)
// Parameters of the network as the fused kernel reads them: bf16 weights (packed W0 W1 W2 W3),
// f32 biases, normalisation of inputs / outputs and the envelope of normalised inputs.
struct SurrogateDev {
    const __nv_bfloat16 *W;  // kNumWeights, order W0, W1, W2, W3
    const float *bias;       // b0 (128), b1, b2, b3 (16)
    const float *in_mean, *in_std, *out_mean, *out_std, *env_lo, *env_hi;  // 16 each
    int enabled;
    int scope;  // 0 every J2 particle, 1 J2 particles whose trial state yields
};

// Shared-memory layout of one block's forward pass over 128 rows: the weights and biases, the
// block's normalised inputs and its outputs; hidden activations stay in registers.  Rows are
// padded (24 and 136 bf16, 48 and 272 bytes) so that the 8 row addresses of an ldmatrix
// phase fall on distinct 16-byte bank groups.
constexpr int kLd16 = kIn + 8, kLd128 = kHid + 8;
struct MlpSmem {
    __nv_bfloat16 W0[kHid][kLd16];
    __nv_bfloat16 W1[kHid][kLd128];
    __nv_bfloat16 W2[kHid][kLd128];
    __nv_bfloat16 W3[kOut][kLd128];
    float bias[3 * kHid + kOut];
    __nv_bfloat16 X[128][kLd16];  // normalised inputs
    float Y[128][kOut + 1];       // outputs
};

__device__ __forceinline__ void mlp_load_params(MlpSmem &sm, const SurrogateDev &s) {
    // global: W0 (128 x 16), W1 (128 x 128), W2 (128 x 128), W3 (16 x 128), unpadded
    const uint4 *w = reinterpret_cast<const uint4 *>(s.W);
    for (int i = threadIdx.x; i < kHid * 2; i += blockDim.x)  // W0: 2 uint4 per row
        reinterpret_cast<uint4 *>(&sm.W0[i >> 1][0])[i & 1] = w[i];
    w += kHid * kIn / 8;
    for (int i = threadIdx.x; i < kHid * 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(&sm.W1[i >> 4][0])[i & 15] = w[i];
    w += kHid * kHid / 8;
    for (int i = threadIdx.x; i < kHid * 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(&sm.W2[i >> 4][0])[i & 15] = w[i];
    w += kHid * kHid / 8;
    for (int i = threadIdx.x; i < kOut * 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(&sm.W3[i >> 4][0])[i & 15] = w[i];
    for (int i = threadIdx.x; i < 3 * kHid + kOut; i += blockDim.x) sm.bias[i] = s.bias[i];
}

// Four 8 x 8 bf16 matrices from shared memory; lane l gives the address of row l % 8 of
// matrix l / 8 and receives in r[q] the pair (row l / 4, columns 2 (l % 4), +1) of matrix q.
__device__ __forceinline__ void ldmatrix_x4(uint32_t r[4], const void *p) {
    const unsigned addr = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// B fragments of two neighbouring n8 tiles (output columns n0 .. n0 + 15) and one k16 tile
// (input columns k0 .. k0 + 15) of W[n][k]: b[0], b[1] for columns n0 .. n0 + 7, b[2], b[3]
// for n0 + 8 .. n0 + 15.
__device__ __forceinline__ void load_b_pair(uint32_t b[4], const __nv_bfloat16 *W, int ldw, int n0, int k0) {
    const int lane = threadIdx.x & 31;
    ldmatrix_x4(b, W + (n0 + (lane & 7) + ((lane >> 4) << 3)) * ldw + k0 + ((lane >> 3) & 1) * 8);
}

// One hidden layer for a warp's 16 rows with the activations in registers: hin holds the A
// fragments of the input (KT tiles of 16 columns), hout receives those of SiLU(in W^T + b)
// (128 columns = 8 tiles).  The accumulator of n8 tiles 2 kk and 2 kk + 1 is, element for
// element, the A fragment of k tile kk of the next layer.
template <int KT>
__device__ __forceinline__ void mlp_layer_regs(const uint32_t (&hin)[KT][4], const __nv_bfloat16 *W, int ldw,
                                               const float *bias, uint32_t (&hout)[8][4]) {
    const int t = threadIdx.x & 3;
    float acc[16][4];
#pragma unroll
    for (int j = 0; j < 16; j++)
#pragma unroll
        for (int q = 0; q < 4; q++) acc[j][q] = 0.0f;
#pragma unroll
    for (int kk = 0; kk < KT; kk++)
#pragma unroll
        for (int jj = 0; jj < 8; jj++) {
            uint32_t b[4];
            load_b_pair(b, W, ldw, 16 * jj, 16 * kk);
            mma_bf16_16816(acc[2 * jj], hin[kk], b);
            mma_bf16_16816(acc[2 * jj + 1], hin[kk], b + 2);
        }
#pragma unroll
    for (int kk = 0; kk < 8; kk++) {
        const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
        const float *a0 = acc[2 * kk], *a1 = acc[2 * kk + 1];
        hout[kk][0] = silu_bf16x2(a0[0] + bias[c0], a0[1] + bias[c0 + 1]);
        hout[kk][1] = silu_bf16x2(a0[2] + bias[c0], a0[3] + bias[c0 + 1]);
        hout[kk][2] = silu_bf16x2(a1[0] + bias[c1], a1[1] + bias[c1 + 1]);
        hout[kk][3] = silu_bf16x2(a1[2] + bias[c1], a1[3] + bias[c1 + 1]);
    }
}

// Forward pass of rows [r0, r0 + 16) of sm.X into sm.Y by one warp.
__device__ __forceinline__ void mlp_forward_rows(MlpSmem &sm, int r0) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    uint32_t x[1][4], h1[8][4], h2[8][4];
    ldmatrix_x4(x[0], &sm.X[r0 + (lane & 15)][(lane >> 4) * 8]);
    mlp_layer_regs<1>(x, &sm.W0[0][0], kLd16, sm.bias, h1);
    mlp_layer_regs<8>(h1, &sm.W1[0][0], kLd128, sm.bias + kHid, h2);
    mlp_layer_regs<8>(h2, &sm.W2[0][0], kLd128, sm.bias + 2 * kHid, h1);
    float acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
#pragma unroll
    for (int kk = 0; kk < 8; kk++) {
        uint32_t b[4];
        load_b_pair(b, &sm.W3[0][0], kLd128, 0, 16 * kk);
        mma_bf16_16816(acc[0], h1[kk], b);
        mma_bf16_16816(acc[1], h1[kk], b + 2);
    }
    const float *b3 = sm.bias + 3 * kHid;
#pragma unroll
    for (int j = 0; j < 2; j++)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int row = r0 + g + 8 * h, col = 8 * j + 2 * t;
            sm.Y[row][col] = acc[j][2 * h] + b3[col];
            sm.Y[row][col + 1] = acc[j][2 * h + 1] + b3[col + 1];
        }
}

// Forward pass of the block's 128 rows of sm.X into sm.Y; warp w owns rows [32 w, 32 w + 32).
// Called by the 4 warps of a 128-thread block; every warp only touches its own rows.
__device__ __forceinline__ void mlp_forward_block(MlpSmem &sm) {
    const int w = threadIdx.x >> 5;
    mlp_forward_rows(sm, 32 * w);
    mlp_forward_rows(sm, 32 * w + 16);
    __syncwarp();
}

// Standalone forward over n rows of raw inputs (normalised / denormalised inside), 128 rows per block.
__global__ void __launch_bounds__(128) k_mlp_forward(int64_t n, const float *x, float *y, SurrogateDev s,
                                                     int *outside) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpSmem &sm = *reinterpret_cast<MlpSmem *>(smraw);
    mlp_load_params(sm, s);
    const int64_t r = blockIdx.x * 128LL + threadIdx.x;
    int out_env = 0;
    for (int c = 0; c < kIn; c++) {
        float v = 0.0f;
        if (r < n) {
            v = (x[r * kIn + c] - s.in_mean[c]) / s.in_std[c];
            out_env |= (v < s.env_lo[c] || v > s.env_hi[c]);
        }
        sm.X[threadIdx.x][c] = __float2bfloat16_rn(v);
    }
    __syncthreads();
    mlp_forward_block(sm);
    __syncthreads();
    if (r < n) {
        for (int c = 0; c < kOut; c++) y[r * kOut + c] = sm.Y[threadIdx.x][c] * s.out_std[c] + s.out_mean[c];
        if (outside) outside[r] = out_env;
    }
}

}  // namespace tl
