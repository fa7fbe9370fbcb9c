// Forward pass of the surrogate network on the 5th-generation tensor cores: tcgen05.mma with
// operands in shared memory and the FP32 accumulator in tensor memory (TMEM).
//
// A group of 128 threads runs tiles of 128 rows.  Each layer is one or eight MMAs of
// M = 128, K = 16 (N = 128, or 16 for the output layer) issued by one thread; the accumulator
// (128 lanes = rows, N columns) is read back with tcgen05.ld, each thread getting the row of its
// own lane, which takes the bias and SiLU and goes back to shared memory in bf16 as the next
// layer's A operand.  The output layer leaves each thread the 16 outputs of its own row.
//
// Operand layout (no swizzle, K-major): core matrices of 8 rows x 16 bytes (8 bf16); element
// (row r, column k) of an R-row operand sits at (k / 8) * (R * 16) + r * 16 + (k % 8) * 2.  The
// descriptor's leading byte offset is the step between core matrices along K (R * 16 bytes),
// its stride byte offset the step between groups of 8 rows (128 bytes).
#pragma once
#include "mlp.cuh"

namespace tl {

// Four groups of 4 warps share a CTA of 512 threads and one copy of the weights; each group runs
// its own tiles with its own operand buffers, barrier and 128 TMEM columns, and synchronises on
// its own named barrier, so the groups' MMAs and epilogues interleave on the SM.
constexpr int kTcGroups = 4;
constexpr int kTcCols = 128;  // TMEM columns per group (the widest accumulator)
struct __align__(16) MlpTcGroup {
    uint8_t H[16 * 2048];  // A of layers 1-3: 128 rows x 128 bf16
    uint8_t X[2 * 2048];   // A of layer 0: 128 rows x 16 bf16
};
struct __align__(16) MlpTcSmem {
    uint8_t W1[16 * 2048];  // B operands W[n][k]: 128 x 128
    uint8_t W2[16 * 2048];
    uint8_t W0[2 * 2048];   // 128 x 16
    uint8_t W3[16 * 256];   // 16 x 128
    MlpTcGroup grp[kTcGroups];
    float bias[3 * kHid + kOut];
    unsigned long long mbar[kTcGroups];
    unsigned tmem;
};

__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory descriptor: start address, leading / stride byte offsets (all >> 4), the fixed
// constant 0b001 in bits 46-48, base offset 0, relative leading offset, no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(const void *p, unsigned lbo, unsigned sbo) {
    return (uint64_t)((smem_addr(p) & 0x3FFFF) >> 4) | ((uint64_t)((lbo & 0x3FFFF) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFF) >> 4) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N / 8, M / 16.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(unsigned tmem, uint64_t da, uint64_t db, uint32_t idesc, unsigned acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                 "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// Wait for completion `parity` of the barrier for about a second at most; true when it completed.
__device__ __forceinline__ bool tc_wait(unsigned long long *mbar, unsigned parity) {
    const long long t0 = clock64();
    while (true) {
        unsigned ok;
        asm volatile("{\n.reg .pred q;\nmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\nselp.u32 %0, 1, 0, q;\n}\n"
                     : "=r"(ok)
                     : "r"(smem_addr(mbar)), "r"(parity));
        if (ok) return true;
        if (clock64() - t0 > 2000000000LL) return false;
    }
}

__device__ __forceinline__ void tc_ld32(uint32_t v[32], unsigned taddr) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tc_ld16(uint32_t v[16], unsigned taddr) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// Barrier of the 128 threads of group g (named barrier 1 + g), plain and with an OR / AND vote.
__device__ __forceinline__ void group_sync(int g) { asm volatile("bar.sync %0, 128;\n" ::"r"(1 + g) : "memory"); }
__device__ __forceinline__ bool group_or(int g, bool v) {
    unsigned r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.or.pred p, %2, 128, q;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(r)
                 : "r"((unsigned)v), "r"(1 + g)
                 : "memory");
    return r != 0;
}
__device__ __forceinline__ bool group_and(int g, bool v) {
    unsigned r;
    asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbar.red.and.pred p, %2, 128, q;\nselp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(r)
                 : "r"((unsigned)v), "r"(1 + g)
                 : "memory");
    return r != 0;
}

// Weights and biases into shared memory (from the packed bf16 W0 | W1 | W2 | W3, row-major [out][in]),
// the groups' barriers, and the TMEM columns of all groups (allocated by warp 0).  Ends with a CTA
// barrier.
__device__ __forceinline__ void mlp_tc_setup(MlpTcSmem &sm, const SurrogateDev &s) {
    const __nv_bfloat16 *w0 = s.W, *w1 = w0 + kHid * kIn, *w2 = w1 + kHid * kHid, *w3 = w2 + kHid * kHid;
    for (int i = threadIdx.x; i < kHid * 2; i += blockDim.x) {
        const int n = i >> 1, g = i & 1;
        *reinterpret_cast<uint4 *>(sm.W0 + g * 2048 + n * 16) = *reinterpret_cast<const uint4 *>(w0 + n * kIn + 8 * g);
    }
    for (int i = threadIdx.x; i < kHid * 16; i += blockDim.x) {
        const int n = i >> 4, g = i & 15;
        *reinterpret_cast<uint4 *>(sm.W1 + g * 2048 + n * 16) = *reinterpret_cast<const uint4 *>(w1 + n * kHid + 8 * g);
        *reinterpret_cast<uint4 *>(sm.W2 + g * 2048 + n * 16) = *reinterpret_cast<const uint4 *>(w2 + n * kHid + 8 * g);
    }
    for (int i = threadIdx.x; i < kOut * 16; i += blockDim.x) {
        const int n = i >> 4, g = i & 15;
        *reinterpret_cast<uint4 *>(sm.W3 + g * 256 + n * 16) = *reinterpret_cast<const uint4 *>(w3 + n * kHid + 8 * g);
    }
    for (int i = threadIdx.x; i < 3 * kHid + kOut; i += blockDim.x) sm.bias[i] = s.bias[i];
    if (threadIdx.x == 0) {
        for (int g = 0; g < kTcGroups; g++) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&sm.mbar[g])));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&sm.tmem)),
                     "r"(kTcCols * kTcGroups));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
}

// Row r of group g's layer-0 operand: the normalised inputs of that row.
__device__ __forceinline__ void mlp_tc_put_row(MlpTcSmem &sm, int g, int r, const float xn[16]) {
    uint4 lo, hi;
    lo.x = pack_bf16(xn[0], xn[1]);
    lo.y = pack_bf16(xn[2], xn[3]);
    lo.z = pack_bf16(xn[4], xn[5]);
    lo.w = pack_bf16(xn[6], xn[7]);
    hi.x = pack_bf16(xn[8], xn[9]);
    hi.y = pack_bf16(xn[10], xn[11]);
    hi.z = pack_bf16(xn[12], xn[13]);
    hi.w = pack_bf16(xn[14], xn[15]);
    *reinterpret_cast<uint4 *>(sm.grp[g].X + r * 16) = lo;
    *reinterpret_cast<uint4 *>(sm.grp[g].X + 2048 + r * 16) = hi;
}

// The four layers on group g's tile (all 128 threads of the group call it; r = thread in the
// group).  Thread r gets in y the 16 outputs of row r before denormalisation.  phase counts the
// group barrier's completions.  Returns false (group-uniform) when a wait ran out; the last MMA
// may then still be in flight.
__device__ __forceinline__ bool mlp_tc_tile(MlpTcSmem &sm, int g, int r, unsigned &phase, float y[16]) {
    const unsigned tcol = sm.tmem + (unsigned)(kTcCols * g);
    const unsigned tlane = tcol + ((unsigned)(32 * (r >> 5)) << 16);
    MlpTcGroup &gr = sm.grp[g];
    constexpr uint32_t id128 = tc_idesc_bf16(128, 128), id16 = tc_idesc_bf16(128, 16);
#pragma unroll 1
    for (int layer = 0; layer < 4; layer++) {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        group_sync(g);
        if (r == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            if (layer == 0) {
                tc_mma(tcol, tc_sdesc(gr.X, 2048, 128), tc_sdesc(sm.W0, 2048, 128), id128, 0u);
            } else {
                const uint8_t *B = layer == 1 ? sm.W1 : layer == 2 ? sm.W2 : sm.W3;
                const unsigned bl = layer == 3 ? 256u : 2048u;
                const uint32_t id = layer == 3 ? id16 : id128;
#pragma unroll
                for (int kk = 0; kk < 8; kk++)
                    tc_mma(tcol, tc_sdesc(gr.H + kk * 4096, 2048, 128), tc_sdesc(B + kk * 2 * bl, bl, 128), id,
                           kk > 0 ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_addr(&sm.mbar[g])));
        }
        const bool done = tc_wait(&sm.mbar[g], phase & 1u);
        if (!group_and(g, done)) return false;
        phase++;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        if (layer < 3) {
            const float *b = sm.bias + layer * kHid;
#pragma unroll 1
            for (int c0 = 0; c0 < kHid; c0 += 32) {
                uint32_t v[32];
                tc_ld32(v, tlane + (unsigned)c0);
#pragma unroll
                for (int q8 = 0; q8 < 4; q8++) {
                    uint32_t p[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int c = c0 + 8 * q8 + 2 * q;
                        p[q] = silu_bf16x2(__uint_as_float(v[8 * q8 + 2 * q]) + b[c],
                                           __uint_as_float(v[8 * q8 + 2 * q + 1]) + b[c + 1]);
                    }
                    *reinterpret_cast<uint4 *>(gr.H + ((c0 >> 3) + q8) * 2048 + r * 16) = make_uint4(p[0], p[1], p[2], p[3]);
                }
            }
        } else {
            uint32_t v[16];
            tc_ld16(v, tlane);
            const float *b = sm.bias + 3 * kHid;
#pragma unroll
            for (int c = 0; c < 16; c++) y[c] = __uint_as_float(v[c]) + b[c];
        }
    }
    return true;
}

// Release the CTA's TMEM (warp 0) once every group is done, after a last bounded wait by a group
// whose MMA may still be in flight.
__device__ __forceinline__ void mlp_tc_finish(MlpTcSmem &sm, int g, unsigned phase, bool pending) {
    if (pending) tc_wait(&sm.mbar[g], phase & 1u);
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(sm.tmem), "r"(kTcCols * kTcGroups));
    }
}

// Standalone forward over n rows of raw inputs (normalised / denormalised inside): CTAs of
// 4 x 128 threads, each group persistent over tiles of 128 rows.  flags[0] counts groups whose
// tensor-core wait ran out.
__global__ void __launch_bounds__(128 * kTcGroups, 1) k_mlp_forward_tc(int64_t n, const float *x, float *y,
                                                                      SurrogateDev s, int *outside, int *flags) {
    extern __shared__ __align__(16) unsigned char smraw[];
    MlpTcSmem &sm = *reinterpret_cast<MlpTcSmem *>(smraw);
    mlp_tc_setup(sm, s);
    const int g = threadIdx.x >> 7, r = threadIdx.x & 127;
    unsigned phase = 0;
    bool pending = false;
    const int64_t ntiles = (n + 127) / 128;
    for (int64_t tile = (int64_t)blockIdx.x * kTcGroups + g; tile < ntiles; tile += (int64_t)gridDim.x * kTcGroups) {
        const int64_t row = tile * 128 + r;
        float xn[16];
        int out_env = 0;
        for (int c = 0; c < kIn; c++) {
            float v = 0.0f;
            if (row < n) {
                v = (x[row * kIn + c] - s.in_mean[c]) / s.in_std[c];
                out_env |= (v < s.env_lo[c] || v > s.env_hi[c]);
            }
            xn[c] = v;
        }
        mlp_tc_put_row(sm, g, r, xn);
        float yr[16];
        if (!mlp_tc_tile(sm, g, r, phase, yr)) {
            if (r == 0) atomicAdd(flags, 1);
            pending = true;
            break;
        }
        if (row < n) {
            for (int c = 0; c < kOut; c++) y[row * kOut + c] = yr[c] * s.out_std[c] + s.out_mean[c];
            if (outside) outside[row] = out_env;
        }
    }
    mlp_tc_finish(sm, g, phase, pending);
}

// ------------------------------------------------------------------ training GEMM on tcgen05
// C[M x N] = A[M x K] B[N x K]^T (+ bias), A and B bf16 row-major (K contiguous), as k_gemm_bf16 with the
// same epilogues (EPI 0: C only; 1: also Aout = SiLU(C) in bf16; 2: Aout = bf16(C)).  N is 16 or a
// multiple of 128 up to the grid's reach, K a multiple of 16, M anything.  One CTA of 128 threads per
// output tile of 128 rows x NT = min(128, N - n0) columns: each K stage of up to 128 columns of A and B
// goes to shared memory in the K-major core-matrix layout, one thread issues its K / 16 MMAs
// (M = 128, N = NT, K = 16) into the tile's TMEM accumulator and commits them to the CTA's barrier;
// after the last stage thread r reads row r of the accumulator (tcgen05.ld) into shared memory, from where
// the CTA writes the outputs in runs of consecutive columns.  A
// wait that runs out adds one to flag and ends the tile without output.
constexpr int kGemmKc = 128;
struct __align__(16) GemmTcSmem {
    uint8_t A[kGemmKc / 8 * 2048];  // 128 rows x kGemmKc bf16
    uint8_t B[kGemmKc / 8 * 2048];  // NT rows x kGemmKc bf16
    unsigned long long mbar;
    unsigned tmem;
};
// The epilogue of the tile's columns col0 .. col0 + NC - 1 (k_gemm_bf16's: v = accumulator + bias to C,
// and SiLU(v) or v in bf16 to Aout).  Thread r puts row r's accumulators (v) into shared memory st (pitch
// NC + 1 floats: no bank conflicts either way), then the 128 threads write whole row segments: C and Aout
// are written in runs of consecutive columns.
template <int EPI, int NC>
__device__ __forceinline__ void gemm_tc_out(const uint32_t (&v)[NC], float *st, int m0, int M, int col0, int N,
                                            const float *bias, float *C, __nv_bfloat16 *Aout) {
    const int r = threadIdx.x;
#pragma unroll
    for (int c = 0; c < NC; c++) st[r * (NC + 1) + c] = __uint_as_float(v[c]);
    __syncthreads();
    constexpr int NP = NC / 2;  // column pairs of a row
    for (int e = r; e < 128 * NP; e += 128) {
        const int row = e / NP, cp = e - row * NP, c = 2 * cp, col = col0 + c;
        if (m0 + row >= M) continue;
        const float a0 = st[row * (NC + 1) + c], a1 = st[row * (NC + 1) + c + 1];
        const float v0 = bias ? a0 + bias[col] : a0, v1 = bias ? a1 + bias[col + 1] : a1;
        *reinterpret_cast<float2 *>(C + (size_t)(m0 + row) * N + col) = make_float2(v0, v1);
        if (EPI == 1) *reinterpret_cast<uint32_t *>(Aout + (size_t)(m0 + row) * N + col) = silu_bf16x2(v0, v1);
        else if (EPI == 2) *reinterpret_cast<uint32_t *>(Aout + (size_t)(m0 + row) * N + col) = pack_bf16(v0, v1);
    }
    __syncthreads();
}
template <int EPI>
__global__ void __launch_bounds__(128) k_gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, const __nv_bfloat16 *B,
                                                 const float *bias, float *C, __nv_bfloat16 *Aout, int *flag) {
    extern __shared__ __align__(16) unsigned char smraw[];
    GemmTcSmem &sm = *reinterpret_cast<GemmTcSmem *>(smraw);
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 128, r = threadIdx.x;
    const int NT = min(128, N - n0);
    const unsigned ncols = NT > 32 ? 128u : 32u;
    if (r == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&sm.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
    }
    if (r < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&sm.tmem)),
                     "r"(ncols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const unsigned tmem = sm.tmem;
    const uint32_t idesc = tc_idesc_bf16(128, NT);
    const unsigned lbo_b = (unsigned)NT * 16u;
    unsigned phase = 0;
    bool ok = true;
    for (int k0 = 0; k0 < K && ok; k0 += kGemmKc) {
        const int kc = min(kGemmKc, K - k0), kb8 = kc / 8;
        for (int u = r; u < 128 * kb8; u += 128) {
            const int row = u / kb8, kb = u - row * kb8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m0 + row < M) v = *reinterpret_cast<const uint4 *>(A + (size_t)(m0 + row) * K + k0 + 8 * kb);
            *reinterpret_cast<uint4 *>(sm.A + kb * 2048 + row * 16) = v;
        }
        for (int u = r; u < NT * kb8; u += 128) {
            const int row = u / kb8, kb = u - row * kb8;
            const uint4 v = *reinterpret_cast<const uint4 *>(B + (size_t)(n0 + row) * K + k0 + 8 * kb);
            *reinterpret_cast<uint4 *>(sm.B + kb * lbo_b + row * 16) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        __syncthreads();
        if (r == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            for (int kk = 0; kk < kc / 16; kk++)
                tc_mma(tmem, tc_sdesc(sm.A + kk * 4096, 2048, 128), tc_sdesc(sm.B + kk * 2 * lbo_b, lbo_b, 128), idesc,
                       (k0 > 0 || kk > 0) ? 1u : 0u);
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                smem_addr(&sm.mbar)));
        }
        ok = __syncthreads_and(tc_wait(&sm.mbar, phase & 1u));
        phase++;
        asm volatile("tcgen05.fence::after_thread_sync;\n");
    }
    if (ok) {  // all MMAs are done: the operand buffers hold the output stage
        const unsigned tl = tmem + ((unsigned)(32 * (r >> 5)) << 16);
        float *st = reinterpret_cast<float *>(sm.A);
        if (NT == 16) {
            uint32_t v[16];
            tc_ld16(v, tl);
            gemm_tc_out<EPI, 16>(v, st, m0, M, n0, N, bias, C, Aout);
        } else {
#pragma unroll 1
            for (int c0 = 0; c0 < NT; c0 += 32) {
                uint32_t v[32];
                tc_ld32(v, tl + (unsigned)c0);
                gemm_tc_out<EPI, 32>(v, st, m0, M, n0 + c0, N, bias, C, Aout);
            }
        }
    } else {
        if (r == 0) atomicAdd(flag, 1);
        tc_wait(&sm.mbar, (phase - 1u) & 1u);  // the last MMAs may still be in flight: wait once more (bounded)
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (r < 32) {
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols));
    }
}

}  // namespace tl
