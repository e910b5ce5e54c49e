// tcgen05 GEMM with fused epilogues for the surrogate MLP.
//
// C (M x N, fp32, in TMEM) = A (M x K) * B (N x K)^T with A and B bf16 in the
// canonical K-major layout (tc05.cuh).  One CTA of 128 threads owns a
// 128-row tile of C and the whole N (<= 256): the 1-D bulk-copy engine moves
// the A and B tiles of one K chunk (<= 256) into shared memory, one thread
// issues K/16 tcgen05.mma instructions into a TMEM accumulator of N fp32
// columns, and after tcgen05.commit every thread reads its row of the
// accumulator (thread t <-> TMEM lane t) and runs the epilogue.
#pragma once

#include "tc05.cuh"

namespace mlpk {

enum Mode : int {
    FWD_HIDDEN = 0,  // z = acc + bias -> Zf; x = silu(z) -> Xc (M x N canonical) and XTc (N x M canonical)
    FWD_OUT = 1,     // y = acc + bias -> Yf (fp32 row-major)
    BWD_DX = 2,      // dz = acc * silu'(Zprev) -> Zf (fp32), Xc (M x N canonical), XTc (N x M canonical)
    BWD_DW = 3,      // acc -> Yf (fp32 row-major, M x N)
};

struct GemmArgs {
    const uint8_t* A;   // canonical bf16, M x K
    const uint8_t* B;   // canonical bf16, N x K
    int M, N, K;        // M % 128 == 0, N in {16, 32, ..., 256} (multiple of 16), K % 16 == 0
    int mode;
    const float* bias;  // [N] (FWD modes)
    const float* zprev; // [M][N] fp32 (BWD_DX)
    float* Zf;          // [M][N] fp32 out
    float* Yf;          // [M][N] fp32 out
    uint8_t* Xc;        // canonical bf16 M x N out
    uint8_t* XTc;       // canonical bf16 N x M out
    int* err;           // set to 1 if a bounded wait expired
};

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void put_bf16(uint8_t* base, int64_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

constexpr int KC = 256;  // K chunk held in shared memory

__global__ void __launch_bounds__(128, 1) k_gemm_tc(GemmArgs g) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar_load, bar_mma;
    __shared__ uint32_t tmem_slot;
    __shared__ int ok_flag;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int mt = blockIdx.x;
    const int N = g.N;
    const int kc = g.K < KC ? g.K : KC;
    uint8_t* sA = smem;                                  // 128 x kc
    uint8_t* sB = smem + (size_t)128 * kc * 2;           // N x kc
    uint32_t ncols = 32;
    while ((int)ncols < N) ncols <<= 1;
    if (tid == 0) {
        tc05::mbar_init(&bar_load, 1);
        tc05::mbar_init(&bar_mma, 1);
        tc05::fence_barrier_init();
        ok_flag = 1;
    }
    if (warp == 0) tc05::tmem_alloc(&tmem_slot, ncols);
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const uint32_t idesc = tc05::idesc_bf16_f32(128, N);
    const int nchunks = g.K / kc;
    for (int ch = 0; ch < nchunks; ++ch) {
        const uint32_t par = (uint32_t)(ch & 1);
        if (tid == 0 && ok_flag) {
            // A tile: rows [128 mt, 128 mt + 128), K chunk ch.  In the canonical
            // layout a row group's K chunk is contiguous (kc/8 core matrices),
            // so copy 16 row groups of kc*16 bytes each; same for B's N/8 groups.
            const uint32_t grp = (uint32_t)kc * 16;
            const uint32_t bytes = grp * (16 + N / 8);
            tc05::mbar_expect_tx(&bar_load, bytes);
            const int64_t srow = (int64_t)g.K * 16;      // bytes per row group in global
            for (int r = 0; r < 16; ++r)
                tc05::bulk_g2s(sA + (size_t)r * grp, g.A + (int64_t)(16 * mt + r) * srow + (int64_t)ch * grp, grp,
                               &bar_load);
            for (int r = 0; r < N / 8; ++r)
                tc05::bulk_g2s(sB + (size_t)r * grp, g.B + (int64_t)r * srow + (int64_t)ch * grp, grp, &bar_load);
            if (!tc05::mbar_wait(&bar_load, par)) {
                ok_flag = 0;
                atomicExch(g.err, 1);
            } else {
                tc05::fence_after_sync();
                for (int kk = 0; kk < kc / 16; ++kk) {
                    const uint64_t ad = tc05::smem_desc(sA + kk * 256, 128, (uint32_t)kc * 16);
                    const uint64_t bd = tc05::smem_desc(sB + kk * 256, 128, (uint32_t)kc * 16);
                    tc05::mma_bf16(tmem, ad, bd, idesc, (ch > 0 || kk > 0) ? 1u : 0u);
                }
                tc05::mma_commit(&bar_mma);
                if (!tc05::mbar_wait(&bar_mma, par)) {
                    ok_flag = 0;
                    atomicExch(g.err, 1);
                }
            }
        }
        __syncthreads();  // shared tiles are free again / MMA done
    }
    tc05::fence_after_sync();
    if (ok_flag) {
        const int row = 128 * mt + tid;
        const uint32_t tbase = tmem + ((uint32_t)(32 * warp) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tc05::tmem_ld16(tbase + (uint32_t)c0, v);
            if (g.mode == FWD_HIDDEN || g.mode == FWD_OUT) {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] += g.bias[c0 + i];
            }
            if (g.mode == FWD_OUT || g.mode == BWD_DW) {
                float4* o = reinterpret_cast<float4*>(g.Yf + (int64_t)row * N + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                continue;
            }
            float x[16];
            if (g.mode == FWD_HIDDEN) {
                float4* o = reinterpret_cast<float4*>(g.Zf + (int64_t)row * N + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
#pragma unroll
                for (int i = 0; i < 16; ++i) x[i] = silu_f(v[i]);
            } else {  // BWD_DX
                const float* zp = g.zprev + (int64_t)row * N + c0;
#pragma unroll
                for (int i = 0; i < 16; ++i) x[i] = v[i] * silu_grad_f(zp[i]);
                float4* o = reinterpret_cast<float4*>(g.Zf + (int64_t)row * N + c0);
#pragma unroll
                for (int i = 0; i < 4; ++i) o[i] = make_float4(x[4 * i], x[4 * i + 1], x[4 * i + 2], x[4 * i + 3]);
            }
            // canonical (M x N): two 16-byte chunks of 8 columns
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                __align__(16) __nv_bfloat16 b8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) b8[i] = __float2bfloat16_rn(x[8 * h + i]);
                *reinterpret_cast<uint4*>(g.Xc + tc05::canon_off(row, c0 + 8 * h, N)) =
                    *reinterpret_cast<const uint4*>(b8);
            }
            // canonical transposed (N x M)
#pragma unroll
            for (int i = 0; i < 16; ++i) put_bf16(g.XTc, tc05::canon_off(c0 + i, row, g.M), x[i]);
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc05::tmem_dealloc(tmem, ncols);
}

}  // namespace mlpk
