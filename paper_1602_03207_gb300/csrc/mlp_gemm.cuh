// tcgen05 GEMM with fused epilogues for the surrogate MLP.
//
// C (M x N, fp32, in TMEM) = A (M x K) * B (N x K)^T with A and B bf16 in the
// canonical K-major layout (tc05.cuh).  A persistent, warp-specialised kernel:
//   * warp 0 (one thread) moves operands with the 1-D bulk-copy engine into a
//     ring of shared-memory stages, one K chunk (<= 64) of a 128-row A tile per
//     stage; B (the weights, N x K <= 128 KB) is copied once per CTA and stays
//     resident, or, for the weight-gradient GEMM whose K is the batch, a K chunk
//     of B travels with each A chunk;
//   * warp 1 (one thread) issues the tcgen05.mma instructions of each stage
//     into one of two TMEM accumulators of N fp32 columns, and frees the stage
//     with tcgen05.commit when its MMAs complete;
//   * warps 2-9 read the finished accumulator (TMEM lane quarter warp % 4,
//     thread <-> tile row; the two warps of a quarter take one half of the
//     columns each) and run the epilogue while the MMAs of the next tile fill
//     the other accumulator.
// A work item is a 128-row tile and a range of K chunks: the weight-gradient
// GEMM (M = 256, K = batch) splits K over the CTAs and writes fp32 partial
// products that a second kernel sums in a fixed order.  Every mbarrier wait
// is bounded; a wait that expires sets an error flag and makes the other roles
// stop, after which the copies and MMAs already issued are drained and the
// TMEM is freed.
#pragma once

#include "tc05.cuh"

namespace mlpk {

enum Mode : int {
    FWD_HIDDEN = 0,  // z = acc + bias -> Zf; x = silu(z) -> Xc (M x N canonical) and XTc (N x M canonical)
    FWD_OUT = 1,     // y = acc + bias -> Yf (fp32 row-major)
    BWD_DX = 2,      // dz = acc * silu'(Zprev) -> Zf (fp32), Xc (M x N canonical), XTc (N x M canonical)
    BWD_DW = 3,      // acc -> Yf (fp32 row-major, M x N), or a partial product when K is split
    FWD_INFER = 4,   // x = silu(acc + bias) -> Xc only (inference: nothing kept for a backward pass)
};

constexpr int EPI_WARPS = 8;           // two per TMEM lane quarter
constexpr int PIPE_THREADS = 64 + 32 * EPI_WARPS;  // warp 0 copies, warp 1 issues MMAs, the rest run the epilogue
constexpr int PIPE_MAX_STAGES = 8;
constexpr int KCH_MAX = 64;            // K elements per stage
constexpr int EPI_BYTES = EPI_WARPS * 1024;  // per epilogue warp: 16 columns x 32 rows of bf16
constexpr int PIPE_SMEM_MAX = 232448 - 2048;  // dynamic shared memory (the static barriers aside)
constexpr uint32_t RESIDENT_B_MAX = 128 * 1024;

struct GemmArgs {
    const uint8_t* A;   // canonical bf16, M x K
    const uint8_t* B;   // canonical bf16, N x K
    int M, N, K;        // M % 128 == 0, N in {16, 32, ..., 256}, K % kch == 0
    int mode;
    const float* bias;  // [N] (forward modes)
    const float* zprev; // [M][N] fp32 (BWD_DX)
    float* Zf;          // [M][N] fp32 out
    float* Yf;          // [M][N] fp32 out
    uint8_t* Xc;        // canonical bf16 M x N out
    uint8_t* XTc;       // canonical bf16 N x M out
    float* part;        // [nsplit][M][N] fp32 partial products (BWD_DW with nsplit > 1)
    int* err;           // set to 1 if a bounded wait expired
    int kch;            // K elements per stage (16, 32, 48 or 64)
    int nsplit, ksplit; // K chunks split into nsplit ranges of ksplit chunks
    int resident;       // B copied once and kept in shared memory
    int stages;
    uint32_t b_tx;      // resident B: bytes copied (N x K x 2)
    uint32_t b_bytes;   // resident B: shared memory reserved (b_tx rounded up to 1024)
    uint32_t a_bytes;   // A part of a stage: 128 x kch bf16
    uint32_t stage_tx;  // bytes copied into one stage
    uint32_t stage_bytes;
};

// fast reciprocal division: the results are rounded to bf16 (8-bit mantissa) or feed a bf16 GEMM
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = __fdividef(1.0f, 1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

__device__ __forceinline__ void put_bf16(uint8_t* base, int64_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool pwait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
    for (uint32_t i = 0; i < tc05::WAIT_LIMIT; ++i) {
        if (tc05::mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicExch(err, 1);
    return false;
}

// bounded wait used on the way out, to let in-flight copies and MMAs finish
__device__ __forceinline__ void drain_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t i = 0; i < tc05::WAIT_LIMIT; ++i)
        if (tc05::mbar_try_wait(bar, parity)) return;
}

__device__ __forceinline__ void store_f32x16(float* dst, const float (&v)[16]) {
    float4* o = reinterpret_cast<float4*>(dst);
#pragma unroll
    for (int i = 0; i < 4; ++i) o[i] = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
}

__global__ void __launch_bounds__(PIPE_THREADS, 1) k_gemm_tc(GemmArgs g) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[PIPE_MAX_STAGES], empty[PIPE_MAX_STAGES];
    __shared__ __align__(8) uint64_t bfull, tfull[2], tempty[2], drain;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = g.stages, N = g.N;
    const int nch = g.K / g.kch;
    const int n_items = (g.M / 128) * g.nsplit;
    uint32_t ncol = 32;  // TMEM columns of one accumulator
    while ((int)ncol < N) ncol <<= 1;
    uint8_t* sB = smem;
    uint8_t* ring = smem + (g.resident ? g.b_bytes : 0u);
    uint8_t* epi = ring + (size_t)S * g.stage_bytes;
    if (tid == 0) {
        for (int s = 0; s < S; ++s) {
            tc05::mbar_init(&full[s], 1);
            tc05::mbar_init(&empty[s], 1);
        }
        tc05::mbar_init(&bfull, 1);
        for (int a = 0; a < 2; ++a) {
            tc05::mbar_init(&tfull[a], 1);
            tc05::mbar_init(&tempty[a], EPI_WARPS);  // one arrival per epilogue warp
        }
        tc05::mbar_init(&drain, 1);
        tc05::fence_barrier_init();
        abort_flag = 0;
    }
    if (warp == 0) tc05::tmem_alloc(&tmem_slot, 2 * ncol);
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    volatile int* ab = &abort_flag;
    const uint32_t rg_bytes = (uint32_t)g.kch * 16;  // one row group's share of a K chunk
    const int64_t rg_stride = (int64_t)g.K * 16;     // one row group of A or B in global memory

    if (warp == 0) {
        if (lane == 0) {  // ---- producer
            uint32_t issued = 0, lastpar = 0;  // per stage: has a copy been issued, parity of the last one
            if (g.resident) {
                tc05::mbar_expect_tx(&bfull, g.b_tx);
                tc05::bulk_g2s(sB, g.B, g.b_tx, &bfull);
            }
            int64_t it = 0;
            bool ok = true;
            for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x) {
                const int mt = item / g.nsplit, sp = item - mt * g.nsplit;
                const int c0 = sp * g.ksplit, c1 = min(nch, c0 + g.ksplit);
                for (int c = c0; c < c1; ++c, ++it) {
                    const int s = (int)(it % S);
                    const uint32_t use = (uint32_t)(it / S);
                    if (use > 0 && !pwait(&empty[s], (use - 1) & 1u, ab, g.err)) {
                        ok = false;
                        break;
                    }
                    uint8_t* st = ring + (size_t)s * g.stage_bytes;
                    tc05::mbar_expect_tx(&full[s], g.stage_tx);
                    for (int r = 0; r < 16; ++r)
                        tc05::bulk_g2s(st + r * rg_bytes, g.A + (int64_t)(16 * mt + r) * rg_stride + (int64_t)c * rg_bytes,
                                       rg_bytes, &full[s]);
                    if (!g.resident)
                        for (int r = 0; r < N / 8; ++r)
                            tc05::bulk_g2s(st + g.a_bytes + r * rg_bytes,
                                           g.B + (int64_t)r * rg_stride + (int64_t)c * rg_bytes, rg_bytes, &full[s]);
                    issued |= 1u << s;
                    lastpar = (lastpar & ~(1u << s)) | ((use & 1u) << s);
                }
            }
            // every copy issued here lands before the CTA may exit
            for (int s = 0; s < S; ++s)
                if ((issued >> s) & 1u) drain_wait(&full[s], (lastpar >> s) & 1u);
            if (g.resident) drain_wait(&bfull, 0);
        }
    } else if (warp == 1) {
        if (lane == 0) {  // ---- MMA issuer
            const uint32_t idesc = tc05::idesc_bf16_f32(128, N);
            bool ok = !g.resident || pwait(&bfull, 0, ab, g.err);
            int64_t it = 0;
            int lt = 0;
            for (int item = blockIdx.x; ok && item < n_items; item += gridDim.x, ++lt) {
                const int mt = item / g.nsplit, sp = item - mt * g.nsplit;
                (void)mt;
                const int c0 = sp * g.ksplit, c1 = min(nch, c0 + g.ksplit);
                const int acc = lt & 1;
                const uint32_t use = (uint32_t)(lt >> 1);
                if (use > 0 && !pwait(&tempty[acc], (use - 1) & 1u, ab, g.err)) break;
                tc05::fence_after_sync();
                const uint32_t td = tmem + (uint32_t)acc * ncol;
                for (int c = c0; c < c1; ++c, ++it) {
                    const int s = (int)(it % S);
                    if (!pwait(&full[s], (uint32_t)(it / S) & 1u, ab, g.err)) {
                        ok = false;
                        break;
                    }
                    tc05::fence_after_sync();
                    const uint8_t* st = ring + (size_t)s * g.stage_bytes;
                    for (int kk = 0; kk < g.kch / 16; ++kk) {
                        const uint64_t ad = tc05::smem_desc(st + kk * 256, 128, rg_bytes);
                        const uint64_t bd =
                            g.resident ? tc05::smem_desc(sB + (size_t)c * rg_bytes + kk * 256, 128, (uint32_t)rg_stride)
                                       : tc05::smem_desc(st + g.a_bytes + kk * 256, 128, rg_bytes);
                        tc05::mma_bf16(td, ad, bd, idesc, (c > c0 || kk > 0) ? 1u : 0u);
                    }
                    tc05::mma_commit(&empty[s]);  // the stage is free once these MMAs complete
                }
                if (!ok) break;
                tc05::mma_commit(&tfull[acc]);
            }
            tc05::mma_commit(&drain);  // all MMAs issued here complete before the TMEM is freed
            drain_wait(&drain, 0);
        }
    } else {  // ---- epilogue: warps 2..9, TMEM lane quarter warp % 4, column half (warp - 2) / 4
        const int q = warp & 3, half = (warp - 2) >> 2;
        const int ngrp = N / 16, gper = (ngrp + 1) / 2;  // 16-column groups, per half
        const int cbeg = 16 * min(ngrp, half * gper), cend = 16 * min(ngrp, (half + 1) * gper);
        uint8_t* tb = epi + (warp - 2) * 1024;
        int lt = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x, ++lt) {
            const int mt = item / g.nsplit, sp = item - mt * g.nsplit;
            const int acc = lt & 1;
            int okw = lane == 0 ? (int)pwait(&tfull[acc], (uint32_t)(lt >> 1) & 1u, ab, g.err) : 0;
            okw = __shfl_sync(0xffffffffu, okw, 0);
            if (!okw) break;
            tc05::fence_after_sync();
            const int rowbase = 128 * mt + 32 * q, row = rowbase + lane;
            const uint32_t taddr = tmem + (uint32_t)acc * ncol + ((uint32_t)(32 * q) << 16);
            for (int c0 = cbeg; c0 < cend; c0 += 16) {
                float v[16];
                tc05::tmem_ld16(taddr + (uint32_t)c0, v);
                if (g.mode == BWD_DW) {
                    float* dst = g.nsplit > 1 ? g.part + ((int64_t)sp * g.M + row) * N + c0 : g.Yf + (int64_t)row * N + c0;
                    store_f32x16(dst, v);
                    continue;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i)
                    if (g.mode != BWD_DX) v[i] += g.bias[c0 + i];
                if (g.mode == FWD_OUT) {
                    store_f32x16(g.Yf + (int64_t)row * N + c0, v);
                    continue;
                }
                float x[16];
                if (g.mode == BWD_DX) {
                    const float4* zp = reinterpret_cast<const float4*>(g.zprev + (int64_t)row * N + c0);
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float4 z = zp[i];
                        x[4 * i] = v[4 * i] * silu_grad_f(z.x);
                        x[4 * i + 1] = v[4 * i + 1] * silu_grad_f(z.y);
                        x[4 * i + 2] = v[4 * i + 2] * silu_grad_f(z.z);
                        x[4 * i + 3] = v[4 * i + 3] * silu_grad_f(z.w);
                    }
                    store_f32x16(g.Zf + (int64_t)row * N + c0, x);
                } else {
                    if (g.mode == FWD_HIDDEN) store_f32x16(g.Zf + (int64_t)row * N + c0, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) x[i] = silu_f(v[i]);
                }
                // canonical (M x N): two 16-byte pieces of 8 columns; lanes 8j..8j+7 fill 128 bytes
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    __align__(16) __nv_bfloat16 b8[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) b8[i] = __float2bfloat16_rn(x[8 * h + i]);
                    *reinterpret_cast<uint4*>(g.Xc + tc05::canon_off(row, c0 + 8 * h, N)) =
                        *reinterpret_cast<const uint4*>(b8);
                }
                if (g.mode == FWD_INFER) continue;
                // canonical transposed (N x M), through shared memory: 8 consecutive rows of one
                // column are 16 contiguous bytes there
                __nv_bfloat16* T = reinterpret_cast<__nv_bfloat16*>(tb);
#pragma unroll
                for (int i = 0; i < 16; ++i) T[i * 32 + lane] = __float2bfloat16_rn(x[i]);
                __syncwarp();
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int cid = lane + 32 * h, col = cid >> 2, grp = cid & 3;
                    const uint4 val = *reinterpret_cast<const uint4*>(tb + col * 64 + grp * 16);
                    *reinterpret_cast<uint4*>(g.XTc + tc05::canon_off(c0 + col, rowbase + 8 * grp, g.M)) = val;
                }
                __syncwarp();
            }
            tc05::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc05::mbar_arrive(&tempty[acc]);
        }
    }
    tc05::fence_before_sync();
    __syncthreads();
    tc05::fence_after_sync();
    if (warp == 0) {
        __syncwarp();
        tc05::tmem_dealloc(tmem, 2 * ncol);
    }
}

// out[i] = sum over s of part[s][i], in order of s (float4 units)
__global__ void k_sum_splits(const float4* __restrict__ part, int nsplit, int64_t n4, float4* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n4) return;
    float4 a = part[i];
    for (int s = 1; s < nsplit; ++s) {
        const float4 b = part[(int64_t)s * n4 + i];
        a.x += b.x;
        a.y += b.y;
        a.z += b.z;
        a.w += b.w;
    }
    out[i] = a;
}

}  // namespace mlpk
