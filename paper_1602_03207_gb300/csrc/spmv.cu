// Kernel (b): BSR (4x4 complex blocks) SpMV and multi-right-hand-side SpMM.
//
// y_r = A x_r for r in a tile of KT right-hand sides.  One thread owns one
// scalar row (node i, component p) and KT accumulators: it streams row p of
// each of the node's blocks once (64 B in FP64, 32 B in FP32, vector loads)
// and applies it to the KT vectors, so the matrix is read once per tile of
// right-hand sides.  The four threads of a node read one block's four rows,
// which are contiguous, and broadcast-share the x segment of each column
// node.  Vectors are stored [k][4N] with leading dimension ld.  The grid is
// one-dimensional with the tile index fastest, so the tiles of a row range
// run side by side and share the matrix blocks through L2.  The launchers
// cover k with full tiles (8, 4, 2, 1), so every row of a tile exists and the
// x loads are unconditional: all of a step's loads can issue before its FMAs.
// Masked right-hand sides are computed and not stored.
#include "common.cuh"

namespace {

template <int KT>
__global__ void __launch_bounds__(256) k_spmv_f64(const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col,
                                                  const double2* __restrict__ val, const double2* __restrict__ x,
                                                  double2* __restrict__ y, int64_t n_rows, int64_t ld,
                                                  const int* __restrict__ active, const double2* __restrict__ b,
                                                  int ntile) {
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t d = (int64_t)(blockIdx.x / ntile) * blockDim.x + threadIdx.x;
    if (d >= 4 * n_rows) return;
    const int row = (int)(d >> 2), p = (int)(d & 3);
    const int r0 = tile * KT;
    bool on[KT], any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = !active || active[r0 + q];
        any |= on[q];
    }
    if (!any) return;  // the whole tile has retired (uniform over the CTA)
    double2 acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = make_double2(0.0, 0.0);
    const int s1 = row_ptr[row + 1];
    for (int s = row_ptr[row]; s < s1; ++s) {
        const int c = col[s];
        const double2* v = val + 16 * (int64_t)s + 4 * p;
        const double2 a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const double2* xv = x + (int64_t)(r0 + q) * ld + 4 * (int64_t)c;
            cfma(acc[q], a0, xv[0]);
            cfma(acc[q], a1, xv[1]);
            cfma(acc[q], a2, xv[2]);
            cfma(acc[q], a3, xv[3]);
        }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) {
            const int64_t e = (int64_t)(r0 + q) * ld + d;
            y[e] = b ? csub(b[e], acc[q]) : acc[q];
        }
}

template <int KT>
__global__ void __launch_bounds__(256, 4) k_spmv_f32(const int32_t* __restrict__ row_ptr,
                                                  const int32_t* __restrict__ col,
                                                  const float2* __restrict__ val, const float2* __restrict__ x,
                                                  float2* __restrict__ y, int64_t n_rows, int64_t ld,
                                                  const int* __restrict__ active, const float2* __restrict__ b,
                                                  int ntile) {
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t d = (int64_t)(blockIdx.x / ntile) * blockDim.x + threadIdx.x;
    if (d >= 4 * n_rows) return;
    const int row = (int)(d >> 2), p = (int)(d & 3);
    const int r0 = tile * KT;
    bool on[KT], any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = !active || active[r0 + q];
        any |= on[q];
    }
    if (!any) return;  // the whole tile has retired (uniform over the CTA)
    float2 acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = make_float2(0.f, 0.f);
    const int s1 = row_ptr[row + 1];
    for (int s = row_ptr[row]; s < s1; ++s) {
        const int c = col[s];
        const float4* v = reinterpret_cast<const float4*>(val + 16 * (int64_t)s + 4 * p);
        const float4 v01 = v[0], v23 = v[1];
        const float2 a0 = make_float2(v01.x, v01.y), a1 = make_float2(v01.z, v01.w);
        const float2 a2 = make_float2(v23.x, v23.y), a3 = make_float2(v23.z, v23.w);
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float4* xv =
                reinterpret_cast<const float4*>(x + (int64_t)(r0 + q) * ld + 4 * (int64_t)c);
            const float4 x01 = xv[0], x23 = xv[1];
            cfma(acc[q], a0, make_float2(x01.x, x01.y));
            cfma(acc[q], a1, make_float2(x01.z, x01.w));
            cfma(acc[q], a2, make_float2(x23.x, x23.y));
            cfma(acc[q], a3, make_float2(x23.z, x23.w));
        }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) {
            const int64_t e = (int64_t)(r0 + q) * ld + d;
            y[e] = b ? csub(b[e], acc[q]) : acc[q];
        }
}

// FP32 SpMM with the right-hand-side tile split across RG thread groups of one
// CTA: each group of 64 threads covers the same 16 block rows for KT of the
// RG*KT right-hand sides, so the matrix values are read from DRAM once and
// served to the other groups from L1, while each thread keeps only KT
// accumulators (few registers, high occupancy, many loads in flight).
template <int KT, int RG>
__global__ void __launch_bounds__(64 * RG) k_spmv_f32_split(const int32_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col,
                                                            const float2* __restrict__ val,
                                                            const float2* __restrict__ x, float2* __restrict__ y,
                                                            int64_t n_rows, int k, int64_t ld,
                                                            const int* __restrict__ active,
                                                            const float2* __restrict__ b) {
    const int lr = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int64_t d = blockIdx.x * 64ll + lr;
    if (d >= 4 * n_rows) return;
    const int row = (int)(d >> 2), p = (int)(d & 3);
    const int r0 = (blockIdx.y * RG + g) * KT;
    bool on[KT];
    bool any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = (r0 + q < k) && (!active || active[r0 + q]);
        any |= on[q];
    }
    if (!any) return;
    float2 acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = make_float2(0.f, 0.f);
    const int s1 = row_ptr[row + 1];
    for (int s = row_ptr[row]; s < s1; ++s) {
        const int c = col[s];
        const float4* v = reinterpret_cast<const float4*>(val + 16 * (int64_t)s + 4 * p);
        const float4 v01 = __ldg(v), v23 = __ldg(v + 1);
        const float2 a0 = make_float2(v01.x, v01.y), a1 = make_float2(v01.z, v01.w);
        const float2 a2 = make_float2(v23.x, v23.y), a3 = make_float2(v23.z, v23.w);
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            if (!on[q]) continue;
            const float4* xv = reinterpret_cast<const float4*>(x + (int64_t)(r0 + q) * ld + 4 * (int64_t)c);
            const float4 x01 = __ldg(xv), x23 = __ldg(xv + 1);
            cfma(acc[q], a0, make_float2(x01.x, x01.y));
            cfma(acc[q], a1, make_float2(x01.z, x01.w));
            cfma(acc[q], a2, make_float2(x23.x, x23.y));
            cfma(acc[q], a3, make_float2(x23.z, x23.w));
        }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) {
            const int64_t e = (int64_t)(r0 + q) * ld + d;
            y[e] = b ? csub(b[e], acc[q]) : acc[q];
        }
}

// Coarse-level SpMM: one warp per block row.  Lane = 4*slice + p: the eight
// slices take every eighth block of the row, each lane keeps KT accumulators
// for scalar row p, and a shuffle tree over the slices sums them (fixed
// order).  Galerkin rows on the coarse levels hold 30-60 blocks while the
// levels have few rows, so splitting the row cuts the serial chain of
// dependent loads per thread by eight.
template <typename T, int KT>
__global__ void __launch_bounds__(256) k_spmv_warp(const int32_t* __restrict__ row_ptr,
                                                   const int32_t* __restrict__ col, const C<T>* __restrict__ val,
                                                   const C<T>* __restrict__ x, C<T>* __restrict__ y, int64_t n_rows,
                                                   int64_t ld, const int* __restrict__ active,
                                                   const C<T>* __restrict__ b, int ntile) {
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t row = ((int64_t)(blockIdx.x / ntile) * blockDim.x + threadIdx.x) >> 5;
    if (row >= n_rows) return;  // uniform over the warp
    const int lane = threadIdx.x & 31, p = lane & 3, sl = lane >> 2;
    const int r0 = tile * KT;
    bool on[KT], any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = !active || active[r0 + q];
        any |= on[q];
    }
    if (!any) return;  // the whole tile has retired (uniform over the CTA)
    C<T> acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = czero<T>();
    const int s1 = row_ptr[row + 1];
    for (int s = row_ptr[row] + sl; s < s1; s += 8) {
        const int c = col[s];
        const C<T>* v = val + 16 * (int64_t)s + 4 * p;
        const C<T> a0 = v[0], a1 = v[1], a2 = v[2], a3 = v[3];
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const C<T>* xv = x + (int64_t)(r0 + q) * ld + 4 * (int64_t)c;
            cfma(acc[q], a0, xv[0]);
            cfma(acc[q], a1, xv[1]);
            cfma(acc[q], a2, xv[2]);
            cfma(acc[q], a3, xv[3]);
        }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, o);
            acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, o);
        }
    if (sl != 0) return;
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) {
            const int64_t e = (int64_t)(r0 + q) * ld + 4 * row + p;
            y[e] = b ? csub(b[e], acc[q]) : acc[q];
        }
}

// Double-float accumulation of one real product (a_hi + a_lo) u into (S, c):
// p = a_hi u rounded, e its exact rounding error plus a_lo u, then Knuth's
// TwoSum adds p to S exactly (the error goes to c).  Round-to-nearest
// intrinsics keep the compiler from fusing the steps.
__device__ __forceinline__ void df32_acc(float& S, float& c, float ah, float al, float u) {
    const float p = __fmul_rn(ah, u);
    float e = __fmaf_rn(ah, u, -p);
    e = __fmaf_rn(al, u, e);
    const float t = __fadd_rn(S, p);
    const float bp = __fsub_rn(t, S);
    const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    S = t;
    c = __fadd_rn(c, __fadd_rn(err, e));
}

// Outer-loop SpMM of the mixed mode: y (FP64) = S u where u is exactly
// representable in FP32 (the inner FP32 solution).  S = S_hi + S_lo, both in
// FP32; every product is formed exactly up to the dropped ~2^-48 terms and
// summed in double-float, so y matches the FP64 product to about 2^-46 of
// sum |S_ij u_j| while the arithmetic runs on the FP32 pipe (GB300's FP64
// rate makes the plain FP64 product ALU-bound at several times the time).
template <int KT>
__global__ void __launch_bounds__(256) k_spmv_df32(const int32_t* __restrict__ row_ptr,
                                                   const int32_t* __restrict__ col,
                                                   const float2* __restrict__ vhi, const float2* __restrict__ vlo,
                                                   const float2* __restrict__ x, double2* __restrict__ y,
                                                   int64_t n_rows, int64_t ld, const int* __restrict__ active,
                                                   int ntile) {
    const int tile = (int)(blockIdx.x % ntile);
    const int64_t d = (int64_t)(blockIdx.x / ntile) * blockDim.x + threadIdx.x;
    if (d >= 4 * n_rows) return;
    const int row = (int)(d >> 2), p = (int)(d & 3);
    const int r0 = tile * KT;
    bool on[KT], any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = !active || active[r0 + q];
        any |= on[q];
    }
    if (!any) return;
    float sr[KT], cr[KT], si[KT], ci[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) sr[q] = cr[q] = si[q] = ci[q] = 0.f;
    const int s1 = row_ptr[row + 1];
    for (int s = row_ptr[row]; s < s1; ++s) {
        const int c = col[s];
        const float4* vh = reinterpret_cast<const float4*>(vhi + 16 * (int64_t)s + 4 * p);
        const float4* vl = reinterpret_cast<const float4*>(vlo + 16 * (int64_t)s + 4 * p);
        const float4 h01 = vh[0], h23 = vh[1], l01 = vl[0], l23 = vl[1];
        const float ahr[4] = {h01.x, h01.z, h23.x, h23.z}, ahi[4] = {h01.y, h01.w, h23.y, h23.w};
        const float alr[4] = {l01.x, l01.z, l23.x, l23.z}, ali[4] = {l01.y, l01.w, l23.y, l23.w};
#pragma unroll
        for (int q = 0; q < KT; ++q) {
            const float4* xv = reinterpret_cast<const float4*>(x + (int64_t)(r0 + q) * ld + 4 * (int64_t)c);
            const float4 x01 = xv[0], x23 = xv[1];
            const float ur[4] = {x01.x, x01.z, x23.x, x23.z}, ui[4] = {x01.y, x01.w, x23.y, x23.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                df32_acc(sr[q], cr[q], ahr[e], alr[e], ur[e]);
                df32_acc(sr[q], cr[q], -ahi[e], -ali[e], ui[e]);
                df32_acc(si[q], ci[q], ahr[e], alr[e], ui[e]);
                df32_acc(si[q], ci[q], ahi[e], ali[e], ur[e]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q])
            y[(int64_t)(r0 + q) * ld + d] =
                make_double2((double)sr[q] + (double)cr[q], (double)si[q] + (double)ci[q]);
}

// FP32 SpMM, one warp per block row, up to 8 right-hand sides per warp.
// Lane (p, q) reads column p of each block (32 contiguous bytes of the
// transposed copy; the four p lanes together read the block's 128 bytes and
// the eight q lanes share them) and the value x_q[4c + p] (the 32 lanes read
// the 8 vectors' 32-byte segments of column node c: one sector per vector),
// and accumulates the four partial rows A[:, p] x_q[4c + p].  At the end of
// the row the partials of the four p lanes are summed with shuffles and lane
// (p, q) stores row p of y_q.  Against the thread-per-row kernel this halves
// the L1 wavefronts per block (the x gather is one 8-sector request per block
// instead of sixteen).
template <bool RESID>
__global__ void __launch_bounds__(256) k_spmm_colwarp(const int32_t* __restrict__ row_ptr,
                                                      const int32_t* __restrict__ col, const float4* __restrict__ valt,
                                                      const float2* __restrict__ x, int64_t ldx, const float2* b,
                                                      float2* y, int64_t ldy, int64_t n_rows, int k,
                                                      const int* __restrict__ active) {
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (i >= n_rows) return;  // uniform over the warp
    const int lane = threadIdx.x & 31, p = lane & 3, q = lane >> 2;
    const int r = blockIdx.y * 8 + q;
    const bool live = r < k && (!active || active[r]);
    if (!__any_sync(0xffffffffu, live)) return;
    const float2* xq = x + (int64_t)min(r, k - 1) * ldx + p;  // lanes past k read the last vector, store nothing
    float2 acc[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[e] = make_float2(0.f, 0.f);
    const int s0 = row_ptr[i], s1 = row_ptr[i + 1];
    for (int sb = s0; sb < s1; sb += 32) {
        const int n = min(32, s1 - sb);
        const int cv = lane < n ? col[sb + lane] : 0;
        const float4* v = valt + (int64_t)sb * 8 + 2 * p;
        int j = 0;
        for (; j + 1 < n; j += 2) {
            const int c0 = __shfl_sync(0xffffffffu, cv, j), c1 = __shfl_sync(0xffffffffu, cv, j + 1);
            const float4 a01 = v[8 * j], a23 = v[8 * j + 1], b01 = v[8 * j + 8], b23 = v[8 * j + 9];
            const float2 x0 = xq[4 * (int64_t)c0], x1 = xq[4 * (int64_t)c1];
            cfma(acc[0], make_float2(a01.x, a01.y), x0);
            cfma(acc[1], make_float2(a01.z, a01.w), x0);
            cfma(acc[2], make_float2(a23.x, a23.y), x0);
            cfma(acc[3], make_float2(a23.z, a23.w), x0);
            cfma(acc[0], make_float2(b01.x, b01.y), x1);
            cfma(acc[1], make_float2(b01.z, b01.w), x1);
            cfma(acc[2], make_float2(b23.x, b23.y), x1);
            cfma(acc[3], make_float2(b23.z, b23.w), x1);
        }
        if (j < n) {
            const int c0 = __shfl_sync(0xffffffffu, cv, j);
            const float4 a01 = v[8 * j], a23 = v[8 * j + 1];
            const float2 x0 = xq[4 * (int64_t)c0];
            cfma(acc[0], make_float2(a01.x, a01.y), x0);
            cfma(acc[1], make_float2(a01.z, a01.w), x0);
            cfma(acc[2], make_float2(a23.x, a23.y), x0);
            cfma(acc[3], make_float2(a23.z, a23.w), x0);
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            acc[e].x += __shfl_xor_sync(0xffffffffu, acc[e].x, o);
            acc[e].y += __shfl_xor_sync(0xffffffffu, acc[e].y, o);
        }
    if (!live) return;
    const float2 mine = p == 0 ? acc[0] : p == 1 ? acc[1] : p == 2 ? acc[2] : acc[3];
    const int64_t e = (int64_t)r * ldy + 4 * i + p;
    y[e] = RESID ? csub(b[e], mine) : mine;
}

}  // namespace

void bsr_spmm_colwarp_f32(cudaStream_t st, const int32_t* rp, const int32_t* col, const float2* valt, int64_t N,
                          const float2* x, int64_t ldx, const float2* b, float2* y, int64_t ldy, int k,
                          const int* active) {
    const dim3 grid(grid_for(32 * N, 256), (unsigned)((k + 7) / 8));
    if (b)
        k_spmm_colwarp<true><<<grid, 256, 0, st>>>(rp, col, reinterpret_cast<const float4*>(valt), x, ldx, b, y, ldy,
                                                   N, k, active);
    else
        k_spmm_colwarp<false><<<grid, 256, 0, st>>>(rp, col, reinterpret_cast<const float4*>(valt), x, ldx, b, y,
                                                    ldy, N, k, active);
    ECT_CHECK_LAUNCH();
}

void bsr_spmv_f64(cudaStream_t st, const int32_t* rp, const int32_t* cl, const double2* val, int64_t N,
                  const double2* x, const double2* b, double2* y, int k, int64_t ldx, int rhs_tile, const int* active) {
    for_tiles(k, rhs_tile, [&](int kt, int r, int nt) {
        const unsigned grid = tile_grid(grid_for(4 * N, 256), nt);
        const double2* xr = x + r * ldx;
        const double2* br = b ? b + r * ldx : nullptr;
        double2* yr = y + r * ldx;
        const int* ar = active ? active + r : nullptr;
        switch (kt) {
            case 8: k_spmv_f64<8><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            case 4: k_spmv_f64<4><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            case 2: k_spmv_f64<2><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            default: k_spmv_f64<1><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
        }
    });
    ECT_CHECK_LAUNCH();
}

void bsr_spmv_f32(cudaStream_t st, const int32_t* rp, const int32_t* cl, const float2* val, int64_t N,
                  const float2* x, const float2* b, float2* y, int k, int64_t ldx, int rhs_tile, const int* active) {
    if (k >= 2 && rhs_tile < 0) {
        // split tiles (rhs_tile == -1): 8 rhs per CTA (4 groups x 2), 4 (4 x 1) or 2 (2 x 1)
        const unsigned gx = grid_for(4 * N, 64);
        if (k >= 8) {
            k_spmv_f32_split<2, 4><<<dim3(gx, (unsigned)((k + 7) / 8)), 256, 0, st>>>(rp, cl, val, x, y, N, k, ldx,
                                                                                      active, b);
        } else if (k >= 4) {
            k_spmv_f32_split<1, 4><<<dim3(gx, (unsigned)((k + 3) / 4)), 256, 0, st>>>(rp, cl, val, x, y, N, k, ldx,
                                                                                      active, b);
        } else {
            k_spmv_f32_split<1, 2><<<dim3(gx, (unsigned)((k + 1) / 2)), 128, 0, st>>>(rp, cl, val, x, y, N, k, ldx,
                                                                                      active, b);
        }
        ECT_CHECK_LAUNCH();
        return;
    }
    for_tiles(k, rhs_tile, [&](int kt, int r, int nt) {
        const unsigned grid = tile_grid(grid_for(4 * N, 256), nt);
        const float2* xr = x + r * ldx;
        const float2* br = b ? b + r * ldx : nullptr;
        float2* yr = y + r * ldx;
        const int* ar = active ? active + r : nullptr;
        switch (kt) {
            case 8: k_spmv_f32<8><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            case 4: k_spmv_f32<4><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            case 2: k_spmv_f32<2><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            default: k_spmv_f32<1><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
        }
    });
    ECT_CHECK_LAUNCH();
}

void spmv_f64(ect_ctx* c, int which, bool scaled, const double2* x, double2* y, int k, int64_t ldx, int rhs_tile,
              const int* active) {
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.assembled, ECT_ERR_STATE, "matrix not assembled");
    const double2* val = scaled ? M.sval.as<double2>() : M.val.as<double2>();
    bsr_spmv_f64(c->stream, c->row_ptr.as<int32_t>(), c->col.as<int32_t>(), val, c->n_nodes, x, nullptr, y, k, ldx,
                 rhs_tile, active);
}

void spmv_f32(ect_ctx* c, int which, const float2* x, float2* y, int k, int64_t ldx, int rhs_tile,
              const int* active) {
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.assembled && M.has_f32, ECT_ERR_STATE, "FP32 matrix not assembled (use ECT_F32 in ect_assemble)");
    if (c->staged_rows == SPMM_COLWARP && rhs_tile != -1) {
        ECT_REQUIRE(M.t_gen == M.val_gen, ECT_ERR_STATE, "transposed FP32 blocks not prepared (internal)");
        bsr_spmm_colwarp_f32(c->stream, c->row_ptr.as<int32_t>(), c->col.as<int32_t>(), M.sval32t.as<float2>(),
                             c->n_nodes, x, ldx, nullptr, y, ldx, k, active);
        return;
    }
    if (c->staged_rows > 0 && rhs_tile != -1 && c->fine_plan.ok && c->fine_plan.rows == c->staged_rows) {
        bsr_spmm_staged_f32(c->stream, c->fine_plan, c->row_ptr.as<int32_t>(), M.sval32p.as<float4>(), x, ldx,
                            nullptr, y, ldx, k, active);
        return;
    }
    bsr_spmv_f32(c->stream, c->row_ptr.as<int32_t>(), c->col.as<int32_t>(), M.sval32.as<float2>(), c->n_nodes, x,
                 nullptr, y, k, ldx, rhs_tile, active);
}

template <typename T>
void bsr_spmv_warp(cudaStream_t st, const int32_t* rp, const int32_t* cl, const C<T>* val, int64_t N, const C<T>* x,
                   const C<T>* b, C<T>* y, int k, int64_t ldx, int rhs_tile, const int* active) {
    for_tiles(k, rhs_tile, [&](int kt, int r, int nt) {
        const unsigned grid = tile_grid(grid_for(32 * N, 256), nt);
        const C<T>* xr = x + r * ldx;
        const C<T>* br = b ? b + r * ldx : nullptr;
        C<T>* yr = y + r * ldx;
        const int* ar = active ? active + r : nullptr;
        switch (kt) {
            case 8: k_spmv_warp<T, 8><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            case 4: k_spmv_warp<T, 4><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            case 2: k_spmv_warp<T, 2><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
            default: k_spmv_warp<T, 1><<<grid, 256, 0, st>>>(rp, cl, val, xr, yr, N, ldx, ar, br, nt); break;
        }
    });
    ECT_CHECK_LAUNCH();
}

template void bsr_spmv_warp<double>(cudaStream_t, const int32_t*, const int32_t*, const double2*, int64_t,
                                    const double2*, const double2*, double2*, int, int64_t, int, const int*);
template void bsr_spmv_warp<float>(cudaStream_t, const int32_t*, const int32_t*, const float2*, int64_t, const float2*,
                                   const float2*, float2*, int, int64_t, int, const int*);

void spmv_df32(ect_ctx* c, int which, const float2* u, double2* y, int k, int64_t ldx, int rhs_tile,
               const int* active) {
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.assembled && M.has_f32, ECT_ERR_STATE, "FP32 matrix not assembled (use ECT_F32 in ect_assemble)");
    const int32_t* rp = c->row_ptr.as<int32_t>();
    const int32_t* cl = c->col.as<int32_t>();
    const float2* hi = M.sval32.as<float2>();
    const float2* lo = M.sval32lo.as<float2>();
    const int64_t N = c->n_nodes;
    for_tiles(k, rhs_tile, [&](int kt, int r, int nt) {
        const unsigned grid = tile_grid(grid_for(4 * N, 256), nt);
        const float2* xr = u + r * ldx;
        double2* yr = y + r * ldx;
        const int* ar = active ? active + r : nullptr;
        switch (kt) {
            case 8: k_spmv_df32<8><<<grid, 256, 0, c->stream>>>(rp, cl, hi, lo, xr, yr, N, ldx, ar, nt); break;
            case 4: k_spmv_df32<4><<<grid, 256, 0, c->stream>>>(rp, cl, hi, lo, xr, yr, N, ldx, ar, nt); break;
            case 2: k_spmv_df32<2><<<grid, 256, 0, c->stream>>>(rp, cl, hi, lo, xr, yr, N, ldx, ar, nt); break;
            default: k_spmv_df32<1><<<grid, 256, 0, c->stream>>>(rp, cl, hi, lo, xr, yr, N, ldx, ar, nt); break;
        }
    });
    ECT_CHECK_LAUNCH();
}
