// Kernel (c): the subdomain-block preconditioner.
//
// The paper partitions the triangulation into subdomains (Sec. 3, Step 2)
// to assemble in parallel; here the same idea, taken to many small
// subdomains on one GPU, defines a block-Jacobi preconditioner: for every
// subdomain s (a contiguous range of nodes, 4 unknowns each) the diagonal
// block S_ss of the scaled matrix is inverted once, and each application
// computes z_s = S_ss^-1 r_s for all subdomains in parallel.
//
// Setup: one CTA per subdomain gathers S_ss (b x b, b <= 64) from the BSR
// blocks into shared memory next to an identity and runs Gauss-Jordan
// elimination with partial (row) pivoting; the inverse is stored
// column-major so that the apply kernel's threads (one per row) read it
// coalesced.  Apply: one CTA per subdomain and tile of right-hand sides.
#include "common.cuh"

namespace {

__global__ void __launch_bounds__(256) k_block_inverse(const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col,
                                                       const double2* __restrict__ sval,
                                                       const int32_t* __restrict__ block_ptr,
                                                       const int64_t* __restrict__ pinv_off,
                                                       double2* __restrict__ pinv, float2* __restrict__ pinv32,
                                                       int* __restrict__ singular) {
    extern __shared__ double2 A[];
    __shared__ double2 fcol[64];
    __shared__ double2 pivinv;
    __shared__ int piv;
    const int blk = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = bd >> 5;
    const int n0 = block_ptr[blk], n1 = block_ptr[blk + 1];
    const int nb = n1 - n0, b = 4 * nb, ld = 2 * b;
    for (int e = tid; e < b * ld; e += bd) {
        int r = e / ld, cc = e - r * ld;
        A[e] = make_double2(cc - b == r ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    for (int il = warp; il < nb; il += nwarps) {
        const int i = n0 + il;
        for (int s = row_ptr[i] + lane; s < row_ptr[i + 1]; s += 32) {
            const int j = col[s];
            if (j >= n0 && j < n1) {
                const int jl = j - n0;
#pragma unroll
                for (int p = 0; p < 4; ++p)
#pragma unroll
                    for (int q = 0; q < 4; ++q) A[(4 * il + p) * ld + 4 * jl + q] = sval[16 * (int64_t)s + 4 * p + q];
            }
        }
    }
    __syncthreads();
    for (int cc = 0; cc < b; ++cc) {
        if (warp == 0) {
            double best = -1.0;
            int bi = cc;
            for (int r = cc + lane; r < b; r += 32) {
                double2 v = A[r * ld + cc];
                double m = v.x * v.x + v.y * v.y;
                if (m > best) {
                    best = m;
                    bi = r;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                double ob = __shfl_xor_sync(0xffffffffu, best, o);
                int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) {
                    best = ob;
                    bi = oi;
                }
            }
            if (lane == 0) {
                piv = bi;
                if (!(best > 0.0)) atomicExch(singular, 1);
            }
        }
        __syncthreads();
        const int pr = piv;
        if (pr != cc)
            for (int j = tid; j < ld; j += bd) {
                double2 t0 = A[cc * ld + j];
                A[cc * ld + j] = A[pr * ld + j];
                A[pr * ld + j] = t0;
            }
        __syncthreads();
        if (tid == 0) {
            double2 v = A[cc * ld + cc];
            double m = v.x * v.x + v.y * v.y;
            pivinv = m > 0.0 ? make_double2(v.x / m, -v.y / m) : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int j = tid; j < ld; j += bd) A[cc * ld + j] = cmul(A[cc * ld + j], pivinv);
        for (int r = tid; r < b; r += bd) fcol[r] = r == cc ? make_double2(0.0, 0.0) : A[r * ld + cc];
        __syncthreads();
        for (int e = tid; e < b * ld; e += bd) {
            int r = e / ld, j = e - r * ld;
            if (r != cc) {
                double2 f = fcol[r], a = A[cc * ld + j], v = A[e];
                v.x -= f.x * a.x - f.y * a.y;
                v.y -= f.x * a.y + f.y * a.x;
                A[e] = v;
            }
        }
        __syncthreads();
    }
    const int64_t off = pinv_off[blk];
    for (int e = tid; e < b * b; e += bd) {
        int cc = e / b, r = e - cc * b;
        double2 v = A[r * ld + b + cc];
        pinv[off + e] = v;
        if (pinv32) pinv32[off + e] = make_float2((float)v.x, (float)v.y);
    }
}

template <typename T, int KT>
__global__ void __launch_bounds__(64) k_block_apply(const int32_t* __restrict__ block_ptr,
                                                    const int64_t* __restrict__ pinv_off,
                                                    const C<T>* __restrict__ pinv, const C<T>* __restrict__ r,
                                                    C<T>* __restrict__ z, int k, int64_t ld,
                                                    const int* __restrict__ active) {
    __shared__ C<T> rs[KT][64];
    const int blk = blockIdx.x, tid = threadIdx.x;
    const int r0 = blockIdx.y * KT;
    const int n0 = block_ptr[blk], n1 = block_ptr[blk + 1];
    const int b = 4 * (n1 - n0);
    const int64_t base = 4 * (int64_t)n0;
    bool on[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = (r0 + q < k) && (!active || active[r0 + q]);
        if (on[q] && tid < b) rs[q][tid] = r[(int64_t)(r0 + q) * ld + base + tid];
    }
    __syncthreads();
    if (tid >= b) return;
    C<T> acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = czero<T>();
    const C<T>* P = pinv + pinv_off[blk] + tid;
    for (int cc = 0; cc < b; ++cc) {
        const C<T> a = P[(int64_t)cc * b];
#pragma unroll
        for (int q = 0; q < KT; ++q) cfma(acc[q], a, rs[q][cc]);
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) z[(int64_t)(r0 + q) * ld + base + tid] = acc[q];
}

int pick_ptile(int k, int rhs_tile) {
    int kt = rhs_tile > 0 ? rhs_tile : 8;
    if (kt > k) kt = k;
    if (kt >= 8) return 8;
    if (kt >= 4) return 4;
    if (kt >= 2) return 2;
    return 1;
}

template <typename T>
void apply_impl(ect_ctx* c, const C<T>* pinv, const C<T>* r, C<T>* z, int k, int64_t ld, int rhs_tile,
                const int* active) {
    const int kt = pick_ptile(k, rhs_tile);
    dim3 grid((unsigned)c->n_blocks, (unsigned)((k + kt - 1) / kt));
    const int32_t* bp = c->block_ptr.as<int32_t>();
    const int64_t* po = c->pinv_off.as<int64_t>();
    cudaStream_t st = c->stream;
    switch (kt) {
        case 8: k_block_apply<T, 8><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active); break;
        case 4: k_block_apply<T, 4><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active); break;
        case 2: k_block_apply<T, 2><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active); break;
        default: k_block_apply<T, 1><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active); break;
    }
    ECT_CHECK_LAUNCH();
}

}  // namespace

void precond_setup(ect_ctx* c, int which, int precision_mask) {
    ECT_REQUIRE(which == ECT_VACUUM || which == ECT_DEFECT, ECT_ERR_ARG, "bad which");
    Matrix& M = c->mat[which];
    ECT_REQUIRE(M.assembled, ECT_ERR_STATE, "ect_assemble must come before ect_precond_setup");
    bool f32 = (precision_mask & ECT_F32) != 0;
    cudaStream_t st = c->stream;
    M.pinv.alloc(sizeof(double2) * c->pinv_total);
    if (f32) M.pinv32.alloc(sizeof(float2) * c->pinv_total);
    else M.pinv32.release();
    const int bmax = 4 * c->max_block_nodes;
    const size_t smem = sizeof(double2) * (size_t)bmax * 2 * bmax;
    ECT_CUDA(cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DevBuf flag;
    flag.alloc(sizeof(int));
    ECT_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    k_block_inverse<<<(unsigned)c->n_blocks, 256, smem, st>>>(
        c->row_ptr.as<int32_t>(), c->col.as<int32_t>(), M.sval.as<double2>(), c->block_ptr.as<int32_t>(),
        c->pinv_off.as<int64_t>(), M.pinv.as<double2>(), f32 ? M.pinv32.as<float2>() : nullptr, flag.as<int>());
    ECT_CHECK_LAUNCH();
    int h = 0;
    ECT_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    ECT_REQUIRE(!h, ECT_ERR_BREAKDOWN, "a subdomain block of the scaled matrix is singular");
    M.pc_f64 = true;
    M.pc_f32 = f32;
}

void precond_apply_f64(ect_ctx* c, int which, const double2* r, double2* z, int k, int64_t ld, int rhs_tile,
                       const int* active) {
    Matrix& M = c->mat[which];
    ECT_REQUIRE(M.pc_f64, ECT_ERR_STATE, "preconditioner not set up");
    apply_impl<double>(c, M.pinv.as<double2>(), r, z, k, ld, rhs_tile, active);
}

void precond_apply_f32(ect_ctx* c, int which, const float2* r, float2* z, int k, int64_t ld, int rhs_tile,
                       const int* active) {
    Matrix& M = c->mat[which];
    ECT_REQUIRE(M.pc_f32, ECT_ERR_STATE, "FP32 preconditioner not set up (use ECT_F32 in ect_precond_setup)");
    apply_impl<float>(c, M.pinv32.as<float2>(), r, z, k, ld, rhs_tile, active);
}
