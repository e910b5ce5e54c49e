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
// elimination with partial (row) pivoting; the FP64 inverse is stored
// column-major so that the apply kernel's threads (one per row) read it
// coalesced, the FP32 copy as the packed upper triangle of the symmetrised
// inverse (S_ss is complex symmetric, so is its inverse), which halves the
// bytes the mixed-precision apply reads.  Apply: one CTA per subdomain and
// tile of right-hand sides.
#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace {

__global__ void __launch_bounds__(256) k_block_inverse(const int32_t* __restrict__ row_ptr,
                                                       const int32_t* __restrict__ col,
                                                       const double2* __restrict__ sval,
                                                       const int32_t* __restrict__ block_ptr,
                                                       const int64_t* __restrict__ pinv_off,
                                                       const int64_t* __restrict__ pinv_off32,
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
        pinv[off + e] = A[r * ld + b + cc];
    }
    if (pinv32) {
        // packed upper triangle of the symmetrised inverse (the exact inverse is symmetric)
        const int64_t off32 = pinv_off32[blk];
        for (int e = tid; e < b * b; e += bd) {
            int cc = e / b, r = e - cc * b;
            if (r > cc) continue;
            const double2 v = A[r * ld + b + cc], u = A[cc * ld + b + r];
            pinv32[off32 + cc * (cc + 1) / 2 + r] =
                make_float2((float)(0.5 * (v.x + u.x)), (float)(0.5 * (v.y + u.y)));
        }
    }
}

template <typename T, int KT>
__global__ void __launch_bounds__(64) k_block_apply(const int32_t* __restrict__ block_ptr,
                                                    const int64_t* __restrict__ pinv_off,
                                                    const C<T>* __restrict__ pinv, const C<T>* __restrict__ r,
                                                    C<T>* __restrict__ z, int k, int64_t ld,
                                                    const int* __restrict__ active,
                                                    const int32_t* __restrict__ blk_c, const C<T>* __restrict__ zc,
                                                    int64_t nc, const T* __restrict__ zv, int accumulate, int ntile) {
    __shared__ C<T> rs[KT][64];
    // one-dimensional grid, tile index fastest: the tiles of a block share its inverse through L2
    const int blk = (int)(blockIdx.x / ntile), tid = threadIdx.x;
    const int r0 = (int)(blockIdx.x % ntile) * KT;
    const int n0 = block_ptr[blk], n1 = block_ptr[blk + 1];
    const int b = 4 * (n1 - n0);
    const int64_t base = 4 * (int64_t)n0;
    bool on[KT], any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = (r0 + q < k) && (!active || active[r0 + q]);
        any |= on[q];
        if (on[q] && tid < b) rs[q][tid] = r[(int64_t)(r0 + q) * ld + base + tid];
    }
    if (!any) return;  // the whole tile has retired (uniform over the CTA, before any barrier)
    __syncthreads();
    if (tid >= b) return;
    C<T> acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = czero<T>();
    const C<T>* P = pinv + pinv_off[blk] + tid;
    // b is a multiple of 4 (four unknowns per node): four independent loads in flight per step
#pragma unroll 4
    for (int cc = 0; cc < b; ++cc) {
        const C<T> a = P[(int64_t)cc * b];
#pragma unroll
        for (int q = 0; q < KT; ++q) cfma(acc[q], a, rs[q][cc]);
    }
    if (zc && (tid & 3) == 3) {
        const int cc = blk_c[blk];
        const T w = zv[n0 + (tid >> 2)];
        if (cc >= 0 && w != T(0))
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                const C<T> v = zc[(int64_t)(r0 + q) * nc + cc];
                acc[q].x += w * v.x;
                acc[q].y += w * v.y;
            }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) {
            C<T>* zp = z + (int64_t)(r0 + q) * ld + base + tid;
            *zp = accumulate ? cadd(*zp, acc[q]) : acc[q];
        }
}

// FP32 block apply from the packed upper triangle of the symmetric inverse.
// The CTA stages its block's packed inverse in shared memory with 16-byte
// loads (about half the bytes of the full inverse), then thread i forms row
// i of the inverse: entries (i, j), j >= i, from column j, entries j < i
// from column i.  Optional coarse-space term as in k_block_apply; one-
// dimensional grid with the tile index fastest.
constexpr int SYM_MAX_F4 = 64 * 65 / 4;  // packed 64 x 64 block in float4 units
template <int KT>
__global__ void __launch_bounds__(64) k_block_apply_sym(const int32_t* __restrict__ block_ptr,
                                                        const int64_t* __restrict__ poff,
                                                        const float2* __restrict__ pinv, const float2* __restrict__ r,
                                                        float2* __restrict__ z, int k, int64_t ld,
                                                        const int* __restrict__ active,
                                                        const int32_t* __restrict__ blk_c,
                                                        const float2* __restrict__ zc, int64_t nc,
                                                        const float* __restrict__ zv, int accumulate, int ntile) {
    __shared__ float4 S4[SYM_MAX_F4];
    __shared__ __align__(16) float2 rs[64][KT];  // [row][rhs]: one step reads its KT values as float4s
    const int blk = (int)(blockIdx.x / ntile), tid = threadIdx.x;
    const int r0 = (int)(blockIdx.x % ntile) * KT;
    const int n0 = block_ptr[blk], n1 = block_ptr[blk + 1];
    const int b = 4 * (n1 - n0);
    const int64_t base = 4 * (int64_t)n0;
    const int n4 = b * (b + 1) / 4;
    bool on[KT], any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = (r0 + q < k) && (!active || active[r0 + q]);
        any |= on[q];
    }
    if (!any) return;  // the whole tile has retired (uniform over the CTA, before any barrier)
    const float4* P4 = reinterpret_cast<const float4*>(pinv + poff[blk]);
    for (int e = tid; e < n4; e += 64) S4[e] = __ldg(P4 + e);
    unsigned onm = 0;
#pragma unroll
    for (int q = 0; q < KT; ++q) onm |= on[q] ? 1u << q : 0u;
    // flat mapping: consecutive threads fill consecutive shared words (no bank conflicts)
    for (int f = tid; f < 64 * KT; f += 64) {
        const int row = f / KT, q = f - row * KT;
        if (row < b && ((onm >> q) & 1u)) rs[row][q] = r[(int64_t)(r0 + q) * ld + base + row];
    }
    __syncthreads();
    if (tid >= b) return;
    const float2* S = reinterpret_cast<const float2*>(S4);
    float2 acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = make_float2(0.f, 0.f);
    const int ti = tid * (tid + 1) / 2;
    int tj = 0;  // j (j + 1) / 2
#pragma unroll 4
    for (int j = 0; j < b; ++j) {
        const float2 a = S[j >= tid ? tj + tid : ti + j];
        if constexpr (KT >= 2) {
            const float4* rj = reinterpret_cast<const float4*>(rs[j]);
#pragma unroll
            for (int h = 0; h < KT / 2; ++h) {
                const float4 v = rj[h];
                cfma(acc[2 * h], a, make_float2(v.x, v.y));
                cfma(acc[2 * h + 1], a, make_float2(v.z, v.w));
            }
        } else {
            cfma(acc[0], a, rs[j][0]);
        }
        tj += j + 1;
    }
    if (zc && (tid & 3) == 3) {
        const int cc = blk_c[blk];
        const float w = zv[n0 + (tid >> 2)];
        if (cc >= 0 && w != 0.f)
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                if (!on[q]) continue;
                const float2 v = zc[(int64_t)(r0 + q) * nc + cc];
                acc[q].x += w * v.x;
                acc[q].y += w * v.y;
            }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) {
            float2* zp = z + (int64_t)(r0 + q) * ld + base + tid;
            *zp = accumulate ? cadd(*zp, acc[q]) : acc[q];
        }
}

// k_block_apply_sym for a full tile of 8 right-hand sides with paired FMAs.
// The tile is kept planar in shared memory (real parts of the 8 right-hand
// sides of a row, then their imaginary parts), so two right-hand sides are
// one 64-bit register pair; with the entry a of the inverse broadcast into
// pairs, a complex multiply-add of two right-hand sides is four paired FMAs:
//   re += (a.x, a.x) (r.re) + (-a.y, -a.y) (r.im),  im += (a.x, a.x) (r.im) + (a.y, a.y) (r.re).
// Half the FMA instructions of the scalar form for the same shared-memory
// loads (the limiting resource of the scalar form was the issue rate).
__global__ void __launch_bounds__(64) k_block_apply_sym8x2(const int32_t* __restrict__ block_ptr,
                                                          const int64_t* __restrict__ poff,
                                                          const float2* __restrict__ pinv, const float2* __restrict__ r,
                                                          float2* __restrict__ z, int k, int64_t ld,
                                                          const int* __restrict__ active,
                                                          const int32_t* __restrict__ blk_c,
                                                          const float2* __restrict__ zc, int64_t nc,
                                                          const float* __restrict__ zv, int accumulate, int ntile,
                                                          int64_t n_blocks, int bpc) {
    constexpr int KT = 8;
    __shared__ float4 S4[SYM_MAX_F4];
    __shared__ __align__(16) float rre[64][KT];
    __shared__ __align__(16) float rim[64][KT];
    // bpc blocks of at most 64 / bpc rows share the CTA: thread group `sub` (64 / bpc threads) takes one
    const int tsub = 64 / bpc, sub = threadIdx.x / tsub, tid = threadIdx.x - sub * tsub;
    const int64_t blk = (int64_t)(blockIdx.x / ntile) * bpc + sub;
    const bool valid = blk < n_blocks;
    const int r0 = (int)(blockIdx.x % ntile) * KT;
    const int n0 = valid ? block_ptr[blk] : 0, n1 = valid ? block_ptr[blk + 1] : 0;
    const int b = 4 * (n1 - n0);
    const int64_t base = 4 * (int64_t)n0;
    const int n4 = b * (b + 1) / 4;
    unsigned onm = 0;
#pragma unroll
    for (int q = 0; q < KT; ++q) onm |= ((r0 + q < k) && (!active || active[r0 + q])) ? 1u << q : 0u;
    if (!onm) return;  // the whole tile has retired (uniform over the CTA, before any barrier)
    float4* S4s = S4 + sub * (SYM_MAX_F4 / bpc);
    float (*rre_s)[KT] = rre + sub * tsub;
    float (*rim_s)[KT] = rim + sub * tsub;
    if (valid) {
        const float4* P4 = reinterpret_cast<const float4*>(pinv + poff[blk]);
        for (int e = tid; e < n4; e += tsub) S4s[e] = __ldg(P4 + e);
    }
    for (int f = tid; f < tsub * KT; f += tsub) {
        const int row = f / KT, q = f - row * KT;
        float2 v = make_float2(0.f, 0.f);
        if (row < b && ((onm >> q) & 1u)) v = r[(int64_t)(r0 + q) * ld + base + row];
        rre_s[row][q] = v.x;
        rim_s[row][q] = v.y;
    }
    __syncthreads();
    if (!valid || tid >= b) return;
    const float2* S = reinterpret_cast<const float2*>(S4s);
    unsigned long long are[4], aim[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) are[h] = aim[h] = 0ull;
    const int ti = tid * (tid + 1) / 2;
    int tj = 0;  // j (j + 1) / 2
#pragma unroll 2
    for (int j = 0; j < b; ++j) {
        const float2 a = S[j >= tid ? tj + tid : ti + j];
        const unsigned long long ax = f2pack(a.x, a.x), ay = f2pack(a.y, a.y), nay = f2pack(-a.y, -a.y);
        const ulonglong2 re01 = *reinterpret_cast<const ulonglong2*>(&rre_s[j][0]);
        const ulonglong2 re23 = *reinterpret_cast<const ulonglong2*>(&rre_s[j][4]);
        const ulonglong2 im01 = *reinterpret_cast<const ulonglong2*>(&rim_s[j][0]);
        const ulonglong2 im23 = *reinterpret_cast<const ulonglong2*>(&rim_s[j][4]);
        const unsigned long long vr[4] = {re01.x, re01.y, re23.x, re23.y};
        const unsigned long long vi[4] = {im01.x, im01.y, im23.x, im23.y};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            are[h] = ffma2(ax, vr[h], are[h]);
            are[h] = ffma2(nay, vi[h], are[h]);
            aim[h] = ffma2(ax, vi[h], aim[h]);
            aim[h] = ffma2(ay, vr[h], aim[h]);
        }
        tj += j + 1;
    }
    float2 acc[KT];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        f2unpack(are[h], acc[2 * h].x, acc[2 * h + 1].x);
        f2unpack(aim[h], acc[2 * h].y, acc[2 * h + 1].y);
    }
    if (zc && (tid & 3) == 3) {
        const int cc = blk_c[blk];
        const float w = zv[n0 + (tid >> 2)];
        if (cc >= 0 && w != 0.f)
#pragma unroll
            for (int q = 0; q < KT; ++q) {
                if (!((onm >> q) & 1u)) continue;
                const float2 v = zc[(int64_t)(r0 + q) * nc + cc];
                acc[q].x += w * v.x;
                acc[q].y += w * v.y;
            }
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if ((onm >> q) & 1u) {
            float2* zp = z + (int64_t)(r0 + q) * ld + base + tid;
            *zp = accumulate ? cadd(*zp, acc[q]) : acc[q];
        }
}

// blocks per 64-thread CTA of k_block_apply_sym8x2: as many as fit one thread per row
inline int sym8_blocks_per_cta(int max_block_nodes) {
    const int b = 4 * max_block_nodes;
    return b <= 16 ? 4 : b <= 32 ? 2 : 1;
}

// coarse restriction: rc[r][c] = sum over the group's nodes of zv[i] * r[r][4i+3]
template <typename T>
__global__ void __launch_bounds__(128) k_coarse_restrict(const C<T>* __restrict__ r, int64_t ld,
                                                         const int32_t* __restrict__ lo, const int32_t* __restrict__ hi,
                                                         const T* __restrict__ zv, int64_t nc,
                                                         const int* __restrict__ active, C<T>* __restrict__ rc) {
    __shared__ double sh[4][2];
    const int cc = blockIdx.x, rr = blockIdx.y;
    if (active && !active[rr]) return;
    double sx = 0.0, sy = 0.0;
    for (int i = lo[cc] + threadIdx.x; i < hi[cc]; i += blockDim.x) {
        const T w = zv[i];
        const C<T> v = r[(int64_t)rr * ld + 4 * (int64_t)i + 3];
        sx += (double)(w * v.x);
        sy += (double)(w * v.y);
    }
    sx = warp_sum(sx);
    sy = warp_sum(sy);
    if ((threadIdx.x & 31) == 0) {
        sh[threadIdx.x >> 5][0] = sx;
        sh[threadIdx.x >> 5][1] = sy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a += sh[w][0];
            b += sh[w][1];
        }
        rc[(int64_t)rr * nc + cc] = from_d<T>(make_double2(a, b));
    }
}

// split dense GEMV: part[s][r][c] = sum over d in chunk s of Einv[d][c] rc[r][d]
constexpr int GEMV_CHUNK = 64;

template <typename T, int KT>
__global__ void __launch_bounds__(256) k_gemv_split(const C<T>* __restrict__ einv, int64_t nc,
                                                    const C<T>* __restrict__ rc, int k,
                                                    const int* __restrict__ active, C<T>* __restrict__ part) {
    __shared__ C<T> rs[KT][GEMV_CHUNK];
    const int64_t cc = blockIdx.x * 256ll + threadIdx.x;
    const int s = blockIdx.y, r0 = blockIdx.z * KT;
    const int64_t d0 = (int64_t)s * GEMV_CHUNK;
    const int dn = (int)((nc - d0) < GEMV_CHUNK ? (nc - d0) : GEMV_CHUNK);
    bool on[KT], any = false;
#pragma unroll
    for (int q = 0; q < KT; ++q) {
        on[q] = (r0 + q < k) && (!active || active[r0 + q]);
        any |= on[q];
    }
    if (!any) return;  // the whole tile has retired (uniform over the CTA, before any barrier)
    for (int e = threadIdx.x; e < KT * GEMV_CHUNK; e += 256) {
        const int q = e / GEMV_CHUNK, d = e % GEMV_CHUNK;
        rs[q][d] = (on[q] && d < dn) ? rc[(int64_t)(r0 + q) * nc + d0 + d] : czero<T>();
    }
    __syncthreads();
    if (cc >= nc) return;
    C<T> acc[KT];
#pragma unroll
    for (int q = 0; q < KT; ++q) acc[q] = czero<T>();
#pragma unroll 8  // independent loads of the chunk's columns in flight together
    for (int d = 0; d < dn; ++d) {
        const C<T> a = einv[(d0 + d) * nc + cc];
#pragma unroll
        for (int q = 0; q < KT; ++q) cfma(acc[q], a, rs[q][d]);
    }
#pragma unroll
    for (int q = 0; q < KT; ++q)
        if (on[q]) part[((int64_t)s * k + r0 + q) * nc + cc] = acc[q];
}

template <typename T>
__global__ void k_gemv_sum(const C<T>* __restrict__ part, int S, int64_t nc, int k, const int* __restrict__ active,
                           C<T>* __restrict__ z) {
    const int64_t e = blockIdx.x * 256ll + threadIdx.x;
    if (e >= (int64_t)k * nc) return;
    const int r = (int)(e / nc);
    if (active && !active[r]) return;
    C<T> s = czero<T>();
    for (int q = 0; q < S; ++q) s = cadd(s, part[(int64_t)q * k * nc + e]);
    z[e] = s;
}

// in-place Gauss-Jordan inversion of the dense coarse matrix, pivot k (no
// pivoting: e^{i pi/4} E has a positive definite Hermitian part).  Step 1
// saves row k (scaled by 1/a_kk) and column k; step 2 updates everything.
__global__ void k_gj_save(double2* __restrict__ a, int64_t n, int64_t k, double2* __restrict__ rowk,
                          double2* __restrict__ colk, int* __restrict__ bad) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double2 piv = a[k * n + k];
    const double m = piv.x * piv.x + piv.y * piv.y;
    if (!(m > 0.0)) {
        if (j == 0) atomicExch(bad, 1);
        return;
    }
    const double2 p = make_double2(piv.x / m, -piv.y / m);
    rowk[j] = j == k ? p : cmul(a[k * n + j], p);
    colk[j] = a[j * n + k];
}

__global__ void k_gj_update(double2* __restrict__ a, int64_t n, int64_t k, const double2* __restrict__ rowk,
                            const double2* __restrict__ colk) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n * n) return;
    const int64_t i = e / n, j = e - i * n;
    const double2 p = rowk[k];
    if (i == k) {
        a[e] = rowk[j];
    } else if (j == k) {
        const double2 v = cmul(colk[i], p);
        a[e] = make_double2(-v.x, -v.y);
    } else {
        a[e] = csub(a[e], cmul(colk[i], rowk[j]));
    }
}

__global__ void k_gather_vv(const double2* __restrict__ val, int64_t nnzb, double2* __restrict__ vv) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s < nnzb) vv[s] = val[16 * s + 15];
}

__global__ void k_make_zv(const double* __restrict__ t, const uint8_t* __restrict__ fixmask, int64_t N,
                          double* __restrict__ zv, float* __restrict__ zv32) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double w = (fixmask[i] & 8) ? 0.0 : 1.0 / t[4 * i + 3];
    zv[i] = w;
    zv32[i] = (float)w;
}

__global__ void k_d2f_vec(const double2* __restrict__ a, float2* __restrict__ b, int64_t n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < n) b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

int pick_ptile(int k, int rhs_tile) {
    int kt = rhs_tile > 0 ? rhs_tile : 8;  // 0 (auto) and -1 use 8 here
    if (kt > k) kt = k;
    if (kt >= 8) return 8;
    if (kt >= 4) return 4;
    if (kt >= 2) return 2;
    return 1;
}

template <typename T>
void apply_impl(ect_ctx* c, Matrix& M, const C<T>* pinv, const C<T>* einv, const T* zv, const C<T>* r, C<T>* z,
                int k, int64_t ld, int rhs_tile, const int* active) {
    const int kt = pick_ptile(k, rhs_tile);
    const int nt = (k + kt - 1) / kt;
    const unsigned grid = tile_grid((unsigned)c->n_blocks, nt);
    const int32_t* bp = c->block_ptr.as<int32_t>();
    const int64_t* po = std::is_same<T, float>::value ? c->pinv_off32.as<int64_t>() : c->pinv_off.as<int64_t>();
    cudaStream_t st = c->stream;
    const int64_t nc = M.nc;
    C<T>* zc = nullptr;
    if (nc > 0) {
        ECT_REQUIRE(M.coarse_k >= k, ECT_ERR_STATE, "coarse scratch too small (internal)");
        C<T>* rc = M.rc.as<C<T>>();
        zc = M.zc.as<C<T>>();
        k_coarse_restrict<T><<<dim3((unsigned)nc, (unsigned)k), 128, 0, st>>>(r, ld, M.agg_lo.as<int32_t>(),
                                                                               M.agg_hi.as<int32_t>(), zv, nc, active, rc);
        dense_gemv<T>(st, einv, nc, rc, zc, k, rhs_tile, active, M.gpart.as<C<T>>());
    }
    const int32_t* bc = M.blk_c.as<int32_t>();
    if constexpr (std::is_same<T, float>::value) {
        const int bpc = sym8_blocks_per_cta(c->max_block_nodes);
        const unsigned grid8 = tile_grid((unsigned)((c->n_blocks + bpc - 1) / bpc), nt);
        switch (kt) {
            case 8: k_block_apply_sym8x2<<<grid8, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt,
                                                                c->n_blocks, bpc); break;
            case 4: k_block_apply_sym<4><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt); break;
            case 2: k_block_apply_sym<2><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt); break;
            default: k_block_apply_sym<1><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt); break;
        }
    } else {
        switch (kt) {
            case 8: k_block_apply<T, 8><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt); break;
            case 4: k_block_apply<T, 4><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt); break;
            case 2: k_block_apply<T, 2><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt); break;
            default: k_block_apply<T, 1><<<grid, 64, 0, st>>>(bp, po, pinv, r, z, k, ld, active, bc, zc, nc, zv, 0, nt); break;
        }
    }
    ECT_CHECK_LAUNCH();
}

// conductor-V coarse space: groups of `group` consecutive subdomains that
// contain a conducting node; E = Z^T S Z = sum of the unscaled V-V couplings
// between the groups' conducting nodes (assembled on the host in a fixed
// order), inverted on the device.
void coarse_setup(ect_ctx* c, int which, int group) {
    Matrix& M = ctx_mat(c, which);
    cudaStream_t st = c->stream;
    const int64_t N = c->n_nodes, nb = c->n_blocks;
    M.nc = 0;
    M.coarse_group = group;
    M.coarse_k = 0;
    for (DevBuf* b : {&M.einv, &M.einv32, &M.blk_c, &M.agg_lo, &M.agg_hi, &M.zv, &M.zv32, &M.rc, &M.zc}) b->release();
    if (group <= 0) return;
    const std::vector<int32_t>& bp = c->h_block_ptr;
    std::vector<int32_t> blk_c(nb, -1), lo, hi;
    std::vector<int32_t> node_c(N, -1);
    int64_t nc = 0;
    for (int64_t g0 = 0; g0 < nb; g0 += group) {
        const int64_t g1 = std::min<int64_t>(nb, g0 + group);
        bool any = false;
        for (int64_t i = bp[g0]; i < bp[g1] && !any; ++i) any = M.h_cond[i] != 0;
        if (!any) continue;
        for (int64_t b = g0; b < g1; ++b) blk_c[b] = (int32_t)nc;
        for (int64_t i = bp[g0]; i < bp[g1]; ++i)
            if (M.h_cond[i]) node_c[i] = (int32_t)nc;
        lo.push_back(bp[g0]);
        hi.push_back(bp[g1]);
        ++nc;
    }
    if (nc == 0) return;
    ECT_REQUIRE(nc <= 16384, ECT_ERR_ARG, "coarse space too large: use a larger coarse group");
    // V-V couplings of the unscaled matrix
    DevBuf vv;
    vv.alloc(sizeof(double2) * c->nnzb);
    k_gather_vv<<<grid_for(c->nnzb, 256), 256, 0, st>>>(M.val.as<double2>(), c->nnzb, vv.as<double2>());
    ECT_CHECK_LAUNCH();
    std::vector<double2> hvv(c->nnzb);
    ECT_CUDA(cudaMemcpyAsync(hvv.data(), vv.p, vv.bytes, cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    std::vector<double2> E((size_t)nc * nc, make_double2(0.0, 0.0));
    for (int64_t i = 0; i < N; ++i) {
        const int ci = node_c[i];
        if (ci < 0) continue;
        for (int32_t s = c->h_row_ptr[i]; s < c->h_row_ptr[i + 1]; ++s) {
            const int cj = node_c[c->h_col[s]];
            if (cj < 0) continue;
            double2& e = E[(size_t)ci * nc + cj];
            e.x += hvv[s].x;
            e.y += hvv[s].y;
        }
    }
    M.einv.alloc(sizeof(double2) * nc * nc);
    ECT_CUDA(cudaMemcpyAsync(M.einv.p, E.data(), M.einv.bytes, cudaMemcpyHostToDevice, st));
    DevBuf rowk, colk, flag;
    rowk.alloc(sizeof(double2) * nc);
    colk.alloc(sizeof(double2) * nc);
    flag.alloc(sizeof(int));
    ECT_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    for (int64_t kk = 0; kk < nc; ++kk) {
        k_gj_save<<<grid_for(nc, 256), 256, 0, st>>>(M.einv.as<double2>(), nc, kk, rowk.as<double2>(),
                                                     colk.as<double2>(), flag.as<int>());
        k_gj_update<<<grid_for(nc * nc, 256), 256, 0, st>>>(M.einv.as<double2>(), nc, kk, rowk.as<double2>(),
                                                            colk.as<double2>());
    }
    ECT_CHECK_LAUNCH();
    int bad = 0;
    ECT_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    ECT_REQUIRE(!bad, ECT_ERR_BREAKDOWN, "the coarse matrix has a zero pivot");
    M.einv32.alloc(sizeof(float2) * nc * nc);
    k_d2f_vec<<<grid_for(nc * nc, 256), 256, 0, st>>>(M.einv.as<double2>(), M.einv32.as<float2>(), nc * nc);
    M.blk_c.alloc(sizeof(int32_t) * nb);
    M.agg_lo.alloc(sizeof(int32_t) * nc);
    M.agg_hi.alloc(sizeof(int32_t) * nc);
    ECT_CUDA(cudaMemcpyAsync(M.blk_c.p, blk_c.data(), M.blk_c.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(M.agg_lo.p, lo.data(), M.agg_lo.bytes, cudaMemcpyHostToDevice, st));
    ECT_CUDA(cudaMemcpyAsync(M.agg_hi.p, hi.data(), M.agg_hi.bytes, cudaMemcpyHostToDevice, st));
    M.zv.alloc(sizeof(double) * N);
    M.zv32.alloc(sizeof(float) * N);
    k_make_zv<<<grid_for(N, 256), 256, 0, st>>>(M.t.as<double>(), M.fixmask.as<uint8_t>(), N, M.zv.as<double>(),
                                                M.zv32.as<float>());
    ECT_CHECK_LAUNCH();
    ECT_CUDA(cudaStreamSynchronize(st));
    M.nc = nc;
}

}  // namespace

void block_inverses(cudaStream_t st, const int32_t* rp, const int32_t* col, const double2* sval, const int32_t* bptr,
                    const int64_t* poff, const int64_t* poff32, int64_t n_blocks, int max_block_nodes, double2* pinv,
                    float2* pinv32) {
    const int bmax = 4 * max_block_nodes;
    ECT_REQUIRE(bmax <= 64, ECT_ERR_ARG, "smoothing block larger than 16 nodes");
    const size_t smem = sizeof(double2) * (size_t)bmax * 2 * bmax;
    ECT_CUDA(cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DevBuf flag;
    flag.alloc(sizeof(int));
    ECT_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    k_block_inverse<<<(unsigned)n_blocks, 256, smem, st>>>(rp, col, sval, bptr, poff, poff32, pinv, pinv32,
                                                           flag.as<int>());
    ECT_CHECK_LAUNCH();
    int h = 0;
    ECT_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    ECT_REQUIRE(!h, ECT_ERR_BREAKDOWN, "a smoothing block is singular");
}

template <typename T>
void block_apply(cudaStream_t st, const int32_t* bptr, const int64_t* poff, const C<T>* pinv, int64_t n_blocks,
                 int max_block_nodes, const C<T>* r, C<T>* z, int k, int64_t ld, int rhs_tile, const int* active,
                 bool accumulate) {
    const int kt = pick_ptile(k, rhs_tile);
    const int nt = (k + kt - 1) / kt;
    const unsigned grid = tile_grid((unsigned)n_blocks, nt);
    const int acc = accumulate ? 1 : 0;
    if constexpr (std::is_same<T, float>::value) {
        const int bpc = sym8_blocks_per_cta(max_block_nodes);
        const unsigned grid8 = tile_grid((unsigned)((n_blocks + bpc - 1) / bpc), nt);
        switch (kt) {
            case 8: k_block_apply_sym8x2<<<grid8, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0,
                                                                nullptr, acc, nt, n_blocks, bpc); break;
            case 4: k_block_apply_sym<4><<<grid, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0, nullptr, acc, nt); break;
            case 2: k_block_apply_sym<2><<<grid, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0, nullptr, acc, nt); break;
            default: k_block_apply_sym<1><<<grid, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0, nullptr, acc, nt); break;
        }
    } else {
        switch (kt) {
            case 8: k_block_apply<T, 8><<<grid, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0, nullptr, acc, nt); break;
            case 4: k_block_apply<T, 4><<<grid, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0, nullptr, acc, nt); break;
            case 2: k_block_apply<T, 2><<<grid, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0, nullptr, acc, nt); break;
            default: k_block_apply<T, 1><<<grid, 64, 0, st>>>(bptr, poff, pinv, r, z, k, ld, active, nullptr, nullptr, 0, nullptr, acc, nt); break;
        }
    }
    ECT_CHECK_LAUNCH();
}
template void block_apply<double>(cudaStream_t, const int32_t*, const int64_t*, const double2*, int64_t, int,
                                  const double2*, double2*, int, int64_t, int, const int*, bool);
template void block_apply<float>(cudaStream_t, const int32_t*, const int64_t*, const float2*, int64_t, int,
                                 const float2*, float2*, int, int64_t, int, const int*, bool);

// in-place dense inverse of a (n x n, complex128, row-major) on the device
void dense_inverse(cudaStream_t st, double2* a, int64_t n) {
    DevBuf rowk, colk, flag;
    rowk.alloc(sizeof(double2) * n);
    colk.alloc(sizeof(double2) * n);
    flag.alloc(sizeof(int));
    ECT_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    for (int64_t kk = 0; kk < n; ++kk) {
        k_gj_save<<<grid_for(n, 256), 256, 0, st>>>(a, n, kk, rowk.as<double2>(), colk.as<double2>(), flag.as<int>());
        k_gj_update<<<grid_for(n * n, 256), 256, 0, st>>>(a, n, kk, rowk.as<double2>(), colk.as<double2>());
    }
    ECT_CHECK_LAUNCH();
    int bad = 0;
    ECT_CUDA(cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    ECT_REQUIRE(!bad, ECT_ERR_BREAKDOWN, "the coarsest matrix has a zero pivot");
}

void to_f32(cudaStream_t st, const double2* a, float2* b, int64_t n) {
    k_d2f_vec<<<grid_for(n, 256), 256, 0, st>>>(a, b, n);
    ECT_CHECK_LAUNCH();
}

// z[r] = Einv r[r] (dense, symmetric Einv) for k vectors of length nc; part:
// scratch of gemv_scratch_elems(nc, k) complex values
int64_t gemv_scratch_elems(int64_t nc, int k) { return ((nc + GEMV_CHUNK - 1) / GEMV_CHUNK) * (int64_t)k * nc; }

template <typename T>
void dense_gemv(cudaStream_t st, const C<T>* einv, int64_t nc, const C<T>* r, C<T>* z, int k, int rhs_tile,
                const int* active, C<T>* part) {
    const int kt = pick_ptile(k, rhs_tile);
    const int S = (int)((nc + GEMV_CHUNK - 1) / GEMV_CHUNK);
    dim3 g1(grid_for(nc, 256), S, (unsigned)((k + kt - 1) / kt));
    switch (kt) {
        case 8: k_gemv_split<T, 8><<<g1, 256, 0, st>>>(einv, nc, r, k, active, part); break;
        case 4: k_gemv_split<T, 4><<<g1, 256, 0, st>>>(einv, nc, r, k, active, part); break;
        case 2: k_gemv_split<T, 2><<<g1, 256, 0, st>>>(einv, nc, r, k, active, part); break;
        default: k_gemv_split<T, 1><<<g1, 256, 0, st>>>(einv, nc, r, k, active, part); break;
    }
    k_gemv_sum<T><<<grid_for((int64_t)k * nc, 256), 256, 0, st>>>(part, S, nc, k, active, z);
    ECT_CHECK_LAUNCH();
}
template void dense_gemv<double>(cudaStream_t, const double2*, int64_t, const double2*, double2*, int, int, const int*,
                                 double2*);
template void dense_gemv<float>(cudaStream_t, const float2*, int64_t, const float2*, float2*, int, int, const int*,
                                float2*);

void precond_setup(ect_ctx* c, int which, int precision_mask, int coarse_group) {
    ECT_REQUIRE(which_valid(c, which), ECT_ERR_ARG, "bad which");
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.assembled, ECT_ERR_STATE, "ect_assemble must come before ect_precond_setup");
    M.pc_mask = precision_mask;
    M.pc_group = coarse_group;
    bool f32 = (precision_mask & ECT_F32) != 0;
    cudaStream_t st = c->stream;
    M.pinv.alloc(sizeof(double2) * c->pinv_total);
    if (f32) M.pinv32.alloc(sizeof(float2) * c->pinv_total32);
    else M.pinv32.release();
    const int bmax = 4 * c->max_block_nodes;
    const size_t smem = sizeof(double2) * (size_t)bmax * 2 * bmax;
    ECT_CUDA(cudaFuncSetAttribute(k_block_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    DevBuf flag;
    flag.alloc(sizeof(int));
    ECT_CUDA(cudaMemsetAsync(flag.p, 0, sizeof(int), st));
    k_block_inverse<<<(unsigned)c->n_blocks, 256, smem, st>>>(
        c->row_ptr.as<int32_t>(), c->col.as<int32_t>(), M.sval.as<double2>(), c->block_ptr.as<int32_t>(),
        c->pinv_off.as<int64_t>(), c->pinv_off32.as<int64_t>(), M.pinv.as<double2>(),
        f32 ? M.pinv32.as<float2>() : nullptr, flag.as<int>());
    ECT_CHECK_LAUNCH();
    int h = 0;
    ECT_CUDA(cudaMemcpyAsync(&h, flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    ECT_CUDA(cudaStreamSynchronize(st));
    ECT_REQUIRE(!h, ECT_ERR_BREAKDOWN, "a subdomain block of the scaled matrix is singular");
    mg_free(M);
    if (coarse_group < 0) {
        coarse_setup(c, which, 0);
        mg_setup(c, which, f32);
        M.pc_f64 = true;
        M.pc_f32 = f32;
        return;
    }
    coarse_setup(c, which, coarse_group);
    M.pc_f64 = true;
    M.pc_f32 = f32;
}

void coarse_scratch(ect_ctx* c, int which, int k) {
    Matrix& M = ctx_mat(c, which);
    if (M.mg && !mg_ready(M, k)) {  // new cycle vectors: captured graphs hold the old ones
        workspace_free(c);
        mg_scratch(M, k);
    }
    if (M.nc == 0 || M.coarse_k >= k) return;
    workspace_free(c);  // captured graphs hold the old scratch pointers
    M.rc.alloc(sizeof(double2) * M.nc * k);
    M.zc.alloc(sizeof(double2) * M.nc * k);
    M.gpart.alloc(sizeof(double2) * gemv_scratch_elems(M.nc, k));
    M.coarse_k = k;
}

void precond_apply_f64(ect_ctx* c, int which, const double2* r, double2* z, int k, int64_t ld, int rhs_tile,
                       const int* active) {
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.pc_f64, ECT_ERR_STATE, "preconditioner not set up");
    if (M.mg) {
        mg_apply_f64(c, which, r, z, k, ld, rhs_tile, active);
        return;
    }
    apply_impl<double>(c, M, M.pinv.as<double2>(), M.einv.as<double2>(), M.zv.as<double>(), r, z, k, ld, rhs_tile,
                       active);
}

void precond_apply_f32(ect_ctx* c, int which, const float2* r, float2* z, int k, int64_t ld, int rhs_tile,
                       const int* active) {
    Matrix& M = ctx_mat(c, which);
    ECT_REQUIRE(M.pc_f32, ECT_ERR_STATE, "FP32 preconditioner not set up (use ECT_F32 in ect_precond_setup)");
    if (M.mg) {
        mg_apply_f32(c, which, r, z, k, ld, rhs_tile, active);
        return;
    }
    apply_impl<float>(c, M, M.pinv32.as<float2>(), M.einv32.as<float2>(), M.zv32.as<float>(), r, z, k, ld, rhs_tile,
                      active);
}
